"""Pins of the scorer oracle: bfloat16 rounding by the format's definition and
against torch's converter, a hand-worked network, the loss at a zero logit,
finite differences of the FP64 network, and Adam's first step in closed form."""
import numpy as np
import pytest

from oracle import mlp as M


def test_bf16_rounding_definition():
    u = 2.0 ** -8                                           # half an ulp of 1 in bfloat16
    cases = {1.0: 1.0, 1 + u: 1.0,                          # tie -> even (1.0)
             1 + 3 * u: 1 + 4 * u,                          # tie between 1+2u and 1+4u -> even mantissa
             1 + u + 2 ** -20: 1 + 2 * u,                   # just above the tie
             -(1 + 3 * u): -(1 + 4 * u), 0.0: 0.0, 3.0: 3.0, 2.0 ** -130: 2.0 ** -130}
    for x, want in cases.items():
        assert M.bf16(np.array([x]))[0] == want, x


def test_bf16_matches_torch_converter():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(1).standard_normal(20000) * 10.0 ** np.random.default_rng(2).integers(-20, 20, 20000)
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16(x), want)


def hand_network():
    """in_dim 2, hidden 8: W1 routes x0 to unit 0 and -x0 to unit 1 and x1 to
    unit 2; W2 = identity; w3 = (1, 2, 3, ...); b1 = (0, 0, 0.25, 0...)."""
    in_dim, H = 2, 8
    flat = np.zeros(M.param_count(in_dim, H), np.float32)
    p = M.split(flat, in_dim, H)
    W1 = np.zeros((16, H))
    W1[0, 0], W1[0, 1], W1[1, 2] = 1.0, -1.0, 1.0
    b1 = np.zeros(H)
    b1[2] = 0.25
    parts = {"W1": W1, "b1": b1, "W2": np.eye(H), "b2": np.zeros(H), "w3": np.arange(1.0, H + 1), "b3": [0.5]}
    flat = np.concatenate([np.ravel(parts[k]) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]).astype(np.float32)
    assert flat.size == sum(v.size for v in p.values())
    return flat, in_dim, H


def test_hand_worked_forward():
    flat, d, H = hand_network()
    x = np.array([[0.5, -2.0], [-1.5, 1.0]])
    # row 0: units (0.5, 0, 0) -> s = 1*0.5 + 0.5 = 1.0
    # row 1: units (0, 1.5, 1.25) -> s = 2*1.5 + 3*1.25 + 0.5 = 7.25
    for quant in (False, True):
        s, _ = M.forward(flat, x, d, H, quant)
        np.testing.assert_array_equal(s, [1.0, 7.25])


def test_loss_at_zero_logit_is_log2():
    flat, d, H = hand_network()
    flat = flat.copy()
    flat[-1 - H:] = 0.0                                     # w3 = 0, b3 = 0 -> every logit is 0
    x = np.random.default_rng(0).standard_normal((3, 2))
    w = np.array([1.0, 2.0, 0.5])
    y = np.array([0.0, 1.0, 1.0])
    assert np.isclose(M.loss(flat, x, y, w, d, H, quant=False), np.log(2) * w.sum())
    # the logit gradient is w (1/2 - y): b3 gets its sum
    _, g = M.gradients(flat, x, y, w, d, H, quant=False)
    assert np.isclose(g[-1], np.sum(w * (0.5 - y)))


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(7)
    d, H, B = 5, 16, 12
    n = M.param_count(d, H)
    flat = rng.standard_normal(n) * 0.5
    P = M.in_pad(d)
    W1 = flat[:P * H].reshape(P, H)
    W1[d:] = 0.0
    x = rng.standard_normal((B, d))
    y = (rng.uniform(size=B) > 0.5).astype(float)
    w = rng.uniform(0.5, 2.0, B)
    L, g = M.gradients(flat, x, y, w, d, H, quant=False)
    assert np.isclose(L, M.loss(flat, x, y, w, d, H, quant=False))
    idx = np.concatenate([rng.choice(d * H, 12, replace=False),                 # W1 (live rows)
                          P * H + rng.choice(H, 4, replace=False),               # b1
                          P * H + H + rng.choice(H * H, 12, replace=False),      # W2
                          P * H + H + H * H + rng.choice(H, 4, replace=False),   # b2
                          P * H + 2 * H + H * H + rng.choice(H, 4, replace=False),   # w3
                          [n - 1]])                                               # b3
    h = 1e-6
    for k in idx:
        e = np.zeros(n)
        e[k] = h
        fd = (M.loss(flat + e, x, y, w, d, H, False) - M.loss(flat - e, x, y, w, d, H, False)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])
    # padded rows of W1 get no gradient
    assert np.all(g[d * H:P * H] == 0)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p0, g = rng.standard_normal(50), rng.standard_normal(50)
    p1, m, v = M.adam(p0, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    # bias-corrected moments are g and g^2 on the first step
    np.testing.assert_allclose(p1, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
    # second step with the same gradient: the corrected moments are again g, g^2
    p2, _, _ = M.adam(p1, g, m, v, 2, 1e-3)
    np.testing.assert_allclose(p2 - p1, -1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)
