"""Learned-proposal kernels on the GPU against the oracle: candidate features,
top-k selection, and the BF16 scorer's forward pass, gradients and Adam step."""
import numpy as np
import pytest
import torch

import paper_2103_14137_gb300 as uvc
from oracle import features as OF
from oracle import mlp as OM
from synth import tiny_room
from synth.batched import batched_room, design_candidates
from tests.gpu_util import T, build

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def check_features(s, cand):
    sc = build(s)
    got = uvc.candidate_features(sc, T(np.asarray(cand, np.float32))).cpu().numpy().astype(np.float64)
    sc.free()
    want, amb = OF.features(s.verts, s.tris, s.centroid, s.area, cand)
    a = np.asarray(s.area, np.float32).astype(np.float64)
    tot = a.sum()
    # a patch within rounding of a bin edge may land in the neighbouring bin;
    # positive-term FP32 sums carry at most (terms - 1) u relative error
    amb_area = (amb * a[None, :]).sum(1) / tot
    terms = -(-s.np_ // 256) + 256 + 2
    tol = amb_area[:, None] + terms * U32 * want[:, :64] + 1e-7 * want[:, :64]
    bad = np.abs(got[:, :64] - want[:, :64]) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], want[:, :64][bad][:5])
    D = float(np.linalg.norm(np.ptp(np.asarray(s.verts, np.float64), axis=0)))
    np.testing.assert_allclose(got[:, 64], want[:, 64], rtol=0, atol=1e-5 * D)
    np.testing.assert_array_equal(got[:, 65], want[:, 65])
    return got


def test_features_tiny_room_all_candidates():
    s = tiny_room()
    got = check_features(s, s.cand)
    np.testing.assert_allclose(got[:, :64].sum(1), 1.0, atol=1e-5)


def test_features_uneven_room_ragged_candidates():
    room = batched_room(105)
    cand = design_candidates(room, 0.8, 1.2, 37, seed=3)
    check_features(room, cand)


def test_features_empty_candidate_set():
    s = tiny_room(n_cand=3)
    sc = build(s)
    out = uvc.candidate_features(sc, torch.empty((0, 3), dtype=torch.float32, device="cuda"))
    assert out.shape == (0, 66)
    sc.free()


def reference_top(score, k):
    key = np.where(np.isnan(score), -np.inf, score.astype(np.float64))
    order = np.lexsort((np.arange(score.size), -key))      # higher score first, then lower index
    return np.sort(order[:k])


@pytest.mark.parametrize("n,k", [(1, 1), (7, 3), (1000, 200), (1000, 0), (5000, 1000), (16384, 3277), (16384, 16384),
                                 (333, 333)])
def test_select_top_bit_exact(n, k):
    rng = np.random.default_rng(n + k)
    score = rng.standard_normal(n).astype(np.float32)
    score[rng.uniform(size=n) < 0.2] = 0.5                  # many ties
    score[rng.uniform(size=n) < 0.01] = np.nan
    score[rng.uniform(size=n) < 0.01] = -0.0
    cand = rng.uniform(-5, 5, (n, 3)).astype(np.float32)
    idx, cs = uvc.select_top(T(score), k, cand=T(cand))
    want = reference_top(score, k)
    np.testing.assert_array_equal(idx.cpu().numpy(), want)
    np.testing.assert_array_equal(cs.cpu().numpy(), cand[want])


def seeded_params(in_dim, H, seed):
    rng = np.random.default_rng(seed)
    flat = np.zeros(OM.param_count(in_dim, H), np.float32)
    p = OM.split(flat, in_dim, H)
    P = OM.in_pad(in_dim)
    parts = {"W1": np.zeros((P, H)), "b1": rng.normal(0, 0.1, H), "W2": rng.normal(0, np.sqrt(2 / H), (H, H)),
             "b2": rng.normal(0, 0.1, H), "w3": rng.normal(0, np.sqrt(1 / H), H), "b3": [0.1]}
    parts["W1"][:in_dim] = rng.normal(0, np.sqrt(2 / in_dim), (in_dim, H))
    flat = np.concatenate([np.ravel(parts[k]) for k in p]).astype(np.float32)
    return flat


def feature_like(B, seed):
    rng = np.random.default_rng(seed)
    h = rng.dirichlet(np.full(64, 0.3), B)
    return np.concatenate([h * 8.0, rng.uniform(0.1, 3, (B, 1)), rng.uniform(0.3, 1.1, (B, 1))], 1).astype(np.float32)


def logit_tol(flat, x, d, H):
    """2^-8 times the absolute magnitude of the terms that feed each logit:
    each BF16 rounding site contributes at most half an ulp (2^-9)."""
    s, c = OM.forward(flat, x, d, H, True)
    p = c["p"]
    pre2 = np.abs(c["H1"]) @ np.abs(c["W2"]) + np.abs(p["b2"])
    scale = (np.abs(c["H2"]) + pre2) @ np.abs(p["w3"]) + abs(p["b3"][0])
    return s, 2.0 ** -8 * scale + 1e-6


@pytest.mark.parametrize("B", [1, 64, 333, 4100])
def test_mlp_forward_matches_oracle(B):
    d, H = 66, 256
    m = uvc.Mlp(d, H, max_batch=4100)
    flat = seeded_params(d, H, 11)
    m.set_params(flat)
    x = feature_like(B, B)
    got = m.forward(T(x)).cpu().numpy().astype(np.float64)
    want, tol = logit_tol(flat, x, d, H)
    assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want) / tol)
    m.close()


def test_mlp_train_step_gradients_and_adam():
    d, H, B, lr = 66, 256, 777, 1e-3
    m = uvc.Mlp(d, H, max_batch=1024)
    flat = seeded_params(d, H, 5)
    m.set_params(flat)
    x = feature_like(B, 9)
    rng = np.random.default_rng(2)
    y = (rng.uniform(size=B) < 0.2).astype(np.float32)
    w = np.where(y > 0, 2.0, 0.5).astype(np.float32) / B
    loss = m.train_step(T(x), T(y), T(w), lr).cpu().numpy()[0]
    g_gpu = m.grads().astype(np.float64)
    L, g_or = OM.gradients(flat, x, y, w, d, H, quant=True)
    assert abs(loss - L) <= 1e-3 * abs(L)
    gp, go = m.split(g_gpu), m.split(g_or)
    for name in gp:
        err = np.linalg.norm(gp[name] - go[name]) / max(np.linalg.norm(go[name]), 1e-30)
        assert err <= 1e-2, (name, err)
    assert np.all(gp["W1"][d:] == 0)                       # padded input rows
    # Adam's first step: -lr g / (|g| + eps) where the gradient is clearly non-zero
    p1 = m.params().astype(np.float64)
    want, _, _ = OM.adam(flat.astype(np.float64), g_or, 0.0, 0.0, 1, lr)
    big = np.abs(g_or) > 1e-2 * np.abs(g_or).max()
    np.testing.assert_allclose(p1[big], want[big], rtol=0, atol=1e-6)
    assert np.all(np.abs(p1 - flat) <= lr * (1 + 1e-6) + 1e-7)
    m.close()


def test_mlp_learns_a_separable_rule():
    d, H, B = 66, 256, 2048
    m = uvc.Mlp(d, H, max_batch=B, seed=1)
    x = feature_like(B, 21)
    y = (x[:, :8].sum(1) > np.median(x[:, :8].sum(1))).astype(np.float32)
    w = np.full(B, 1.0 / B, np.float32)
    xd, yd, wd = T(x), T(y), T(w)
    first = float(m.train_step(xd, yd, wd, 3e-3).item())
    for _ in range(300):
        last = m.train_step(xd, yd, wd, 3e-3)
    last = float(last.item())
    s = m.forward(xd).cpu().numpy()
    acc = np.mean((s > 0) == (y > 0))
    assert last < 0.3 * first and acc > 0.95, (first, last, acc)
    m.close()


def test_mlp_rejects_oversized_batch():
    m = uvc.Mlp(66, 64, max_batch=8)
    with pytest.raises(uvc.UvcError):
        m.forward(T(np.zeros((9, 66), np.float32)))
    m.close()


@pytest.mark.parametrize("nc,np_,k", [(1, 1, 1), (50, 333, 10), (1200, 3000, 240), (7, 0, 3)])
def test_probe_lost_matches_definition(nc, np_, k):
    rng = np.random.default_rng(nc + np_)
    A = rng.uniform(0, 1, (nc, np_)).astype(np.float32)
    A[rng.uniform(size=A.shape) < 0.97] = 0.0
    area = rng.uniform(0.001, 0.02, np_).astype(np.float32)
    idx = np.sort(rng.choice(nc, k, replace=False)).astype(np.int32)
    got = float(uvc.probe_lost(T(A), T(idx), T(area)).item())
    lit_all = (A > 0).any(0)
    lit_kept = (A[idx] > 0).any(0)
    want = float((area * (lit_all & ~lit_kept)).sum() / area.sum()) if np_ else 0.0
    assert abs(got - want) <= 1e-6 * max(want, 1e-30) + 1e-9


@pytest.mark.parametrize("nc,np_", [(1, 1), (37, 200), (1200, 3001), (5, 0)])
def test_probe_features_match_oracle(nc, np_):
    rng = np.random.default_rng(nc * 7 + np_)
    A = (rng.uniform(0, 3, (nc, np_)) ** 3).astype(np.float32)
    A[rng.uniform(size=A.shape) < 0.4] = 0.0
    if np_ > 4:
        A[:, :3] = 0.0                                      # unlit patches
        A[: max(1, nc // 2), 3] = 1.5                       # a tie for the best candidate
    area = rng.uniform(0.001, 0.02, np_).astype(np.float32)
    got = uvc.probe_features(T(A), T(area)).cpu().numpy().astype(np.float64)
    want, amb = OF.probe_features(A, area)
    lit = A.max(0) > 0 if np_ else np.zeros(0, bool)
    tol_amb = float(area[amb & lit].sum() / max(area[lit].sum(), 1e-30)) if np_ else 0.0
    tol = tol_amb + (np_ / 32 + 34) * U32 * want + 1e-7
    assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want) - tol)


def test_feature_columns_share_one_buffer():
    s = tiny_room()
    sc = build(s)
    cand = T(s.cand)
    rng = np.random.default_rng(0)
    A = rng.uniform(0, 1, (s.nc, 300)).astype(np.float32)
    area = rng.uniform(0.001, 0.02, 300).astype(np.float32)
    wide = torch.full((s.nc, 128), -7.0, device="cuda")
    uvc.candidate_features(sc, cand, feat=wide[:, :66])
    uvc.probe_features(T(A)[:, 100:], T(area[100:]), feat=wide[:, 66:114])
    a = uvc.candidate_features(sc, cand)
    b = uvc.probe_features(T(np.ascontiguousarray(A[:, 100:])), T(area[100:]))
    torch.testing.assert_close(wide[:, :66], a, rtol=0, atol=0)
    torch.testing.assert_close(wide[:, 66:114], b, rtol=0, atol=0)
    assert bool((wide[:, 114:] == -7.0).all())
    sc.free()


@pytest.mark.parametrize("nc,np_,rare", [(1, 5, 0), (40, 300, 0), (3000, 257, 0), (9, 0, 0), (40, 300, 3),
                                         (3000, 257, 2)])
def test_mark_best_bit_exact(nc, np_, rare):
    rng = np.random.default_rng(nc + 3 * np_)
    A = rng.integers(0, 5, (nc, np_)).astype(np.float32)    # many ties
    if np_:
        A[:, 0] = 0.0                                        # an unlit patch marks nothing
    if np_ > 10:
        for j in range(1, 8):                                # patches lit by j candidates only
            A[:, j] = 0.0
            A[rng.choice(nc, min(j, nc), replace=False), j] = 2.0
    score = rng.standard_normal(nc).astype(np.float32)
    got = uvc.mark_best(T(A), T(score), value=9.5, rare=rare).cpu().numpy()
    want = score.copy()
    for j in range(np_):
        if A[:, j].max() > 0:
            want[int(np.argmax(A[:, j]))] = 9.5              # first maximum = lowest index
            if (A[:, j] > 0).sum() <= rare:
                want[A[:, j] > 0] = 9.5
    np.testing.assert_array_equal(got, want)


def test_learned_selection_keeps_best_sources():
    """The shipped scorer end to end on one room: 20% kept, ascending indices,
    every sketch patch's best source among them, the check in [0, 1]."""
    from paper_2103_14137_gb300 import proposal as prop
    from synth.batched import designs
    from synth.scenes import line_lamp
    room = batched_room(131)
    h, L, K = designs()[4]
    cand = design_candidates(room, h, L, 700, seed=5)
    sc = build(room)
    lamp = line_lamp(L, K, 120.0)
    cd = T(cand)
    probe, half = prop.probe_columns(room.np_, seed=9)
    pi = torch.from_numpy(probe).cuda()
    A, _ = uvc.irradiance_matrix(sc, cd, uvc.Lamp(lamp.offsets, lamp.weights, lamp.power))
    Ap = A.index_select(1, pi).contiguous()
    area = T(np.asarray(room.area, np.float32)).index_select(0, pi).contiguous()
    scorer = prop.Scorer.load()
    feat = prop.features(sc, cd, Ap[:, :half], area[:half])
    assert bool(torch.isfinite(feat).all())
    idx, kept = scorer.select(feat, cd, A_sketch=Ap[:, :half])
    idx = idx.cpu().numpy()
    assert idx.size == prop.keep_count(cand.shape[0]) and np.all(np.diff(idx) > 0)
    np.testing.assert_array_equal(kept.cpu().numpy(), cand[idx])
    Ah = Ap[:, :half].cpu().numpy()
    lit = Ah.max(0) > 0
    best = np.unique(Ah.argmax(0)[lit])
    if best.size <= idx.size:
        assert np.isin(best, idx).all()
    lost = float(uvc.probe_lost(Ap[:, half:], T(idx.astype(np.int32)), area[half:]).item())
    assert 0.0 <= lost <= 1.0
    scorer.close()
    sc.free()


@pytest.mark.parametrize("n,group", [(1, 10), (95, 10), (1000, 7), (333, 1)])
def test_group_boost_bit_exact(n, group):
    rng = np.random.default_rng(n + group)
    score = rng.integers(-3, 3, n).astype(np.float32)        # ties within groups
    score[rng.uniform(size=n) < 0.05] = np.nan
    got = uvc.group_boost(T(score), group, bonus=1000.0).cpu().numpy()
    want = score.copy()
    for g0 in range(0, n, group):
        seg = np.where(np.isnan(score[g0:g0 + group]), -np.inf, score[g0:g0 + group])
        w = g0 + int(np.argmax(seg))                          # first maximum
        want[w] = np.float32(score[w] + np.float32(1000.0))
    np.testing.assert_array_equal(got, want)
