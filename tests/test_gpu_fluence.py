"""Fluence (Eq. (5)), streamed fluence and coverage on the GPU against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2103_14137_gb300 as uvc
from synth import dwell_vectors, tiny_room
from tests.gpu_util import T, build, build_arrays, lamp_of

pytestmark = pytest.mark.gpu
MU_TOL = 1e-5


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-30)))


def test_fluence_random_matrix_ragged_sizes():
    rng = np.random.default_rng(4)
    s = tiny_room(n_cand=3)
    sc = build(s)
    np_ = s.np_
    for nc, nvec in ((1, 1), (77, 3), (2000, 16), (301, 37)):
        A = rng.uniform(0, 10, size=(nc, np_)).astype(np.float32)
        A[rng.uniform(size=A.shape) < 0.3] = 0.0
        t = rng.uniform(0, 60, size=(nvec, nc)).astype(np.float32)
        mu = uvc.fluence(sc, T(A), T(t)).cpu().numpy()
        assert _rel(mu, oracle.fluence(A, t)) <= MU_TOL, (nc, nvec)
    sc.free()


def _rows_of(nc, n, lda):
    """(nc, n) view of a (nc, lda) buffer (padded rows)."""
    return torch.empty((nc, lda), dtype=torch.float32, device="cuda")[:, :n]


@pytest.mark.parametrize("n", [3, 640, 641, 643, 988])
def test_fluence_padded_rows_match_unpadded(n):
    """On the CUDA cores, A given as a view of wider rows (row stride a
    multiple of 4 floats: the tensor-map kernel) and with odd or unpadded
    strides (register-fed kernel) give the same fluence bit for bit and match
    the oracle, including column tiles with 1-3 leftover columns and fewer
    than 4 patches."""
    rng = np.random.default_rng(n)
    s = tiny_room(n_cand=3)
    sc = build_arrays(s.verts, s.tris, s.centroid[:n], s.normal[:n], s.area[:n], s.excl[:n])
    for nc, nvec in ((1, 1), (77, 3), (2000, 16), (301, 37)):
        A = rng.uniform(0, 10, size=(nc, n)).astype(np.float32)
        A[rng.uniform(size=A.shape) < 0.3] = 0.0
        t = rng.uniform(0, 60, size=(nvec, nc)).astype(np.float32)
        Ab = _rows_of(nc, n, (n + 3) // 4 * 4)
        Ab.copy_(T(A))
        Ap = _rows_of(nc, n, n if n % 2 else n + 1)   # odd stride: 4-byte loads
        Ap.copy_(T(A))
        prev = uvc.set_fluence_tensor_cores(False)
        try:
            mu_b = uvc.fluence(sc, Ab, T(t))
            mu_p = uvc.fluence(sc, Ap, T(t))
        finally:
            uvc.set_fluence_tensor_cores(prev)
        torch.cuda.synchronize()
        assert uvc.scene_status(sc) == 0
        assert torch.equal(mu_b, mu_p), (n, nc, nvec)
        assert _rel(mu_b.cpu().numpy(), oracle.fluence(A, t)) <= MU_TOL, (n, nc, nvec)
    sc.free()


def test_fluence_padded_rows_ward_size():
    """The ward's shape (2,000 x 102,030, 16 vectors, ragged last tile of 14
    columns) with even and odd row strides on the CUDA cores: bit-identical."""
    from synth import ward_room
    s = ward_room(n_cand=4)
    sc = build(s)
    g = torch.Generator(device="cuda").manual_seed(3)
    Ab = _rows_of(2000, s.np_, (s.np_ + 3) // 4 * 4)
    Ab.copy_(torch.rand((2000, s.np_), generator=g, device="cuda"))
    Ap = _rows_of(2000, s.np_, s.np_ + 1)
    Ap.copy_(Ab)
    t = torch.rand((16, 2000), generator=g, device="cuda") * 60
    prev = uvc.set_fluence_tensor_cores(False)
    try:
        mu_b, mu_p = uvc.fluence(sc, Ab, t), uvc.fluence(sc, Ap, t)
    finally:
        uvc.set_fluence_tensor_cores(prev)
    torch.cuda.synchronize()
    assert uvc.scene_status(sc) == 0 and torch.equal(mu_b, mu_p)
    sc.free()


@pytest.mark.parametrize("n", [3, 128, 129, 641, 988])
def test_fluence_tensor_cores_against_oracle(n):
    """The tensor-core kernel (rows on 16-byte boundaries) against the FP64
    product, element by element within the same 1e-5 relative bound as the
    CUDA cores: candidate counts below, at and across the 32-row stage (1, 31,
    32, 33, 77, 301, 2,000), vector counts across the 16-vector pass (1, 16,
    17, 37), strips with a ragged tail, values over six decades and exact
    zeros; and against the CUDA-core kernel on the same buffer."""
    rng = np.random.default_rng(100 + n)
    s = tiny_room(n_cand=3)
    sc = build_arrays(s.verts, s.tris, s.centroid[:n], s.normal[:n], s.area[:n], s.excl[:n])
    for nc, nvec in ((1, 1), (31, 2), (32, 16), (33, 17), (77, 3), (2000, 16), (301, 37)):
        A = np.exp(rng.uniform(np.log(1e-4), np.log(1e2), size=(nc, n))).astype(np.float32)
        A[rng.uniform(size=A.shape) < 0.3] = 0.0
        t = rng.uniform(0, 60, size=(nvec, nc)).astype(np.float32)
        Ab = _rows_of(nc, n, (n + 3) // 4 * 4)
        Ab.copy_(T(A))
        mu_tc = uvc.fluence(sc, Ab, T(t))
        prev = uvc.set_fluence_tensor_cores(False)
        try:
            mu_cc = uvc.fluence(sc, Ab, T(t))
        finally:
            uvc.set_fluence_tensor_cores(prev)
        torch.cuda.synchronize()
        assert uvc.scene_status(sc) == 0
        ref = oracle.fluence(A, t)
        got = mu_tc.cpu().numpy()
        assert np.all(got[ref == 0] == 0), (n, nc, nvec)
        assert _rel(got, ref) <= MU_TOL, (n, nc, nvec, _rel(got, ref))
        assert _rel(got, mu_cc.cpu().numpy()) <= 2 * MU_TOL, (n, nc, nvec)
    sc.free()


def test_fluence_tensor_cores_ward_size():
    """The ward's shape (2,000 x 102,030, 16 vectors) on the tensor cores
    against the FP64 product and the CUDA-core kernel; all-zero A gives zeros."""
    from synth import ward_room
    s = ward_room(n_cand=4)
    sc = build(s)
    g = torch.Generator(device="cuda").manual_seed(5)
    Ab = _rows_of(2000, s.np_, (s.np_ + 3) // 4 * 4)
    Ab.copy_(torch.rand((2000, s.np_), generator=g, device="cuda") * 20)
    t = torch.rand((16, 2000), generator=g, device="cuda") * 60
    mu_tc = uvc.fluence(sc, Ab, t)
    prev = uvc.set_fluence_tensor_cores(False)
    try:
        mu_cc = uvc.fluence(sc, Ab, t)
    finally:
        uvc.set_fluence_tensor_cores(prev)
    torch.cuda.synchronize()
    assert uvc.scene_status(sc) == 0
    ref = oracle.fluence(Ab.cpu().numpy(), t.cpu().numpy())
    got = mu_tc.cpu().numpy()
    err = _rel(got, ref)
    print(f"tensor-core fluence, ward shape: max relative error {err:.3e} "
          f"(CUDA cores {_rel(mu_cc.cpu().numpy(), ref):.3e})")
    assert err <= MU_TOL
    Ab.zero_()
    assert torch.count_nonzero(uvc.fluence(sc, Ab, t)).item() == 0
    sc.free()


def test_fluence_and_streamed_match_oracle_end_to_end():
    s = tiny_room()
    sc = build(s)
    t = dwell_vectors(16, s.nc)
    A, _ = uvc.irradiance_matrix(sc, T(s.cand), lamp_of(s.lamp))
    mu = uvc.fluence(sc, A, T(t)).cpu().numpy()
    mus = uvc.fluence_streamed(sc, T(s.cand), lamp_of(s.lamp), T(t)).cpu().numpy()
    E, _, flag = oracle.irradiance_scene(s, flags=True)
    assert not flag.any()
    mu_o = oracle.fluence(E, t)
    assert _rel(mu, mu_o) <= MU_TOL
    assert _rel(mus, mu_o) <= MU_TOL
    sc.free()


def test_streamed_many_vectors_and_chunks():
    s = tiny_room(n_cand=150)
    sc = build(s)
    t = dwell_vectors(64, s.nc, seed=9)
    A, _ = uvc.irradiance_matrix(sc, T(s.cand), lamp_of(s.lamp))
    mus = uvc.fluence_streamed(sc, T(s.cand), lamp_of(s.lamp), T(t)).cpu().numpy()
    mu_o = oracle.fluence(A.cpu().numpy(), t)     # same A: isolates the streamed summation
    assert _rel(mus, mu_o) <= MU_TOL
    sc.free()


def test_coverage_matches_oracle_decisions():
    rng = np.random.default_rng(2)
    s = tiny_room(n_cand=3)
    sc = build(s)
    mu = rng.uniform(0, 200, size=(5, s.np_)).astype(np.float32)
    mu[1] = 100.0                       # all exactly at the threshold: inclusive
    mu[2] = 0.0
    ca, cc = uvc.coverage(sc, T(mu), 100.0)
    oa, oc = oracle.coverage(mu, s.area, 100.0)
    assert np.allclose(ca.cpu().numpy(), oa, rtol=1e-6, atol=0)
    assert np.allclose(cc.cpu().numpy(), oc, rtol=1e-6, atol=0)
    assert ca[1].item() == pytest.approx(1.0, abs=1e-6) and ca[2].item() == 0.0
    sc.free()


def _streamed_vs_oracle(s, sc, cand, L, t, bvh):
    """Streamed fluence of a vertical line lamp (the wedge search) against
    mu = t E with E from the oracle.  Columns where some pair of a candidate
    with t > 0 is flagged as grazing may legitimately differ by that pair's
    term; they are counted and left out, every other column must agree
    within the fluence tolerance."""
    mus = uvc.fluence_streamed(sc, T(cand), lamp_of(L), T(t)).cpu().numpy()
    torch.cuda.synchronize()
    assert uvc.scene_status(sc) == 0
    E, _, flag = oracle.irradiance(s.verts, s.tris, s.centroid, s.normal, s.excl, cand, L.offsets, L.weights,
                                   L.power, flags=True, bvh=bvh)
    mu_o = oracle.fluence(E, t)
    used = (t > 0).any(axis=0)
    excused = (flag[used] != 0).any(axis=0)
    ok = ~excused
    assert _rel(mus[:, ok], mu_o[:, ok]) <= MU_TOL
    return int(excused.sum())


def test_streamed_line_lamp_against_oracle_tiny_room_three_heights():
    """K = 8 vertical line lamp (1.2 m) on the tiny room from candidates at
    three lamp-bottom heights (0.3 m and 0.62 m put the tube across the table
    top's plane), 64 dwell vectors: the streamed wedge kernel against the
    brute-force oracle's E."""
    from synth.scenes import line_lamp
    s = tiny_room(n_cand=60)
    sc = build(s)
    cand = s.cand.copy()
    cand[:, 2] = np.where(np.arange(60) % 3 == 0, 0.3, np.where(np.arange(60) % 3 == 1, 0.62, 1.0))
    L = line_lamp(1.2, 8, 120.0)
    t = dwell_vectors(64, 60, seed=17)
    n_excused = _streamed_vs_oracle(s, sc, cand.astype(np.float32), L, t, bvh=False)
    assert n_excused <= 0.01 * s.np_
    sc.free()


def test_streamed_line_lamp_against_oracle_ward_rows():
    """24 whole rows of the full-size ward (candidates spread over the list x
    all 102,030 patches, the benchmark's K = 8 lamp, 16 dwell vectors) through
    the streamed wedge kernel, against mu from the oracle's CPU-BVH entries."""
    from synth import ward_room
    s = ward_room()
    sc = build(s)
    rows = np.linspace(0, s.nc - 1, 24).astype(np.int64)
    cand = np.ascontiguousarray(s.cand[rows])
    t = dwell_vectors(16, rows.size, seed=23)
    n_excused = _streamed_vs_oracle(s, sc, cand, s.lamp, t, bvh=True)
    assert n_excused <= 0.05 * s.np_
    sc.free()
