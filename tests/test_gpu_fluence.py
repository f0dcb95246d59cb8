"""Fluence (Eq. (5)), streamed fluence and coverage on the GPU against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2103_14137_gb300 as uvc
from synth import dwell_vectors, tiny_room
from tests.gpu_util import T, build, lamp_of

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
