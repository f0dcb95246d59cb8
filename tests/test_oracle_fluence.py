"""Pins of the fluence (Eq. (5)) and coverage oracles: hand-computed values,
unit dwell vectors, rank-one matrices, inclusive threshold."""
import numpy as np

import oracle


def test_fluence_hand_example():
    A = np.array([[1, 2], [3, 4], [5, 6]], np.float32)       # 3 candidates x 2 patches
    t = np.array([[1, 0, 2], [0, 1, 0]], np.float32)          # 2 dwell vectors
    mu = oracle.fluence(A, t)
    assert mu.tolist() == [[11.0, 14.0], [3.0, 4.0]]


def test_fluence_unit_vector_and_rank_one():
    rng = np.random.default_rng(0)
    A = rng.uniform(0, 5, size=(7, 11))
    for k in range(7):
        e = np.zeros(7)
        e[k] = 1.0
        assert np.array_equal(oracle.fluence(A, e)[0], A[k])
    u = rng.uniform(size=7)
    w = rng.uniform(size=11)
    t = rng.uniform(size=(3, 7))
    mu = oracle.fluence(np.outer(u, w), t)
    assert np.allclose(mu, (t @ u)[:, None] * w[None, :], rtol=1e-14)


def test_coverage_hand_example():
    area = np.array([1, 2, 3, 4], np.float32)
    mu = np.array([[5, 10, 10, 20], [0, 0, 0, 0], [100, 100, 100, 100]], np.float32)
    by_area, by_count = oracle.coverage(mu, area, 10.0)
    assert by_area.tolist() == [0.9, 0.0, 1.0]
    assert by_count.tolist() == [0.75, 0.0, 1.0]
