"""The relaxed LP of Eq. (9) on problems whose optimum is known in closed form."""
import numpy as np
import pytest

pytest.importorskip("scipy")
from paper_2103_14137_gb300.lp import lp_dwell, patch_sample, support  # noqa: E402


def test_separate_candidates_each_cover_their_patch():
    # candidate 0 lights patch 0 at 1 W/m^2, candidate 1 lights patch 1 at 2 W/m^2
    t, s = lp_dwell([[1.0, 0.0], [0.0, 2.0]], [1.0, 1.0], mu_min=100.0)
    np.testing.assert_allclose(t, [100.0, 50.0], rtol=1e-7)
    np.testing.assert_allclose(s, 0.0, atol=1e-7)


def test_a_candidate_seeing_both_patches_wins():
    t, _ = lp_dwell([[1.0, 0.0], [0.0, 2.0], [1.0, 1.0]], [1.0, 1.0], mu_min=100.0)
    np.testing.assert_allclose(t, [0.0, 0.0, 100.0], atol=1e-6)
    assert support(t).tolist() == [False, False, True]


def test_invisible_patch_takes_the_slack():
    t, s = lp_dwell([[2.0, 0.0]], [1.0, 1.0], mu_min=100.0)
    np.testing.assert_allclose(t, [50.0], rtol=1e-7)
    np.testing.assert_allclose(s, [0.0, 100.0], atol=1e-6)


def test_time_budget_binds():
    t, s = lp_dwell([[1.0, 1.0]], [1.0, 1.0], mu_min=100.0, t_max=60.0)
    np.testing.assert_allclose(t, [60.0], rtol=1e-7)
    np.testing.assert_allclose(s, [40.0, 40.0], rtol=1e-6)


def test_patch_sample_is_seeded_sorted_and_complete_when_small():
    a = patch_sample(1000, 100, 3)
    assert a.size == 100 and np.all(np.diff(a) > 0) and np.array_equal(a, patch_sample(1000, 100, 3))
    assert np.array_equal(patch_sample(50, 100, 3), np.arange(50))


def test_dual_prices_give_unit_efficiency_on_the_support():
    from paper_2103_14137_gb300.lp import efficiency
    rng = np.random.default_rng(4)
    A = rng.uniform(0, 3, (60, 40))
    A[rng.uniform(size=A.shape) < 0.6] = 0
    A[0] = 0.05                                            # every patch lit by someone: no slack
    t, s, y = lp_dwell(A, rng.uniform(0.5, 1.5, 40), mu_min=100.0, duals=True)
    eta = efficiency(A, y)
    assert np.all(eta <= 1 + 1e-6)                         # dual feasibility
    np.testing.assert_allclose(eta[support(t)], 1.0, atol=1e-6)   # complementary slackness
    np.testing.assert_allclose(s, 0.0, atol=1e-7)
    assert np.isclose(t.sum(), 100.0 * y.sum(), rtol=1e-6)          # strong duality


def test_first_example_duals():
    # two separate candidates: prices 1/1 and 1/2 seconds per J/m^2
    from paper_2103_14137_gb300.lp import efficiency
    t, s, y = lp_dwell([[1.0, 0.0], [0.0, 2.0], [0.5, 0.5]], [1.0, 1.0], mu_min=100.0, duals=True)
    np.testing.assert_allclose(y, [1.0, 0.5], rtol=1e-7)
    np.testing.assert_allclose(efficiency([[1.0, 0.0], [0.0, 2.0], [0.5, 0.5]], y), [1.0, 1.0, 0.75], rtol=1e-7)
