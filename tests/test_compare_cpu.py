"""The comparison the GPU parity tests rely on (tests/_compare.py) rejects every
kind of disagreement it is meant to catch and accepts what the parity bar
allows: checked here on the CPU with an oracle result and planted departures."""
import numpy as np
import pytest

from tests._compare import compare_irradiance


def _case(rng, P=2_000_000, K=1):
    ovis = rng.uniform(size=(P, K)) < 0.6
    E = np.where(ovis.any(axis=1), rng.uniform(0.5, 50.0, P), 0.0)
    flag = np.zeros(P, np.uint8)
    flag[rng.choice(P, 20, replace=False)] = 1
    return E.astype(np.float32).astype(np.float64), ovis, flag


def test_identical_results_pass_and_report():
    rng = np.random.default_rng(0)
    E, ovis, flag = _case(rng)
    st = compare_irradiance(E.astype(np.float32), ovis, E, ovis, flag)
    assert st["pairs"] == E.size and st["excused_bits"] == 0 and st["flagged"] == 20 and st["max_rel"] == 0.0


def test_allowed_departures_pass():
    rng = np.random.default_rng(1)
    E, ovis, flag = _case(rng)
    A = E * (1 + 0.9e-5 * rng.choice([-1, 1], E.size))          # within 1e-5
    g = ovis.copy()
    f = np.flatnonzero(flag)[:2]                                 # 2 bits on flagged pairs <= cap floor(1e-6 * 2e6) = 2
    g[f, 0] = ~g[f, 0]
    compare_irradiance(A, g, E, ovis, flag)


@pytest.mark.parametrize("kind", ["bit_on_unflagged_pair", "bits_over_the_cap", "entry_off_by_2e-5",
                                  "light_where_the_oracle_has_none", "nan_entry"])
def test_each_departure_is_rejected(kind):
    rng = np.random.default_rng(2)
    E, ovis, flag = _case(rng)
    A, g = E.copy(), ovis.copy()
    unflagged_visible = np.flatnonzero((flag == 0) & (E > 0))
    if kind == "bit_on_unflagged_pair":
        g[unflagged_visible[0], 0] = ~g[unflagged_visible[0], 0]
    elif kind == "bits_over_the_cap":
        f = np.flatnonzero(flag)[:3]
        g[f, 0] = ~g[f, 0]
    elif kind == "entry_off_by_2e-5":
        A[unflagged_visible[5]] *= 1 + 2e-5
    elif kind == "light_where_the_oracle_has_none":
        A[np.flatnonzero((flag == 0) & (E == 0))[0]] = 1e-30
    else:
        A[unflagged_visible[7]] = np.nan
    with pytest.raises(AssertionError):
        compare_irradiance(A, g, E, ovis, flag)
