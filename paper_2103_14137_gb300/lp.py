"""Dwell times from the relaxed linear program of Sec. IV-D, Eq. (9).

    minimise  sum_k t_k + sum_i p_i sigma_i
    subject to  mu_i + sigma_i >= mu_min   (mu_i = sum_k A[k, i] t_k, Eq. (5))
                sum_k t_k <= T_max,  t >= 0, sigma >= 0

Host code, as in the paper (which calls a commercial interior-point solver);
here HiGHS's interior-point method with crossover, through SciPy, so the
solution is a vertex and the dwell-time support {k : t_k > 0} is well defined.
The penalty follows the paper's advice p_i > ||A||_F: p_i = 10 ||A||_F a_i /
mean(a) (area-weighted, so that every patch counts by its size).
No torch import: the module runs in worker processes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog

MU_MIN = 100.0            # J/m^2 (10 mJ/cm^2)
T_MAX = 100.0 * 3600.0    # s


def lp_dwell(A, area, mu_min: float = MU_MIN, t_max: float = T_MAX, duals: bool = False):
    """Dwell times t (nc,) and slacks sigma (m,) for irradiance rows A (nc, m)
    in W/m^2 and patch areas (m,); with duals=True also the dose prices
    y (m,) >= 0 of the constraints mu_j + sigma_j >= mu_min (seconds per J/m^2).
    Raises RuntimeError if HiGHS fails."""
    A = np.asarray(A, np.float64)
    a = np.asarray(area, np.float64)
    nc, m = A.shape
    if nc == 0:
        return (np.zeros(0), np.full(m, mu_min)) + ((np.zeros(m),) if duals else ())
    p = 10.0 * max(np.linalg.norm(A), 1e-30) * a / a.mean()
    c = np.concatenate([np.ones(nc), p])
    At = sp.csr_matrix(A.T)
    A_ub = sp.vstack([sp.hstack([-At, -sp.identity(m, format="csr")]),
                      sp.hstack([sp.csr_matrix(np.ones((1, nc))), sp.csr_matrix((1, m))])]).tocsr()
    b_ub = np.concatenate([np.full(m, -mu_min), [t_max]])
    r = linprog(c, A_ub=A_ub, b_ub=b_ub, bounds=(0, None), method="highs-ipm")
    if r.status != 0:
        raise RuntimeError(f"HiGHS: {r.message}")
    t = np.maximum(r.x[:nc], 0.0)
    if duals:
        y = np.maximum(-np.asarray(r.ineqlin.marginals[:m], np.float64), 0.0)
        return t, np.maximum(r.x[nc:], 0.0), y
    return t, np.maximum(r.x[nc:], 0.0)


def efficiency(A, y):
    """eta_k = sum_j A[k, j] y_j: the dose value per second of candidate k at the
    LP's dual prices.  Complementary slackness gives eta_k = 1 wherever
    t_k > 0 (when the time budget does not bind) and eta_k <= 1 elsewhere, so
    eta ranks the candidates by how nearly they could replace the chosen ones."""
    return np.asarray(A, np.float64) @ np.asarray(y, np.float64)


def support(t, rel: float = 1e-6):
    """Candidates with non-zero dwell time (relative to the largest)."""
    t = np.asarray(t, np.float64)
    if t.size == 0 or t.max() <= 0:
        return np.zeros(t.shape, bool)
    return t > rel * t.max()


def patch_sample(np_: int, m: int, seed: int):
    """Seeded subset of m patch indices (sorted); all patches if np_ <= m."""
    if np_ <= m:
        return np.arange(np_)
    return np.sort(np.random.default_rng(seed).choice(np_, size=m, replace=False))


def solve_job(args):
    """Worker entry: (A_rows, area, mu_min, t_max) -> (t, seconds, eta)."""
    import time
    A, area, mu_min, t_max = args
    t0 = time.perf_counter()
    t, _, y = lp_dwell(A, area, mu_min, t_max, duals=True)
    return t, time.perf_counter() - t0, efficiency(A, y)
