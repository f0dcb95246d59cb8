"""Comparison of the CUDA path with the oracle.

Visibility: per (pair, source) bits must be identical except on pairs the
oracle flags as grazing; excused mismatches are capped at floor(1e-6 * pairs
* K).  Irradiance: on pairs whose bits all agree, relative error <= 1e-5 where
the oracle is positive, and exactly 0 where the oracle is 0.
"""
import math

import numpy as np

REL_TOL = 1e-5          # irradiance, relative (agreeing pairs)
GRAZE_CAP = 1e-6        # excused visibility mismatches per (pair, source)


def compare_irradiance(Ag, visg, E, ovis, flag, rel_tol=REL_TOL):
    """Ag (P,), visg (P,K) bool, E (P,), ovis (P,K), flag (P,) over P pairs."""
    Ag = np.asarray(Ag, np.float64).reshape(-1)
    E = np.asarray(E, np.float64).reshape(-1)
    K = ovis.shape[-1]
    visg = np.asarray(visg, bool).reshape(-1, K)
    ovis = np.asarray(ovis).astype(bool).reshape(-1, K)
    flag = np.asarray(flag).reshape(-1)
    bit_mism = visg != ovis
    pair_mism = bit_mism.any(axis=1)
    unexcused = int((pair_mism & (flag == 0)).sum())
    excused_bits = int(bit_mism[flag != 0].sum())
    cap = math.floor(GRAZE_CAP * E.size * K)
    assert unexcused == 0, f"{unexcused} visibility mismatches on non-grazing pairs"
    assert excused_bits <= cap, f"{excused_bits} grazing mismatches > cap {cap}"
    agree = ~pair_mism
    pos = agree & (E > 0)
    rel = np.abs(Ag[pos] - E[pos]) / E[pos] if pos.any() else np.zeros(1)
    assert np.all(np.isfinite(Ag)), "non-finite irradiance"
    assert rel.max() <= rel_tol, f"max relative error {rel.max():.3e} > {rel_tol}"
    zero = agree & (E == 0)
    assert np.all(Ag[zero] == 0.0), "nonzero irradiance where the oracle has none"
    return dict(pairs=E.size, max_rel=float(rel.max()), flagged=int((flag != 0).sum()),
                excused_bits=excused_bits, visible_frac=float(ovis.mean()))
