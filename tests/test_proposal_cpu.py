"""Host logic of the learned proposal: folding the input standardisation into
the first layer, keep counts, and the probe split."""
import numpy as np

from oracle import mlp as OM
from paper_2103_14137_gb300.proposal import fold_standardisation, keep_count, probe_columns


def test_folded_parameters_take_raw_features():
    rng = np.random.default_rng(0)
    d, H, B = 114, 32, 50
    flat = rng.standard_normal(OM.param_count(d, H)) * 0.3
    P = OM.in_pad(d)
    flat[d * H:P * H] = 0.0
    mean, std = rng.uniform(-2, 2, d), rng.uniform(0.01, 3, d)
    x = rng.standard_normal((B, d)) * std + mean
    s_std, _ = OM.forward(flat, (x - mean) / std, d, H, quant=False)
    s_raw, _ = OM.forward(fold_standardisation(flat, mean, std, d, H).astype(np.float64), x, d, H, quant=False)
    np.testing.assert_allclose(s_raw, s_std, rtol=1e-4, atol=1e-4)


def test_keep_count_and_probe_split():
    assert keep_count(0) == 0 and keep_count(1) == 1 and keep_count(10) == 2 and keep_count(11) == 3
    cols, half = probe_columns(100000, 3)
    assert cols.size == 1000 and half == 500 and np.unique(cols).size == 1000
    assert np.all(np.diff(cols[:half]) > 0) and np.all(np.diff(cols[half:]) > 0)
