"""Planted mistakes in the Python oracles (LBVH, candidate features, the
scorer network, fluence and coverage), each of which must make one of that
oracle's pins fail: evidence that the pins constrain every step.  A mutant is
one function's source with one text replacement, compiled in the module's
namespace and swapped in for the duration of the test.  Runs on the CPU."""
import inspect
import textwrap

import pytest

import oracle
from oracle import features, lbvh, mlp
from tests import test_oracle_features, test_oracle_fluence, test_oracle_lbvh, test_oracle_mlp

# (pin module, oracle module, function, old text, new text)
MUTANTS = {
    # LBVH
    "morton_axes_in_wrong_bits": (test_oracle_lbvh, lbvh, "morton_keys", "((0, 2), (1, 1), (2, 0))",
                                  "((0, 0), (1, 1), (2, 2))"),
    "morton_not_clamped": (test_oracle_lbvh, lbvh, "morton_keys",
                           "np.minimum(np.floor(q).astype(np.int64), 2 ** BITS - 1)", "np.floor(q).astype(np.int64)"),
    "reference_point_is_box_corner": (test_oracle_lbvh, lbvh, "reference_points",
                                      "return (lo + hi) * np.float32(0.5)", "return lo"),
    "ties_in_reverse_order": (test_oracle_lbvh, lbvh, "sort_keys", 'order = np.argsort(keys, kind="stable")',
                              "order = np.lexsort((-np.arange(len(keys)), keys))"),
    "split_at_first_longer_prefix": (test_oracle_lbvh, lbvh, "radix_tree",
                                     "while g + 1 <= b - 1 and _prefix(sorted_keys, a, g + 1) > whole:",
                                     "while g + 1 <= b - 1 and _prefix(sorted_keys, a, g + 1) > whole + 1:"),
    "equal_keys_ignore_position": (test_oracle_lbvh, lbvh, "_prefix",
                                   "return 64 + 32 - (int(i) ^ int(j)).bit_length()", "return 64"),
    "box_lower_corner_by_max": (test_oracle_lbvh, lbvh, "boxes", "node_lo[node] = np.minimum(llo, rlo)",
                                "node_lo[node] = np.maximum(llo, rlo)"),
    # candidate features
    "bin_edges_not_squared": (test_oracle_features, features, "bin_edges_sq", "return (e * e).astype(np.float32)",
                              "return e.astype(np.float32)"),
    "histogram_by_count": (test_oracle_features, features, "features",
                           "np.bincount(b, weights=a, minlength=NBINS) / tot",
                           "np.bincount(b, minlength=NBINS) / len(b)"),
    "edge_region_wrong_vertex": (test_oracle_features, features, "_point_triangle_distance",
                                 "put((d3 >= 0) & (d4 <= d3), b)", "put((d3 >= 0) & (d4 <= d3), a)"),
    "hardness_offset_lost": (test_oracle_features, features, "probe_features", "h = np.clip(ex - 1 + 4, 0, HARD_BINS - 1)",
                             "h = np.clip(ex - 1 + 3, 0, HARD_BINS - 1)"),
    "efficiency_edges_exclusive": (test_oracle_features, features, "probe_features",
                                   'eb = np.searchsorted(EFF_EDGES, eff, side="right")',
                                   'eb = np.searchsorted(EFF_EDGES, eff, side="left")'),
    # scorer network
    "bf16_truncates": (test_oracle_mlp, mlp, "bf16", "r = ((u + 0x7FFF + lsb) & 0xFFFF0000)", "r = (u & 0xFFFF0000)"),
    "no_hidden_relu": (test_oracle_mlp, mlp, "forward", "H2 = q(np.maximum(H1 @ W2 + p[\"b2\"], 0.0))",
                       "H2 = q(H1 @ W2 + p[\"b2\"])"),
    "loss_sign": (test_oracle_mlp, mlp, "loss", "(softplus(s) - np.asarray(y, np.float64) * s)",
                  "(softplus(s) + np.asarray(y, np.float64) * s)"),
    "gradient_bias_dropped": (test_oracle_mlp, mlp, "gradients", 'g["b1"] = dZ1.sum(0)', 'g["b1"] = 0.0 * dZ1.sum(0)'),
    "adam_without_bias_correction": (test_oracle_mlp, mlp, "adam", "mh = m / (1 - b1 ** step)", "mh = m"),
    # fluence and coverage
    "fluence_transposed_dwell": (test_oracle_fluence, oracle, "fluence", "return t @ A", "return t[:, ::-1] @ A"),
    "coverage_strict_threshold": (test_oracle_fluence, oracle, "coverage", "ok = mu >= np.float32(mu_min)",
                                  "ok = mu > np.float32(mu_min)"),
    "coverage_by_count": (test_oracle_fluence, oracle, "coverage",
                          "by_area = (ok * area[None, :]).sum(axis=1) / total if total > 0 else np.zeros(mu.shape[0])",
                          "by_area = ok.mean(axis=1)"),
}


def _pins(module):
    """The module's test functions that take no arguments."""
    out = []
    for name in sorted(dir(module)):
        fn = getattr(module, name)
        if name.startswith("test_") and callable(fn) and not inspect.signature(fn).parameters:
            out.append(fn)
    return out


def _failing(module):
    failed = []
    for fn in _pins(module):
        try:
            fn()
        except Exception:   # noqa: BLE001 - an assertion or a crash both reject the mutant
            failed.append(fn.__name__)
    return failed


@pytest.mark.parametrize("pins", [test_oracle_lbvh, test_oracle_features, test_oracle_mlp, test_oracle_fluence],
                         ids=lambda m: m.__name__.split(".")[-1])
def test_unmutated_oracles_pass_their_pins(pins):
    assert _pins(pins) and _failing(pins) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_python_oracle_mutant_is_caught(name, monkeypatch):
    pins, module, func, old, new = MUTANTS[name]
    src = textwrap.dedent(inspect.getsource(getattr(module, func)))
    assert src.count(old) == 1, f"mutation anchor not unique in {func}: {old!r}"
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), ns)   # noqa: S102 - test-only source edit
    monkeypatch.setattr(module, func, ns[func])
    assert _failing(pins), f"mutant {name} passed every pin of {pins.__name__}"
