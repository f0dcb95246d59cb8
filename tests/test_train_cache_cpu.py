"""The scorer's training resumes from its cache of solved chunks (host code,
no GPU): a chunk written by save_chunk is read back job by job, bit for bit,
and training_data takes a fully cached run without building a scene; a chunk
made under other settings, or missing, is not used."""
import os

import numpy as np

from paper_2103_14137_gb300 import train_scorer as ts


def _chunk(rng, sizes, d=114):
    feats = [rng.normal(size=(n, d)).astype(np.float32) for n in sizes]
    ys = [rng.uniform(size=n).astype(np.float32) for n in sizes]
    etas = [rng.uniform(size=n).astype(np.float32) for n in sizes]
    sups = [rng.uniform(size=n) < 0.1 for n in sizes]
    lp_s = [float(x) for x in rng.uniform(1, 9, len(sizes))]
    return feats, ys, etas, sups, lp_s


def test_chunk_round_trip_and_settings(tmp_path):
    rng = np.random.default_rng(0)
    feats, ys, etas, sups, lp_s = _chunk(rng, [5, 0, 7])
    ts.save_chunk(str(tmp_path), 0, 2, 1200, feats, ys, etas, sups, lp_s)
    assert sorted(os.listdir(tmp_path)) == ["train_rooms_10000-10001.npz"]      # no temporary file left
    f, y, e, sp, ls = ts.load_chunk(str(tmp_path), 0, 2, 1200)
    for a, b in ((f, feats), (y, ys), (e, etas), (sp, sups)):
        assert len(a) == len(b) and all(np.array_equal(u, v) and u.dtype == v.dtype for u, v in zip(a, b))
    assert ls == lp_s
    assert ts.load_chunk(str(tmp_path), 0, 2, 800) is None                       # another candidate cap
    assert ts.load_chunk(str(tmp_path), 2, 4, 1200) is None                      # not solved yet
    assert ts.load_chunk(None, 0, 2, 1200) is None


def test_training_data_resumes_from_the_cache(tmp_path):
    rng = np.random.default_rng(1)
    want = [_chunk(rng, [3, 4, 2]), _chunk(rng, [6])]
    ts.save_chunk(str(tmp_path), 0, 2, 1200, *want[0])
    ts.save_chunk(str(tmp_path), 2, 3, 1200, *want[1])
    logs = []
    feats, ys, lp_s, etas, sups = ts.training_data(3, 1200, None, 1, logs.append, chunk=2, cache=str(tmp_path))
    assert len(logs) == 2 and all("read from" in m for m in logs)
    exp_f = want[0][0] + want[1][0]
    assert len(feats) == 4 and all(np.array_equal(a, b) for a, b in zip(feats, exp_f))
    assert all(np.array_equal(a, b) for a, b in zip(ys, want[0][1] + want[1][1]))
    assert lp_s == want[0][4] + want[1][4]
