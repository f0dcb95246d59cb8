"""Host logic of the counting replay (replay/): the closed-form source range
is decided as the library decides it, tasks are sampled without repeats
inside the matrix, and the byte model adds up as documented."""
import numpy as np

import replay
from synth.scenes import line_lamp


def test_uniform_lamp_decision():
    L = line_lamp(1.2, 8, 120.0)
    wu, wz0, wrdz = replay.uniform_lamp(L.offsets[:, 2], coord_bound=10.0)
    assert wu == 1 and wz0 == np.float32(0.075) and abs(float(wrdz) - 1 / 0.15) < 1e-5
    # uneven spacing: no closed form
    oz = L.offsets[:, 2].copy()
    oz[3] += 0.01
    assert replay.uniform_lamp(oz, 10.0)[0] == 0
    # a step below 2^-16 (16 B + 3 max|oz|) of the coordinates: no closed form
    assert replay.uniform_lamp(L.offsets[:, 2], coord_bound=1e6)[0] == 0


def test_sample_tasks_distinct_and_in_range():
    t = replay.sample_tasks(2000, 102030, 3000, seed=11)
    assert t.shape == (3000, 2)
    assert t[:, 0].max() < 500 and t[:, 1].max() < (102030 + 31) // 32 and t.min() >= 0
    assert len({(a, b) for a, b in t}) == 3000
    assert np.array_equal(t, replay.sample_tasks(2000, 102030, 3000, seed=11))
    small = replay.sample_tasks(5, 40, 100, seed=1)   # fewer tasks than asked: all of them
    assert small.shape == (2 * 2, 2)


def test_bytes_per_pair_model():
    c = dict.fromkeys(replay.COUNTERS, 0)
    c.update(pairs=128, tasks=1, node_visits=10, lane_node_visits=100, leaf_loads=40, leaf_step_unique=20,
             cache_loads=4, leaf_steps=5, leaf_step_lanes=40)
    b = replay.bytes_per_pair(c, K=8)
    assert b["output"] == 5.0
    assert np.isclose(b["per_warp"], (10 * 128 + 20 * 48 + 4 * 48 + 32 * 40) / 128 + 5.0)
    assert np.isclose(b["per_lane"], (100 * 128 + 40 * 48 + 4 * 48 + 32 * 40) / 128 + 5.0)
    assert np.isclose(b["leaf_step_lane_occupancy"], 40 / 5 / 32)
