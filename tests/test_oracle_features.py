"""Pins of the feature oracle: bin edges by their definition, a histogram of
hand-placed patches, and the point-triangle distance against closed forms and
dense sampling of the triangle."""
import numpy as np

from oracle import features as F


def test_bin_edges():
    E = F.bin_edges_sq()
    assert E.shape == (63,) and np.all(np.diff(E) > 0)
    assert np.isclose(np.sqrt(E[0]), 0.1 * 250 ** (1 / 64)) and np.isclose(np.sqrt(E[31]), 0.1 * 250 ** 0.5)


def test_histogram_hand_placed():
    c = np.array([[0.0, 0.0, 0.0]])
    # distances 0.05 (bin 0), 1.0, 30 (last bin); areas 1, 2, 3
    s = np.array([[0.05, 0, 0], [0, 1.0, 0], [0, 0, 30.0]], np.float32)
    f, amb = F.features(np.zeros((3, 3)), np.zeros((0, 3), np.int64), s, [1, 2, 3], c)
    b1 = int(np.floor(64 * np.log(1.0 / 0.1) / np.log(250)))    # d = 1 m lies in bin floor(64 log10 / log250)
    assert f[0, 0] == 1 / 6 and f[0, 63] == 3 / 6 and f[0, b1] == 2 / 6
    assert np.isclose(f[0, :64].sum(), 1.0)


def test_point_triangle_distance():
    a, b, c = np.array([[0.0, 0, 0]]), np.array([[2.0, 0, 0]]), np.array([[0.0, 2, 0]])
    d = lambda p: F._point_triangle_distance(np.array(p, float), a, b, c)[0]  # noqa: E731
    assert np.isclose(d([0.5, 0.5, 3.0]), 3.0)                     # above the interior
    assert np.isclose(d([-1.0, -1.0, 0.0]), np.sqrt(2))            # nearest to vertex a
    assert np.isclose(d([1.0, -2.0, 0.0]), 2.0)                    # nearest to edge ab
    assert np.isclose(d([2.0, 2.0, 0.0]), np.sqrt(2))              # nearest to edge bc (x+y=2)
    assert np.isclose(d([3.0, -1.0, 0.0]), np.sqrt(2))             # nearest to vertex b
    assert np.isclose(d([-1.0, 3.0, 1.0]), np.sqrt(3))             # nearest to vertex c
    assert np.isclose(d([-2.0, 1.0, 0.0]), 2.0)                    # nearest to edge ca (x = 0)
    rng = np.random.default_rng(0)
    uv = rng.uniform(size=(20000, 2))
    uv = np.where(uv.sum(1, keepdims=True) > 1, 1 - uv, uv)
    pts = a + uv[:, :1] * (b - a) + uv[:, 1:] * (c - a)
    for p in rng.uniform(-3, 3, size=(10, 3)):
        assert d(p) <= np.linalg.norm(pts - p, axis=1).min() + 1e-12
        assert d(p) >= np.linalg.norm(pts - p, axis=1).min() - 0.03


def test_probe_features_hand_worked():
    # E* = (1, 2, 0.5), all lit; Ebar = (1*1 + 1*2 + 2*0.5) / 4 = 1
    # hardness: log2 (1, 2, 0.5) = (0, 1, -1) -> bins (4, 5, 3)
    # efficiencies: cand 0 (1, 0, 1) -> (5, 0, 5); cand 1 (0.5, 1, 1) -> (1, 5, 5)
    A = [[1.0, 0.0, 0.5], [0.5, 2.0, 0.5]]
    f, amb = F.probe_features(A, [1.0, 1.0, 2.0])
    want = np.zeros((2, 48))
    want[0, 4 * 6 + 5], want[0, 5 * 6 + 0], want[0, 3 * 6 + 5] = 0.25, 0.25, 0.5
    want[1, 4 * 6 + 1], want[1, 5 * 6 + 5], want[1, 3 * 6 + 5] = 0.25, 0.25, 0.5
    np.testing.assert_array_equal(f, want)
    assert amb.all()                                        # every ratio is an exact power of two


def test_probe_features_invariants():
    rng = np.random.default_rng(5)
    A = rng.uniform(0, 3, (40, 500)).astype(np.float32)
    A[rng.uniform(size=A.shape) < 0.5] = 0
    A[:, :20] = 0                                          # unlit probe patches are left out
    area = rng.uniform(0.001, 0.01, 500)
    f, _ = F.probe_features(A, area)
    np.testing.assert_allclose(f.sum(1), 1.0)              # every lit patch counted once per candidate
    best = A.argmax(0)
    # a candidate's top efficiency bin holds at least the patches it is best for
    for i in range(5):
        mine = (best == i) & (A.max(0) > 0)
        assert f[i, 5::6].sum() >= area[mine].sum() / area[A.max(0) > 0].sum() - 1e-12
    # scaling all irradiance leaves the sketch unchanged (bins are ratios)
    f2, _ = F.probe_features(A * 4.0, area)
    np.testing.assert_array_equal(f, f2)
