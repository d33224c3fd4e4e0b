"""Seeded generator: determinism, the SplitMix64 definition, distributions and shapes."""
import numpy as np

from paper_2509_26581_gb300 import synth


def _splitmix64_python(state: int, n: int):
    """SplitMix64 written with Python integers (Steele, Lea and Flood 2014)."""
    out = []
    m = (1 << 64) - 1
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & m
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        out.append(z ^ (z >> 31))
    return out


def test_stream_is_splitmix64_sequence():
    s = synth.Stream(7, 3)
    key = int(s.key)
    got = [int(v) for v in s.u64(5)] + [int(v) for v in s.u64(3)]
    assert got == _splitmix64_python(key, 8)


def test_streams_deterministic_and_distinct():
    a = synth.Stream(1, 1).normal(1000)
    b = synth.Stream(1, 1).normal(1000)
    c = synth.Stream(1, 2).normal(1000)
    d = synth.Stream(2, 1).normal(1000)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c) and not np.array_equal(a, d)


def test_distribution_moments():
    s = synth.Stream(5, 0)
    u = s.uniform(200_000)
    z = s.normal(200_000)
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert u.min() >= 0.0 and u.max() < 1.0


def test_track_length_laws():
    L = synth.track_lengths(synth.Stream(3, 0), 400_000, "pareto")
    assert L.min() == 2 and L.max() <= 40 and abs(L.mean() - 6.0) < 0.05
    G = synth.track_lengths(synth.Stream(3, 1), 400_000, "geom")
    assert G.min() == 2 and G.max() <= 200 and abs(G.mean() - 6.5) < 0.05


def test_ba_tiny_shape_and_determinism():
    p = synth.ba_tiny(0)
    q = synth.ba_tiny(0)
    assert p.n_cams == 10 and p.n_pts == 500 and p.n_edges == 3000
    for name in ("cams_gt", "pts_gt", "cams0", "pts0", "cam_idx", "pt_idx", "obs"):
        assert np.array_equal(getattr(p, name), getattr(q, name)), name
    # every point seen by 6 distinct cameras
    pairs = set(zip(p.cam_idx.tolist(), p.pt_idx.tolist()))
    assert len(pairs) == 3000
    assert np.all(np.bincount(p.pt_idx, minlength=500) == 6)


def test_ba_path_small_locality_and_outliers():
    p = synth.ba_path(4, 60, 3000, "pareto", outlier_frac=0.01)
    cnt = np.bincount(p.pt_idx, minlength=p.n_pts)
    assert cnt.min() >= 2 and cnt.max() <= 40
    # each point's cameras form a window of consecutive cameras (locality)
    order = np.lexsort((p.cam_idx, p.pt_idx))
    ci, pi = p.cam_idx[order], p.pt_idx[order]
    first = np.r_[True, pi[1:] != pi[:-1]]
    span = np.maximum.reduceat(ci, np.nonzero(first)[0]) - np.minimum.reduceat(ci, np.nonzero(first)[0])
    assert np.all(span <= 40)
    assert 0.002 < p.is_outlier.mean() < 0.03
    assert p.huber_delta == 2.0
