"""Seeded synthetic problems shaped like the paper's bundle-adjustment workloads.

This module only synthesises scenes: camera placements, 3-D points, which camera
sees which point, measurement noise, outliers and the initial perturbation of the
state.  To produce observations it renders the ground-truth scene through its own
forward camera model (a world simulator, written here independently of both the
optimiser and the oracle).  It holds no part of the optimiser: no residual
Jacobians, no normal equations, no linear solver, no update rule.  It is imported
by the tests, the benchmark and the oracle checks alike; neither the oracle nor the
CUDA path imports the other.

Camera convention (the Bundle Adjustment in the Large format the paper evaluates
on, Sec. V): a camera is the 9-vector [w, t, f, k1, k2] with w an angle-axis
rotation; a world point X maps to P = R(w) X + t, p = -P_xy / P_z (P_z < 0 in
front), u = f (1 + k1 |p|^2 + k2 |p|^4) p.

Random numbers come from counter-based SplitMix64 streams (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), so one seed gives
the same bytes on every machine and numpy version.  Normals use the Box-Muller
transform.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to a uint64 array."""
    z = np.atleast_1d(np.asarray(x, dtype=np.uint64)).copy()
    z ^= z >> np.uint64(30)
    z *= _MIX1
    z ^= z >> np.uint64(27)
    z *= _MIX2
    z ^= z >> np.uint64(31)
    return z


class Stream:
    """One counter-based random stream, keyed by (seed, stream id).

    Draw i of the stream is splitmix64(key + (i + 1) * golden), exactly the
    SplitMix64 sequence started from state `key`.
    """

    def __init__(self, seed: int, stream: int):
        base = splitmix64(np.array([int(seed) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
        self.key = splitmix64(base + np.array([int(stream)], dtype=np.uint64) * _GOLDEN)[0]
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        return splitmix64(self.key + idx * _GOLDEN)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """n doubles uniform on [lo, hi) with 53 random bits each."""
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, sigma: float = 1.0) -> np.ndarray:
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)  # (0, 1]
        u2 = self.uniform(m)
        rad = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)])
        return sigma * z[:n]

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """n integers uniform on [lo, hi)."""
        return (lo + np.floor(self.uniform(n) * (hi - lo))).astype(np.int64)

    def unit_vectors(self, n: int) -> np.ndarray:
        v = self.normal(3 * n).reshape(n, 3)
        return v / np.linalg.norm(v, axis=1, keepdims=True)


# --------------------------------------------------------------------------
# rotation helpers of the world simulator (frame <-> quaternion <-> angle-axis)
# --------------------------------------------------------------------------

def _quat_from_matrix(R: np.ndarray) -> np.ndarray:
    """Unit quaternions (w, x, y, z) from rotation matrices (n,3,3), Shepperd's method."""
    n = R.shape[0]
    q = np.empty((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    cand = np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], axis=1)
    k = np.argmax(cand, axis=1)
    for case in range(4):
        m = k == case
        if not np.any(m):
            continue
        Rm = R[m]
        if case == 0:
            s = 2.0 * np.sqrt(1.0 + tr[m])
            q[m, 0] = 0.25 * s
            q[m, 1] = (Rm[:, 2, 1] - Rm[:, 1, 2]) / s
            q[m, 2] = (Rm[:, 0, 2] - Rm[:, 2, 0]) / s
            q[m, 3] = (Rm[:, 1, 0] - Rm[:, 0, 1]) / s
        elif case == 1:
            s = 2.0 * np.sqrt(1.0 + Rm[:, 0, 0] - Rm[:, 1, 1] - Rm[:, 2, 2])
            q[m, 0] = (Rm[:, 2, 1] - Rm[:, 1, 2]) / s
            q[m, 1] = 0.25 * s
            q[m, 2] = (Rm[:, 0, 1] + Rm[:, 1, 0]) / s
            q[m, 3] = (Rm[:, 0, 2] + Rm[:, 2, 0]) / s
        elif case == 2:
            s = 2.0 * np.sqrt(1.0 + Rm[:, 1, 1] - Rm[:, 0, 0] - Rm[:, 2, 2])
            q[m, 0] = (Rm[:, 0, 2] - Rm[:, 2, 0]) / s
            q[m, 1] = (Rm[:, 0, 1] + Rm[:, 1, 0]) / s
            q[m, 2] = 0.25 * s
            q[m, 3] = (Rm[:, 1, 2] + Rm[:, 2, 1]) / s
        else:
            s = 2.0 * np.sqrt(1.0 + Rm[:, 2, 2] - Rm[:, 0, 0] - Rm[:, 1, 1])
            q[m, 0] = (Rm[:, 1, 0] - Rm[:, 0, 1]) / s
            q[m, 1] = (Rm[:, 0, 2] + Rm[:, 2, 0]) / s
            q[m, 2] = (Rm[:, 1, 2] + Rm[:, 2, 1]) / s
            q[m, 3] = 0.25 * s
    q[q[:, 0] < 0] *= -1.0
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _angle_axis_from_quat(q: np.ndarray) -> np.ndarray:
    v = q[:, 1:]
    s = np.linalg.norm(v, axis=1)
    ang = 2.0 * np.arctan2(s, q[:, 0])
    scale = np.where(s > 1e-12, ang / np.where(s > 1e-12, s, 1.0), 2.0)
    return v * scale[:, None]


def _quat_from_angle_axis(w: np.ndarray) -> np.ndarray:
    th = np.linalg.norm(w, axis=1)
    half = 0.5 * th
    k = np.where(th > 1e-12, np.sin(half) / np.where(th > 1e-12, th, 1.0), 0.5)
    return np.concatenate([np.cos(half)[:, None], w * k[:, None]], axis=1)


def _quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    aw, ax, ay, az = a.T
    bw, bx, by, bz = b.T
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=1)


def _matrix_from_quat(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], axis=1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], axis=1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], axis=1)], axis=1)


def _look_frames(forward: np.ndarray) -> np.ndarray:
    """World-to-camera rotations whose camera -z axis points along `forward` (n,3)."""
    z = -forward / np.linalg.norm(forward, axis=1, keepdims=True)
    up = np.tile(np.array([0.0, 0.0, 1.0]), (len(z), 1))
    x = np.cross(up, z)
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=1)  # rows are the camera axes in world coordinates


def render(R: np.ndarray, t: np.ndarray, f: np.ndarray, k1: np.ndarray, k2: np.ndarray,
           X: np.ndarray) -> np.ndarray:
    """Noise-free pixel coordinates of points X (n,3) seen by cameras (R (n,3,3), t (n,3), ...)."""
    Pc = np.einsum("nij,nj->ni", R, X) + t
    p = -Pc[:, :2] / Pc[:, 2:3]
    rr = np.sum(p * p, axis=1)
    return (f * (1.0 + k1 * rr + k2 * rr * rr))[:, None] * p


# --------------------------------------------------------------------------
# bundle-adjustment problems
# --------------------------------------------------------------------------

@dataclass
class BAProblem:
    """A seeded synthetic BA problem.  Edge k observes point pt_idx[k] from camera cam_idx[k]."""
    name: str
    seed: int
    cams_gt: np.ndarray   # (C, 9) float64  [w(3), t(3), f, k1, k2]
    pts_gt: np.ndarray    # (P, 3) float64
    cams0: np.ndarray     # (C, 9) initial state
    pts0: np.ndarray      # (P, 3) initial state
    cam_idx: np.ndarray   # (E,) int32
    pt_idx: np.ndarray    # (E,) int32
    obs: np.ndarray       # (E, 2) float64 pixels
    is_outlier: np.ndarray  # (E,) bool
    huber_delta: float | None
    meta: dict = field(default_factory=dict)

    @property
    def n_cams(self) -> int:
        return self.cams_gt.shape[0]

    @property
    def n_pts(self) -> int:
        return self.pts_gt.shape[0]

    @property
    def n_edges(self) -> int:
        return self.cam_idx.shape[0]


def _intrinsics(rng: Stream, n: int, k_sigma: float) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    f = 500.0 + rng.uniform(n, -10.0, 10.0)
    k1 = rng.normal(n, k_sigma)
    k2 = rng.normal(n, k_sigma)
    return f, k1, k2


def _observe(rng_noise: Stream, R, t, f, k1, k2, X, cam_idx, pt_idx, pixel_sigma,
             outlier_frac, outlier_range, block=4_000_000):
    E = cam_idx.shape[0]
    obs = np.empty((E, 2))
    for s in range(0, E, block):
        c = cam_idx[s:s + block]
        p = pt_idx[s:s + block]
        obs[s:s + block] = render(R[c], t[c], f[c], k1[c], k2[c], X[p])
    noise = rng_noise.normal(2 * E, pixel_sigma).reshape(E, 2)
    if outlier_frac > 0:
        is_out = rng_noise.uniform(E) < outlier_frac
        n_out = int(is_out.sum())
        noise[is_out] = rng_noise.uniform(2 * n_out, -outlier_range, outlier_range).reshape(n_out, 2)
    else:
        is_out = np.zeros(E, dtype=bool)
    return obs + noise, is_out


def _perturb(rng: Stream, cams_gt, R_gt, pts_gt, rot_noise, trans_noise, point_noise):
    """Initial state: each camera is turned by rot_noise radians about a uniformly random
    axis through its own centre (the centre stays put), then t gets N(0, trans_noise^2)
    per axis; points get N(0, point_noise^2) per axis."""
    C, P = cams_gt.shape[0], pts_gt.shape[0]
    cams0 = cams_gt.copy()
    centers = -np.einsum("nji,nj->ni", R_gt, cams_gt[:, 3:6])        # c = -R^T t
    dq = _quat_from_angle_axis(rot_noise * rng.unit_vectors(C))
    q0 = _quat_mul(dq, _quat_from_matrix(R_gt))
    R0 = _matrix_from_quat(q0)
    cams0[:, 0:3] = _angle_axis_from_quat(q0 / np.linalg.norm(q0, axis=1, keepdims=True))
    cams0[:, 3:6] = -np.einsum("nij,nj->ni", R0, centers) + rng.normal(3 * C, trans_noise).reshape(C, 3)
    pts0 = pts_gt + rng.normal(3 * P, point_noise).reshape(P, 3)
    return cams0, pts0


def ba_ring(seed: int, n_cams: int = 10, n_pts: int = 500, views: int = 6, radius: float = 15.0,
            pixel_sigma: float = 1.0, rot_noise: float = 0.02, trans_noise: float = 0.05,
            point_noise: float = 0.1, k_sigma: float = 1e-3, outlier_frac: float = 0.0,
            huber_delta: float | None = None, name: str = "ba_ring") -> BAProblem:
    """Cameras on a ring of `radius` looking at the origin; points uniform in [-5, 5]^3;
    every point seen by `views` distinct random cameras."""
    if views > n_cams:
        raise ValueError("views must not exceed n_cams")
    rng_geo, rng_vis = Stream(seed, 1), Stream(seed, 2)
    rng_noise, rng_init = Stream(seed, 3), Stream(seed, 4)
    phi = 2.0 * np.pi * np.arange(n_cams) / n_cams + rng_geo.uniform(n_cams, -0.1, 0.1)
    centers = np.stack([radius * np.cos(phi), radius * np.sin(phi),
                        rng_geo.uniform(n_cams, -2.0, 2.0)], axis=1)
    R = _look_frames(-centers)
    t = -np.einsum("nij,nj->ni", R, centers)
    f, k1, k2 = _intrinsics(rng_geo, n_cams, k_sigma)
    X = rng_geo.uniform(3 * n_pts, -5.0, 5.0).reshape(n_pts, 3)
    keys = rng_vis.uniform(n_pts * n_cams).reshape(n_pts, n_cams)
    chosen = np.argsort(keys, axis=1, kind="stable")[:, :views]
    pt_idx = np.repeat(np.arange(n_pts), views).astype(np.int32)
    cam_idx = chosen.reshape(-1).astype(np.int32)
    order = np.argsort(cam_idx, kind="stable")       # file order: grouped by camera
    cam_idx, pt_idx = cam_idx[order], pt_idx[order]
    obs, is_out = _observe(rng_noise, R, t, f, k1, k2, X, cam_idx, pt_idx, pixel_sigma,
                           outlier_frac, 50.0)
    w = _angle_axis_from_quat(_quat_from_matrix(R))
    cams_gt = np.concatenate([w, t, f[:, None], k1[:, None], k2[:, None]], axis=1)
    cams0, pts0 = _perturb(rng_init, cams_gt, R, X, rot_noise, trans_noise, point_noise)
    return BAProblem(name, seed, cams_gt, X, cams0, pts0, cam_idx, pt_idx, obs, is_out,
                     huber_delta, dict(kind="ring", views=views, pixel_sigma=pixel_sigma))


def _pareto_alpha(lo: int, hi: int, mean: float) -> float:
    k = np.arange(lo, hi + 1, dtype=np.float64)
    a, b = 0.0, 10.0
    for _ in range(200):
        m = 0.5 * (a + b)
        w = k ** (-m)
        if (k * w).sum() / w.sum() > mean:
            a = m
        else:
            b = m
    return 0.5 * (a + b)


def track_lengths(rng: Stream, n: int, law: str) -> np.ndarray:
    """Track lengths (views per point).

    'pareto': discrete power law P(L=k) ~ k^-a on [2, 40] with mean 6.
    'geom':   L = 2 + G, G geometric on {0, 1, ...} with mean 4.5 (mean L = 6.5), capped at 200.
    """
    u = rng.uniform(n)
    if law == "pareto":
        k = np.arange(2, 41)
        w = k ** (-_pareto_alpha(2, 40, 6.0))
        cdf = np.cumsum(w / w.sum())
        return k[np.minimum(np.searchsorted(cdf, u, side="right"), len(k) - 1)].astype(np.int64)
    if law == "geom":
        q = 4.5 / 5.5
        g = np.floor(np.log1p(-u) / np.log(q)).astype(np.int64)
        return np.minimum(2 + g, 200)
    raise ValueError(law)


def ba_path(seed: int, n_cams: int, n_pts: int, law: str = "pareto", spacing: float = 0.3,
            depth_lo: float = 2.0, depth_hi: float = 20.0,
            pixel_sigma: float = 1.0, rot_noise: float = 0.02, trans_noise: float = 0.05,
            point_noise: float = 0.1, k_sigma: float = 1e-3, outlier_frac: float = 0.01,
            huber_delta: float | None = 2.0, name: str = "ba_path") -> BAProblem:
    """Cameras along a smooth random path, looking sideways; each point is anchored at a
    random camera at depth U[2, 20] and seen by a window of consecutive cameras around
    the anchor (spatial locality), with track lengths drawn from `law`."""
    rng_geo, rng_vis = Stream(seed, 11), Stream(seed, 12)
    rng_noise, rng_init = Stream(seed, 13), Stream(seed, 14)
    s = np.arange(n_cams) / max(n_cams, 1)
    amp = rng_geo.uniform(3, 0.1, 0.4)
    cyc = rng_geo.integers(3, 1, 5)
    ph = rng_geo.uniform(3, 0.0, 2.0 * np.pi)
    heading = sum(amp[i] * np.sin(2.0 * np.pi * cyc[i] * s + ph[i]) for i in range(3))
    tang = np.stack([-np.sin(heading), np.cos(heading), np.zeros(n_cams)], axis=1)
    centers = np.cumsum(spacing * tang, axis=0)
    centers[:, 2] = 0.5 * np.sin(2.0 * np.pi * 2.0 * s + ph[0])
    fwd = np.stack([np.cos(heading), np.sin(heading), np.zeros(n_cams)], axis=1)
    R = _look_frames(fwd)
    t = -np.einsum("nij,nj->ni", R, centers)
    f, k1, k2 = _intrinsics(rng_geo, n_cams, k_sigma)

    anchor = rng_vis.integers(n_pts, 0, n_cams)
    L = np.minimum(track_lengths(rng_vis, n_pts, law), n_cams)
    # depth U[depth_lo, depth_hi], raised so that the whole window of observing cameras
    # sees the point within a +-35 degree cone (half window <= 0.7 depth)
    depth = np.maximum(rng_vis.uniform(n_pts, depth_lo, depth_hi), 0.5 * L * spacing / 0.7)
    lat = rng_vis.uniform(n_pts, -0.4, 0.4) * depth
    up = rng_vis.uniform(n_pts, -0.3, 0.3) * depth
    X = centers[anchor] + depth[:, None] * fwd[anchor] + lat[:, None] * tang[anchor]
    X[:, 2] += up
    start = np.clip(anchor - L // 2, 0, n_cams - L)

    E0 = int(L.sum())
    pt_e = np.repeat(np.arange(n_pts, dtype=np.int64), L)
    first = np.repeat(np.cumsum(L) - L, L)
    cam_e = np.repeat(start, L) + (np.arange(E0, dtype=np.int64) - first)
    # an observer keeps the observation only if the point lies in front (depth >= 0.5)
    # and inside a +-45 degree field of view about the viewing direction
    rel = X[pt_e] - centers[cam_e]
    dep = np.einsum("ni,ni->n", rel, fwd[cam_e])
    lat_x = np.abs(np.einsum("ni,ni->n", rel, R[cam_e, 0]))
    lat_y = np.abs(np.einsum("ni,ni->n", rel, R[cam_e, 1]))
    keep = (dep >= 0.5) & (lat_x <= dep) & (lat_y <= dep)
    del rel, dep, lat_x, lat_y
    pt_e, cam_e = pt_e[keep], cam_e[keep]
    cnt = np.bincount(pt_e, minlength=n_pts)
    good = cnt >= 2
    new_id = np.cumsum(good) - 1
    sel = good[pt_e]
    pt_e, cam_e = new_id[pt_e[sel]], cam_e[sel]
    X = X[good]
    order = np.argsort(cam_e, kind="stable")         # file order: grouped by camera
    cam_idx = cam_e[order].astype(np.int32)
    pt_idx = pt_e[order].astype(np.int32)
    obs, is_out = _observe(rng_noise, R, t, f, k1, k2, X, cam_idx, pt_idx, pixel_sigma,
                           outlier_frac, 50.0)
    w = _angle_axis_from_quat(_quat_from_matrix(R))
    cams_gt = np.concatenate([w, t, f[:, None], k1[:, None], k2[:, None]], axis=1)
    cams0, pts0 = _perturb(rng_init, cams_gt, R, X, rot_noise, trans_noise, point_noise)
    return BAProblem(name, seed, cams_gt, X, cams0, pts0, cam_idx, pt_idx, obs, is_out,
                     huber_delta, dict(kind="path", law=law, pixel_sigma=pixel_sigma))


# Workload presets (sizes of the paper-shaped synthetic inputs).
def ba_tiny(seed: int = 0, **kw) -> BAProblem:
    """10 cameras, 500 points, 6 views per point (3,000 observations); no outliers."""
    return ba_ring(seed, 10, 500, 6, name="ba_tiny_c10_p500", **kw)


def ba_medium(seed: int = 1, **kw) -> BAProblem:
    """1,000 cameras, 500,000 points, 2-40 views per point (mean 6, ~3M observations),
    1% outliers at U[-50, 50] px, Huber delta 2."""
    return ba_path(seed, 1000, 500_000, "pareto", name="ba_medium_c1000_p500k", **kw)


def ba_large(seed: int = 2, **kw) -> BAProblem:
    """13,000 cameras, 4.5M points, geometric tracks (mean 6.5, max 200, ~29M observations),
    1% outliers, Huber delta 2."""
    return ba_path(seed, 13_000, 4_500_000, "geom", name="ba_large_c13000_p4500k", **kw)


def ba_window(seed: int, n_kf: int, n_pts: int, **kw) -> BAProblem:
    """A local bundle-adjustment window: n_kf keyframes along a path and n_pts landmarks
    (tracks of 2-40 views, 1% outliers, Huber delta 2), generated as the medium problem."""
    return ba_path(seed, n_kf, n_pts, "pareto", name=f"ba_window_k{n_kf}_p{n_pts}", **kw)


def window_pool(seed: int, n: int, kf=(5, 40), pts=(300, 8000)) -> list:
    """n windows with keyframes ~ U{kf} and landmarks ~ U{pts} (edges follow from the
    track lengths: about 6 per landmark, 2k-60k per window)."""
    rng = Stream(seed, 21)
    k = rng.integers(n, kf[0], kf[1] + 1)
    m = rng.integers(n, pts[0], pts[1] + 1)
    return [ba_window(seed * 1000003 + i, int(k[i]), int(m[i])) for i in range(n)]


def fresh_request(base: BAProblem, seed: int, i: int, pixel_sigma: float = 0.5,
                  trans_noise: float = 0.02, point_noise: float = 0.05) -> BAProblem:
    """Request i of a served stream built on the window topology `base`: the same
    cameras, landmarks and visibility, with observation noise and an initial state of
    its own (N(0, pixel_sigma^2) added to every pixel, N(0, trans_noise^2) to every
    camera translation, N(0, point_noise^2) to every landmark), drawn from counter-based
    streams keyed by (seed, i).  Every request is a distinct problem with a distinct
    optimum, at a cost of a few array operations (generating a new window topology takes
    milliseconds, too slow for thousands of requests per second)."""
    rng = Stream(int(seed) * 1000003 + int(i), 23)
    E, C, P = base.n_edges, base.n_cams, base.n_pts
    obs = base.obs + rng.normal(2 * E, pixel_sigma).reshape(E, 2)
    cams0 = base.cams0.copy()
    cams0[:, 3:6] += rng.normal(3 * C, trans_noise).reshape(C, 3)
    pts0 = base.pts0 + rng.normal(3 * P, point_noise).reshape(P, 3)
    return BAProblem(f"{base.name}_r{i}", base.seed, base.cams_gt, base.pts_gt, cams0, pts0, base.cam_idx,
                     base.pt_idx, obs, base.is_outlier, base.huber_delta, dict(base.meta))


def poisson_arrivals(seed: int, rate: float, duration: float) -> np.ndarray:
    """Arrival times of a Poisson process of `rate` per second over [0, duration)."""
    rng = Stream(seed, 22)
    n_max = int(rate * duration * 1.5 + 100)
    gaps = -np.log1p(-rng.uniform(n_max)) / rate
    t = np.cumsum(gaps)
    return t[t < duration]


# --------------------------------------------------------------------------
# visual-inertial problems
# --------------------------------------------------------------------------

GRAVITY = np.array([0.0, 0.0, -9.81])


def _rodrigues(w: np.ndarray) -> np.ndarray:
    """Rotation matrix of one angle-axis vector (world simulator)."""
    t = float(np.linalg.norm(w))
    K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    if t < 1e-9:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + np.sin(t) / t * K + (1.0 - np.cos(t)) / (t * t) * K @ K


@dataclass
class VIProblem:
    """Keyframe states x = [q (x y z w), p, v, bg, ba] (16), landmarks, stereo edges and, per
    consecutive keyframe pair, the raw IMU samples between them."""
    name: str
    seed: int
    nav_gt: np.ndarray        # (K, 16)
    pts_gt: np.ndarray        # (P, 3)
    nav0: np.ndarray          # (K, 16) initial state (zero bias estimates)
    pts0: np.ndarray          # (P, 3)
    kf_idx: np.ndarray        # (E,) int32 keyframe of each stereo edge
    pt_idx: np.ndarray        # (E,) int32
    obs: np.ndarray           # (E, 3) [u_l, v_l, u_r]
    imu_gyro: np.ndarray      # (K-1, N, 3) measured angular rates between keyframes k, k+1
    imu_acc: np.ndarray       # (K-1, N, 3) measured specific forces
    dt: float
    camera: dict              # fx fy cx cy baseline R_cb t_cb width height
    noise: dict               # sigma_g sigma_a sigma_bg sigma_ba pixel
    huber_delta: float
    meta: dict = field(default_factory=dict)

    @property
    def n_kf(self) -> int:
        return self.nav_gt.shape[0]

    @property
    def n_pts(self) -> int:
        return self.pts_gt.shape[0]

    @property
    def n_edges(self) -> int:
        return self.kf_idx.shape[0]


def vi_problem(seed: int, n_kf: int = 3000, n_pts: int = 200_000, rate: float = 200.0,
               kf_gap: float = 0.25, sigma_g: float = 1.7e-4, sigma_a: float = 2e-3,
               sigma_bg: float = 2e-5, sigma_ba: float = 3e-3, pixel_sigma: float = 1.0,
               imu_noise: bool = True, mean_track: float = 10.0, name: str = "vi") -> VIProblem:
    """Stereo-inertial trajectory: smooth random body rates and world accelerations sampled
    at `rate` Hz; ground-truth keyframe states are the discrete integration of the true
    samples (R <- R Exp(w dt), v <- v + (g + R f) dt, p <- p + v dt + (g + R f) dt^2 / 2 with
    f the specific force), one keyframe every kf_gap seconds.  Landmarks are back-projected
    from random pixels of a keyframe at depth U[2, 20] and observed by nearby keyframes whose
    left and right images contain them."""
    rng_traj, rng_vis = Stream(seed, 31), Stream(seed, 32)
    rng_noise, rng_init = Stream(seed, 33), Stream(seed, 34)
    dt = 1.0 / rate
    N = int(round(kf_gap * rate))
    S = (n_kf - 1) * N
    t = np.arange(S + 1) * dt
    # smooth world velocity v(t) = v_init + sum of sinusoids (periods 2-20 s); a = dv/dt
    amp = rng_traj.uniform(9, 0.05, 0.4).reshape(3, 3) * np.array([[1.0], [1.0], [0.2]])
    frq = 2.0 * np.pi / rng_traj.uniform(9, 2.0, 20.0).reshape(3, 3)
    phs = rng_traj.uniform(9, 0.0, 2.0 * np.pi).reshape(3, 3)
    a_world = np.zeros((S + 1, 3))
    for ax in range(3):
        for j in range(3):
            a_world[:, ax] += amp[ax, j] * frq[ax, j] * np.cos(frq[ax, j] * t + phs[ax, j])
    v_init = np.array([1.0, 0.0, 0.0]) + (amp * np.sin(phs)).sum(axis=1) * 0.0
    # smooth body rates, yaw dominated
    wamp = rng_traj.uniform(9, 0.02, 0.1).reshape(3, 3) * np.array([[0.3], [0.3], [1.0]])
    wfrq = 2.0 * np.pi / rng_traj.uniform(9, 2.0, 20.0).reshape(3, 3)
    wphs = rng_traj.uniform(9, 0.0, 2.0 * np.pi).reshape(3, 3)
    w_body = np.zeros((S + 1, 3))
    for ax in range(3):
        for j in range(3):
            w_body[:, ax] += wamp[ax, j] * np.sin(wfrq[ax, j] * t + wphs[ax, j])
    bg_true = rng_traj.normal(3, 1e-3)
    ba_true = rng_traj.normal(3, 1e-2)
    # discrete integration of the true samples -> ground truth at every keyframe
    Rk = np.eye(3)
    pk = np.zeros(3)
    vk = v_init.copy()
    gyro = np.empty((S, 3))
    accm = np.empty((S, 3))
    nav_gt = np.zeros((n_kf, 16))
    for k in range(S + 1):
        if k % N == 0:
            i = k // N
            nav_gt[i, 0:4] = _quat_from_matrix(Rk[None])[0][[1, 2, 3, 0]]
            nav_gt[i, 4:7] = pk
            nav_gt[i, 7:10] = vk
            nav_gt[i, 10:13] = bg_true
            nav_gt[i, 13:16] = ba_true
        if k == S:
            break
        f_body = Rk.T @ (a_world[k] - GRAVITY)
        gyro[k] = w_body[k] + bg_true
        accm[k] = f_body + ba_true
        acc_w = GRAVITY + Rk @ (accm[k] - ba_true)
        pk = pk + vk * dt + 0.5 * acc_w * dt * dt
        vk = vk + acc_w * dt
        Rk = Rk @ _rodrigues((gyro[k] - bg_true) * dt)
    if imu_noise:
        gyro = gyro + rng_noise.normal(3 * S, sigma_g / np.sqrt(dt)).reshape(S, 3)
        accm = accm + rng_noise.normal(3 * S, sigma_a / np.sqrt(dt)).reshape(S, 3)

    # stereo rig: camera z = body x (forward), camera x = -body y, camera y = -body z
    R_cb = np.array([[0.0, -1.0, 0.0], [0.0, 0.0, -1.0], [1.0, 0.0, 0.0]])
    t_cb = np.array([0.02, -0.01, 0.05])
    cam = dict(fx=450.0, fy=450.0, cx=320.0, cy=240.0, baseline=0.11, R_cb=R_cb, t_cb=t_cb,
               width=640.0, height=480.0)
    Rq = _matrix_from_quat(nav_gt[:, [3, 0, 1, 2]])          # (K,3,3) body-to-world
    # landmarks
    anchor = rng_vis.integers(n_pts, 0, n_kf)
    u = rng_vis.uniform(n_pts, 40.0, 600.0)
    v = rng_vis.uniform(n_pts, 40.0, 440.0)
    depth = rng_vis.uniform(n_pts, 2.0, 20.0)
    Xc = np.stack([(u - cam["cx"]) / cam["fx"] * depth, (v - cam["cy"]) / cam["fy"] * depth, depth], axis=1)
    Xb = (Xc - t_cb) @ R_cb
    X = np.einsum("nij,nj->ni", Rq[anchor], Xb) + nav_gt[anchor, 4:7]
    q_geo = (mean_track - 2.0) / (mean_track - 1.0)
    L = np.minimum(2 + np.floor(np.log1p(-rng_vis.uniform(n_pts)) / np.log(q_geo)).astype(np.int64), 40)
    L = np.minimum(L, n_kf)
    start = np.clip(anchor - L // 2, 0, n_kf - L)
    E0 = int(L.sum())
    pt_e = np.repeat(np.arange(n_pts), L)
    kf_e = np.repeat(start, L) + (np.arange(E0) - np.repeat(np.cumsum(L) - L, L))
    Xbe = np.einsum("nji,nj->ni", Rq[kf_e], X[pt_e] - nav_gt[kf_e, 4:7])
    Xce = Xbe @ R_cb.T + t_cb
    z = Xce[:, 2]
    ok = z > 0.5
    zs = np.where(ok, z, 1.0)
    ul = cam["fx"] * Xce[:, 0] / zs + cam["cx"]
    vl = cam["fy"] * Xce[:, 1] / zs + cam["cy"]
    ur = cam["fx"] * (Xce[:, 0] - cam["baseline"]) / zs + cam["cx"]
    ok &= (ul >= 0) & (ul < cam["width"]) & (vl >= 0) & (vl < cam["height"]) & (ur >= 0)
    pt_e, kf_e = pt_e[ok], kf_e[ok]
    obs = np.stack([ul, vl, ur], axis=1)[ok]
    cnt = np.bincount(pt_e, minlength=n_pts)
    good = cnt >= 2
    new_id = np.cumsum(good) - 1
    sel = good[pt_e]
    pt_e, kf_e, obs = new_id[pt_e[sel]], kf_e[sel], obs[sel]
    X = X[good]
    obs = obs + rng_noise.normal(obs.size, pixel_sigma).reshape(obs.shape)
    order = np.argsort(kf_e, kind="stable")
    kf_e, pt_e, obs = kf_e[order].astype(np.int32), pt_e[order].astype(np.int32), obs[order]

    # initial state: rotation turned by 0.02 rad (random axis, right), position and velocity
    # N(0, 0.05^2) per axis, biases zero, points N(0, 0.1^2) per axis
    nav0 = nav_gt.copy()
    dq = _quat_from_angle_axis(0.02 * rng_init.unit_vectors(n_kf))
    q = _quat_mul(nav_gt[:, [3, 0, 1, 2]], dq)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    nav0[:, 0:4] = q[:, [1, 2, 3, 0]]
    nav0[:, 4:7] += rng_init.normal(3 * n_kf, 0.05).reshape(n_kf, 3)
    nav0[:, 7:10] += rng_init.normal(3 * n_kf, 0.05).reshape(n_kf, 3)
    nav0[:, 10:16] = 0.0
    pts0 = X + rng_init.normal(3 * len(X), 0.1).reshape(len(X), 3)
    return VIProblem(name, seed, nav_gt, X, nav0, pts0, kf_e, pt_e, obs,
                     gyro.reshape(n_kf - 1, N, 3), accm.reshape(n_kf - 1, N, 3), dt, cam,
                     dict(sigma_g=sigma_g, sigma_a=sigma_a, sigma_bg=sigma_bg, sigma_ba=sigma_ba,
                          pixel=pixel_sigma), float(np.sqrt(7.815)))


def vi_global(seed: int = 3, **kw) -> VIProblem:
    """3,000 stereo keyframes, 200,000 landmarks, ~2M stereo observations, IMU at 200 Hz
    over 0.25 s gaps."""
    return vi_problem(seed, 3000, 200_000, name="vi_global_k3000_p200k", **kw)
