"""Visual-inertial terms of the FP64 oracle (test infrastructure).

Eq. 8 adds an inertial residual r_I between consecutive keyframes and a bias residual
r_b; Sec. V-C lists the constraints (stereo reprojection, inertial, gyro and
accelerometer bias random walks, bias priors).  The paper gives no formulas, so
these are the standard ones of on-manifold IMU preintegration (Forster, Carlone,
Dellaert and Scaramuzza, "On-Manifold Preintegration for Real-Time Visual-Inertial
Odometry", T-RO 2017), restated here from their definitions.

Keyframe state ("navigation state", tangent size 15):
    x = [q (qx qy qz qw, body-to-world rotation R), p (3), v (3), bg (3), ba (3)]
    update: R <- R Exp(dtheta), p <- p + R dp, v <- v + dv, bg <- bg + dbg, ba <- ba + dba
Gravity g = (0, 0, -9.81).

Stereo reprojection (pose i, world point X; extrinsic body-to-camera R_cb, t_cb):
    X_b = R^T (X - p),  X_c = R_cb X_b + t_cb,
    r = [fx X_c/Z_c + cx, fy Y_c/Z_c + cy, fx (X_c - b)/Z_c + cx] - [u_l, v_l, u_r].

Preintegration of samples (w_k, a_k), k < N, step dt, at bias estimates (bg0, ba0):
    dR_{k+1} = dR_k Exp((w_k - bg0) dt)
    dv_{k+1} = dv_k + dR_k (a_k - ba0) dt
    dp_{k+1} = dp_k + dv_k dt + 1/2 dR_k (a_k - ba0) dt^2
with first-order bias Jacobians and the covariance of (dphi, dv, dp) propagated from
the discrete noise densities sigma_g / sqrt(dt), sigma_a / sqrt(dt).

Inertial residual between keyframes i and j (T = N dt), with bias deviations
dbg = bg_i - bg0, dba = ba_i - ba0:
    r_R = Log((dR Exp(J_R^g dbg))^T R_i^T R_j)
    r_v = R_i^T (v_j - v_i - g T) - (dv + J_v^g dbg + J_v^a dba)
    r_p = R_i^T (p_j - p_i - v_i T - 1/2 g T^2) - (dp + J_p^g dbg + J_p^a dba)
Bias random walk between i and j: r = [bg_j - bg_i, ba_j - ba_i].
Bias prior on keyframe i: r = [bg_i - bg_prior, ba_i - ba_prior].
"""
import numpy as np

from . import so3

GRAVITY = np.array([0.0, 0.0, -9.81])


# ---------------------------------------------------------------- rotation helpers

def quat_to_R(q: np.ndarray) -> np.ndarray:
    """Rotation matrices of unit quaternions stored as (x, y, z, w)."""
    q = np.atleast_2d(q)
    x, y, z, w = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], axis=1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], axis=1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], axis=1)], axis=1)


def R_to_quat(R: np.ndarray) -> np.ndarray:
    """(x, y, z, w) with w >= 0, through the angle-axis of R."""
    w = so3.log(R)
    th = np.linalg.norm(w, axis=1)
    s = np.where(th > 1e-12, np.sin(0.5 * th) / np.where(th > 1e-12, th, 1.0), 0.5)
    q = np.concatenate([w * s[:, None], np.cos(0.5 * th)[:, None]], axis=1)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def right_jacobian(phi: np.ndarray) -> np.ndarray:
    """Jr(phi) = I - (1 - cos t)/t^2 [phi]x + (t - sin t)/t^3 [phi]x^2 (series for small t)."""
    phi = np.atleast_2d(phi)
    t2 = np.sum(phi * phi, axis=1)
    t = np.sqrt(t2)
    small = t < 1e-4
    ts = np.where(small, 1.0, t)
    a = np.where(small, 0.5 - t2 / 24.0, (1.0 - np.cos(ts)) / (ts * ts))
    b = np.where(small, 1.0 / 6.0 - t2 / 120.0, (ts - np.sin(ts)) / (ts ** 3))
    K = so3.hat(phi)
    return np.eye(3)[None] - a[:, None, None] * K + b[:, None, None] * (K @ K)


def right_jacobian_inv(phi: np.ndarray) -> np.ndarray:
    """Jr^-1(phi) = I + 1/2 [phi]x + (1/t^2 - (1 + cos t)/(2 t sin t)) [phi]x^2."""
    phi = np.atleast_2d(phi)
    t2 = np.sum(phi * phi, axis=1)
    t = np.sqrt(t2)
    small = t < 1e-4
    ts = np.where(small, 1.0, t)
    c = np.where(small, 1.0 / 12.0 + t2 / 720.0,
                 1.0 / (ts * ts) - (1.0 + np.cos(ts)) / (2.0 * ts * np.sin(ts)))
    K = so3.hat(phi)
    return np.eye(3)[None] + 0.5 * K + c[:, None, None] * (K @ K)


# ---------------------------------------------------------------- navigation state

def nav_parts(x: np.ndarray):
    x = np.atleast_2d(x)
    return quat_to_R(x[:, 0:4]), x[:, 4:7], x[:, 7:10], x[:, 10:13], x[:, 13:16]


def retract_nav(x: np.ndarray, d: np.ndarray) -> np.ndarray:
    """x [+] d on the navigation-state chart (right rotation update, p += R dp)."""
    R, p, v, bg, ba = nav_parts(x)
    R2 = R @ so3.exp(d[:, 0:3])
    out = np.empty_like(np.atleast_2d(x))
    out[:, 0:4] = R_to_quat(R2)
    out[:, 4:7] = p + np.einsum("nij,nj->ni", R, d[:, 3:6])
    out[:, 7:10] = v + d[:, 6:9]
    out[:, 10:13] = bg + d[:, 9:12]
    out[:, 13:16] = ba + d[:, 12:15]
    return out


# ---------------------------------------------------------------- stereo reprojection

def kb_project(x, y, z, fx, fy, cx, cy, k):
    """Kannala-Brandt (equidistant) fisheye projection of camera-frame points and its
    Jacobian d(u, v)/d(x, y, z): theta = atan2(r, z), r = |(x, y)|,
    theta_d = theta (1 + k1 theta^2 + k2 theta^4 + k3 theta^6 + k4 theta^8),
    (u, v) = (fx theta_d x / r + cx, fy theta_d y / r + cy)."""
    k1, k2, k3, k4 = k
    r = np.sqrt(x * x + y * y)
    th = np.arctan2(r, z)
    t2 = th * th
    thd = th * (1 + t2 * (k1 + t2 * (k2 + t2 * (k3 + t2 * k4))))
    dthd = 1 + t2 * (3 * k1 + t2 * (5 * k2 + t2 * (7 * k3 + t2 * 9 * k4)))
    s = thd / r
    q = r * r + z * z
    dth = np.stack([x * z / (r * q), y * z / (r * q), -r / q], axis=-1)      # dtheta/d(x, y, z)
    ds = dthd[..., None] * dth / r[..., None]
    ds[..., 0] -= thd * x / r ** 3
    ds[..., 1] -= thd * y / r ** 3
    u = fx * s * x + cx
    v = fy * s * y + cy
    J = np.zeros(x.shape + (2, 3))
    J[..., 0, :] = fx * x[..., None] * ds
    J[..., 0, 0] += fx * s
    J[..., 1, :] = fy * y[..., None] * ds
    J[..., 1, 1] += fy * s
    return u, v, J


class StereoCamera:
    """Pinhole stereo rig, or Kannala-Brandt fisheye when `fisheye` holds k1..k4 (both
    cameras, the right one `baseline` along x)."""

    def __init__(self, fx, fy, cx, cy, baseline, R_cb, t_cb, fisheye=None):
        self.fx, self.fy, self.cx, self.cy, self.b = fx, fy, cx, cy, baseline
        self.R_cb = np.asarray(R_cb, dtype=np.float64)
        self.t_cb = np.asarray(t_cb, dtype=np.float64)
        self.fisheye = None if fisheye is None else np.asarray(fisheye, dtype=np.float64)

    def point_in_camera(self, nav, X):
        R, p, _, _, _ = nav_parts(nav)
        Xb = np.einsum("nji,nj->ni", R, np.atleast_2d(X) - p)
        return Xb, Xb @ self.R_cb.T + self.t_cb

    def project(self, nav, X):
        _, Xc = self.point_in_camera(nav, X)
        x, y, z = Xc[:, 0], Xc[:, 1], Xc[:, 2]
        if self.fisheye is not None:
            ul, vl, _ = kb_project(x, y, z, self.fx, self.fy, self.cx, self.cy, self.fisheye)
            ur, _, _ = kb_project(x - self.b, y, z, self.fx, self.fy, self.cx, self.cy, self.fisheye)
            return np.stack([ul, vl, ur], axis=1)
        return np.stack([self.fx * x / z + self.cx, self.fy * y / z + self.cy,
                         self.fx * (x - self.b) / z + self.cx], axis=1)

    def evaluate(self, states, obs):
        """Edge evaluator: states = [nav (n,16), points (n,3)] -> r (n,3), [J_nav (n,3,15), J_pt (n,3,3)]."""
        nav, X = states
        R, _, _, _, _ = nav_parts(nav)
        Xb, Xc = self.point_in_camera(nav, X)
        x, y, z = Xc[:, 0], Xc[:, 1], Xc[:, 2]
        r = self.project(nav, X) - obs
        n = len(z)
        D = np.zeros((n, 3, 3))          # dr / dX_c
        if self.fisheye is not None:
            _, _, Jl = kb_project(x, y, z, self.fx, self.fy, self.cx, self.cy, self.fisheye)
            _, _, Jr = kb_project(x - self.b, y, z, self.fx, self.fy, self.cx, self.cy, self.fisheye)
            D[:, 0:2] = Jl
            D[:, 2] = Jr[:, 0]
        else:
            D[:, 0, 0] = self.fx / z
            D[:, 0, 2] = -self.fx * x / z ** 2
            D[:, 1, 1] = self.fy / z
            D[:, 1, 2] = -self.fy * y / z ** 2
            D[:, 2, 0] = self.fx / z
            D[:, 2, 2] = -self.fx * (x - self.b) / z ** 2
        DR = D @ self.R_cb
        Jn = np.zeros((n, 3, 15))
        Jn[:, :, 0:3] = DR @ so3.hat(Xb)      # dX_b/dtheta = [X_b]x
        Jn[:, :, 3:6] = -DR                    # dX_b/dp = -I
        Jp = DR @ np.transpose(R, (0, 2, 1))   # dX_b/dX = R^T
        return r, [Jn, Jp]


# ---------------------------------------------------------------- IMU preintegration

def preintegrate(omega, acc, dt, bg0, ba0, sigma_g, sigma_a):
    """Preintegrated measurement of samples (N,3) at bias estimates bg0, ba0 (see module doc)."""
    omega = np.asarray(omega, dtype=np.float64)
    acc = np.asarray(acc, dtype=np.float64)
    dR = np.eye(3)
    dv = np.zeros(3)
    dp = np.zeros(3)
    JRg = np.zeros((3, 3))
    Jvg = np.zeros((3, 3))
    Jva = np.zeros((3, 3))
    Jpg = np.zeros((3, 3))
    Jpa = np.zeros((3, 3))
    cov = np.zeros((9, 9))
    Qg = (sigma_g ** 2 / dt) * np.eye(3)
    Qa = (sigma_a ** 2 / dt) * np.eye(3)
    for k in range(len(omega)):
        w = (omega[k] - bg0) * dt
        a = acc[k] - ba0
        dRk = so3.exp(w)[0]
        Jr = right_jacobian(w)[0]
        ahat = so3.hat(a)
        # covariance of (dphi, dv, dp)
        A = np.eye(9)
        A[0:3, 0:3] = dRk.T
        A[3:6, 0:3] = -dR @ ahat * dt
        A[6:9, 0:3] = -0.5 * dR @ ahat * dt * dt
        A[6:9, 3:6] = np.eye(3) * dt
        Bg = np.zeros((9, 3))
        Bg[0:3] = Jr * dt
        Ba = np.zeros((9, 3))
        Ba[3:6] = dR * dt
        Ba[6:9] = 0.5 * dR * dt * dt
        cov = A @ cov @ A.T + Bg @ Qg @ Bg.T + Ba @ Qa @ Ba.T
        # bias Jacobians (position first: it uses the previous velocity Jacobians)
        Jpa = Jpa + Jva * dt - 0.5 * dR * dt * dt
        Jpg = Jpg + Jvg * dt - 0.5 * dR @ ahat @ JRg * dt * dt
        Jva = Jva - dR * dt
        Jvg = Jvg - dR @ ahat @ JRg * dt
        JRg = dRk.T @ JRg - Jr * dt
        # the measurement itself
        dp = dp + dv * dt + 0.5 * dR @ a * dt * dt
        dv = dv + dR @ a * dt
        dR = dR @ dRk
    return dict(dR=dR, dv=dv, dp=dp, T=dt * len(omega), JRg=JRg, Jvg=Jvg, Jva=Jva, Jpg=Jpg,
                Jpa=Jpa, cov=cov, bg0=np.asarray(bg0, float).copy(), ba0=np.asarray(ba0, float).copy())


def imu_residual_one(pim, xi, xj):
    """9-vector inertial residual [r_R, r_v, r_p] of one edge."""
    Ri, pi, vi, bgi, bai = [a[0] for a in nav_parts(xi)]
    Rj, pj, vj, _, _ = [a[0] for a in nav_parts(xj)]
    dbg = bgi - pim["bg0"]
    dba = bai - pim["ba0"]
    T = pim["T"]
    dRc = pim["dR"] @ so3.exp(pim["JRg"] @ dbg)[0]
    dvc = pim["dv"] + pim["Jvg"] @ dbg + pim["Jva"] @ dba
    dpc = pim["dp"] + pim["Jpg"] @ dbg + pim["Jpa"] @ dba
    rR = so3.log(dRc.T @ Ri.T @ Rj)[0]
    rv = Ri.T @ (vj - vi - GRAVITY * T) - dvc
    rp = Ri.T @ (pj - pi - vi * T - 0.5 * GRAVITY * T * T) - dpc
    return np.concatenate([rR, rv, rp])


def imu_jacobians_one(pim, xi, xj):
    """(J_i (9,15), J_j (9,15)) of the inertial residual on the navigation-state chart."""
    Ri, pi, vi, bgi, bai = [a[0] for a in nav_parts(xi)]
    Rj, pj, vj, _, _ = [a[0] for a in nav_parts(xj)]
    dbg = bgi - pim["bg0"]
    T = pim["T"]
    dRc = pim["dR"] @ so3.exp(pim["JRg"] @ dbg)[0]
    rR = so3.log(dRc.T @ Ri.T @ Rj)[0]
    Jri = right_jacobian_inv(rR)[0]
    Ji = np.zeros((9, 15))
    Jj = np.zeros((9, 15))
    # rotation row
    Ji[0:3, 0:3] = -Jri @ Rj.T @ Ri
    Jj[0:3, 0:3] = Jri
    Ji[0:3, 9:12] = -Jri @ so3.exp(rR)[0].T @ right_jacobian(pim["JRg"] @ dbg)[0] @ pim["JRg"]
    # velocity row
    Ji[3:6, 0:3] = so3.hat(Ri.T @ (vj - vi - GRAVITY * T))
    Ji[3:6, 6:9] = -Ri.T
    Jj[3:6, 6:9] = Ri.T
    Ji[3:6, 9:12] = -pim["Jvg"]
    Ji[3:6, 12:15] = -pim["Jva"]
    # position row
    Ji[6:9, 0:3] = so3.hat(Ri.T @ (pj - pi - vi * T - 0.5 * GRAVITY * T * T))
    Ji[6:9, 3:6] = -np.eye(3)
    Jj[6:9, 3:6] = Ri.T @ Rj
    Ji[6:9, 6:9] = -Ri.T * T
    Ji[6:9, 9:12] = -pim["Jpg"]
    Ji[6:9, 12:15] = -pim["Jpa"]
    return Ji, Jj


def imu_evaluate(pims):
    """Edge evaluator over a list of preintegrated measurements (one per edge)."""
    def ev(states, data):
        xi, xj = states
        idx = data
        r = np.stack([imu_residual_one(pims[k], xi[n:n + 1], xj[n:n + 1]) for n, k in enumerate(idx)])
        Js = [imu_jacobians_one(pims[k], xi[n:n + 1], xj[n:n + 1]) for n, k in enumerate(idx)]
        return r, [np.stack([a for a, _ in Js]), np.stack([b for _, b in Js])]
    return ev


def bias_rw_evaluate(states, data):
    """r = [bg_j - bg_i, ba_j - ba_i] (6), Jacobians +-I on the bias columns."""
    xi, xj = states
    n = xi.shape[0]
    r = np.concatenate([xj[:, 10:13] - xi[:, 10:13], xj[:, 13:16] - xi[:, 13:16]], axis=1)
    Ji = np.zeros((n, 6, 15))
    Jj = np.zeros((n, 6, 15))
    Ji[:, :, 9:15] = -np.eye(6)
    Jj[:, :, 9:15] = np.eye(6)
    return r, [Ji, Jj]


def bias_prior_evaluate(states, data):
    """r = [bg - bg_prior, ba - ba_prior] (6); data = priors (n, 6)."""
    (x,) = states
    n = x.shape[0]
    r = x[:, 10:16] - data
    J = np.zeros((n, 6, 15))
    J[:, :, 9:15] = np.eye(6)
    return r, [J]


# ---------------------------------------------------------------- problem builder

def mono_evaluate(cam: StereoCamera):
    """Monocular reprojection in the rig's left camera: the first two rows of the stereo
    residual and its Jacobians (obs: n x 2 pixels)."""
    def ev(states, obs):
        o3 = np.concatenate([np.asarray(obs, float), np.zeros((len(obs), 1))], axis=1)
        r, (Jn, Jp) = cam.evaluate(states, o3)
        return r[:, :2], [Jn[:, :2], Jp[:, :2]]
    return ev


def camera_of(cam: dict) -> StereoCamera:
    return StereoCamera(cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["baseline"], cam["R_cb"],
                        cam["t_cb"], cam.get("fisheye"))


def preintegrate_all(p, bg0=None, ba0=None):
    """Preintegrated measurement of every consecutive keyframe pair of a VIProblem-like
    record, at bias estimates (default: the initial state's)."""
    out = []
    for k in range(p.imu_gyro.shape[0]):
        b_g = p.nav0[k, 10:13] if bg0 is None else bg0
        b_a = p.nav0[k, 13:16] if ba0 is None else ba0
        out.append(preintegrate(p.imu_gyro[k], p.imu_acc[k], p.dt, b_g, b_a,
                                p.noise["sigma_g"], p.noise["sigma_a"]))
    return out


def problem(p, nav, pts, pims, prior_sigma=(1e-2, 1e-1), huber=True, imu_huber=None, mono=None):
    """Generic-LM problem of the VI objective: stereo reprojection (Huber), inertial
    (optionally Huber on its whitened residual, threshold imu_huber), bias random walk
    between consecutive keyframes, bias prior on keyframe 0.  mono: boolean mask of the
    observations kept as monocular (left-camera) edges instead of stereo ones."""
    from . import lm
    K = nav.shape[0]
    vs = {"nav": lm.VertexSet("nav", 15, nav, retract_nav, False),
          "pt": lm.VertexSet("pt", 3, pts, lambda s, d: s + d, True)}
    cam = camera_of(p.camera)
    loss = ("huber", p.huber_delta) if huber else None
    keep = np.ones(len(p.kf_idx), bool) if mono is None else ~np.asarray(mono, bool)
    ids = np.stack([p.kf_idx, p.pt_idx], axis=1)
    obs = np.asarray(p.obs, float)
    sets = []
    if keep.any():
        sets.append(lm.EdgeSet("stereo", ["nav", "pt"], ids[keep], cam.evaluate, obs[keep], None, loss))
    if mono is not None and (~keep).any():
        sets.append(lm.EdgeSet("mono", ["nav", "pt"], ids[~keep], mono_evaluate(cam), obs[~keep, :2], None, loss))
    ij = np.stack([np.arange(K - 1), np.arange(1, K)], axis=1)
    U = np.stack([np.linalg.cholesky(np.linalg.inv(pm["cov"])).T for pm in pims])
    imu = lm.EdgeSet("imu", ["nav", "nav"], ij, imu_evaluate(pims), np.arange(K - 1), U,
                     None if imu_huber is None else ("huber", float(imu_huber)))
    T = np.array([pm["T"] for pm in pims])
    w = np.concatenate([np.tile(1.0 / np.sqrt(p.noise["sigma_bg"] ** 2 * T)[:, None], (1, 3)),
                        np.tile(1.0 / np.sqrt(p.noise["sigma_ba"] ** 2 * T)[:, None], (1, 3))], axis=1)
    rw = lm.EdgeSet("bias_rw", ["nav", "nav"], ij, bias_rw_evaluate, None,
                    np.stack([np.diag(x) for x in w]), None)
    pw = np.diag(np.r_[np.full(3, 1.0 / prior_sigma[0]), np.full(3, 1.0 / prior_sigma[1])])
    prior = lm.EdgeSet("bias_prior", ["nav"], np.array([[0]]), bias_prior_evaluate,
                       np.zeros((1, 6)), pw[None], None)
    return lm.Problem(vs, sets + [imu, rw, prior])
