// Visual-inertial kernel set: the Schur-complement LM kernels instantiated for the
// stereo reprojection model on 15-dimensional navigation states, plus the kernels of
// the camera-side edges between keyframes (Eq. 8: inertial residual r_I and bias
// residual r_b; Sec. V-C: inertial, bias random-walk and bias-prior constraints).
//
// Navigation state x = [qx qy qz qw, p, v, bg, ba] (body-to-world rotation R),
// tangent [dtheta, dp, dv, dbg, dba]: R <- R Exp(dtheta), p <- p + R dp, the rest
// additive.  Gravity g = (0, 0, -9.81).
//
// The inertial residual is that of on-manifold IMU preintegration (Forster, Carlone,
// Dellaert, Scaramuzza, T-RO 2017) with first-order bias correction, between
// keyframes i and j with preintegrated (dR, dv, dp) over T at bias estimates
// (bg0, ba0), dbg = bg_i - bg0, dba = ba_i - ba0:
//   r_R = Log((dR Exp(JRg dbg))^T R_i^T R_j)
//   r_v = R_i^T (v_j - v_i - g T) - (dv + Jvg dbg + Jva dba)
//   r_p = R_i^T (p_j - p_i - v_i T - g T^2 / 2) - (dp + Jpg dbg + Jpa dba)
// Bias random walk: [bg_j - bg_i, ba_j - ba_i]; bias prior: [bg_i, ba_i] - prior.
// All are whitened by the upper-triangular square root of their information matrix.
// Camera-side edges are few (one or two per keyframe), so they are evaluated in FP64
// by one thread each, and their Jacobians are kept in FP64.
#include "schur_kernels.cuh"

namespace gpo {

namespace {

// ---------------------------------------------------------------- 3x3 helpers (row-major)

__device__ __forceinline__ void mm3(const double* A, const double* B, double* C) {   // C = A B
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}
__device__ __forceinline__ void mtm3(const double* A, const double* B, double* C) {  // C = A^T B
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[i] * B[j] + A[3 + i] * B[3 + j] + A[6 + i] * B[6 + j];
}
__device__ __forceinline__ void mv3(const double* A, const double* v, double* o) {
  for (int i = 0; i < 3; ++i) o[i] = A[3 * i] * v[0] + A[3 * i + 1] * v[1] + A[3 * i + 2] * v[2];
}
__device__ __forceinline__ void mtv3(const double* A, const double* v, double* o) {  // A^T v
  for (int i = 0; i < 3; ++i) o[i] = A[i] * v[0] + A[3 + i] * v[1] + A[6 + i] * v[2];
}
__device__ __forceinline__ void hat3(const double* v, double* K) {
  K[0] = 0.0;   K[1] = -v[2]; K[2] = v[1];
  K[3] = v[2];  K[4] = 0.0;   K[5] = -v[0];
  K[6] = -v[1]; K[7] = v[0];  K[8] = 0.0;
}

// Unit quaternion (w, x, y, z) of a rotation matrix, from the largest of the four
// squared components (Shepperd's method).
__device__ void R_to_q(const double* R, double* q) {
  const double tr = R[0] + R[4] + R[8];
  if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
    const double s = 2.0 * sqrt(1.0 + tr);   // 4 w
    q[0] = 0.25 * s; q[1] = (R[7] - R[5]) / s; q[2] = (R[2] - R[6]) / s; q[3] = (R[3] - R[1]) / s;
  } else if (R[0] >= R[4] && R[0] >= R[8]) {
    const double s = 2.0 * sqrt(1.0 + R[0] - R[4] - R[8]);   // 4 x
    q[0] = (R[7] - R[5]) / s; q[1] = 0.25 * s; q[2] = (R[1] + R[3]) / s; q[3] = (R[2] + R[6]) / s;
  } else if (R[4] >= R[8]) {
    const double s = 2.0 * sqrt(1.0 + R[4] - R[0] - R[8]);   // 4 y
    q[0] = (R[2] - R[6]) / s; q[1] = (R[1] + R[3]) / s; q[2] = 0.25 * s; q[3] = (R[5] + R[7]) / s;
  } else {
    const double s = 2.0 * sqrt(1.0 + R[8] - R[0] - R[4]);   // 4 z
    q[0] = (R[3] - R[1]) / s; q[1] = (R[2] + R[6]) / s; q[2] = (R[5] + R[7]) / s; q[3] = 0.25 * s;
  }
  const double n = 1.0 / sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) q[k] *= n;
}

// SO(3) logarithm.  With v = vee(R - R^T) / 2 = sin(t) a and cos(t) = (tr R - 1) / 2,
// t = atan2(|v|, cos t) and w = t / sin(t) v (series 1 + t^2 / 6 for small t); near
// t = pi the axis is taken from the quaternion of R.
__device__ void so3_log(const double* R, double* w) {
  const double v0 = 0.5 * (R[7] - R[5]), v1 = 0.5 * (R[2] - R[6]), v2 = 0.5 * (R[3] - R[1]);
  const double s = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
  const double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  const double t = atan2(s, c);
  if (t > 3.14059265358979) {   // within 1e-3 of pi
    double q[4];
    R_to_q(R, q);
    q_to_aa(q, w);
    return;
  }
  const double k = t < 1e-4 ? 1.0 + t * t / 6.0 : t / s;
  w[0] = k * v0;
  w[1] = k * v1;
  w[2] = k * v2;
}

// Right Jacobian of SO(3): Jr(phi) = I - (1 - cos t)/t^2 [phi]x + (t - sin t)/t^3 [phi]x^2,
// and its inverse I + [phi]x / 2 + (1/t^2 - (1 + cos t)/(2 t sin t)) [phi]x^2 (Taylor
// coefficients below t = 1e-4).
__device__ void so3_jr(const double* phi, double* J, bool inverse) {
  const double t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  const double t = sqrt(t2);
  double a, b;
  if (!inverse) {
    if (t < 1e-4) {
      a = -(0.5 - t2 / 24.0);
      b = 1.0 / 6.0 - t2 / 120.0;
    } else {
      double sn, cs;
      sincos(t, &sn, &cs);
      a = -(1.0 - cs) / t2;
      b = (t - sn) / (t2 * t);
    }
  } else {
    a = 0.5;
    if (t < 1e-4) {
      b = 1.0 / 12.0 + t2 / 720.0;
    } else {
      double sn, cs;
      sincos(t, &sn, &cs);
      b = 1.0 / t2 - (1.0 + cs) / (2.0 * t * sn);
    }
  }
  double K[9], K2[9];
  hat3(phi, K);
  mm3(K, K, K2);
  for (int i = 0; i < 9; ++i) J[i] = a * K[i] + b * K2[i];
  J[0] += 1.0;
  J[4] += 1.0;
  J[8] += 1.0;
}

struct Nav {
  double R[9], p[3], v[3], bg[3], ba[3];
};
__device__ __forceinline__ void nav_load(const double* x, const double* rb, Nav& n) {
  for (int i = 0; i < 9; ++i) n.R[i] = rb[i];
  for (int i = 0; i < 3; ++i) {
    n.p[i] = x[4 + i];
    n.v[i] = x[7 + i];
    n.bg[i] = x[10 + i];
    n.ba[i] = x[13 + i];
  }
}

// J (row-major kXRows x kXCols) block setters: rows r0.., columns c0.. of a 3x3 block.
__device__ __forceinline__ void put3(double* J, int r0, int c0, const double* B, double s) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) J[(r0 + i) * kXCols + c0 + j] = s * B[3 * i + j];
}

// Inertial residual r (9) and, if J is given, its Jacobians on both navigation
// charts (columns 0-14: keyframe i, 15-29: keyframe j).
__device__ void imu_eval(const double* rec, const Nav& a, const Nav& b, double* r, double* J) {
  const double* dR = rec;
  const double* dv = rec + 9;
  const double* dp = rec + 12;
  const double* JRg = rec + 15;
  const double* Jvg = rec + 24;
  const double* Jva = rec + 33;
  const double* Jpg = rec + 42;
  const double* Jpa = rec + 51;
  const double T = rec[60];
  const double* bg0 = rec + 61;
  const double* ba0 = rec + 64;
  const double gz = -9.81;
  double dbg[3], dba[3];
  for (int k = 0; k < 3; ++k) {
    dbg[k] = a.bg[k] - bg0[k];
    dba[k] = a.ba[k] - ba0[k];
  }
  double phi[3], E[9], dRc[9];
  mv3(JRg, dbg, phi);
  aa_to_R(phi, E);
  mm3(dR, E, dRc);
  double A[9], Q[9], rR[3];
  mtm3(a.R, b.R, A);     // R_i^T R_j
  mtm3(dRc, A, Q);       // dRc^T R_i^T R_j
  so3_log(Q, rR);
  double u[3], w[3], Ru[3], Rw[3];
  for (int k = 0; k < 3; ++k) {
    const double gk = k == 2 ? gz : 0.0;
    u[k] = b.v[k] - a.v[k] - gk * T;
    w[k] = b.p[k] - a.p[k] - a.v[k] * T - 0.5 * gk * T * T;
  }
  mtv3(a.R, u, Ru);
  mtv3(a.R, w, Rw);
  double t1[3], t2[3];
  mv3(Jvg, dbg, t1);
  mv3(Jva, dba, t2);
  for (int k = 0; k < 3; ++k) {
    r[k] = rR[k];
    r[3 + k] = Ru[k] - (dv[k] + t1[k] + t2[k]);
  }
  mv3(Jpg, dbg, t1);
  mv3(Jpa, dba, t2);
  for (int k = 0; k < 3; ++k) r[6 + k] = Rw[k] - (dp[k] + t1[k] + t2[k]);
  if (!J) return;
  for (int k = 0; k < kXJ; ++k) J[k] = 0.0;
  double Jri[9], B[9], C[9], D[9];
  so3_jr(rR, Jri, true);
  // rotation rows: d/dtheta_i = -Jr^-1 R_j^T R_i, d/dtheta_j = Jr^-1,
  // d/dbg_i = -Jr^-1 Exp(r_R)^T Jr(JRg dbg) JRg
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[3 * i + j] = A[3 * j + i];   // R_j^T R_i = A^T
  mm3(Jri, B, C);
  put3(J, 0, 0, C, -1.0);
  put3(J, 0, 15, Jri, 1.0);
  double ER[9], Jrp[9];
  aa_to_R(rR, ER);
  so3_jr(phi, Jrp, false);
  mtm3(ER, Jrp, B);      // Exp(r_R)^T Jr(phi)
  mm3(B, JRg, C);
  mm3(Jri, C, D);
  put3(J, 0, 9, D, -1.0);
  // velocity rows
  double K[9], Rt[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Rt[3 * i + j] = a.R[3 * j + i];
  hat3(Ru, K);
  put3(J, 3, 0, K, 1.0);
  put3(J, 3, 6, Rt, -1.0);
  put3(J, 3, 15 + 6, Rt, 1.0);
  put3(J, 3, 9, Jvg, -1.0);
  put3(J, 3, 12, Jva, -1.0);
  // position rows
  hat3(Rw, K);
  put3(J, 6, 0, K, 1.0);
  for (int k = 0; k < 3; ++k) J[(6 + k) * kXCols + 3 + k] = -1.0;
  put3(J, 6, 15 + 3, A, 1.0);
  put3(J, 6, 6, Rt, -T);
  put3(J, 6, 9, Jpg, -1.0);
  put3(J, 6, 12, Jpa, -1.0);
}

// Residual (and Jacobian) of one camera-side edge, whitened; returns its row count.
__device__ int xedge_eval(const DevBA& d, int x, const double* cams, const double* rbs, double* r, double* J) {
  const int kind = d.xe_kind[x], i = d.xe_i[x], j = d.xe_j[x];
  const double* rec = d.xe_rec + (size_t)x * kXRec;
  Nav a, b;
  nav_load(cams + 16 * (size_t)i, rbs + 16 * (size_t)i, a);
  if (j >= 0) nav_load(cams + 16 * (size_t)j, rbs + 16 * (size_t)j, b);
  int m;
  if (kind == XK_IMU) {
    m = 9;
    imu_eval(rec, a, b, r, J);
  } else if (kind == XK_BIAS_RW) {
    m = 6;
    for (int k = 0; k < 3; ++k) {
      r[k] = b.bg[k] - a.bg[k];
      r[3 + k] = b.ba[k] - a.ba[k];
    }
    if (J) {
      for (int k = 0; k < kXJ; ++k) J[k] = 0.0;
      for (int k = 0; k < 6; ++k) {
        J[k * kXCols + 9 + k] = -1.0;
        J[k * kXCols + 15 + 9 + k] = 1.0;
      }
    }
  } else {
    m = 6;
    for (int k = 0; k < 3; ++k) {
      r[k] = a.bg[k] - rec[k];
      r[3 + k] = a.ba[k] - rec[3 + k];
    }
    if (J) {
      for (int k = 0; k < kXJ; ++k) J[k] = 0.0;
      for (int k = 0; k < 6; ++k) J[k * kXCols + 9 + k] = 1.0;
    }
  }
  // whitening by the upper-triangular U (row-major kXRows x kXRows), top row first
  // so that each row only reads rows not yet overwritten
  const double* U = rec + kXU;
  for (int p = 0; p < m; ++p) {
    double s = 0.0;
    for (int q = p; q < m; ++q) s += U[p * kXRows + q] * r[q];
    r[p] = s;
  }
  if (J) {
    for (int col = 0; col < kXCols; ++col)
      for (int p = 0; p < m; ++p) {
        double s = 0.0;
        for (int q = p; q < m; ++q) s += U[p * kXRows + q] * J[q * kXCols + col];
        J[p * kXCols + col] = s;
      }
    const bool fi = d.cam_fixed[i], fj = j >= 0 && d.cam_fixed[j];
    for (int p = 0; p < m; ++p)
      for (int k = 0; k < 15; ++k) {
        if (fi) J[p * kXCols + k] = 0.0;
        if (fj) J[p * kXCols + 15 + k] = 0.0;
      }
  }
  for (int p = m; p < kXRows; ++p) r[p] = 0.0;
  return m;
}

// One thread per camera-side edge, the edges whose first keyframe lies in the CTA's
// block of cameras.  mode 0: linearise (r, J) at the current state; 1: cost at the
// candidate state; 2: cost at the current state.
__global__ void __launch_bounds__(kCamPerBlock * 32) k_extra_eval(LaunchSet ls, int mode, int force) {
  GPO_BIND(cb, cbl)
  const Scalars* sc = d.sc;
  if (!sc->active || d.NX == 0) return;
  if (mode == 0 && !force && !sc->need_lin) return;
  const int c0 = cbl * kCamPerBlock, c1 = min(c0 + kCamPerBlock, d.C);
  const int x0 = d.xo_off[c0], x1 = d.xo_off[c1];
  const bool cand = mode == 1;
  const double* cams = cand ? d.cam_cand : d.cam;
  const double* rbs = cand ? d.camrb_cand : d.camrb;
  for (int x = x0 + (int)threadIdx.x; x < x1; x += blockDim.x) {
    double r[kXRows];
    double* J = mode == 0 ? d.xe_J + (size_t)x * kXJ : nullptr;
    const int m = xedge_eval(d, x, cams, rbs, r, J);
    double s = 0.0;
    for (int p = 0; p < m; ++p) s += r[p] * r[p];
    // Huber loss on the whitened residual (inertial edges): IRLS rows scaled by
    // sqrt(rho'), cost 1/2 rho(s), as for the observation edges
    const double delta = d.xe_rec[(size_t)x * kXRec + kXDelta];
    if (mode == 0) {
      const double sw = huber_weight<double>(s, delta);
      if (sw != 1.0) {
        for (int p = 0; p < m; ++p) r[p] *= sw;
        for (int k = 0; k < m * kXCols; ++k) J[k] *= sw;
      }
      for (int p = 0; p < kXRows; ++p) d.xe_r[(size_t)x * kXRows + p] = r[p];
    } else {
      d.xe_cost[x] = 0.5 * huber_rho(s, delta);
    }
  }
}

// -1/2 |J_e dx|^2 of every camera-side edge (FP64), for the model decrease.
template <class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_extra_md(LaunchSet ls) {
  GPO_BIND(cb, cbl)
  const Scalars* sc = d.sc;
  if (!sc->active || d.NX == 0) return;
  const int c0 = cbl * kCamPerBlock, c1 = min(c0 + kCamPerBlock, d.C);
  const int x0 = d.xo_off[c0], x1 = d.xo_off[c1];
  const AT* xs = reinterpret_cast<const AT*>(sc->use_best ? d.xbest : d.x);
  for (int x = x0 + (int)threadIdx.x; x < x1; x += blockDim.x) {
    const int i = d.xe_i[x], j = d.xe_j[x], m = xrows(d.xe_kind[x]);
    const double* J = d.xe_J + (size_t)x * kXJ;
    double s = 0.0;
    for (int p = 0; p < m; ++p) {
      double v = 0.0;
      for (int k = 0; k < 15; ++k) v += J[p * kXCols + k] * (double)xs[15 * (size_t)i + k];
      if (j >= 0)
        for (int k = 0; k < 15; ++k) v += J[p * kXCols + 15 + k] * (double)xs[15 * (size_t)j + k];
      s += v * v;
    }
    d.xe_md[x] = -0.5 * s;
  }
}

using LS = Launch<ModelStereo>;

int vi_linearize(const LaunchSet& ls, Prec pr, bool force, cudaStream_t st) {
  int n = LS::linearize(ls, pr, force, st);
  if (ls.n_cb) {
    launch_pdl(k_extra_eval, ls.n_cb, kCamPerBlock * 32, 0, st, ls, 0, force ? 1 : 0);
    ++n;
  }
  return n;
}

int vi_cost(const LaunchSet& ls, bool candidate, cudaStream_t st) {
  int n = LS::cost(ls, candidate, st);
  if (ls.n_cb) {
    launch_pdl(k_extra_eval, ls.n_cb, kCamPerBlock * 32, 0, st, ls, candidate ? 1 : 2, 0);
    ++n;
  }
  return n;
}

int vi_backsub(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  int n = LS::backsub(ls, pr, st);
  if (ls.n_cb) {
    if (pr == Prec::F64) launch_pdl(k_extra_md<double>, ls.n_cb, kCamPerBlock * 32, 0, st, ls);
    else launch_pdl(k_extra_md<float>, ls.n_cb, kCamPerBlock * 32, 0, st, ls);
    ++n;
  }
  return n;
}

}  // namespace

const KernelSet& kernels_stereo() {
  static const KernelSet k = [] {
    KernelSet s = make_kernel_set<ModelStereo>(ModelKind::STEREO);
    s.linearize = &vi_linearize;
    s.cost = &vi_cost;
    s.backsub = &vi_backsub;
    return s;
  }();
  return k;
}

}  // namespace gpo
