// Forward-mode automatic differentiation of the edge residuals (dual numbers), the
// checker and prototyping path for edge kinds (Sec. IV-D: the paper differentiates its
// edges with a forward-mode generator and offers analytic Jacobians beside it).  Every
// observation edge's residual is evaluated on dual numbers carrying the derivatives
// with respect to the camera's tangent coordinates (the chart of the analytic
// Jacobians: left rotation update for BA cameras, right update of rotation and
// position for navigation states) and the point, at the current state, in FP64.  The
// whitening, the Huber IRLS weight (a constant of the linearisation, not
// differentiated) and the fixed-vertex zero columns are those of the analytic path, so
// both give the same rows up to rounding.
#pragma once

#include "schur_common.cuh"

namespace gpo {

// A value and its derivatives with respect to N seeded variables (first order: the
// product of two derivative parts is dropped, which is exact for first derivatives).
template <int N>
struct Dual {
  double v;
  double g[N];
};
template <int N>
__device__ __forceinline__ Dual<N> dconst(double v) {
  Dual<N> a;
  a.v = v;
#pragma unroll
  for (int i = 0; i < N; ++i) a.g[i] = 0.0;
  return a;
}
template <int N>
__device__ __forceinline__ Dual<N> dvar(double v, int i) {
  Dual<N> a = dconst<N>(v);
  a.g[i] = 1.0;
  return a;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> c;
  c.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.g[i] = a.g[i] + b.g[i];
  return c;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> c;
  c.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.g[i] = a.g[i] - b.g[i];
  return c;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
  Dual<N> c;
  c.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.g[i] = -a.g[i];
  return c;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> c;
  c.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.g[i] = a.g[i] * b.v + a.v * b.g[i];
  return c;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(double s, const Dual<N>& a) {
  Dual<N> c;
  c.v = s * a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.g[i] = s * a.g[i];
  return c;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, double s) {
  Dual<N> c = a;
  c.v += s;
  return c;
}
// a / b: (a' b - a b') / b^2
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> c;
  const double ib = 1.0 / b.v;
  c.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) c.g[i] = (a.g[i] - c.v * b.g[i]) * ib;
  return c;
}

template <int N>
__device__ __forceinline__ Dual<N> dsqrt(const Dual<N>& a) {
  Dual<N> c;
  c.v = sqrt(a.v);
  const double h = 0.5 / c.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.g[i] = a.g[i] * h;
  return c;
}
// atan2(y, x): derivative (x dy - y dx) / (x^2 + y^2)
template <int N>
__device__ __forceinline__ Dual<N> datan2(const Dual<N>& y, const Dual<N>& x) {
  Dual<N> c;
  c.v = atan2(y.v, x.v);
  const double q = 1.0 / (x.v * x.v + y.v * y.v);
#pragma unroll
  for (int i = 0; i < N; ++i) c.g[i] = (x.v * y.g[i] - y.v * x.g[i]) * q;
  return c;
}

// Kannala-Brandt fisheye projection (u, v) of a camera-frame point on duals.
template <int N>
__device__ void kb_project_ad(const double* camk, const Dual<N>& x, const Dual<N>& y, const Dual<N>& z,
                              Dual<N>& u, Dual<N>& v) {
  const double k1 = camk[18], k2 = camk[19], k3 = camk[20], k4 = camk[21];
  const Dual<N> r = dsqrt(x * x + y * y);
  const Dual<N> th = datan2(r, z), t2 = th * th;
  const Dual<N> poly = t2 * (t2 * (t2 * (k4 * t2 + k3) + k2) + k1) + 1.0;
  const Dual<N> s = (th * poly) / r;
  u = camk[0] * (s * x) + camk[2];
  v = camk[1] * (s * y) + camk[3];
}

// BA reprojection on duals: variables 0..8 the camera tangent (left rotation update dw,
// translation, f, k1, k2), 9..11 the point.  P = (I + [dw]_x) R X + t, p = -P_xy / P_z,
// u = f (1 + k1 |p|^2 + k2 |p|^4) p, r = u - z.
template <int N>
__device__ void ba_residual_ad(const double* rb, const double* X0, const double* z, Dual<N> (&r)[2]) {
  Dual<N> X[3], w[3], y[3], P[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    X[j] = dvar<N>(X0[j], 9 + j);
    w[j] = dvar<N>(0.0, j);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = rb[3 * i] * X[0] + rb[3 * i + 1] * X[1] + rb[3 * i + 2] * X[2];
  const Dual<N> wy[3] = {w[1] * y[2] - w[2] * y[1], w[2] * y[0] - w[0] * y[2], w[0] * y[1] - w[1] * y[0]};
#pragma unroll
  for (int i = 0; i < 3; ++i) P[i] = y[i] + wy[i] + dvar<N>(rb[9 + i], 3 + i);
  const Dual<N> p0 = -(P[0] / P[2]), p1 = -(P[1] / P[2]);
  const Dual<N> f = dvar<N>(rb[12], 6), k1 = dvar<N>(rb[13], 7), k2 = dvar<N>(rb[14], 8);
  const Dual<N> r2 = p0 * p0 + p1 * p1;
  const Dual<N> dd = (k1 * r2 + k2 * r2 * r2) + 1.0;
  const Dual<N> fd = f * dd;
  r[0] = fd * p0 + (-z[0]);
  r[1] = fd * p1 + (-z[1]);
}

// Stereo reprojection of a navigation state on duals: variables 0..2 the rotation
// update dtheta (R <- R Exp(dtheta)), 3..5 the position update dp (p <- p + R dp),
// 6..8 the point.  X_b = (I - [dtheta]_x)(R^T (X - p) - dp), X_c = R_cb X_b + t_cb,
// u = (fx x / z + cx, fy y / z + cy, fx (x - b) / z + cx), r = u - z_obs.
template <int N>
__device__ void stereo_residual_ad(const DevBA& d, const double* rb, const double* X0, const double* z,
                                   Dual<N> (&r)[3]) {
  Dual<N> a[3], v[3], th[3], xb[3], xc[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    a[j] = dvar<N>(X0[j], 6 + j) + (-rb[9 + j]);
    th[j] = dvar<N>(0.0, j);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] = (rb[i] * a[0] + rb[3 + i] * a[1] + rb[6 + i] * a[2]) - dvar<N>(0.0, 3 + i);
  const Dual<N> tv[3] = {th[1] * v[2] - th[2] * v[1], th[2] * v[0] - th[0] * v[2], th[0] * v[1] - th[1] * v[0]};
#pragma unroll
  for (int i = 0; i < 3; ++i) xb[i] = v[i] - tv[i];
  const double* Rc = d.camk + 5;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    xc[i] = (Rc[3 * i] * xb[0] + Rc[3 * i + 1] * xb[1] + Rc[3 * i + 2] * xb[2]) + d.camk[14 + i];
  const double fx = d.camk[0], fy = d.camk[1], cx = d.camk[2], cy = d.camk[3], b = d.camk[4];
  if (d.camk[17] != 0.0) {   // fisheye rig
    Dual<N> u, v, ur, vr;
    kb_project_ad<N>(d.camk, xc[0], xc[1], xc[2], u, v);
    kb_project_ad<N>(d.camk, xc[0] + (-b), xc[1], xc[2], ur, vr);
    r[0] = u + (-z[0]);
    r[1] = v + (-z[1]);
    r[2] = ur + (-z[2]);
    return;
  }
  r[0] = fx * (xc[0] / xc[2]) + (cx - z[0]);
  r[1] = fy * (xc[1] / xc[2]) + (cy - z[1]);
  r[2] = fx * ((xc[0] + (-b)) / xc[2]) + (cx - z[2]);
}

template <class Mo>
struct AdModel;
template <>
struct AdModel<ModelBA> {
  static constexpr int M = 2, N = 12;
  __device__ static void residual(const DevBA& d, int e, const double* rb, const double* X, Dual<N> (&r)[M]) {
    ba_residual_ad<N>(rb, X, d.obs + 2 * (size_t)e, r);
  }
};
template <>
struct AdModel<ModelStereo> {
  static constexpr int M = 3, N = 9;
  __device__ static void residual(const DevBA& d, int e, const double* rb, const double* X, Dual<N> (&r)[M]) {
    stereo_residual_ad<N>(d, rb, X, d.obs + 3 * (size_t)e, r);
  }
};

// One thread per observation edge (sorted order): the weighted, whitened residual
// r_out[M e + a] and Jacobian rows J_out[(M e + a) N + j] (camera tangent columns, then
// the point's three), FP64.
template <class Mo>
__global__ void __launch_bounds__(256) k_autodiff(LaunchSet ls, double* r_out, double* J_out) {
  using A = AdModel<Mo>;
  constexpr int M = A::M, N = A::N, DC = Mo::DC;
  __shared__ DevBA d;
  pdl_trigger();
  bind_problem(d, ls.probs);
  pdl_wait();
  const int e = blockIdx.x * 256 + threadIdx.x;
  if (e >= d.E) return;
  const int c = d.e_cam[e], p = d.e_pt[e];
  double rb[16];
  load_rb(d.camrb + 16 * (size_t)c, rb);
  const double X[3] = {d.pt[3 * (size_t)p], d.pt[3 * (size_t)p + 1], d.pt[3 * (size_t)p + 2]};
  Dual<N> r[M];
  A::residual(d, e, rb, X, r);
  if (d.e_sqinfo) {   // r <- U r with U upper triangular, packed row by row
    const double* U = d.e_sqinfo + Mo::NQ * (size_t)e;
    int q = 0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
      Dual<N> s = dconst<N>(0.0);
      for (int j = i; j < M; ++j) s = s + U[q++] * r[j];
      r[i] = s;
    }
  }
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) s += r[a].v * r[a].v;
  const double sw = huber_weight<double>(s, d.e_delta[e]);
  const bool cf = d.cam_fixed[c] != 0, pf = d.pt_fixed[p] != 0;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    r_out[(size_t)M * e + a] = sw * r[a].v;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const bool zero = j < DC ? cf : pf;
      J_out[((size_t)M * e + a) * N + j] = zero ? 0.0 : sw * r[a].g[j];
    }
  }
}

}  // namespace gpo
