// Bundle-adjustment hot path on sm_103a: edge linearisation, point and camera
// accumulation, camera Schur complement, matrix-free block-Jacobi PCG, point
// back-substitution, FP64 retraction, cost and the LM gain-ratio decision.
//
// Paper mapping: Eq. 1 and Eq. 7 (cost with Huber), Eq. 3-6 (LM normal equations),
// Sec. IV-B (analytic Jacobians), Sec. IV-E (PCG on implicit products of the
// Jacobians, block-Jacobi preconditioner kept at FP32 or higher, Hessian-diagonal
// clamping, residual normalisation), Sec. IV-E last paragraph (kernels walk the
// graph structure; no sparse-matrix format).  The PCG runs on the camera Schur
// complement S = H_cc + lambda D_c - H_cp H_pp^-1 H_pc; its product with a vector is
// formed from the stored Jacobians in one pass per chunk of point-major edges.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "gpo_internal.h"

namespace gpo {

// ---------------------------------------------------------------- numeric helpers

template <class JT> struct AccOf { using T = float; };
template <> struct AccOf<double> { using T = double; };

__device__ __forceinline__ float ldj(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ldj(const float* p) { return *p; }
__device__ __forceinline__ double ldj(const double* p) { return *p; }
__device__ __forceinline__ __nv_bfloat16 cvj(float v, const __nv_bfloat16*) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float cvj(float v, const float*) { return v; }
__device__ __forceinline__ double cvj(double v, const double*) { return v; }

// Edge-major Jacobian rows: 24 values per edge, [Jc row 0 (9), Jc row 1 (9),
// Jp row 0 (3), Jp row 1 (3)], contiguous in point-major edge order.  A row is 48,
// 96 or 192 bytes (BF16 / FP32 / FP64): three, six or twelve 16-byte accesses.
template <class AT>
__device__ __forceinline__ void load_row(const __nv_bfloat16* src, AT (&v)[kJComp]) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const uint4 w = s4[i];
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&w);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 f = __bfloat1622float2(h[j]);
      v[8 * i + 2 * j] = (AT)f.x;
      v[8 * i + 2 * j + 1] = (AT)f.y;
    }
  }
}
template <class AT>
__device__ __forceinline__ void load_row(const float* src, AT (&v)[kJComp]) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float4 w = s4[i];
    v[4 * i] = (AT)w.x; v[4 * i + 1] = (AT)w.y; v[4 * i + 2] = (AT)w.z; v[4 * i + 3] = (AT)w.w;
  }
}
template <class AT>
__device__ __forceinline__ void load_row(const double* src, AT (&v)[kJComp]) {
  const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const double2 w = s2[i];
    v[2 * i] = (AT)w.x; v[2 * i + 1] = (AT)w.y;
  }
}
__device__ __forceinline__ void store_row(__nv_bfloat16* dst, const __nv_bfloat16 (&v)[kJComp]) {
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  const uint4* s4 = reinterpret_cast<const uint4*>(v);
#pragma unroll
  for (int i = 0; i < 3; ++i) d4[i] = s4[i];
}
__device__ __forceinline__ void store_row(float* dst, const float (&v)[kJComp]) {
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < 6; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
__device__ __forceinline__ void store_row(double* dst, const double (&v)[kJComp]) {
  double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
  for (int i = 0; i < 12; ++i) d2[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

// Upper triangle of a 9x9 symmetric block, row-major: entry t is (c_ti[t], c_tj[t]).
__constant__ unsigned char c_ti[kCamTri] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1,
                                            2, 2, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 4, 4, 4, 4,
                                            4, 5, 5, 5, 5, 6, 6, 6, 7, 7, 8};
__constant__ unsigned char c_tj[kCamTri] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 1, 2, 3, 4, 5, 6, 7, 8,
                                            2, 3, 4, 5, 6, 7, 8, 3, 4, 5, 6, 7, 8, 4, 5, 6, 7,
                                            8, 5, 6, 7, 8, 6, 7, 8, 7, 8, 8};
__host__ __device__ __forceinline__ int tri9(int i, int j) {  // i <= j
  return i * 9 - (i * (i - 1)) / 2 + (j - i);
}
__host__ __device__ __forceinline__ int sym9(int i, int j) { return i <= j ? tri9(i, j) : tri9(j, i); }

// ---------------------------------------------------------------- SO(3) (FP64)

// Rodrigues: R = I + a [w]_x + b [w]_x^2 with a = sin t / t, b = (1 - cos t)/t^2,
// [w]_x^2 = w w^T - t^2 I; Taylor coefficients below t = 1e-4.
__device__ void aa_to_R(const double* w, double* R) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, b;
  if (t2 < 1e-8) {
    a = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
    b = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
  } else {
    const double t = sqrt(t2);
    double s, c;
    sincos(t, &s, &c);
    a = s / t;
    b = (1.0 - c) / t2;
  }
  R[0] = 1.0 + b * (w[0] * w[0] - t2);
  R[1] = -a * w[2] + b * w[0] * w[1];
  R[2] = a * w[1] + b * w[0] * w[2];
  R[3] = a * w[2] + b * w[1] * w[0];
  R[4] = 1.0 + b * (w[1] * w[1] - t2);
  R[5] = -a * w[0] + b * w[1] * w[2];
  R[6] = -a * w[1] + b * w[2] * w[0];
  R[7] = a * w[0] + b * w[2] * w[1];
  R[8] = 1.0 + b * (w[2] * w[2] - t2);
}

// Unit quaternion (w, x, y, z) of an angle-axis vector.
__device__ void aa_to_q(const double* w, double* q) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double c, sdt;  // cos(t/2), sin(t/2)/t
  if (t2 < 1e-8) {
    c = 1.0 - t2 / 8.0 + t2 * t2 / 384.0;
    sdt = 0.5 - t2 / 48.0 + t2 * t2 / 3840.0;
  } else {
    const double t = sqrt(t2);
    double s;
    sincos(0.5 * t, &s, &c);
    sdt = s / t;
  }
  q[0] = c;
  q[1] = sdt * w[0];
  q[2] = sdt * w[1];
  q[3] = sdt * w[2];
}

// Angle-axis of a unit quaternion, angle in [0, pi].
__device__ void q_to_aa(const double* qin, double* w) {
  double q0 = qin[0], q1 = qin[1], q2 = qin[2], q3 = qin[3];
  if (q0 < 0) { q0 = -q0; q1 = -q1; q2 = -q2; q3 = -q3; }
  const double s = sqrt(q1 * q1 + q2 * q2 + q3 * q3);
  double k;
  if (s < 1e-8) {
    k = 2.0 / q0 * (1.0 - s * s / (3.0 * q0 * q0));   // 2 atan(s/q0)/s, series
  } else {
    k = 2.0 * atan2(s, q0) / s;
  }
  w[0] = k * q1;
  w[1] = k * q2;
  w[2] = k * q3;
}

// Left update w' = Log(Exp(dw) Exp(w)) via quaternion product.
__device__ void aa_left_update(const double* dw, const double* w, double* out) {
  double a[4], b[4], c[4];
  aa_to_q(dw, a);
  aa_to_q(w, b);
  c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  c[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  c[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  c[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
  const double n = 1.0 / sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2] + c[3] * c[3]);
  c[0] *= n; c[1] *= n; c[2] *= n; c[3] *= n;
  q_to_aa(c, out);
}

// ---------------------------------------------------------------- BA edge model

// Camera render block rb[16]: R (row-major, 9), t (3), f, k1, k2, pad.
struct Geom {
  double y[3];   // R X
  double P[3];   // R X + t
  double p[2];   // -P_xy / P_z
  double iz;     // 1 / P_z
  double r2, d;  // |p|^2, 1 + k1 r2 + k2 r2^2
  double u[2];   // f d p
};

__device__ __forceinline__ void load_rb(const double* __restrict__ src, double* rb) {
  const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const double2 v = __ldg(s2 + i);
    rb[2 * i] = v.x;
    rb[2 * i + 1] = v.y;
  }
}

__device__ __forceinline__ void ba_geom(const double* rb, const double* X, Geom& g) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    g.y[i] = rb[3 * i] * X[0] + rb[3 * i + 1] * X[1] + rb[3 * i + 2] * X[2];
    g.P[i] = g.y[i] + rb[9 + i];
  }
  g.iz = 1.0 / g.P[2];
  g.p[0] = -g.P[0] * g.iz;
  g.p[1] = -g.P[1] * g.iz;
  g.r2 = g.p[0] * g.p[0] + g.p[1] * g.p[1];
  g.d = 1.0 + rb[13] * g.r2 + rb[14] * g.r2 * g.r2;
  const double fd = rb[12] * g.d;
  g.u[0] = fd * g.p[0];
  g.u[1] = fd * g.p[1];
}

// Whitened residual, squared norm, Huber value and sqrt of the first-order weight.
struct Robust {
  double r[2];   // whitened residual U (u - z)
  double rho;    // rho(s)
  double sw;     // sqrt(rho'(s))
};

__device__ __forceinline__ void ba_residual(const DevBA& d, int e, const Geom& g, Robust& o) {
  const double2 z = __ldg(reinterpret_cast<const double2*>(d.obs) + e);
  double r0 = g.u[0] - z.x, r1 = g.u[1] - z.y;
  if (d.e_sqinfo) {
    const double* U = d.e_sqinfo + 3 * (size_t)e;
    const double a = U[0] * r0 + U[1] * r1;
    r1 = U[2] * r1;
    r0 = a;
  }
  o.r[0] = r0;
  o.r[1] = r1;
  const double s = r0 * r0 + r1 * r1;
  const double delta = __ldg(d.e_delta + e);
  if (delta > 0.0 && s > delta * delta) {
    const double sq = sqrt(s);
    o.rho = 2.0 * delta * sq - delta * delta;
    o.sw = sqrt(delta / sq);
  } else {
    o.rho = s;
    o.sw = 1.0;
  }
}

// Jacobian rows of the residual on the chart (left rotation update, additive rest):
// Jc (2x9) and Jp (2x3), whitened and scaled by sqrt(rho').  Computed in AT from
// the FP64 geometry.
template <class AT>
__device__ __forceinline__ void ba_jacobian(const DevBA& d, int e, const double* rb, const Geom& g,
                                            double sw, AT (&Jc)[2][9], AT (&Jp)[2][3]) {
  const AT f = (AT)rb[12], k1 = (AT)rb[13], k2 = (AT)rb[14];
  const AT p0 = (AT)g.p[0], p1 = (AT)g.p[1], r2 = (AT)g.r2, dd = (AT)g.d, iz = (AT)g.iz;
  const AT c2 = (AT)2 * k1 + (AT)4 * k2 * r2;
  // du/dp = f (d I + c2 p p^T)
  const AT A00 = f * (dd + c2 * p0 * p0), A01 = f * c2 * p0 * p1, A11 = f * (dd + c2 * p1 * p1);
  // dp/dP = [[-iz, 0, -p0 iz], [0, -iz, -p1 iz]]  (P_x / P_z^2 = -p0 / P_z)
  const AT B02 = -p0 * iz, B12 = -p1 * iz;
  AT D[2][3];
  D[0][0] = -A00 * iz; D[0][1] = -A01 * iz; D[0][2] = A00 * B02 + A01 * B12;
  D[1][0] = -A01 * iz; D[1][1] = -A11 * iz; D[1][2] = A01 * B02 + A11 * B12;
  const AT y0 = (AT)g.y[0], y1 = (AT)g.y[1], y2 = (AT)g.y[2];
  const AT pp[2] = {p0, p1};
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    // dP/d(dw) = -[y]_x : column k is e_k x y
    Jc[a][0] = -D[a][1] * y2 + D[a][2] * y1;
    Jc[a][1] = D[a][0] * y2 - D[a][2] * y0;
    Jc[a][2] = -D[a][0] * y1 + D[a][1] * y0;
    Jc[a][3] = D[a][0];
    Jc[a][4] = D[a][1];
    Jc[a][5] = D[a][2];
    Jc[a][6] = dd * pp[a];
    Jc[a][7] = f * r2 * pp[a];
    Jc[a][8] = f * r2 * r2 * pp[a];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Jp[a][j] = D[a][0] * (AT)rb[j] + D[a][1] * (AT)rb[3 + j] + D[a][2] * (AT)rb[6 + j];
  }
  if (d.e_sqinfo) {
    const double* U = d.e_sqinfo + 3 * (size_t)e;
    const AT u00 = (AT)U[0], u01 = (AT)U[1], u11 = (AT)U[2];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const AT a = u00 * Jc[0][k] + u01 * Jc[1][k];
      Jc[1][k] = u11 * Jc[1][k];
      Jc[0][k] = a;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const AT a = u00 * Jp[0][k] + u01 * Jp[1][k];
      Jp[1][k] = u11 * Jp[1][k];
      Jp[0][k] = a;
    }
  }
  const AT s = (AT)sw;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
#pragma unroll
    for (int k = 0; k < 9; ++k) Jc[a][k] *= s;
#pragma unroll
    for (int k = 0; k < 3; ++k) Jp[a][k] *= s;
  }
}

// Deterministic CTA sum of one double per thread (fixed tree).
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double out = red[0];
  __syncthreads();
  return out;
}

// Last-CTA detection for grid-wide reductions in a fixed order.
// Call after thread 0 has written the CTA's partial; true in the CTA that finishes last.
__device__ bool last_cta(unsigned int* ticket, int ctas) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == (unsigned int)ctas - 1u);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Sums the n per-CTA partial pairs (stride 2) with all threads of the CTA in a fixed
// order (strided per thread, then a fixed tree); the result is valid in thread 0.
__device__ void sum_partials(const double* part, int n, double& a, double& b) {
  __shared__ double ra[256], rb[256];
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    x += part[2 * i];
    y += part[2 * i + 1];
  }
  ra[threadIdx.x] = x;
  rb[threadIdx.x] = y;
  __syncthreads();
  for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
    if ((int)threadIdx.x < s2) {
      ra[threadIdx.x] += ra[threadIdx.x + s2];
      rb[threadIdx.x] += rb[threadIdx.x + s2];
    }
    __syncthreads();
  }
  a = ra[0];
  b = rb[0];
}

struct ChunkRange {
  int e0, nE, p0, nP, s0, nS;
};
__device__ __forceinline__ ChunkRange chunk_range(const DevBA& d, int k) {
  ChunkRange c;
  c.e0 = d.ch_e0[k];
  c.nE = d.ch_e0[k + 1] - c.e0;
  c.p0 = d.ch_p0[k];
  c.nP = d.ch_p0[k + 1] - c.p0;
  c.s0 = d.ch_s0[k];
  c.nS = d.ch_s0[k + 1] - c.s0;
  return c;
}

// ---------------------------------------------------------------- problem binding

// Copies problem q's descriptor into shared memory (all threads cooperate).
__device__ __forceinline__ void bind_problem(DevBA& dst, const DevBA* src) {
  static_assert(sizeof(DevBA) % 4 == 0, "DevBA must be a whole number of words");
  const int* s4 = reinterpret_cast<const int*>(src);
  int* d4 = reinterpret_cast<int*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(DevBA) / 4); i += blockDim.x) d4[i] = s4[i];
  __syncthreads();
}

// Programmatic dependent launch: every kernel lets the next one in the stream start
// its prologue early (launch_dependents) and waits for its predecessor to complete
// before touching anything the predecessor writes (wait).  The problem descriptor and
// the schedule tables are written by the host before the launches.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

#define GPO_BIND(KIND, LOCAL)                              \
  __shared__ DevBA d;                                      \
  pdl_trigger();                                           \
  const int prob_ = ls.KIND##_prob[blockIdx.x];            \
  const int LOCAL = blockIdx.x - ls.KIND##_base[prob_];    \
  bind_problem(d, ls.probs + prob_);                       \
  pdl_wait();

// ---------------------------------------------------------------- camera render blocks

__global__ void __launch_bounds__(kCamPerBlock * 32) k_cam_prepare(LaunchSet ls, int candidate) {
  GPO_BIND(cb, cbl)
  if (!d.sc->active) return;
  const int c = cbl * kCamPerBlock + (threadIdx.x >> 5);
  if (c >= d.C || (threadIdx.x & 31) != 0) return;
  const double* cam = (candidate ? d.cam_cand : d.cam) + 9 * (size_t)c;
  double* rb = (candidate ? d.camrb_cand : d.camrb) + 16 * (size_t)c;
  double R[9];
  aa_to_R(cam, R);
  for (int i = 0; i < 9; ++i) rb[i] = R[i];
  for (int i = 0; i < 6; ++i) rb[9 + i] = cam[3 + i];
  rb[15] = 0.0;
}

// ---------------------------------------------------------------- cost F(x)

__global__ void __launch_bounds__(kThreads) k_cost(LaunchSet ls, int candidate) {
  __shared__ double red[kThreads];
  GPO_BIND(ch, kl)
  if (!d.sc->active) return;
  const ChunkRange cr = chunk_range(d, kl);
  const double* rbs = candidate ? d.camrb_cand : d.camrb;
  const double* pts = candidate ? d.pt_cand : d.pt;
  double acc = 0.0;
  for (int i = threadIdx.x; i < cr.nE; i += kThreads) {
    const int e = cr.e0 + i;
    double rb[16];
    load_rb(rbs + 16 * (size_t)__ldg(d.e_cam + e), rb);
    const double* Xp = pts + 3 * (size_t)__ldg(d.e_pt + e);
    const double X[3] = {Xp[0], Xp[1], Xp[2]};
    Geom g;
    ba_geom(rb, X, g);
    Robust o;
    ba_residual(d, e, g, o);
    acc += 0.5 * o.rho;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.cost_part[kl] = s;
}

__global__ void k_cost_init(LaunchSet ls) {
  __shared__ double red[kThreads];
  __shared__ DevBA d;
  pdl_trigger();
  bind_problem(d, ls.probs + blockIdx.x);
  pdl_wait();
  if (!d.sc->active) return;
  double acc = 0.0;
  for (int k = threadIdx.x; k < d.NCH; k += kThreads) acc += d.cost_part[k];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.sc->cost = s;
}

// ---------------------------------------------------------------- linearisation

// One CTA per chunk.  Writes the chunk's Jacobian tile, the undamped point blocks
// H_pp = sum Jp^T Jp and gradients b_p, and per-slot camera partials
// (H_cc = sum Jc^T Jc, b_c = sum Jc^T r).  H uses the stored (rounded) Jacobian; the
// gradient uses the unrounded one, so BF16 storage leaves the LM fixed point intact.
template <class JT>
__global__ void __launch_bounds__(kThreads) k_linearize(LaunchSet ls, int force) {
  using AT = typename AccOf<JT>::T;
  constexpr bool kSplit = !std::is_same<JT, AT>::value;
  GPO_BIND(ch, kl)
  if (!d.sc->active || (!force && !d.sc->need_lin)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int CH = d.ch_max;
  JT* Js = reinterpret_cast<JT*>(smem);               // [24][CH]
  AT* rs = reinterpret_cast<AT*>(Js + kJComp * CH);   // [2][CH]
  AT* bce = rs + 2 * CH;                              // [9][CH]  (kSplit only)
  AT* bpe = bce + 9 * CH;                             // [3][CH]  (kSplit only)
  uint16_t* srt = reinterpret_cast<uint16_t*>(kSplit ? bpe + 3 * CH : bce);   // [CH]
  const ChunkRange cr = chunk_range(d, kl);
  JT* Jg = reinterpret_cast<JT*>(d.J) + (size_t)cr.e0 * kJComp;

  for (int i = threadIdx.x; i < cr.nE; i += kThreads) {
    const int e = cr.e0 + i;
    const int c = __ldg(d.e_cam + e), p = __ldg(d.e_pt + e);
    double rb[16];
    load_rb(d.camrb + 16 * (size_t)c, rb);
    const double X[3] = {d.pt[3 * (size_t)p], d.pt[3 * (size_t)p + 1], d.pt[3 * (size_t)p + 2]};
    Geom g;
    ba_geom(rb, X, g);
    Robust o;
    ba_residual(d, e, g, o);
    AT Jc[2][9], Jp[2][3];
    ba_jacobian<AT>(d, e, rb, g, o.sw, Jc, Jp);
    if (d.cam_fixed[c]) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Jc[0][k] = Jc[1][k] = (AT)0;
    }
    if (d.pt_fixed[p]) {
#pragma unroll
      for (int k = 0; k < 3; ++k) Jp[0][k] = Jp[1][k] = (AT)0;
    }
    const AT rw0 = (AT)(o.sw * o.r[0]), rw1 = (AT)(o.sw * o.r[1]);
    __align__(16) JT row[kJComp];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      row[k] = cvj(Jc[0][k], (const JT*)nullptr);
      row[9 + k] = cvj(Jc[1][k], (const JT*)nullptr);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      row[18 + k] = cvj(Jp[0][k], (const JT*)nullptr);
      row[21 + k] = cvj(Jp[1][k], (const JT*)nullptr);
    }
    store_row(Jg + (size_t)i * kJComp, row);
#pragma unroll
    for (int k = 0; k < kJComp; ++k) Js[k * CH + i] = row[k];
    srt[i] = d.ch_sorted[e];
    rs[i] = rw0;
    rs[CH + i] = rw1;
    if constexpr (kSplit) {
#pragma unroll
      for (int k = 0; k < 9; ++k) bce[k * CH + i] = Jc[0][k] * rw0 + Jc[1][k] * rw1;
#pragma unroll
      for (int k = 0; k < 3; ++k) bpe[k * CH + i] = Jp[0][k] * rw0 + Jp[1][k] * rw1;
    }
    if (d.dbg_r) {
      d.dbg_r[2 * (size_t)e] = o.sw * o.r[0];
      d.dbg_r[2 * (size_t)e + 1] = o.sw * o.r[1];
    }
  }
  __syncthreads();

  // point blocks
  AT* Hpp = reinterpret_cast<AT*>(d.Hpp);
  AT* bp = reinterpret_cast<AT*>(d.bp);
  for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
    const int pj = cr.p0 + j;
    const int a = d.pt_off[pj] - cr.e0, b = d.pt_off[pj + 1] - cr.e0;
    AT h[6] = {0, 0, 0, 0, 0, 0}, bb[3] = {0, 0, 0};
    for (int i = a; i < b; ++i) {
      AT J0[3], J1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        J0[k] = ldj(Js + (18 + k) * CH + i);
        J1[k] = ldj(Js + (21 + k) * CH + i);
      }
      h[0] += J0[0] * J0[0] + J1[0] * J1[0];
      h[1] += J0[0] * J0[1] + J1[0] * J1[1];
      h[2] += J0[0] * J0[2] + J1[0] * J1[2];
      h[3] += J0[1] * J0[1] + J1[1] * J1[1];
      h[4] += J0[1] * J0[2] + J1[1] * J1[2];
      h[5] += J0[2] * J0[2] + J1[2] * J1[2];
      if constexpr (kSplit) {
#pragma unroll
        for (int k = 0; k < 3; ++k) bb[k] += bpe[k * CH + i];
      } else {
        const AT r0 = rs[i], r1 = rs[CH + i];
#pragma unroll
        for (int k = 0; k < 3; ++k) bb[k] += J0[k] * r0 + J1[k] * r1;
      }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) Hpp[6 * (size_t)pj + k] = h[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) bp[3 * (size_t)pj + k] = bb[k];
  }

  // camera slots: 6 groups of 9 outputs (5 groups of H_cc entries, 1 of b_c)
  AT* partA = reinterpret_cast<AT*>(d.partA);
  for (int w = threadIdx.x; w < cr.nS * 6; w += kThreads) {
    const int sl = w / 6, grp = w - sl * 6;
    const int a = d.slot_e0[cr.s0 + sl], b = d.slot_e0[cr.s0 + sl + 1];
    AT acc[9];
#pragma unroll
    for (int o = 0; o < 9; ++o) acc[o] = (AT)0;
    for (int q = a; q < b; ++q) {
      const int i = srt[q - cr.e0];
      if (grp < 5) {
#pragma unroll
        for (int o = 0; o < 9; ++o) {
          const int ti = c_ti[9 * grp + o], tj = c_tj[9 * grp + o];
          acc[o] += ldj(Js + ti * CH + i) * ldj(Js + tj * CH + i) +
                    ldj(Js + (9 + ti) * CH + i) * ldj(Js + (9 + tj) * CH + i);
        }
      } else {
        if constexpr (kSplit) {
#pragma unroll
          for (int o = 0; o < 9; ++o) acc[o] += bce[o * CH + i];
        } else {
          const AT r0 = rs[i], r1 = rs[CH + i];
#pragma unroll
          for (int o = 0; o < 9; ++o)
            acc[o] += ldj(Js + o * CH + i) * r0 + ldj(Js + (9 + o) * CH + i) * r1;
        }
      }
    }
    AT* out = partA + (size_t)d.slot_pos[cr.s0 + sl] * kPartA + 9 * grp;
#pragma unroll
    for (int o = 0; o < 9; ++o) out[o] = acc[o];
  }
}

// ---------------------------------------------------------------- Schur preparation

// 3x3 SPD inverse by cofactors; h = (a b c d e f) packed upper triangle.
template <class AT>
__device__ __forceinline__ void inv3(const AT* h, AT* o) {
  const AT a = h[0], b = h[1], c = h[2], dd = h[3], e = h[4], f = h[5];
  const AT A = dd * f - e * e, B = c * e - b * f, C = b * e - c * dd;
  const AT D = a * f - c * c, E = b * c - a * e, F = a * dd - b * b;
  const AT det = a * A + b * B + c * C;
  if (det > (AT)0 && isfinite(det)) {
    const AT id = (AT)1 / det;
    o[0] = A * id; o[1] = B * id; o[2] = C * id; o[3] = D * id; o[4] = E * id; o[5] = F * id;
  } else {  // not positive definite in this precision: Jacobi fallback
    o[0] = a > (AT)0 ? (AT)1 / a : (AT)0;
    o[3] = dd > (AT)0 ? (AT)1 / dd : (AT)0;
    o[5] = f > (AT)0 ? (AT)1 / f : (AT)0;
    o[1] = o[2] = o[4] = (AT)0;
  }
}

template <class AT>
__device__ __forceinline__ void mul3(const AT* h, const AT* v, AT* o) {
  o[0] = h[0] * v[0] + h[1] * v[1] + h[2] * v[2];
  o[1] = h[1] * v[0] + h[3] * v[1] + h[4] * v[2];
  o[2] = h[2] * v[0] + h[4] * v[1] + h[5] * v[2];
}

template <class AT>
__device__ __forceinline__ AT damp_diag(AT h, const Scalars* sc) {
  if (sc->damping_mode == 1) return (AT)1;
  return fmin(fmax(h, (AT)sc->diag_min), (AT)sc->diag_max);
}

// One CTA per chunk: damped point inverses H_pp^-1 and per-slot partials of
// sum_e W_e H_pp^-1 W_e^T (= Jc^T (Jp Hinv Jp^T) Jc) and sum_e W_e H_pp^-1 b_p.
template <class JT>
__global__ void __launch_bounds__(kThreads) k_schur_prepare(LaunchSet ls) {
  using AT = typename AccOf<JT>::T;
  GPO_BIND(ch, kl)
  if (!d.sc->active) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int CH = d.ch_max;
  JT* Jcs = reinterpret_cast<JT*>(smem);              // [18][CH]
  AT* Ae = reinterpret_cast<AT*>(Jcs + 18 * CH);      // [3][CH]
  AT* qe = Ae + 3 * CH;                               // [2][CH]
  uint16_t* srt = reinterpret_cast<uint16_t*>(qe + 2 * CH);   // [CH]
  const ChunkRange cr = chunk_range(d, kl);
  const JT* Jg = reinterpret_cast<const JT*>(d.J) + (size_t)cr.e0 * kJComp;
  const Scalars* sc = d.sc;
  const AT lam = (AT)sc->lambda;
  const AT* Hpp = reinterpret_cast<const AT*>(d.Hpp);
  const AT* bp = reinterpret_cast<const AT*>(d.bp);
  AT* Hinv = reinterpret_cast<AT*>(d.Hinv);

  for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
    const int pj = cr.p0 + j;
    AT h[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = Hpp[6 * (size_t)pj + k];
    h[0] += lam * damp_diag(h[0], sc);
    h[3] += lam * damp_diag(h[3], sc);
    h[5] += lam * damp_diag(h[5], sc);
    AT o[6];
    inv3(h, o);
#pragma unroll
    for (int k = 0; k < 6; ++k) Hinv[6 * (size_t)pj + k] = o[k];
  }
  __syncthreads();

  for (int i = threadIdx.x; i < cr.nE; i += kThreads) {
    const int pj = __ldg(d.e_pt + cr.e0 + i);
    AT hi[6], bb[3], hb[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) hi[k] = Hinv[6 * (size_t)pj + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) bb[k] = bp[3 * (size_t)pj + k];
    mul3(hi, bb, hb);
    AT row[kJComp];
    load_row(Jg + (size_t)i * kJComp, row);
    AT J0[3], J1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      J0[k] = row[18 + k];
      J1[k] = row[21 + k];
    }
#pragma unroll
    for (int k = 0; k < 18; ++k) Jcs[k * CH + i] = cvj(row[k], (const JT*)nullptr);
    srt[i] = d.ch_sorted[cr.e0 + i];
    AT t0[3], t1[3];
    mul3(hi, J0, t0);
    mul3(hi, J1, t1);
    Ae[i] = J0[0] * t0[0] + J0[1] * t0[1] + J0[2] * t0[2];
    Ae[CH + i] = J0[0] * t1[0] + J0[1] * t1[1] + J0[2] * t1[2];
    Ae[2 * CH + i] = J1[0] * t1[0] + J1[1] * t1[1] + J1[2] * t1[2];
    qe[i] = J0[0] * hb[0] + J0[1] * hb[1] + J0[2] * hb[2];
    qe[CH + i] = J1[0] * hb[0] + J1[1] * hb[1] + J1[2] * hb[2];
  }
  __syncthreads();

  AT* partB = reinterpret_cast<AT*>(d.partB);
  for (int w = threadIdx.x; w < cr.nS * 6; w += kThreads) {
    const int sl = w / 6, grp = w - sl * 6;
    const int a = d.slot_e0[cr.s0 + sl], b = d.slot_e0[cr.s0 + sl + 1];
    AT acc[9];
#pragma unroll
    for (int o = 0; o < 9; ++o) acc[o] = (AT)0;
    for (int q = a; q < b; ++q) {
      const int i = srt[q - cr.e0];
      if (grp < 5) {
        const AT a00 = Ae[i], a01 = Ae[CH + i], a11 = Ae[2 * CH + i];
#pragma unroll
        for (int o = 0; o < 9; ++o) {
          const int ti = c_ti[9 * grp + o], tj = c_tj[9 * grp + o];
          const AT c0i = ldj(Jcs + ti * CH + i), c1i = ldj(Jcs + (9 + ti) * CH + i);
          const AT c0j = ldj(Jcs + tj * CH + i), c1j = ldj(Jcs + (9 + tj) * CH + i);
          acc[o] += c0i * (a00 * c0j + a01 * c1j) + c1i * (a01 * c0j + a11 * c1j);
        }
      } else {
        const AT q0 = qe[i], q1 = qe[CH + i];
#pragma unroll
        for (int o = 0; o < 9; ++o)
          acc[o] += ldj(Jcs + o * CH + i) * q0 + ldj(Jcs + (9 + o) * CH + i) * q1;
      }
    }
    AT* out = partB + (size_t)d.slot_pos[cr.s0 + sl] * kPartA + 9 * grp;
#pragma unroll
    for (int o = 0; o < 9; ++o) out[o] = acc[o];
  }
}

// ---------------------------------------------------------------- camera blocks + PCG start

// 9x9 SPD inverse via Cholesky: S (packed upper) -> M = S^-1 (packed upper).
// If S is not positive definite in this precision, M = diag(1 / S_ii) (Jacobi).
template <class AT>
__device__ void spd_inverse9(const AT* S, AT* M) {
  AT L[9][9];
  bool ok = true;
  for (int j = 0; j < 9 && ok; ++j) {
    AT s = S[tri9(j, j)];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > (AT)0)) { ok = false; break; }
    const AT ljj = sqrt(s);
    L[j][j] = ljj;
    for (int i = j + 1; i < 9; ++i) {
      AT t = S[tri9(j, i)];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / ljj;
    }
  }
  if (!ok) {
    for (int t = 0; t < kCamTri; ++t) M[t] = (AT)0;
    for (int i = 0; i < 9; ++i) {
      const AT v = S[tri9(i, i)];
      M[tri9(i, i)] = v > (AT)0 ? (AT)1 / v : (AT)1;
    }
    return;
  }
  // W = L^-1 (lower triangular)
  AT W[9][9];
  for (int i = 0; i < 9; ++i) {
    W[i][i] = (AT)1 / L[i][i];
    for (int j = 0; j < i; ++j) {
      AT s = (AT)0;
      for (int k = j; k < i; ++k) s += L[i][k] * W[k][j];
      W[i][j] = -s / L[i][i];
    }
  }
  // M = W^T W
  for (int i = 0; i < 9; ++i)
    for (int j = i; j < 9; ++j) {
      AT s = (AT)0;
      for (int k = j; k < 9; ++k) s += W[k][i] * W[k][j];
      M[tri9(i, j)] = s;
    }
}

// One warp per camera: reduces the slot partials into H_cc, b_c and the Schur
// terms, forms H_cc + lambda D_c, S_cc, g_c and M_c = S_cc^-1, and starts the PCG
// (x = 0, r = g, z = M g, p = z).  The last CTA reduces r^T z and |r|^2.
template <class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_cam_finalize(LaunchSet ls) {
  __shared__ AT vals[kCamPerBlock][2 * kPartA];
  __shared__ double red[kCamPerBlock][2];
  GPO_BIND(cb, cbl)
  if (!d.sc->active) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = cbl * kCamPerBlock + warp;
  Scalars* sc = d.sc;
  const AT lam = (AT)sc->lambda;
  const AT* partA = reinterpret_cast<const AT*>(d.partA);
  const AT* partB = reinterpret_cast<const AT*>(d.partB);
  double rz_c = 0.0, rr_c = 0.0;
  if (c < d.C) {
    const int sa = d.cam_s_off[c], sb = d.cam_s_off[c + 1];
    // 12 groups of 9 outputs; lanes stride over the camera's slots, then a fixed
    // shuffle tree sums the lanes
    for (int grp = 0; grp < 12; ++grp) {
      const AT* base = (grp < 6 ? partA : partB) + 9 * (grp % 6);
      AT acc[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[k] = (AT)0;
      for (int s = sa + lane; s < sb; s += 32) {
        const AT* src = base + (size_t)s * kPartA;   // camera-major rows
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] += src[k];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k) vals[warp][9 * grp + k] = acc[k];
      }
    }
    __syncwarp();
    AT* Hcl = reinterpret_cast<AT*>(d.Hcl) + (size_t)c * kCamTri;
    AT* S = reinterpret_cast<AT*>(d.S) + (size_t)c * kCamTri;
    AT* M = reinterpret_cast<AT*>(d.Minv) + (size_t)c * kCamTri;
    if (lane == 0) {
      AT Sl[kCamTri], Ml[kCamTri];
      for (int t = 0; t < kCamTri; ++t) Sl[t] = vals[warp][t];
      for (int i = 0; i < 9; ++i) Sl[tri9(i, i)] += lam * damp_diag(vals[warp][tri9(i, i)], sc);
      for (int t = 0; t < kCamTri; ++t) {
        Hcl[t] = Sl[t];
        Sl[t] -= vals[warp][kPartA + t];
        S[t] = Sl[t];
      }
      spd_inverse9(Sl, Ml);
      for (int t = 0; t < kCamTri; ++t) M[t] = Ml[t];
    }
    __syncwarp();
    AT* g = reinterpret_cast<AT*>(d.g) + 9 * (size_t)c;
    AT* bc = reinterpret_cast<AT*>(d.bc) + 9 * (size_t)c;
    if (lane < 9) {
      const AT gi = -vals[warp][45 + lane] + vals[warp][kPartA + 45 + lane];
      g[lane] = gi;
      bc[lane] = vals[warp][45 + lane];
      reinterpret_cast<AT*>(d.x)[9 * (size_t)c + lane] = (AT)0;
      reinterpret_cast<AT*>(d.xbest)[9 * (size_t)c + lane] = (AT)0;
      reinterpret_cast<AT*>(d.r)[9 * (size_t)c + lane] = gi;
    }
    __syncwarp();
    if (lane < 9) {
      AT zi = (AT)0;
      for (int j = 0; j < 9; ++j) zi += M[sym9(lane, j)] * g[j];
      reinterpret_cast<AT*>(d.z)[9 * (size_t)c + lane] = zi;
      reinterpret_cast<AT*>(d.p)[9 * (size_t)c + lane] = (AT)0;   // p_{-1}: p_0 = z_0
      const AT gi = g[lane];
      rz_c = (double)gi * (double)zi;
      rr_c = (double)gi * (double)gi;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rz_c += __shfl_down_sync(0xffffffffu, rz_c, o);
    rr_c += __shfl_down_sync(0xffffffffu, rr_c, o);
  }
  if (lane == 0) {
    red[warp][0] = rz_c;
    red[warp][1] = rr_c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kCamPerBlock; ++w) { a += red[w][0]; b += red[w][1]; }
    d.cblk_part[2 * cbl] = a;
    d.cblk_part[2 * cbl + 1] = b;
  }
  if (!last_cta(&sc->ticket, d.ncblk)) return;
  double rz, rr;
  sum_partials(d.cblk_part, d.ncblk, rz, rr);
  if (threadIdx.x == 0) {
    const double gn = sqrt(rr);
    sc->rz = rz;
    sc->gnorm = gn;
    sc->rnorm = gn;
    sc->rmin = gn;
    sc->sigma = 1.0;
    sc->inv_n = 1.0;
    sc->beta = 0.0;
    sc->pidx = 0;
    sc->pcg_it = 0;
    sc->use_best = 0;
    sc->save_best = 0;
    sc->tol_abs = sc->pcg_rel ? sc->pcg_tol * gn : sc->pcg_tol;
    sc->pcg_done = (rr == 0.0 || !(rz > 0.0) || !isfinite(rz)) ? 1 : 0;
    if (!sc->pcg_done) atomicAdd(ls.running, 1);
    sc->ticket = 0u;
  }
}

// ---------------------------------------------------------------- PCG

// Matrix-free Schur product, one CTA per chunk (the hot loop).  With t_p =
// H_pp^-1 sum_e Jp_e^T Jc_e x_c(e), each edge contributes v_e = Jc_e^T Jp_e t_p(e) to
// its camera.  The CTA first issues every load it needs at once (its edges'
// Jacobian rows, kept in registers when they fit; the camera vector of each slot,
// staged once per slot instead of once per edge; point offsets, point inverses and
// slot ranges), then runs three barrier-separated passes in shared memory: point
// sums, per-edge camera terms scattered to slot-sorted positions, and contiguous
// per-slot sums.  Each chunk's Jacobian bytes are read from HBM once.
template <class JT, int EPT>
__global__ void __launch_bounds__(kThreads) k_spmv(LaunchSet ls) {
  using AT = typename AccOf<JT>::T;
  constexpr int RV = (int)(sizeof(JT) * kJComp / 16);          // 16-byte vectors per row
  constexpr bool kKeep = false;                                 // re-read rows (L1/L2) in pass 3
  GPO_BIND(ch, kl)
  if (!d.sc->active || d.sc->pcg_done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int CH = d.ch_max, LD = CH + 1;
  AT* vv = reinterpret_cast<AT*>(smem);        // [9][LD]; [0..2] hold a_e in pass 1
  AT* tp = vv + 9 * LD;                        // [3][LD] point solutions
  AT* xs = tp + 3 * LD;                        // [ls.ns_max][9] slot camera vectors
  AT* hv = xs + 9 * ls.ns_max;                 // [ls.np_max][6] point inverses
  int* po = reinterpret_cast<int*>(hv + 6 * ls.np_max);   // [np + 1] local point offsets
  int* so = po + ls.np_max + 1;                           // [ns + 1] local slot offsets
  int* sp = so + ls.ns_max + 1;                           // [ns] camera-major slot rows
  const ChunkRange cr = chunk_range(d, kl);
  const JT* Jg = reinterpret_cast<const JT*>(d.J) + (size_t)cr.e0 * kJComp;

  // ---- prefetch
  uint4 raw[kKeep ? EPT : 1][kKeep ? RV : 1];
  int pos[EPT], slot[EPT], ptl[EPT];
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const int i = threadIdx.x + m * kThreads;
    if (i < cr.nE) {
      if constexpr (kKeep) {
        const uint4* src = reinterpret_cast<const uint4*>(Jg + (size_t)i * kJComp);
#pragma unroll
        for (int v = 0; v < RV; ++v) raw[m][v] = __ldg(src + v);
      }
      pos[m] = __ldg(d.e_pos + cr.e0 + i);
      slot[m] = __ldg(d.e_slot + cr.e0 + i);
      ptl[m] = __ldg(d.e_pt + cr.e0 + i) - cr.p0;
    }
  }
  // the search direction p_k = (z_k + beta_k p_{k-1}) / n_k, formed per slot camera
  const AT* zv = reinterpret_cast<const AT*>(d.z);
  const AT* pold = reinterpret_cast<const AT*>(d.sc->pidx ? d.p2 : d.p);
  const AT beta = (AT)d.sc->beta, inv_n = (AT)d.sc->inv_n;
  for (int w = threadIdx.x; w < cr.nS * 9; w += kThreads) {
    const int sl = w / 9, k = w - sl * 9;
    const size_t o = 9 * (size_t)__ldg(d.slot_cam + cr.s0 + sl) + k;
    xs[w] = (zv[o] + beta * pold[o]) * inv_n;
  }
  for (int t = threadIdx.x; t < cr.nS; t += kThreads) sp[t] = __ldg(d.slot_pos + cr.s0 + t);
  const AT* Hinv = reinterpret_cast<const AT*>(d.Hinv) + 6 * (size_t)cr.p0;
  for (int w = threadIdx.x; w < cr.nP * 6; w += kThreads) hv[w] = Hinv[w];
  for (int j = threadIdx.x; j <= cr.nP; j += kThreads) po[j] = __ldg(d.pt_off + cr.p0 + j) - cr.e0;
  for (int t = threadIdx.x; t <= cr.nS; t += kThreads) so[t] = __ldg(d.slot_e0 + cr.s0 + t) - cr.e0;
  __syncthreads();

  // ---- pass 1: a_e = Jp^T (Jc x_c)
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const int i = threadIdx.x + m * kThreads;
    if (i >= cr.nE) break;
    AT row[kJComp];
    if constexpr (kKeep) load_row(reinterpret_cast<const JT*>(raw[m]), row);
    else load_row(Jg + (size_t)i * kJComp, row);
    const AT* xc = xs + 9 * slot[m];
    AT q0 = (AT)0, q1 = (AT)0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      q0 += row[k] * xc[k];
      q1 += row[9 + k] * xc[k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) vv[k * LD + i] = row[18 + k] * q0 + row[21 + k] * q1;
  }
  __syncthreads();
  // ---- pass 2: t_p = H_pp^-1 sum_e a_e
  for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
    AT u[3] = {0, 0, 0};
    for (int i = po[j]; i < po[j + 1]; ++i) {
#pragma unroll
      for (int k = 0; k < 3; ++k) u[k] += vv[k * LD + i];
    }
    AT t[3];
    mul3(hv + 6 * j, u, t);
#pragma unroll
    for (int k = 0; k < 3; ++k) tp[k * LD + j] = t[k];
  }
  __syncthreads();
  // ---- pass 3: v_e = Jc^T (Jp t_p), scattered to the edge's slot-sorted position
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const int i = threadIdx.x + m * kThreads;
    if (i >= cr.nE) break;
    AT row[kJComp];
    if constexpr (kKeep) load_row(reinterpret_cast<const JT*>(raw[m]), row);
    else load_row(Jg + (size_t)i * kJComp, row);
    const int pl = ptl[m];
    const AT t0 = tp[pl], t1 = tp[LD + pl], t2 = tp[2 * LD + pl];
    const AT s0 = row[18] * t0 + row[19] * t1 + row[20] * t2;
    const AT s1 = row[21] * t0 + row[22] * t1 + row[23] * t2;
#pragma unroll
    for (int k = 0; k < 9; ++k) vv[k * LD + pos[m]] = row[k] * s0 + row[9 + k] * s1;
  }
  __syncthreads();
  // ---- pass 4: per-slot sums over contiguous positions
  AT* partV = reinterpret_cast<AT*>(d.partV);
  for (int w = threadIdx.x; w < cr.nS * 9; w += kThreads) {
    const int sl = w / 9, comp = w - sl * 9;
    const AT* src = vv + comp * LD;
    AT acc = (AT)0;
    for (int q = so[sl]; q < so[sl + 1]; ++q) acc += src[q];
    partV[(size_t)sp[sl] * 9 + comp] = acc;
  }
}

// y_c = (H_cc + lambda D_c) p_c - sum_slots v, four warps per camera (each sums a
// quarter of the camera's slot partials; the quarters are added in a fixed order).
// The CTAs of camera block b are 4b .. 4b + 3, two cameras each.  The last CTA of
// the problem reduces p^T y and sets alpha = r^T z / p^T y.
constexpr int kApplySplit = 4;
template <class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_cam_apply(LaunchSet ls) {
  __shared__ double red[kCamPerBlock];
  __shared__ AT quarter[kCamPerBlock][9];
  __shared__ DevBA d;
  pdl_trigger();
  const int cb = blockIdx.x / kApplySplit, part = blockIdx.x % kApplySplit;
  const int prob_ = ls.cb_prob[cb];
  const int cbl = cb - ls.cb_base[prob_];
  bind_problem(d, ls.probs + prob_);
  pdl_wait();
  Scalars* sc = d.sc;
  if (!sc->active || sc->pcg_done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cams_per_cta = kCamPerBlock / kApplySplit;             // 2
  const int c = cbl * kCamPerBlock + part * cams_per_cta + warp / kApplySplit;
  const int q = warp % kApplySplit;                                // quarter of the slots
  double dot = 0.0;
  AT pi = (AT)0;
  if (c < d.C) {   // warp-uniform
    const AT* partV = reinterpret_cast<const AT*>(d.partV);
    const int sa = d.cam_s_off[c], sb = d.cam_s_off[c + 1];
    AT acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = (AT)0;
#pragma unroll 4
    for (int s = sa + q * 32 + lane; s < sb; s += 32 * kApplySplit) {
      const AT* src = partV + (size_t)s * 9;   // camera-major rows
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[k] += src[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) quarter[warp][k] = acc[k];
    }
  }
  __syncthreads();
  if (c < d.C && q == 0) {
    AT sv = (AT)0;
    if (lane < 9) {
      sv = quarter[warp][lane];
      for (int j = 1; j < kApplySplit; ++j) sv += quarter[warp + j][lane];
    }
    // p_k = (z_k + beta_k p_{k-1}) / n_k for this camera (the same values the Schur
    // product gathered), written to the other direction buffer
    const AT* pold = reinterpret_cast<const AT*>(sc->pidx ? d.p2 : d.p) + 9 * (size_t)c;
    AT* pnew = reinterpret_cast<AT*>(sc->pidx ? d.p : d.p2) + 9 * (size_t)c;
    const AT* zc = reinterpret_cast<const AT*>(d.z) + 9 * (size_t)c;
    pi = lane < 9 ? (zc[lane] + (AT)sc->beta * pold[lane]) * (AT)sc->inv_n : (AT)0;
    if (lane < 9) {
      pnew[lane] = pi;
      if (sc->save_best)
        reinterpret_cast<AT*>(d.xbest)[9 * (size_t)c + lane] = reinterpret_cast<const AT*>(d.x)[9 * (size_t)c + lane];
    }
    const AT* H = reinterpret_cast<const AT*>(d.Hcl) + (size_t)c * kCamTri;
    AT yi = (AT)0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const AT pj = __shfl_sync(0xffffffffu, pi, j);
      if (lane < 9) yi += H[sym9(lane, j)] * pj;
    }
    if (lane < 9) {
      yi -= sv;
      reinterpret_cast<AT*>(d.y)[9 * (size_t)c + lane] = yi;
      dot = (double)pi * (double)yi;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
  if (lane == 0) red[warp] = dot;
  __syncthreads();
  const int ctas = d.ncblk * kApplySplit, me = cbl * kApplySplit + part;
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < kCamPerBlock; ++w) a += red[w];
    d.cblk_part[2 * me] = a;
    d.cblk_part[2 * me + 1] = 0.0;
  }
  if (!last_cta(&sc->ticket, ctas)) return;
  double pAp, unused;
  sum_partials(d.cblk_part, ctas, pAp, unused);
  if (threadIdx.x == 0) {
    sc->pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) {
      sc->alpha = 0.0;
      sc->pcg_done = 1;
      atomicSub(ls.running, 1);
    } else {
      sc->alpha = sc->rz / pAp;
    }
    sc->ticket = 0u;
  }
}

// One warp per camera: x += sigma alpha p, r -= alpha y, z = M r; the last CTA of
// the problem reduces r^T z and |r|^2, applies the stopping rules (tolerance,
// rejection ratio, iteration cap) and computes beta and the normalisation factor.
template <class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_pcg_update(LaunchSet ls) {
  __shared__ double red[kCamPerBlock][2];
  GPO_BIND(cb, cbl)
  Scalars* sc = d.sc;
  if (!sc->active || sc->pcg_done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = cbl * kCamPerBlock + warp;
  double rz_c = 0.0, rr_c = 0.0;
  if (c < d.C) {   // warp-uniform
    const AT alpha = (AT)sc->alpha, sa = (AT)(sc->sigma * sc->alpha), sn = (AT)sc->inv_n;
    AT* x = reinterpret_cast<AT*>(d.x) + 9 * (size_t)c;
    AT* r = reinterpret_cast<AT*>(d.r) + 9 * (size_t)c;
    AT* z = reinterpret_cast<AT*>(d.z) + 9 * (size_t)c;
    const AT* pv = reinterpret_cast<const AT*>(sc->pidx ? d.p : d.p2) + 9 * (size_t)c;
    const AT* yv = reinterpret_cast<const AT*>(d.y) + 9 * (size_t)c;
    const AT* M = reinterpret_cast<const AT*>(d.Minv) + (size_t)c * kCamTri;
    AT ri = (AT)0;
    if (lane < 9) {
      x[lane] += sa * pv[lane];
      ri = r[lane] * sn - alpha * yv[lane];
      r[lane] = ri;
    }
    AT zi = (AT)0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const AT rj = __shfl_sync(0xffffffffu, ri, j);
      if (lane < 9) zi += M[sym9(lane, j)] * rj;
    }
    if (lane < 9) {
      z[lane] = zi;
      rz_c = (double)ri * (double)zi;
      rr_c = (double)ri * (double)ri;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rz_c += __shfl_down_sync(0xffffffffu, rz_c, o);
    rr_c += __shfl_down_sync(0xffffffffu, rr_c, o);
  }
  if (lane == 0) {
    red[warp][0] = rz_c;
    red[warp][1] = rr_c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kCamPerBlock; ++w) { a += red[w][0]; b += red[w][1]; }
    d.cblk_part[2 * cbl] = a;
    d.cblk_part[2 * cbl + 1] = b;
  }
  if (!last_cta(&sc->ticket, d.ncblk)) return;
  double rz, rr;
  sum_partials(d.cblk_part, d.ncblk, rz, rr);
  if (threadIdx.x == 0) {
    const double n = sqrt(rr);
    const double rtrue = sc->sigma * n;
    sc->pcg_it += 1;
    sc->pcg_total += 1;
    sc->rnorm = rtrue;
    int done = 0;
    sc->save_best = 0;
    if (sc->ratio > 0.0) {
      if (rtrue < sc->rmin) {
        sc->rmin = rtrue;
        sc->save_best = 1;
      } else if (rtrue > sc->ratio * sc->rmin) {
        done = 1;
        sc->use_best = 1;
      }
    }
    if (rtrue <= sc->tol_abs || sc->pcg_it >= sc->max_it || !isfinite(rtrue) || !(rz > 0.0)) {
      done = 1;
      if (!isfinite(rtrue)) sc->use_best = 1;
    }
    sc->beta = rz / sc->rz;
    if (sc->normalize && n > 0.0) {
      sc->inv_n = 1.0 / n;
      sc->sigma *= n;
      sc->rz = rz / (n * n);
    } else {
      sc->inv_n = 1.0;
      sc->rz = rz;
    }
    sc->pidx ^= 1;
    sc->pcg_done = done;
    if (done) atomicSub(ls.running, 1);
    sc->ticket = 0u;
  }
}

// ---------------------------------------------------------------- back-substitution

// One CTA per chunk: dp = H_pp^-1 (-b_p - sum_e Jp^T Jc dc) and the chunk's share of
// the model decrease -b_p^T dp - 1/2 sum_e |Jc dc + Jp dp|^2 (FP64 accumulation).
template <class JT>
__global__ void __launch_bounds__(kThreads) k_backsub(LaunchSet ls) {
  using AT = typename AccOf<JT>::T;
  __shared__ double red[kThreads];
  GPO_BIND(ch, kl)
  if (!d.sc->active) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int CH = d.ch_max;
  AT* qv = reinterpret_cast<AT*>(smem);   // [2][CH]
  AT* av = qv + 2 * CH;                   // [3][CH]
  const ChunkRange cr = chunk_range(d, kl);
  const JT* Jg = reinterpret_cast<const JT*>(d.J) + (size_t)cr.e0 * kJComp;
  const AT* xs = reinterpret_cast<const AT*>(d.sc->use_best ? d.xbest : d.x);
  const AT* Hinv = reinterpret_cast<const AT*>(d.Hinv);
  const AT* bp = reinterpret_cast<const AT*>(d.bp);
  AT* dp = reinterpret_cast<AT*>(d.dp);
  for (int i = threadIdx.x; i < cr.nE; i += kThreads) {
    const int c = __ldg(d.e_cam + cr.e0 + i);
    AT row[kJComp];
    load_row(Jg + (size_t)i * kJComp, row);
    AT q0 = (AT)0, q1 = (AT)0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const AT xk = xs[9 * (size_t)c + k];
      q0 += row[k] * xk;
      q1 += row[9 + k] * xk;
    }
    qv[i] = q0;
    qv[CH + i] = q1;
#pragma unroll
    for (int k = 0; k < 3; ++k) av[k * CH + i] = row[18 + k] * q0 + row[21 + k] * q1;
  }
  __syncthreads();
  double md = 0.0;
  for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
    const int pj = cr.p0 + j;
    const int a = d.pt_off[pj] - cr.e0, b = d.pt_off[pj + 1] - cr.e0;
    AT u[3] = {0, 0, 0};
    for (int i = a; i < b; ++i) {
#pragma unroll
      for (int k = 0; k < 3; ++k) u[k] += av[k * CH + i];
    }
    AT hi[6], rhs[3], t[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) hi[k] = Hinv[6 * (size_t)pj + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) rhs[k] = -bp[3 * (size_t)pj + k] - u[k];
    mul3(hi, rhs, t);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dp[3 * (size_t)pj + k] = t[k];
      md -= (double)bp[3 * (size_t)pj + k] * (double)t[k];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cr.nE; i += kThreads) {
    const int pj = __ldg(d.e_pt + cr.e0 + i);
    const AT t0 = dp[3 * (size_t)pj], t1 = dp[3 * (size_t)pj + 1], t2 = dp[3 * (size_t)pj + 2];
    AT row[kJComp];
    load_row(Jg + (size_t)i * kJComp, row);
    const double j0 = (double)(qv[i] + row[18] * t0 + row[19] * t1 + row[20] * t2);
    const double j1 = (double)(qv[CH + i] + row[21] * t0 + row[22] * t1 + row[23] * t2);
    md -= 0.5 * (j0 * j0 + j1 * j1);
  }
  const double s = block_sum(md, red);
  if (threadIdx.x == 0) d.md_part[kl] = s;
}

// ---------------------------------------------------------------- retraction (FP64)

template <class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_retract_cams(LaunchSet ls) {
  GPO_BIND(cb, cbl)
  if (!d.sc->active) return;
  const int c = cbl * kCamPerBlock + (threadIdx.x >> 5);
  if (c >= d.C || (threadIdx.x & 31) != 0) return;
  const double* cur = d.cam + 9 * (size_t)c;
  double* nxt = d.cam_cand + 9 * (size_t)c;
  double* rb = d.camrb_cand + 16 * (size_t)c;
  if (d.cam_fixed[c]) {
    for (int i = 0; i < 9; ++i) nxt[i] = cur[i];
    for (int i = 0; i < 16; ++i) rb[i] = d.camrb[16 * (size_t)c + i];
    return;
  }
  const AT* xs = reinterpret_cast<const AT*>(d.sc->use_best ? d.xbest : d.x) + 9 * (size_t)c;
  double dl[9];
  for (int i = 0; i < 9; ++i) dl[i] = (double)xs[i];
  double w[3];
  aa_left_update(dl, cur, w);
  nxt[0] = w[0];
  nxt[1] = w[1];
  nxt[2] = w[2];
  for (int i = 3; i < 9; ++i) nxt[i] = cur[i] + dl[i];
  double R[9];
  aa_to_R(w, R);
  for (int i = 0; i < 9; ++i) rb[i] = R[i];
  for (int i = 0; i < 6; ++i) rb[9 + i] = nxt[3 + i];
  rb[15] = 0.0;
}

template <class AT>
__global__ void __launch_bounds__(256) k_retract_pts(LaunchSet ls) {
  GPO_BIND(pb, pbl)
  if (!d.sc->active) return;
  const int p = pbl * 256 + threadIdx.x;
  if (p >= d.P) return;
  const AT* dp = reinterpret_cast<const AT*>(d.dp) + 3 * (size_t)p;
  for (int i = 0; i < 3; ++i)
    d.pt_cand[3 * (size_t)p + i] = d.pt[3 * (size_t)p + i] + (d.pt_fixed[p] ? 0.0 : (double)dp[i]);
}

// ---------------------------------------------------------------- LM decision (FP64)

template <class AT>
__global__ void __launch_bounds__(kThreads) k_decide(LaunchSet ls) {
  __shared__ double red[kThreads];
  __shared__ DevBA d;
  pdl_trigger();
  bind_problem(d, ls.probs + blockIdx.x);
  pdl_wait();
  Scalars* sc = d.sc;
  if (!sc->active) return;
  double fc = 0.0, md = 0.0;
  for (int k = threadIdx.x; k < d.NCH; k += kThreads) {
    fc += d.cost_part[k];
    md += d.md_part[k];
  }
  const AT* xs = reinterpret_cast<const AT*>(sc->use_best ? d.xbest : d.x);
  const AT* bc = reinterpret_cast<const AT*>(d.bc);
  for (int i = threadIdx.x; i < 9 * d.C; i += kThreads) md -= (double)bc[i] * (double)xs[i];
  const double Fc = block_sum(fc, red);
  const double L = block_sum(md, red);
  if (threadIdx.x != 0) return;
  const double F = sc->cost;
  const bool acc = L > 0.0 && isfinite(Fc) && Fc < F;
  const double rho = L != 0.0 ? (F - Fc) / L : 0.0;
  const int it = sc->iter;
  if (it < kMaxHistory) {
    IterRecord& h = d.hist[it];
    h.cost = F;
    h.cand_cost = Fc;
    h.model_decrease = L;
    h.rho = rho;
    h.lambda = sc->lambda;
    h.pcg_residual = sc->gnorm > 0.0 ? sc->rnorm / sc->gnorm : 0.0;
    h.accepted = acc ? 1 : 0;
    h.pcg_iters = sc->pcg_it;
  }
  double lam = sc->lambda, nu = sc->nu;
  if (acc) {
    const double t = 2.0 * rho - 1.0;
    lam *= fmax(1.0 / 3.0, 1.0 - t * t * t);
    nu = 2.0;
    sc->cost = Fc;
    sc->n_accepted += 1;
  } else {
    lam *= nu;
    nu *= 2.0;
  }
  sc->lambda = fmin(fmax(lam, sc->lambda_min), sc->lambda_max);
  sc->nu = nu;
  sc->cand_cost = Fc;
  sc->model_dec = L;
  sc->rho = rho;
  sc->accepted = acc ? 1 : 0;
  sc->need_lin = acc ? 1 : 0;
  sc->iter = it + 1;
}

__global__ void __launch_bounds__(kCamPerBlock * 32) k_commit_cams(LaunchSet ls) {
  GPO_BIND(cb, cbl)
  if (!d.sc->active || !d.sc->accepted) return;
  const int lane = threadIdx.x & 31;
  const int c = cbl * kCamPerBlock + (threadIdx.x >> 5);
  if (c >= d.C) return;
  if (lane < 9) d.cam[9 * (size_t)c + lane] = d.cam_cand[9 * (size_t)c + lane];
  if (lane < 16) d.camrb[16 * (size_t)c + lane] = d.camrb_cand[16 * (size_t)c + lane];
}

__global__ void __launch_bounds__(256) k_commit_pts(LaunchSet ls) {
  GPO_BIND(pb, pbl)
  if (!d.sc->active || !d.sc->accepted) return;
  const int p = pbl * 256 + threadIdx.x;
  if (p >= d.P) return;
  for (int k = 0; k < 3; ++k) d.pt[3 * (size_t)p + k] = d.pt_cand[3 * (size_t)p + k];
}

// ---------------------------------------------------------------- launchers


int default_ch_max(Prec) { return 512; }

static size_t lin_smem(Prec pr, int ch) {
  const size_t sJ = pr == Prec::F64 ? 8 : (pr == Prec::F32 ? 4 : 2);
  const size_t sA = pr == Prec::F64 ? 8 : 4;
  const size_t per = kJComp * sJ + 2 * sA + (pr == Prec::BF16 ? 12 * sA : 0) + 2;
  return per * (size_t)ch;
}
static size_t schur_smem(Prec pr, int ch) {
  const size_t sJ = pr == Prec::F64 ? 8 : (pr == Prec::F32 ? 4 : 2);
  const size_t sA = pr == Prec::F64 ? 8 : 4;
  return (18 * sJ + 5 * sA + 2) * (size_t)ch;
}
static size_t spmv_smem(Prec pr, const LaunchSet& ls) {
  const size_t sA = pr == Prec::F64 ? 8 : 4;
  return sA * (12 * (size_t)(ls.ch_max + 1) + 9 * (size_t)ls.ns_max + 6 * (size_t)ls.np_max) +
         4 * (size_t)(ls.np_max + 2 * ls.ns_max + 2);
}
static size_t backsub_smem(Prec pr, int ch) {
  const size_t sA = pr == Prec::F64 ? 8 : 4;
  return 5 * sA * (size_t)ch;
}
size_t smem_bytes_linearize(Prec pr, int ch) { return lin_smem(pr, ch); }

int max_supported_ch(Prec pr) {
  // largest chunk whose linearisation tile fits the 227 KB opt-in shared memory
  const size_t limit = 227 * 1024;
  int ch = 64;
  while (lin_smem(pr, ch * 2) <= limit && schur_smem(pr, ch * 2) <= limit) ch *= 2;
  return ch;
}

// Launches with programmatic stream serialization, so the kernel may begin while
// its predecessor in the stream finishes (the kernels order themselves with
// griddepcontrol).
template <class... KArgs, class... Args>
static void launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Raises a kernel's dynamic shared-memory limit once per (kernel, size).
static void set_smem(const void* kernel, size_t bytes) {
  static const void* keys[32];
  static size_t vals[32];
  static int n = 0;
  for (int i = 0; i < n; ++i)
    if (keys[i] == kernel) {
      if (vals[i] >= bytes) return;
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      vals[i] = bytes;
      return;
    }
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (n < 32) { keys[n] = kernel; vals[n] = bytes; ++n; }
}

int launch_cam_prepare(const LaunchSet& ls, bool candidate, cudaStream_t st) {
  if (ls.n_cb == 0) return 0;
  launch_pdl(k_cam_prepare, ls.n_cb, kCamPerBlock * 32, 0, st, ls, candidate ? 1 : 0);
  return 1;
}

int launch_cost(const LaunchSet& ls, bool candidate, cudaStream_t st) {
  if (ls.n_ch == 0) return 0;
  launch_pdl(k_cost, ls.n_ch, kThreads, 0, st, ls, candidate ? 1 : 0);
  return 1;
}

int launch_cost_init(const LaunchSet& ls, cudaStream_t st) {
  launch_pdl(k_cost_init, ls.nprob, kThreads, 0, st, ls);
  return 1;
}

template <class JT>
static void lin_t(const LaunchSet& ls, Prec pr, bool force, cudaStream_t st) {
  const size_t sm = lin_smem(pr, ls.ch_max);
  set_smem(reinterpret_cast<const void*>(k_linearize<JT>), sm);
  launch_pdl(k_linearize<JT>, ls.n_ch, kThreads, sm, st, ls, force ? 1 : 0);
}
int launch_linearize(const LaunchSet& ls, Prec pr, bool force, cudaStream_t st) {
  if (ls.n_ch == 0) return 0;
  if (pr == Prec::F64) lin_t<double>(ls, pr, force, st);
  else if (pr == Prec::F32) lin_t<float>(ls, pr, force, st);
  else lin_t<__nv_bfloat16>(ls, pr, force, st);
  return 1;
}

template <class JT>
static void schur_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  const size_t sm = schur_smem(pr, ls.ch_max);
  set_smem(reinterpret_cast<const void*>(k_schur_prepare<JT>), sm);
  launch_pdl(k_schur_prepare<JT>, ls.n_ch, kThreads, sm, st, ls);
}
int launch_schur_prepare(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  if (ls.n_ch == 0) return 0;
  if (pr == Prec::F64) schur_t<double>(ls, pr, st);
  else if (pr == Prec::F32) schur_t<float>(ls, pr, st);
  else schur_t<__nv_bfloat16>(ls, pr, st);
  return 1;
}

int launch_cam_finalize(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  if (ls.n_cb == 0) return 0;
  if (pr == Prec::F64) launch_pdl(k_cam_finalize<double>, ls.n_cb, kCamPerBlock * 32, 0, st, ls);
  else launch_pdl(k_cam_finalize<float>, ls.n_cb, kCamPerBlock * 32, 0, st, ls);
  return 1;
}

template <class JT, int EPT>
static void spmv_e(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  const size_t sm = spmv_smem(pr, ls);
  set_smem(reinterpret_cast<const void*>(k_spmv<JT, EPT>), sm);
  launch_pdl(k_spmv<JT, EPT>, ls.n_ch, kThreads, sm, st, ls);
}
template <class JT>
static void spmv_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  const int ept = (ls.ch_max + kThreads - 1) / kThreads;
  if (ept <= 1) spmv_e<JT, 1>(ls, pr, st);
  else if (ept <= 2) spmv_e<JT, 2>(ls, pr, st);
  else if (ept <= 4) spmv_e<JT, 4>(ls, pr, st);
  else spmv_e<JT, 8>(ls, pr, st);
}
int launch_pcg_spmv(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  if (ls.n_ch == 0) return 0;
  if (pr == Prec::F64) spmv_t<double>(ls, pr, st);
  else if (pr == Prec::F32) spmv_t<float>(ls, pr, st);
  else spmv_t<__nv_bfloat16>(ls, pr, st);
  return 1;
}
int launch_cam_apply(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  if (ls.n_cb == 0) return 0;
  if (pr == Prec::F64) launch_pdl(k_cam_apply<double>, ls.n_cb * kApplySplit, kCamPerBlock * 32, 0, st, ls);
  else launch_pdl(k_cam_apply<float>, ls.n_cb * kApplySplit, kCamPerBlock * 32, 0, st, ls);
  return 1;
}
int launch_pcg_update(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  if (ls.n_cb == 0) return 0;
  if (pr == Prec::F64) launch_pdl(k_pcg_update<double>, ls.n_cb, kCamPerBlock * 32, 0, st, ls);
  else launch_pdl(k_pcg_update<float>, ls.n_cb, kCamPerBlock * 32, 0, st, ls);
  return 1;
}

template <class JT>
static void backsub_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  const size_t sm = backsub_smem(pr, ls.ch_max);
  set_smem(reinterpret_cast<const void*>(k_backsub<JT>), sm);
  launch_pdl(k_backsub<JT>, ls.n_ch, kThreads, sm, st, ls);
}
int launch_backsub(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  if (ls.n_ch == 0) return 0;
  if (pr == Prec::F64) backsub_t<double>(ls, pr, st);
  else if (pr == Prec::F32) backsub_t<float>(ls, pr, st);
  else backsub_t<__nv_bfloat16>(ls, pr, st);
  return 1;
}

int launch_retract(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  int n = 0;
  if (pr == Prec::F64) {
    if (ls.n_cb) { launch_pdl(k_retract_cams<double>, ls.n_cb, kCamPerBlock * 32, 0, st, ls); ++n; }
    if (ls.n_pb) { launch_pdl(k_retract_pts<double>, ls.n_pb, 256, 0, st, ls); ++n; }
  } else {
    if (ls.n_cb) { launch_pdl(k_retract_cams<float>, ls.n_cb, kCamPerBlock * 32, 0, st, ls); ++n; }
    if (ls.n_pb) { launch_pdl(k_retract_pts<float>, ls.n_pb, 256, 0, st, ls); ++n; }
  }
  return n;
}

int launch_decide(const LaunchSet& ls, Prec pr, cudaStream_t st) {
  if (pr == Prec::F64) launch_pdl(k_decide<double>, ls.nprob, kThreads, 0, st, ls);
  else launch_pdl(k_decide<float>, ls.nprob, kThreads, 0, st, ls);
  return 1;
}

int launch_commit(const LaunchSet& ls, cudaStream_t st) {
  int n = 0;
  if (ls.n_cb) { launch_pdl(k_commit_cams, ls.n_cb, kCamPerBlock * 32, 0, st, ls); ++n; }
  if (ls.n_pb) { launch_pdl(k_commit_pts, ls.n_pb, 256, 0, st, ls); ++n; }
  return n;
}

}  // namespace gpo
