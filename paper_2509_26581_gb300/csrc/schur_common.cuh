// Shared device helpers of the Schur-complement LM kernels: storage conversions,
// packed symmetric indexing, SO(3) / quaternion maths in FP64, deterministic
// reductions, problem binding for launch sets, and the two edge models:
//  * ModelBA: BAL reprojection (Sec. V; 2 residual rows, 9-dim camera);
//  * ModelStereo: stereo reprojection on a 15-dim navigation state (Sec. V-C; 3 rows,
//    the pose part (6) of the state carries the Jacobian).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "gpo_internal.h"

namespace gpo {

// ---------------------------------------------------------------- storage types

template <class JT> struct AccOf { using T = float; };
template <> struct AccOf<double> { using T = double; };

__device__ __forceinline__ float ldj(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ldj(const float* p) { return *p; }
__device__ __forceinline__ double ldj(const double* p) { return *p; }
__device__ __forceinline__ __nv_bfloat16 cvj(float v, const __nv_bfloat16*) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float cvj(float v, const float*) { return v; }
__device__ __forceinline__ double cvj(double v, const double*) { return v; }

// Edge-major Jacobian rows of NJ values (NJ a multiple of 8): the camera-side rows
// (M x DC), then the point rows (M x 3), then padding.  Rows are 16-byte aligned and
// moved with 16-byte vector accesses.
template <int NJ, class AT>
__device__ __forceinline__ void load_row(const __nv_bfloat16* src, AT (&v)[NJ]) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int i = 0; i < NJ / 8; ++i) {
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
template <int NJ, class AT>
__device__ __forceinline__ void load_row(const float* src, AT (&v)[NJ]) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < NJ / 4; ++i) {
    const float4 w = s4[i];
    v[4 * i] = (AT)w.x; v[4 * i + 1] = (AT)w.y; v[4 * i + 2] = (AT)w.z; v[4 * i + 3] = (AT)w.w;
  }
}
template <int NJ, class AT>
__device__ __forceinline__ void load_row(const double* src, AT (&v)[NJ]) {
  const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int i = 0; i < NJ / 2; ++i) {
    const double2 w = s2[i];
    v[2 * i] = (AT)w.x; v[2 * i + 1] = (AT)w.y;
  }
}
// Jacobian rows live in tiles of 32 consecutive edges.  Inside a tile the rows are cut
// into Q 16-byte pieces and piece q of the tile's rows is one contiguous 512-byte
// block ([tile][q][e mod 32]): a warp that reads the rows of 32 consecutive edges
// reads Q whole blocks, one per 16-byte vector access, instead of Q scattered 16-byte
// pieces per 48-byte row.  J is allocated in whole tiles.
template <class JT, int NJ>
struct JTiles {
  static constexpr int Q = NJ * (int)sizeof(JT) / 16;   // pieces per row
  static_assert(NJ * sizeof(JT) % 16 == 0, "rows are whole 16-byte pieces");
  // index (in 16-byte units) of piece q of row e
  __host__ __device__ static __forceinline__ size_t piece(size_t e, int q) {
    return ((e >> 5) * Q + q) * kJTile + (e & 31);
  }
};
template <int NJ, class JT, class AT>
__device__ __forceinline__ void load_row_t(const JT* J, size_t e, AT (&v)[NJ]) {
  using T = JTiles<JT, NJ>;
  const uint4* J4 = reinterpret_cast<const uint4*>(J);
  uint4 w[T::Q];
#pragma unroll
  for (int q = 0; q < T::Q; ++q) w[q] = J4[T::piece(e, q)];
  load_row<NJ>(reinterpret_cast<const JT*>(w), v);
}
template <int NJ, class JT>
__device__ __forceinline__ void store_row_t(JT* J, size_t e, const JT (&v)[NJ]) {
  using T = JTiles<JT, NJ>;
  uint4* J4 = reinterpret_cast<uint4*>(J);
  const uint4* s4 = reinterpret_cast<const uint4*>(v);
#pragma unroll
  for (int q = 0; q < T::Q; ++q) J4[T::piece(e, q)] = s4[q];
}

template <int NJ>
__device__ __forceinline__ void store_row(__nv_bfloat16* dst, const __nv_bfloat16 (&v)[NJ]) {
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  const uint4* s4 = reinterpret_cast<const uint4*>(v);
#pragma unroll
  for (int i = 0; i < NJ / 8; ++i) d4[i] = s4[i];
}
template <int NJ>
__device__ __forceinline__ void store_row(float* dst, const float (&v)[NJ]) {
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < NJ / 4; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
template <int NJ>
__device__ __forceinline__ void store_row(double* dst, const double (&v)[NJ]) {
  double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
  for (int i = 0; i < NJ / 2; ++i) d2[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

// ---------------------------------------------------------------- packed symmetric blocks

// Upper triangle of an n x n symmetric block, row-major packed: (i, j), i <= j.
__host__ __device__ constexpr int tri_n(int n) { return n * (n + 1) / 2; }
__host__ __device__ __forceinline__ int tri_idx(int n, int i, int j) { return i * n - (i * (i - 1)) / 2 + (j - i); }
__host__ __device__ __forceinline__ int sym_idx(int n, int i, int j) { return i <= j ? tri_idx(n, i, j) : tri_idx(n, j, i); }
__device__ __forceinline__ void tri_ij(int n, int t, int& i, int& j) {
  i = 0;
  while (t >= n - i) { t -= n - i; ++i; }
  j = i + t;
}

// ---------------------------------------------------------------- SO(3) and quaternions (FP64)

// Rodrigues: R = I + a [w]_x + b [w]_x^2 with a = sin t / t, b = (1 - cos t)/t^2,
// [w]_x^2 = w w^T - t^2 I; Taylor coefficients below t = 1e-4.
__device__ __forceinline__ void aa_to_R(const double* w, double* R) {
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
__device__ __forceinline__ void aa_to_q(const double* w, double* q) {
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

// Angle-axis of a unit quaternion (w, x, y, z), angle in [0, pi].
__device__ __forceinline__ void q_to_aa(const double* qin, double* w) {
  double q0 = qin[0], q1 = qin[1], q2 = qin[2], q3 = qin[3];
  if (q0 < 0) { q0 = -q0; q1 = -q1; q2 = -q2; q3 = -q3; }
  const double s = sqrt(q1 * q1 + q2 * q2 + q3 * q3);
  double k;
  if (s < 1e-8) k = 2.0 / q0 * (1.0 - s * s / (3.0 * q0 * q0));   // 2 atan(s/q0)/s, series
  else k = 2.0 * atan2(s, q0) / s;
  w[0] = k * q1;
  w[1] = k * q2;
  w[2] = k * q3;
}

// Hamilton product c = a b of (w, x, y, z) quaternions.
__device__ __forceinline__ void q_mul(const double* a, const double* b, double* c) {
  c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  c[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  c[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  c[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Rotation matrix (row-major) of a unit quaternion (w, x, y, z).
__device__ __forceinline__ void q_to_R(const double* q, double* R) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
  R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
  R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

// Left update w' = Log(Exp(dw) Exp(w)) via the quaternion product.
__device__ __forceinline__ void aa_left_update(const double* dw, const double* w, double* out) {
  double a[4], b[4], c[4];
  aa_to_q(dw, a);
  aa_to_q(w, b);
  q_mul(a, b, c);
  const double n = 1.0 / sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2] + c[3] * c[3]);
  c[0] *= n; c[1] *= n; c[2] *= n; c[3] *= n;
  q_to_aa(c, out);
}

// ---------------------------------------------------------------- reductions and binding

// Deterministic CTA sum of one double per thread (fixed tree, blockDim == kThreads).
__device__ __forceinline__ double block_sum(double v, double* red) {
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

// GPU-scope synchronising accesses (PTX memory model): an add that is both a release of
// the thread's earlier writes (and of the writes it has observed, such as its CTA's
// before a barrier) and an acquire of the writes released to the same location; a
// release add that returns nothing; an acquire load.
__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_add_release(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Call after thread 0 has written the CTA's partial (after a barrier if other threads
// wrote it); true in the CTA that finishes last.  Thread 0 takes the ticket with an
// acquire-release add: it releases the CTA's writes, and in the last CTA it acquires
// every other CTA's, which the barrier then orders before the CTA's later reads.
__device__ __forceinline__ bool last_cta(unsigned int* ticket, int ctas) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) is_last = atom_add_acq_rel(ticket, 1u) == (unsigned int)ctas - 1u;
  __syncthreads();
  return is_last;
}

// The PCG's beta and 1/n in the accumulation type: the FP32 copies the update stores
// beside the FP64 values (the same rounding a conversion here would give).
template <class AT>
__device__ __forceinline__ AT sc_beta(const Scalars* sc) {
  if constexpr (sizeof(AT) == 4) return sc->beta_f;
  else return sc->beta;
}
template <class AT>
__device__ __forceinline__ AT sc_inv_n(const Scalars* sc) {
  if constexpr (sizeof(AT) == 4) return sc->inv_n_f;
  else return sc->inv_n;
}

// Width of the reduction trees below: the smallest power of two holding the threads
// that loaded a partial (the threads past them hold zeros, which the full-width tree
// would only add, exactly; FP64 adds are scarce on this part).
__device__ __forceinline__ int tree_width(int n) {
  int m = 1;
  while (m < n && m < (int)blockDim.x) m <<= 1;
  return m;
}

// Sums the n per-CTA partial pairs (stride 2) with all threads of the CTA in a fixed
// order (strided per thread, then a fixed tree); the result is valid in every thread.
__device__ __forceinline__ void sum_partials(const double* part, int n, double& a, double& b) {
  __shared__ double ra[256], rb[256];
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    x += part[2 * i];
    y += part[2 * i + 1];
  }
  ra[threadIdx.x] = x;
  rb[threadIdx.x] = y;
  __syncthreads();
  for (int s2 = tree_width(n) / 2; s2 > 0; s2 >>= 1) {
    if ((int)threadIdx.x < s2) {
      ra[threadIdx.x] += ra[threadIdx.x + s2];
      rb[threadIdx.x] += rb[threadIdx.x + s2];
    }
    __syncthreads();
  }
  a = ra[0];
  b = rb[0];
}

// The first members of n partial pairs (stride 2), summed exactly as sum_partials sums
// them (the same value as its a) without the FP64 work of the second members, which
// matters on a part whose FP64 rate is a small fraction of its FP32 rate.
__device__ __forceinline__ double sum_partials_first(const double* part, int n) {
  __shared__ double ra[256];
  double x = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x += part[2 * i];
  ra[threadIdx.x] = x;
  __syncthreads();
  for (int s2 = tree_width(n) / 2; s2 > 0; s2 >>= 1) {
    if ((int)threadIdx.x < s2) ra[threadIdx.x] += ra[threadIdx.x + s2];
    __syncthreads();
  }
  return ra[0];
}

// Sums n single per-CTA partials with all threads in a fixed order (as sum_partials);
// the result is valid in every thread.
__device__ __forceinline__ double sum_singles(const double* part, int n) {
  __shared__ double rs[256];
  double x = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x += part[i];
  rs[threadIdx.x] = x;
  __syncthreads();
  for (int s2 = tree_width(n) / 2; s2 > 0; s2 >>= 1) {
    if ((int)threadIdx.x < s2) rs[threadIdx.x] += rs[threadIdx.x + s2];
    __syncthreads();
  }
  return rs[0];
}

// Point blocks of 256 points (the point kernels' CTAs) of a problem.
__device__ __forceinline__ int point_blocks(const DevBA& d) { return (d.P + 255) / 256; }
// Points per update CTA of the full-system PCG, and that update's point CTAs.
constexpr int kUpdatePoints = 2048;
__host__ __device__ inline int update_point_blocks(int P) { return (P + kUpdatePoints - 1) / kUpdatePoints; }

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

// Copies a problem's descriptor into shared memory (all threads cooperate).
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

// A launch over one problem needs no schedule lookup (CTA b is local block b), which
// takes two dependent global loads off the start of every CTA.
#define GPO_BIND(KIND, LOCAL)                                                    \
  __shared__ DevBA d;                                                            \
  pdl_trigger();                                                                 \
  const int prob_ = ls.nprob == 1 ? 0 : ls.KIND##_prob[blockIdx.x];              \
  const int LOCAL = ls.nprob == 1 ? (int)blockIdx.x                              \
                                  : (int)blockIdx.x - ls.KIND##_base[prob_];     \
  bind_problem(d, ls.probs + prob_);                                             \
  pdl_wait();

__device__ __forceinline__ void load_rb(const double* __restrict__ src, double* rb) {
  const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const double2 v = __ldg(s2 + i);
    rb[2 * i] = v.x;
    rb[2 * i + 1] = v.y;
  }
}

// IRLS weight sqrt(rho'(s)) = sqrt(delta / sqrt(s)) of a whitened squared norm s for
// s > delta^2 (1 inside), in the accumulation type: FP32 for the mixed forms (the
// Jacobian it scales is FP32), FP64 otherwise.
template <class AT>
__device__ __forceinline__ double huber_weight(double s, double delta) {
  if (!(delta > 0.0 && s > delta * delta)) return 1.0;
  if constexpr (std::is_same<AT, float>::value) {
    return (double)sqrtf((float)delta * rsqrtf((float)s));
  } else {
    return sqrt(delta / sqrt(s));
  }
}
// Huber value rho(s) (FP64): s inside delta^2, 2 delta sqrt(s) - delta^2 outside.
__device__ __forceinline__ double huber_rho(double s, double delta) {
  if (delta > 0.0 && s > delta * delta) return 2.0 * delta * sqrt(s) - delta * delta;
  return s;
}

// ---------------------------------------------------------------- BA model

// Camera render block rb[16]: R (row-major, 9), t (3), f, k1, k2, pad.
struct ModelBA {
  static constexpr int M = 2, DC = 9, DB = 9, SS = 9, NJ = 24, NQ = 3;   // NQ: packed sqrt-info
  static constexpr bool kExtra = false;

  // Not inlined: the retraction and the camera preparation call the same compiled body,
  // so a state renders to the same bits on both paths (inlined copies may contract the
  // arithmetic into FMAs differently and differ in the last bit).
  __device__ static __noinline__ void render(const DevBA&, const double* cam, double* rb) {
    aa_to_R(cam, rb);
    for (int i = 0; i < 6; ++i) rb[9 + i] = cam[3 + i];
    rb[15] = 0.0;
  }

  // x <- x [+] dx: w <- Log(Exp(dw) Exp(w)), the rest additive.
  __device__ static void retract(const double* cur, const double* dl, double* nxt) {
    double w[3];
    aa_left_update(dl, cur, w);
    nxt[0] = w[0]; nxt[1] = w[1]; nxt[2] = w[2];
    for (int i = 3; i < 9; ++i) nxt[i] = cur[i] + dl[i];
  }

  struct Geom {
    double y[3], P[3], p[2], iz, r2, d, u[2];
  };
  __device__ static void geom(const double* rb, const double* X, Geom& g) {
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

  // Whitened residual U (u - z).
  __device__ static void residual(const DevBA& d, int e, const Geom& g, double (&r)[M]) {
    const double2 z = __ldg(reinterpret_cast<const double2*>(d.obs) + e);
    double r0 = g.u[0] - z.x, r1 = g.u[1] - z.y;
    if (d.e_sqinfo) {
      const double* U = d.e_sqinfo + NQ * (size_t)e;
      const double a = U[0] * r0 + U[1] * r1;
      r1 = U[2] * r1;
      r0 = a;
    }
    r[0] = r0;
    r[1] = r1;
  }

  // 1/2 rho of an edge (cost only).
  __device__ static double cost(const DevBA& d, int e, const double* rb, const double* X) {
    Geom g;
    geom(rb, X, g);
    double r[M];
    residual(d, e, g, r);
    return 0.5 * huber_rho(r[0] * r[0] + r[1] * r[1], __ldg(d.e_delta + e));
  }

  // Whitened residual, Huber, and the whitened, sqrt(rho')-scaled Jacobian rows on the
  // chart (left rotation update, additive rest).  FP64 accumulation: everything in FP64.
  // FP32 accumulation (the mixed modes): only the camera-frame point P = R X + t is
  // formed in FP64 (world coordinates of hundreds of units cancel there down to depths
  // of a few); the projection, distortion, residual and rows follow in FP32 from it.
  // rb: the render block; rbf: the same rounded to FP32 (read by the FP32 path).  The
  // residual r and the square root of the IRLS weight sw come out in AT.
  template <class AT>
  __device__ static void eval(const DevBA& d, int e, const double* rb, const float* rbf, const double* X,
                              AT (&r)[M], AT& sw, AT (&Jc)[M][DC], AT (&Jp)[M][3]) {
    AT y[3], p0, p1, r2, dd, iz, f, k1, k2, R[9];
    if constexpr (std::is_same<AT, float>::value) {
      float P[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        P[i] = (float)(rb[3 * i] * X[0] + rb[3 * i + 1] * X[1] + rb[3 * i + 2] * X[2] + rb[9 + i]);
      float4 q[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) q[i] = __ldg(reinterpret_cast<const float4*>(rbf) + i);
      const float* fb = reinterpret_cast<const float*>(q);
#pragma unroll
      for (int i = 0; i < 9; ++i) R[i] = fb[i];
#pragma unroll
      for (int i = 0; i < 3; ++i) y[i] = P[i] - fb[9 + i];   // R X, far from any cancellation
      f = fb[12];
      k1 = fb[13];
      k2 = fb[14];
      iz = 1.0f / P[2];
      p0 = -P[0] * iz;
      p1 = -P[1] * iz;
      r2 = p0 * p0 + p1 * p1;
      dd = 1.0f + r2 * (k1 + k2 * r2);
      const float fd = f * dd;
      const double2 z = __ldg(reinterpret_cast<const double2*>(d.obs) + e);
      float r0 = fmaf(fd, p0, -(float)z.x), r1 = fmaf(fd, p1, -(float)z.y);
      if (d.e_sqinfo) {
        const double* U = d.e_sqinfo + NQ * (size_t)e;
        const float a = (float)U[0] * r0 + (float)U[1] * r1;
        r1 = (float)U[2] * r1;
        r0 = a;
      }
      r[0] = r0;
      r[1] = r1;
      const float dl = (float)__ldg(d.e_delta + e), sq = r0 * r0 + r1 * r1;
      sw = (dl > 0.0f && sq > dl * dl) ? sqrtf(dl * rsqrtf(sq)) : 1.0f;
    } else {
      Geom g;
      geom(rb, X, g);
      double rd[M];
      residual(d, e, g, rd);
      sw = huber_weight<AT>(rd[0] * rd[0] + rd[1] * rd[1], __ldg(d.e_delta + e));
      r[0] = rd[0];
      r[1] = rd[1];
      p0 = g.p[0];
      p1 = g.p[1];
      r2 = g.r2;
      dd = g.d;
      iz = g.iz;
      f = rb[12];
      k1 = rb[13];
      k2 = rb[14];
#pragma unroll
      for (int i = 0; i < 3; ++i) y[i] = g.y[i];
#pragma unroll
      for (int i = 0; i < 9; ++i) R[i] = rb[i];
    }
    const AT c2 = (AT)2 * k1 + (AT)4 * k2 * r2;
    // du/dp = f (d I + c2 p p^T)
    const AT A00 = f * (dd + c2 * p0 * p0), A01 = f * c2 * p0 * p1, A11 = f * (dd + c2 * p1 * p1);
    // dp/dP = [[-iz, 0, -p0 iz], [0, -iz, -p1 iz]]  (P_x / P_z^2 = -p0 / P_z)
    const AT B02 = -p0 * iz, B12 = -p1 * iz;
    AT D[2][3];
    D[0][0] = -A00 * iz; D[0][1] = -A01 * iz; D[0][2] = A00 * B02 + A01 * B12;
    D[1][0] = -A01 * iz; D[1][1] = -A11 * iz; D[1][2] = A01 * B02 + A11 * B12;
    const AT pp[2] = {p0, p1};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      // dP/d(dw) = -[y]_x : column k is e_k x y
      Jc[a][0] = -D[a][1] * y[2] + D[a][2] * y[1];
      Jc[a][1] = D[a][0] * y[2] - D[a][2] * y[0];
      Jc[a][2] = -D[a][0] * y[1] + D[a][1] * y[0];
      Jc[a][3] = D[a][0];
      Jc[a][4] = D[a][1];
      Jc[a][5] = D[a][2];
      Jc[a][6] = dd * pp[a];
      Jc[a][7] = f * r2 * pp[a];
      Jc[a][8] = f * r2 * r2 * pp[a];
#pragma unroll
      for (int j = 0; j < 3; ++j) Jp[a][j] = D[a][0] * R[j] + D[a][1] * R[3 + j] + D[a][2] * R[6 + j];
    }
    if (d.e_sqinfo) {
      const double* U = d.e_sqinfo + NQ * (size_t)e;
      const AT u00 = (AT)U[0], u01 = (AT)U[1], u11 = (AT)U[2];
#pragma unroll
      for (int k = 0; k < DC; ++k) {
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
    const AT s = sw;
#pragma unroll
    for (int a = 0; a < M; ++a) {
#pragma unroll
      for (int k = 0; k < DC; ++k) Jc[a][k] *= s;
#pragma unroll
      for (int k = 0; k < 3; ++k) Jp[a][k] *= s;
    }
  }
};

// ---------------------------------------------------------------- stereo / navigation model

// Kannala-Brandt (equidistant) fisheye projection of a camera-frame point by the rig's
// intrinsics and coefficients k1..k4 (camk[18..21]): theta = atan2(r, z), r = |(x, y)|,
// theta_d = theta (1 + k1 theta^2 + k2 theta^4 + k3 theta^6 + k4 theta^8),
// (u, v) = (fx theta_d x / r + cx, fy theta_d y / r + cy); with D also d(u, v)/d(x, y, z).
// On the optical axis (r = 0) the model's limit is the pinhole projection.
__device__ __forceinline__ void kb_project(const double* camk, double x, double y, double z, double& u,
                                          double& v, double (*D)[3]) {
  const double fx = camk[0], fy = camk[1], cx = camk[2], cy = camk[3];
  const double k1 = camk[18], k2 = camk[19], k3 = camk[20], k4 = camk[21];
  const double r = sqrt(x * x + y * y);
  if (!(r > 1e-12 * fabs(z))) {
    const double iz = 1.0 / z;
    u = fx * x * iz + cx;
    v = fy * y * iz + cy;
    if (D) {
      D[0][0] = fx * iz; D[0][1] = 0.0; D[0][2] = -fx * x * iz * iz;
      D[1][0] = 0.0; D[1][1] = fy * iz; D[1][2] = -fy * y * iz * iz;
    }
    return;
  }
  const double th = atan2(r, z), t2 = th * th;
  const double thd = th * (1.0 + t2 * (k1 + t2 * (k2 + t2 * (k3 + t2 * k4))));
  const double s = thd / r;
  u = fx * s * x + cx;
  v = fy * s * y + cy;
  if (D) {
    const double dthd = 1.0 + t2 * (3.0 * k1 + t2 * (5.0 * k2 + t2 * (7.0 * k3 + t2 * 9.0 * k4)));
    const double q = r * r + z * z;
    const double dth[3] = {x * z / (r * q), y * z / (r * q), -r / q};
    double ds[3];
    for (int i = 0; i < 3; ++i) ds[i] = dthd * dth[i] / r;
    ds[0] -= thd * x / (r * r * r);
    ds[1] -= thd * y / (r * r * r);
    for (int i = 0; i < 3; ++i) {
      D[0][i] = fx * x * ds[i];
      D[1][i] = fy * y * ds[i];
    }
    D[0][0] += fx * s;
    D[1][1] += fy * s;
  }
}

// Navigation state x = [qx qy qz qw, p (3), v (3), bg (3), ba (3)] (16 doubles), tangent
// [dtheta, dp, dv, dbg, dba] (15): R <- R Exp(dtheta), p <- p + R dp, rest additive.
// Render block rb[16]: R (body-to-world, row-major, 9), p (3), pad.
// d.camk: fx fy cx cy baseline, R_cb (9, body-to-camera), t_cb (3).
struct ModelStereo {
  static constexpr int M = 3, DC = 6, DB = 15, SS = 16, NJ = 32, NQ = 6;
  static constexpr bool kExtra = true;

  __device__ static __noinline__ void render(const DevBA&, const double* x, double* rb) {   // not inlined: see ModelBA
    const double q[4] = {x[3], x[0], x[1], x[2]};
    q_to_R(q, rb);
    rb[9] = x[4]; rb[10] = x[5]; rb[11] = x[6];
    rb[12] = rb[13] = rb[14] = rb[15] = 0.0;
  }

  __device__ static void retract(const double* cur, const double* dl, double* nxt) {
    const double q[4] = {cur[3], cur[0], cur[1], cur[2]};
    double dq[4], qn[4], R[9];
    aa_to_q(dl, dq);
    q_mul(q, dq, qn);
    double n = 1.0 / sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
    if (qn[0] < 0) n = -n;
    nxt[0] = qn[1] * n; nxt[1] = qn[2] * n; nxt[2] = qn[3] * n; nxt[3] = qn[0] * n;
    q_to_R(q, R);
    for (int i = 0; i < 3; ++i)
      nxt[4 + i] = cur[4 + i] + R[3 * i] * dl[3] + R[3 * i + 1] * dl[4] + R[3 * i + 2] * dl[5];
    for (int i = 7; i < 16; ++i) nxt[i] = cur[i] + dl[i - 1];
  }

  struct Geom {
    double Xb[3], Xc[3], iz, u[3];
  };
  __device__ static void geom(const DevBA& d, const double* rb, const double* X, Geom& g) {
    const double a0 = X[0] - rb[9], a1 = X[1] - rb[10], a2 = X[2] - rb[11];
#pragma unroll
    for (int i = 0; i < 3; ++i) g.Xb[i] = rb[i] * a0 + rb[3 + i] * a1 + rb[6 + i] * a2;   // R^T (X - p)
    const double* Rc = d.camk + 5;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      g.Xc[i] = Rc[3 * i] * g.Xb[0] + Rc[3 * i + 1] * g.Xb[1] + Rc[3 * i + 2] * g.Xb[2] + d.camk[14 + i];
    g.iz = 1.0 / g.Xc[2];
    if (d.camk[17] != 0.0) {   // fisheye rig: both cameras Kannala-Brandt
      double vr;
      kb_project(d.camk, g.Xc[0], g.Xc[1], g.Xc[2], g.u[0], g.u[1], nullptr);
      kb_project(d.camk, g.Xc[0] - d.camk[4], g.Xc[1], g.Xc[2], g.u[2], vr, nullptr);
      return;
    }
    g.u[0] = d.camk[0] * g.Xc[0] * g.iz + d.camk[2];
    g.u[1] = d.camk[1] * g.Xc[1] * g.iz + d.camk[3];
    g.u[2] = d.camk[0] * (g.Xc[0] - d.camk[4]) * g.iz + d.camk[2];
  }

  __device__ static void residual(const DevBA& d, int e, const Geom& g, double (&r)[M]) {
    const double* z = d.obs + 3 * (size_t)e;
    double e0 = g.u[0] - z[0], e1 = g.u[1] - z[1], e2 = g.u[2] - z[2];
    if (d.e_sqinfo) {   // U upper triangular, packed (u00 u01 u02 u11 u12 u22)
      const double* U = d.e_sqinfo + NQ * (size_t)e;
      const double w0 = U[0] * e0 + U[1] * e1 + U[2] * e2;
      const double w1 = U[3] * e1 + U[4] * e2;
      const double w2 = U[5] * e2;
      e0 = w0; e1 = w1; e2 = w2;
    }
    r[0] = e0; r[1] = e1; r[2] = e2;
  }

  __device__ static double cost(const DevBA& d, int e, const double* rb, const double* X) {
    Geom g;
    geom(d, rb, X, g);
    double r[M];
    residual(d, e, g, r);
    return 0.5 * huber_rho(r[0] * r[0] + r[1] * r[1] + r[2] * r[2], __ldg(d.e_delta + e));
  }

  // dr/dX_c rows: [fx/Z, 0, -fx X/Z^2], [0, fy/Z, -fy Y/Z^2], [fx/Z, 0, -fx (X-b)/Z^2];
  // dX_b/dtheta = [X_b]_x, dX_b/dp = -I, dX_b/dX = R^T; dX_c/dX_b = R_cb.
  // (rbf, the FP32 copy of the render block, is not used: the stereo rows come from FP64
  // geometry in every precision.)
  template <class AT>
  __device__ static void eval(const DevBA& d, int e, const double* rb, const float* rbf, const double* X,
                              AT (&rr)[M], AT& swr, AT (&Jc)[M][DC], AT (&Jp)[M][3]) {
    Geom g;
    geom(d, rb, X, g);
    double r[M];
    residual(d, e, g, r);
    const double sw = huber_weight<AT>(r[0] * r[0] + r[1] * r[1] + r[2] * r[2], __ldg(d.e_delta + e));
#pragma unroll
    for (int a = 0; a < M; ++a) rr[a] = (AT)r[a];
    swr = (AT)sw;
    const AT fx = (AT)d.camk[0], fy = (AT)d.camk[1], b = (AT)d.camk[4];
    const AT iz = (AT)g.iz, x = (AT)g.Xc[0], y = (AT)g.Xc[1];
    AT D[3][3];
    if (d.camk[17] != 0.0) {   // fisheye: rows of the left projection, u-row of the right
      double Dl[2][3], Dr[2][3], uu, vv;
      kb_project(d.camk, g.Xc[0], g.Xc[1], g.Xc[2], uu, vv, Dl);
      kb_project(d.camk, g.Xc[0] - d.camk[4], g.Xc[1], g.Xc[2], uu, vv, Dr);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        D[0][j] = (AT)Dl[0][j];
        D[1][j] = (AT)Dl[1][j];
        D[2][j] = (AT)Dr[0][j];
      }
    } else {
      D[0][0] = fx * iz; D[0][1] = (AT)0; D[0][2] = -fx * x * iz * iz;
      D[1][0] = (AT)0;   D[1][1] = fy * iz; D[1][2] = -fy * y * iz * iz;
      D[2][0] = fx * iz; D[2][1] = (AT)0; D[2][2] = -fx * (x - b) * iz * iz;
    }
    AT DR[3][3];   // D R_cb
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        DR[a][j] = D[a][0] * (AT)d.camk[5 + j] + D[a][1] * (AT)d.camk[8 + j] + D[a][2] * (AT)d.camk[11 + j];
    const AT b0 = (AT)g.Xb[0], b1 = (AT)g.Xb[1], b2 = (AT)g.Xb[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // DR [X_b]_x : column k is DR (X_b x e_k)
      Jc[a][0] = DR[a][1] * b2 - DR[a][2] * b1;
      Jc[a][1] = -DR[a][0] * b2 + DR[a][2] * b0;
      Jc[a][2] = DR[a][0] * b1 - DR[a][1] * b0;
      Jc[a][3] = -DR[a][0];
      Jc[a][4] = -DR[a][1];
      Jc[a][5] = -DR[a][2];
#pragma unroll
      for (int j = 0; j < 3; ++j)   // DR R^T: R^T[i][j] = R[j][i]
        Jp[a][j] = DR[a][0] * (AT)rb[3 * j] + DR[a][1] * (AT)rb[3 * j + 1] + DR[a][2] * (AT)rb[3 * j + 2];
    }
    if (d.e_sqinfo) {
      const double* U = d.e_sqinfo + NQ * (size_t)e;
      const AT u00 = (AT)U[0], u01 = (AT)U[1], u02 = (AT)U[2], u11 = (AT)U[3], u12 = (AT)U[4], u22 = (AT)U[5];
#pragma unroll
      for (int k = 0; k < DC; ++k) {
        const AT w0 = u00 * Jc[0][k] + u01 * Jc[1][k] + u02 * Jc[2][k];
        const AT w1 = u11 * Jc[1][k] + u12 * Jc[2][k];
        Jc[2][k] = u22 * Jc[2][k];
        Jc[0][k] = w0; Jc[1][k] = w1;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const AT w0 = u00 * Jp[0][k] + u01 * Jp[1][k] + u02 * Jp[2][k];
        const AT w1 = u11 * Jp[1][k] + u12 * Jp[2][k];
        Jp[2][k] = u22 * Jp[2][k];
        Jp[0][k] = w0; Jp[1][k] = w1;
      }
    }
    const AT s = (AT)sw;
#pragma unroll
    for (int a = 0; a < M; ++a) {
#pragma unroll
      for (int k = 0; k < DC; ++k) Jc[a][k] *= s;
#pragma unroll
      for (int k = 0; k < 3; ++k) Jp[a][k] *= s;
    }
  }
};

// ---------------------------------------------------------------- model sizes and shared helpers

template <class Mo>
struct Dims {
  static constexpr int M = Mo::M, DC = Mo::DC, DB = Mo::DB, SS = Mo::SS, NJ = Mo::NJ;
  static constexpr int JP0 = M * DC;            // first point-row value of a Jacobian row
  static constexpr int NJU = JP0 + 3 * M;       // values in use (the rest is padding)
  static constexpr int TC = tri_n(DC);          // H entries of a slot partial
  static constexpr int NA = TC + DC;            // H + b entries of a slot partial
  static constexpr int NG = (NA + 8) / 9;       // groups of nine
  static constexpr int NPA = 9 * NG;            // slot partial row
  static constexpr int TB = tri_n(DB);          // packed camera block
  static constexpr int TM = tri_n(M);           // packed M x M point-side weights
  static constexpr int VW = DC > 3 ? DC : 3;    // rows of the Schur-product scratch
  static_assert(NJ % 8 == 0 && NJU <= NJ, "Jacobian rows are whole 16-byte vectors");
  static_assert(DB <= 32, "one lane per camera-block component");
};

// The two per-edge terms of the matrix-free Schur product (Sec. IV-E), shared by every
// Schur-product kernel so that all of them round alike.  `row` is the edge's unpacked
// Jacobian row (Jc row-major, then Jp row-major).  Every sum runs in a fixed order,
// spelled out as fused multiply-adds:
//   point term   q_a = sum_k Jc[a][k] x_k (k ascending), a_k = sum_a Jp[a][k] q_a;
//   camera term  s_a = sum_k Jp[a][k] t_k (k ascending), v_k = sum_a Jc[a][k] s_a.
// For two residual rows in FP32 the two rows' (or two components') chains run side by
// side in packed FP32x2 instructions; each lane performs the scalar chain's operations,
// so the packed and scalar forms give the same values.
template <class Mo, class AT>
__device__ __forceinline__ void edge_point_term(const AT* row, const AT* xc, AT (&a)[3]) {
  constexpr int M = Mo::M, DC = Mo::DC, JP0 = M * DC;
  if constexpr (M == 2 && std::is_same<AT, float>::value) {
    float2 q = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < DC; ++k) {
      const float xk = xc[k];
      q = __ffma2_rn(make_float2(row[k], row[DC + k]), make_float2(xk, xk), q);
    }
    const float2 s = __ffma2_rn(make_float2(row[JP0 + 3], row[JP0 + 4]), make_float2(q.y, q.y),
                                __fmul2_rn(make_float2(row[JP0], row[JP0 + 1]), make_float2(q.x, q.x)));
    a[0] = s.x;
    a[1] = s.y;
    a[2] = fmaf(row[JP0 + 5], q.y, row[JP0 + 2] * q.x);
  } else {
    AT q[M];
#pragma unroll
    for (int r = 0; r < M; ++r) q[r] = (AT)0;
#pragma unroll
    for (int k = 0; k < DC; ++k) {
      const AT xk = xc[k];
#pragma unroll
      for (int r = 0; r < M; ++r) q[r] = fma(row[r * DC + k], xk, q[r]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      AT s = row[JP0 + k] * q[0];
#pragma unroll
      for (int r = 1; r < M; ++r) s = fma(row[JP0 + 3 * r + k], q[r], s);
      a[k] = s;
    }
  }
}
template <class Mo, class AT>
__device__ __forceinline__ void edge_camera_term(const AT* row, AT t0, AT t1, AT t2, AT (&v)[Mo::DC]) {
  constexpr int M = Mo::M, DC = Mo::DC, JP0 = M * DC;
  if constexpr (M == 2 && std::is_same<AT, float>::value) {
    float2 s = __fmul2_rn(make_float2(row[JP0], row[JP0 + 3]), make_float2(t0, t0));
    s = __ffma2_rn(make_float2(row[JP0 + 1], row[JP0 + 4]), make_float2(t1, t1), s);
    s = __ffma2_rn(make_float2(row[JP0 + 2], row[JP0 + 5]), make_float2(t2, t2), s);
#pragma unroll
    for (int k = 0; k + 1 < DC; k += 2) {
      const float2 w = __ffma2_rn(make_float2(row[DC + k], row[DC + k + 1]), make_float2(s.y, s.y),
                                  __fmul2_rn(make_float2(row[k], row[k + 1]), make_float2(s.x, s.x)));
      v[k] = w.x;
      v[k + 1] = w.y;
    }
    if constexpr (DC % 2 == 1) v[DC - 1] = fmaf(row[2 * DC - 1], s.y, row[DC - 1] * s.x);
  } else {
    AT s[M];
#pragma unroll
    for (int r = 0; r < M; ++r) s[r] = fma(row[JP0 + 3 * r + 2], t2, fma(row[JP0 + 3 * r + 1], t1, row[JP0 + 3 * r] * t0));
#pragma unroll
    for (int k = 0; k < DC; ++k) {
      AT w = row[k] * s[0];
#pragma unroll
      for (int r = 1; r < M; ++r) w = fma(row[r * DC + k], s[r], w);
      v[k] = w;
    }
  }
}

template <class AT>
__device__ __forceinline__ void mul3(const AT* h, const AT* v, AT* o) {
  o[0] = h[0] * v[0] + h[1] * v[1] + h[2] * v[2];
  o[1] = h[1] * v[0] + h[3] * v[1] + h[4] * v[2];
  o[2] = h[2] * v[0] + h[4] * v[1] + h[5] * v[2];
}

// Sum of src[a .. b) with four interleaved partial sums (more loads in flight than a
// single running sum), combined as (s0 + s1) + (s2 + s3).
template <class AT>
__device__ __forceinline__ AT seg_sum(const AT* src, int a, int b) {
  AT s0 = (AT)0, s1 = (AT)0, s2 = (AT)0, s3 = (AT)0;
  int q = a;
  for (; q + 4 <= b; q += 4) {
    s0 += src[q];
    s1 += src[q + 1];
    s2 += src[q + 2];
    s3 += src[q + 3];
  }
  for (; q < b; ++q) s0 += src[q];
  return (s0 + s1) + (s2 + s3);
}

// Point sums of the Schur product's pass 2: u_k = sum_{i in [a, b)} v[k LD + i].  FP32
// storage takes the interleaved sums (measured faster on the 1,000-camera BA workload);
// BF16 and FP64 keep one running sum per component (the interleaved form raises their
// register count past six resident CTAs per SM, which costs more than it gains).
template <class JT, class AT>
__device__ __forceinline__ void point_sum(const AT* v, int LD, int a, int b, AT (&u)[3]) {
  if constexpr (std::is_same<JT, float>::value) {
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = seg_sum(v + k * LD, a, b);
  } else {
    u[0] = u[1] = u[2] = (AT)0;
    for (int i = a; i < b; ++i) {
#pragma unroll
      for (int k = 0; k < 3; ++k) u[k] += v[k * LD + i];
    }
  }
}

}  // namespace gpo
