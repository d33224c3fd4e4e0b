// Schur-complement Levenberg-Marquardt kernels on sm_103a, generic over the edge
// model: observation-edge linearisation, point and camera accumulation, the camera
// Schur complement, matrix-free block-Jacobi PCG, point back-substitution, FP64
// retraction, cost and the LM gain-ratio decision.
//
// Paper mapping: Eq. 1 and Eq. 7 (cost with Huber), Eq. 3-6 (LM normal equations),
// Sec. IV-B (analytic Jacobians), Sec. IV-E (PCG on implicit products of the
// Jacobians, block-Jacobi preconditioner kept at FP32 or higher, Hessian-diagonal
// clamping, residual normalisation), Sec. IV-E last paragraph (kernels walk the
// graph structure; no sparse-matrix format).  The PCG runs on the camera Schur
// complement S = H_cc + lambda D_c - H_cp H_pp^-1 H_pc; its product with a vector is
// formed from the stored Jacobians in one pass per chunk of point-major edges.
//
// A model (schur_common.cuh) fixes M observation rows, DC camera columns of an
// observation's Jacobian (the first DC dimensions of the DB-dimensional camera
// block) and NJ stored values per edge.  Models with camera-side edges (kExtra:
// inertial and bias edges of the navigation model) add their diagonal blocks and
// gradients in the camera finalisation and their off-diagonal products in the
// camera half of the Schur product; their linearisation, cost and model-decrease
// kernels live with the model (vi_kernels.cu).
#pragma once
#include <algorithm>
#include <atomic>
#include <mutex>

#include "schur_common.cuh"
#include "schur_spmv.cuh"
#include "schur_wg.cuh"
#include "schur_dynamic.cuh"

namespace gpo {

// Packed upper triangles of 9x9 and 6x6 blocks: entry t is (row[t], col[t]).
static __constant__ unsigned char c_t9i[45] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1,
                                               2, 2, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 4, 4, 4, 4,
                                               4, 5, 5, 5, 5, 6, 6, 6, 7, 7, 8};
static __constant__ unsigned char c_t9j[45] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 1, 2, 3, 4, 5, 6, 7, 8,
                                               2, 3, 4, 5, 6, 7, 8, 3, 4, 5, 6, 7, 8, 4, 5, 6, 7,
                                               8, 5, 6, 7, 8, 6, 7, 8, 7, 8, 8};
static __constant__ unsigned char c_t6i[21] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
static __constant__ unsigned char c_t6j[21] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};

template <int N>
__device__ __forceinline__ int tri_row(int t) {
  static_assert(N == 9 || N == 6, "no table for this block size");
  if constexpr (N == 9) return c_t9i[t];
  else return c_t6i[t];
}
template <int N>
__device__ __forceinline__ int tri_col(int t) {
  if constexpr (N == 9) return c_t9j[t];
  else return c_t6j[t];
}

// ---------------------------------------------------------------- small dense helpers

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
__device__ __forceinline__ AT damp_diag(AT h, const Scalars* sc) {
  if (sc->damping_mode == 1) return (AT)1;
  return fmin(fmax(h, (AT)sc->diag_min), (AT)sc->diag_max);
}

// Inverse of an N x N SPD block by one warp, lane i holding row i (N <= 32): the block
// is first scaled to unit diagonal (A' = D^-1/2 A D^-1/2, which removes the spread of
// scales between rotation, translation, intrinsics or bias coordinates), then
// Gauss-Jordan elimination without pivoting runs on [A' | I] (stable for SPD matrices:
// each pivot is a Schur-complement diagonal, positive exactly when A is positive
// definite).  M = D^-1/2 A'^-1 D^-1/2, written as the packed upper triangle.  If A is
// not positive definite in this precision, M = diag(1 / A_ii) (Jacobi; 1 where
// A_ii <= 0).  A is a full row-major N x N block in shared memory; every lane calls.
template <int N, class AT>
__device__ void warp_spd_inverse(const AT* A, AT* M, int lane) {
  const unsigned full = 0xffffffffu;
  const AT dii = lane < N ? A[lane * N + lane] : (AT)1;
  const bool pos = __all_sync(full, dii > (AT)0);
  const AT sc = pos ? (AT)1 / sqrt(dii) : (AT)0;
  AT a[N], b[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const AT sj = __shfl_sync(full, sc, j);
    a[j] = lane < N ? A[lane * N + j] * sc * sj : (AT)0;
    b[j] = lane == j ? (AT)1 : (AT)0;
  }
  bool ok = pos;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const AT pk = __shfl_sync(full, a[k], k);
    ok = ok && pk > (AT)0;
    const AT inv = ok ? (AT)1 / pk : (AT)0;
    const AT f = a[k];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const AT akj = __shfl_sync(full, a[j], k) * inv;
      const AT bkj = __shfl_sync(full, b[j], k) * inv;
      if (lane == k) {
        a[j] = akj;
        b[j] = bkj;
      } else {
        a[j] -= f * akj;
        b[j] -= f * bkj;
      }
    }
  }
  if (ok) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const AT sj = __shfl_sync(full, sc, j);
      if (lane < N && j >= lane) M[tri_idx(N, lane, j)] = sc * b[j] * sj;
    }
  } else if (lane < N) {
    for (int j = lane; j < N; ++j) M[tri_idx(N, lane, j)] = (AT)0;
    M[tri_idx(N, lane, lane)] = dii > (AT)0 ? (AT)1 / dii : (AT)1;
  }
}

__device__ __forceinline__ int xrows(int kind) { return kind == XK_IMU ? 9 : 6; }

// ---------------------------------------------------------------- camera render blocks

template <class Mo>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_cam_prepare(LaunchSet ls, int candidate) {
  GPO_BIND(cb, cbl)
  if (!d.sc->active) return;
  const int c = cbl * kCamPerBlock + (threadIdx.x >> 5);
  if (c >= d.C || (threadIdx.x & 31) != 0) return;
  const double* cam = (candidate ? d.cam_cand : d.cam) + Mo::SS * (size_t)c;
  double* rb = (candidate ? d.camrb_cand : d.camrb) + 16 * (size_t)c;
  float* rbf = (candidate ? d.camrbf_cand : d.camrbf) + 16 * (size_t)c;
  Mo::render(d, cam, rb);
  for (int i = 0; i < 16; ++i) rbf[i] = (float)rb[i];
}

// ---------------------------------------------------------------- cost F(x)

template <class Mo>
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
    acc += Mo::cost(d, e, rb, X);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.cost_part[kl] = s;
}

template <class Mo>
__global__ void k_cost_init(LaunchSet ls) {
  __shared__ double red[kThreads];
  __shared__ DevBA d;
  pdl_trigger();
  bind_problem(d, ls.probs + blockIdx.x);
  pdl_wait();
  if (!d.sc->active) return;
  double acc = 0.0;
  for (int k = threadIdx.x; k < d.NCH; k += kThreads) acc += d.cost_part[k];
  if constexpr (Mo::kExtra)
    for (int x = threadIdx.x; x < d.NX; x += kThreads) acc += d.xe_cost[x];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.sc->cost = s;
}

// ---------------------------------------------------------------- per-edge records and slot rows

// Both accumulation kernels first turn each edge of the chunk into records in shared
// memory, then reduce the records of each camera slot into that slot's partial row.
// Per edge: Y[k * M + a] (k < DC camera coordinates, a < M rows; type YT) and, in a
// second array of AT values, the DC-vector g followed by kernel-specific terms.  Rows
// are an odd number of 4-byte words apart (8-byte values: an odd number of values) so
// that the edge-per-thread stores do not collide in a bank.  The slot row is the packed
// upper triangle of sum_e Y_e^T Y_e (TC entries), then sum_e g_e (DC entries), then
// zero padding up to NPA.
template <int N>
struct OddStride {
  static constexpr int value = N | 1;
};
template <class T, int N>
struct OddRow {   // row length in values, N rounded up so the row spans an odd count of banks
  static constexpr int value = sizeof(T) == 2 ? ((N / 2) % 2 == 1 ? N : N + 2) : (N | 1);
  static_assert(sizeof(T) != 2 || N % 2 == 0, "two-byte rows hold whole words");
};

// One warp per slot (slots handed out by a shared counter, so long slots do not hold
// up a fixed set of warps).  The camera indices are cut into blocks of three; a lane
// has a role -- one 3 x 3 tile of the upper block triangle of sum_e Y_e^T Y_e, and the
// entries role, role + NT, ... of sum_e g_e -- and an edge group: the warp's NT roles
// repeat NG = 32 / NT times, group j takes the slot's edges j, j + NG, ... in slot
// order, and at the end group 0 adds the other groups' sums in group order (shuffles).
// A lane reads its 2 x 3 record values per row of Y once per edge and forms nine
// products from them, so the reduction costs a fraction of the instructions of one
// output per lane.
template <class Mo, class YT, class AT, int RSY, int RSG>
__device__ __forceinline__ void slot_rows(const DevBA& d, const ChunkRange& cr, const YT* Y, const AT* G,
                                          const uint16_t* srt, AT* part, int* next) {
  using Dm = Dims<Mo>;
  constexpr int M = Mo::M, DC = Mo::DC, TC = Dm::TC, NPA = Dm::NPA;
  constexpr int NB = (DC + 2) / 3;           // index blocks of three
  constexpr int NT = NB * (NB + 1) / 2;      // tiles of the upper block triangle: the roles
  constexpr int KG = (DC + NT - 1) / NT;     // gradient entries per role
  constexpr int NG = 32 / NT;                // edge groups
  constexpr int NA = 9 + KG;                 // sums per lane
  static_assert(NG >= 1, "a warp holds every role");
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, role = lane % NT, grp = lane / NT;   // grp == NG: idle
  int bi = 0, t = role;
  while (t >= NB - bi) {
    t -= NB - bi;
    ++bi;
  }
  const int bj = bi + t;
  for (;;) {
    int sl = 0;
    if (lane == 0) sl = atomicAdd(next, 1);
    sl = __shfl_sync(full, sl, 0);
    if (sl >= cr.nS) break;
    const int qa = d.slot_e0[cr.s0 + sl] - cr.e0, qb = d.slot_e0[cr.s0 + sl + 1] - cr.e0;
    AT acc[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) acc[c] = (AT)0;
    if (grp < NG) {
      for (int q = qa + grp; q < qb; q += NG) {
        const int e = srt[q];
        const YT* y = Y + (size_t)e * RSY;
        const AT* g = G + (size_t)e * RSG;
        AT yi[3][M], yj[3][M];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int i = 3 * bi + u, j = 3 * bj + u;
#pragma unroll
          for (int r = 0; r < M; ++r) {
            yi[u][r] = i < DC ? (AT)ldj(y + i * M + r) : (AT)0;
            yj[u][r] = j < DC ? (AT)ldj(y + j * M + r) : (AT)0;
          }
        }
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
          for (int v = 0; v < 3; ++v)
#pragma unroll
            for (int r = 0; r < M; ++r) acc[3 * u + v] = fma(yi[u][r], yj[v][r], acc[3 * u + v]);
#pragma unroll
        for (int m = 0; m < KG; ++m)
          if (role + NT * m < DC) acc[9 + m] += g[role + NT * m];
      }
    }
#pragma unroll
    for (int j = 1; j < NG; ++j) {
#pragma unroll
      for (int c = 0; c < NA; ++c) {
        const AT o = __shfl_sync(full, acc[c], role + NT * j);
        if (grp == 0) acc[c] += o;
      }
    }
    AT* out = part + (size_t)d.slot_pos[cr.s0 + sl] * NPA;
    if (grp == 0) {
#pragma unroll
      for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const int i = 3 * bi + u, j = 3 * bj + v;
          if (i < DC && j < DC && i <= j) out[tri_idx(DC, i, j)] = acc[3 * u + v];
        }
#pragma unroll
      for (int m = 0; m < KG; ++m)
        if (role + NT * m < DC) out[TC + role + NT * m] = acc[9 + m];
    }
    for (int o = TC + DC + lane; o < NPA; o += 32) out[o] = (AT)0;
  }
}

// ---------------------------------------------------------------- linearisation

// Records of the linearisation: Y = the stored camera rows in the storage type (exact:
// they are the rounded values), and in AT g = Jc^T r from the unrounded rows, then the
// point terms: packed Jp^T Jp of the stored rows (6) and Jp^T r from the unrounded rows
// (3).  BF16 rows keep the records at 112 bytes per edge (three CTAs per SM).
template <class Mo, class JT>
struct LinRec {
  static constexpr int RSY = OddRow<JT, Mo::M * Mo::DC>::value;
  static constexpr int G = 0, H = Mo::DC, B = H + 6;
  static constexpr int RSG = OddStride<B + 3>::value;
};

// One CTA per chunk.  Writes the chunk's Jacobian rows, the undamped point blocks
// H_pp = sum Jp^T Jp and gradients b_p, and per-slot camera partials
// (H_cc = sum Jc^T Jc, b_c = sum Jc^T r).  H uses the stored (rounded) Jacobian; the
// gradient uses the unrounded one, so BF16 storage leaves the LM fixed point intact.
template <class Mo, class JT>
__global__ void __launch_bounds__(kThreads) k_linearize(LaunchSet ls, int force) {
  using AT = typename AccOf<JT>::T;
  using Dm = Dims<Mo>;
  using R = LinRec<Mo, JT>;
  constexpr int M = Mo::M, DC = Mo::DC, NJ = Mo::NJ, JP0 = Dm::JP0, NJU = Dm::NJU;
  constexpr int RSY = R::RSY, RSG = R::RSG;
  GPO_BIND(ch, kl)
  if (!d.sc->active || (!force && !d.sc->need_lin)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int next_slot;
  const int CH = d.ch_max;
  AT* rec = reinterpret_cast<AT*>(smem);                       // [CH][RSG]
  JT* yrec = reinterpret_cast<JT*>(rec + (size_t)RSG * CH);     // [CH][RSY]
  uint16_t* srt = reinterpret_cast<uint16_t*>(yrec + (size_t)RSY * CH);   // [CH]
  const ChunkRange cr = chunk_range(d, kl);
  JT* Jg = reinterpret_cast<JT*>(d.J);
  if (threadIdx.x == 0) next_slot = 0;

  for (int i = threadIdx.x; i < cr.nE; i += kThreads) {
    const int e = cr.e0 + i;
    const int c = __ldg(d.e_cam + e), p = __ldg(d.e_pt + e);
    double rb[16];
    load_rb(d.camrb + 16 * (size_t)c, rb);
    const double X[3] = {d.pt[3 * (size_t)p], d.pt[3 * (size_t)p + 1], d.pt[3 * (size_t)p + 2]};
    AT r[M], sw;
    AT Jc[M][DC], Jp[M][3];
    Mo::template eval<AT>(d, e, rb, d.camrbf + 16 * (size_t)c, X, r, sw, Jc, Jp);
    if (d.cam_fixed[c]) {
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int k = 0; k < DC; ++k) Jc[a][k] = (AT)0;
    }
    if (d.pt_fixed[p]) {
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) Jp[a][k] = (AT)0;
    }
    AT rw[M];
#pragma unroll
    for (int a = 0; a < M; ++a) rw[a] = sw * r[a];
    __align__(16) JT row[NJ];
#pragma unroll
    for (int a = 0; a < M; ++a) {
#pragma unroll
      for (int k = 0; k < DC; ++k) row[a * DC + k] = cvj(Jc[a][k], (const JT*)nullptr);
#pragma unroll
      for (int k = 0; k < 3; ++k) row[JP0 + 3 * a + k] = cvj(Jp[a][k], (const JT*)nullptr);
    }
#pragma unroll
    for (int k = NJU; k < NJ; ++k) row[k] = cvj((AT)0, (const JT*)nullptr);
    if (Jg) store_row_t<NJ>(Jg, (size_t)e, row);   // dynamic Jacobians keep no rows
    srt[i] = d.ch_sorted[e];
    AT* re = rec + (size_t)i * RSG;
    JT* ye = yrec + (size_t)i * RSY;
#pragma unroll
    for (int k = 0; k < DC; ++k) {
#pragma unroll
      for (int a = 0; a < M; ++a) ye[k * M + a] = row[a * DC + k];
      AT s = Jc[0][k] * rw[0];
#pragma unroll
      for (int a = 1; a < M; ++a) s += Jc[a][k] * rw[a];
      re[R::G + k] = s;
    }
    AT Jq[M][3];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) Jq[a][k] = ldj(&row[JP0 + 3 * a + k]);
    AT hs[6];
    hs[0] = Jq[0][0] * Jq[0][0]; hs[1] = Jq[0][0] * Jq[0][1]; hs[2] = Jq[0][0] * Jq[0][2];
    hs[3] = Jq[0][1] * Jq[0][1]; hs[4] = Jq[0][1] * Jq[0][2]; hs[5] = Jq[0][2] * Jq[0][2];
#pragma unroll
    for (int a = 1; a < M; ++a) {
      hs[0] += Jq[a][0] * Jq[a][0]; hs[1] += Jq[a][0] * Jq[a][1]; hs[2] += Jq[a][0] * Jq[a][2];
      hs[3] += Jq[a][1] * Jq[a][1]; hs[4] += Jq[a][1] * Jq[a][2]; hs[5] += Jq[a][2] * Jq[a][2];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) re[R::H + k] = hs[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      AT s = Jp[0][k] * rw[0];
#pragma unroll
      for (int a = 1; a < M; ++a) s += Jp[a][k] * rw[a];
      re[R::B + k] = s;
    }
    if (d.dbg_r) {
#pragma unroll
      for (int a = 0; a < M; ++a) d.dbg_r[M * (size_t)e + a] = sw * r[a];
    }
  }
  __syncthreads();

  // point blocks: the point's edges are contiguous in the chunk
  AT* Hpp = reinterpret_cast<AT*>(d.Hpp);
  AT* bp = reinterpret_cast<AT*>(d.bp);
  for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
    const int pj = cr.p0 + j;
    const int a0 = d.pt_off[pj] - cr.e0, b0 = d.pt_off[pj + 1] - cr.e0;
    AT h[6] = {0, 0, 0, 0, 0, 0}, bb[3] = {0, 0, 0};
    for (int i = a0; i < b0; ++i) {
      const AT* re = rec + (size_t)i * RSG;
#pragma unroll
      for (int k = 0; k < 6; ++k) h[k] += re[R::H + k];
#pragma unroll
      for (int k = 0; k < 3; ++k) bb[k] += re[R::B + k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) Hpp[6 * (size_t)pj + k] = h[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) bp[3 * (size_t)pj + k] = bb[k];
  }

  // camera slots
  slot_rows<Mo, JT, AT, RSY, RSG>(d, cr, yrec, rec, srt, reinterpret_cast<AT*>(d.partA), &next_slot);
}

// ---------------------------------------------------------------- Schur preparation

// Upper Cholesky-style factor of an M x M positive semi-definite block: A = L L^T with L
// lower triangular (a non-positive pivot, possible only through rounding of a singular
// block, gives a zero column).
template <int M, class AT>
__device__ __forceinline__ void psd_cholesky(const AT (&A)[M][M], AT (&L)[M][M]) {
#pragma unroll
  for (int j = 0; j < M; ++j) {
#pragma unroll
    for (int i = 0; i < M; ++i) L[i][j] = (AT)0;
  }
#pragma unroll
  for (int j = 0; j < M; ++j) {
    AT dj = A[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) dj -= L[j][k] * L[j][k];
    const AT ljj = dj > (AT)0 ? sqrt(dj) : (AT)0;
    const AT inv = ljj > (AT)0 ? (AT)1 / ljj : (AT)0;
    L[j][j] = ljj;
#pragma unroll
    for (int i = j + 1; i < M; ++i) {
      AT v = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v * inv;
    }
  }
}

// Record layout of the Schur preparation: Y = K = L^T Jc, where L L^T = Jp H_pp^-1 Jp^T,
// so that sum_e K^T K = sum_e W_e H_pp^-1 W_e^T; g = Jc^T Jp H_pp^-1 b_p.
template <class Mo, class AT>
struct SchurRec {
  static constexpr int RSY = OddRow<AT, Mo::M * Mo::DC>::value;
  static constexpr int RSG = OddStride<Mo::DC>::value;
};

// One CTA per chunk: damped point inverses H_pp^-1 (and the point records of the Schur
// product), then per-slot partials of sum_e W_e H_pp^-1 W_e^T and sum_e W_e H_pp^-1 b_p
// (W_e = Jc^T Jp, from the stored Jacobian rows).
template <class Mo, class JT, bool kDyn = false>
__global__ void __launch_bounds__(kThreads) k_schur_prepare(LaunchSet ls) {
  using AT = typename AccOf<JT>::T;
  using Dm = Dims<Mo>;
  using R = SchurRec<Mo, AT>;
  constexpr int M = Mo::M, DC = Mo::DC, NJ = Mo::NJ, JP0 = Dm::JP0, RSY = R::RSY, RSG = R::RSG;
  GPO_BIND(ch, kl)
  if (!d.sc->active) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int next_slot;
  const int CH = d.ch_max;
  AT* rec = reinterpret_cast<AT*>(smem);                   // [CH][RSY]: K
  AT* grec = rec + (size_t)RSY * CH;                       // [CH][RSG]: g
  AT* pv = grec + (size_t)RSG * CH;                        // [np_max][9]: H_pp^-1 (6), H_pp^-1 b_p (3)
  uint16_t* srt = reinterpret_cast<uint16_t*>(pv + 9 * (size_t)ls.np_max);   // [CH]
  const ChunkRange cr = chunk_range(d, kl);
  const JT* Jg = reinterpret_cast<const JT*>(d.J);
  const Scalars* sc = d.sc;
  const AT lam = (AT)sc->lambda;
  const AT* Hpp = reinterpret_cast<const AT*>(d.Hpp);
  const AT* bp = reinterpret_cast<const AT*>(d.bp);
  AT* Hinv = reinterpret_cast<AT*>(d.Hinv);
  constexpr size_t PRB = (6 * sizeof(AT) + 8 + 15) & ~(size_t)15;
  if (threadIdx.x == 0) next_slot = 0;

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
    unsigned char* prec = static_cast<unsigned char*>(d.pt_rec) + (size_t)pj * PRB;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      Hinv[6 * (size_t)pj + k] = o[k];
      reinterpret_cast<AT*>(prec)[k] = o[k];
      pv[9 * j + k] = o[k];
    }
    int* se = reinterpret_cast<int*>(prec + 6 * sizeof(AT));
    se[0] = d.pt_off[pj] - cr.e0;
    se[1] = d.pt_off[pj + 1] - cr.e0;
    AT bb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) bb[k] = bp[3 * (size_t)pj + k];
    mul3(o, bb, pv + 9 * j + 6);
  }
  __syncthreads();

  const bool packed = ls.ch_max <= 1024;
  for (int i = threadIdx.x; i < cr.nE; i += kThreads) {
    const int pl = packed ? (int)(__ldg(d.e_meta + cr.e0 + i) >> 20) : __ldg(d.e_pt + cr.e0 + i) - cr.p0;
    const AT* hi = pv + 9 * pl;
    const AT* hb = hi + 6;
    AT row[NJ];
    row_of<Mo, JT, AT, kDyn>(d, Jg, cr.e0 + i, row);
    srt[i] = d.ch_sorted[cr.e0 + i];
    AT t[M][3];
#pragma unroll
    for (int a = 0; a < M; ++a) mul3(hi, row + JP0 + 3 * a, t[a]);
    AT A[M][M], qe[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const AT* Ja = row + JP0 + 3 * a;
#pragma unroll
      for (int b = a; b < M; ++b) A[a][b] = A[b][a] = Ja[0] * t[b][0] + Ja[1] * t[b][1] + Ja[2] * t[b][2];
      qe[a] = Ja[0] * hb[0] + Ja[1] * hb[1] + Ja[2] * hb[2];
    }
    AT L[M][M];
    psd_cholesky<M>(A, L);
    AT* re = rec + (size_t)i * RSY;
    AT* ge = grec + (size_t)i * RSG;
#pragma unroll
    for (int k = 0; k < DC; ++k) {
#pragma unroll
      for (int a = 0; a < M; ++a) {           // K[a][k] = sum_{b >= a} L[b][a] Jc[b][k]
        AT v = L[a][a] * row[a * DC + k];
#pragma unroll
        for (int b = a + 1; b < M; ++b) v += L[b][a] * row[b * DC + k];
        re[k * M + a] = v;
      }
      AT s = row[k] * qe[0];
#pragma unroll
      for (int a = 1; a < M; ++a) s += row[a * DC + k] * qe[a];
      ge[k] = s;
    }
  }
  __syncthreads();

  slot_rows<Mo, AT, AT, RSY, RSG>(d, cr, rec, grec, srt, reinterpret_cast<AT*>(d.partB), &next_slot);
}

// ---------------------------------------------------------------- camera blocks + PCG start

// One warp per camera: reduces the slot partials into H_cc, b_c and the Schur
// terms, adds the camera-side edges' blocks, forms H_cc + lambda D_c, S_cc, g_c and
// M_c = S_cc^-1, and starts the PCG (x = 0, r = g, z = M g, p = z).  The last CTA
// reduces r^T z and |r|^2.
template <class Mo, class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_cam_finalize(LaunchSet ls) {
  using Dm = Dims<Mo>;
  constexpr int DB = Mo::DB, DC = Mo::DC, TC = Dm::TC, TB = Dm::TB, NG = Dm::NG, NPA = Dm::NPA;
  constexpr int NHX = Mo::kExtra ? TB + DB : 1;
  __shared__ AT vals[kCamPerBlock][2 * NPA];
  __shared__ AT hx[kCamPerBlock][NHX];
  __shared__ AT Sf[kCamPerBlock][DB * DB];
  __shared__ double red[kCamPerBlock][2];
  GPO_BIND(cb, cbl)
  if (!d.sc->active) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = cbl * kCamPerBlock + warp;
  Scalars* sc = d.sc;
  const AT lam = (AT)sc->lambda;
  const AT* partA = reinterpret_cast<const AT*>(d.partA);
  const AT* partB = reinterpret_cast<const AT*>(d.partB);
  AT rz_c = (AT)0, rr_c = (AT)0;   // per-warp partials in AT, accumulated across warps in FP64
  if (c < d.C) {
    const int sa = d.cam_s_off[c], sb = d.cam_s_off[c + 1];
    // 2 NG groups of nine outputs; lanes stride over the camera's slots, then a fixed
    // shuffle tree sums the lanes
    for (int grp = 0; grp < 2 * NG; ++grp) {
      const AT* base = (grp < NG ? partA : partB) + 9 * (grp % NG);
      AT acc[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[k] = (AT)0;
      for (int s = sa + lane; s < sb; s += 32) {
        const AT* src = base + (size_t)s * NPA;   // camera-major rows
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
    if constexpr (Mo::kExtra) {
      // diagonal blocks J_c^T J_c and gradients J_c^T r of the camera-side edges
      // touching c, in edge order (FP64 products, one rounding per edge)
      const int xa = d.xk_off[c], xb = d.xk_off[c + 1];
      for (int t = lane; t < TB + DB; t += 32) {
        int ti = 0, tj = 0;
        if (t < TB) tri_ij(DB, t, ti, tj);
        AT acc = (AT)0;
        for (int u = xa; u < xb; ++u) {
          const int code = d.xk_list[u], x = code >> 1, off = (code & 1) * DB;
          const double* J = d.xe_J + (size_t)x * kXJ;
          const int m = xrows(d.xe_kind[x]);
          double s = 0.0;
          if (t < TB) {
            for (int a = 0; a < m; ++a) s += J[a * kXCols + off + ti] * J[a * kXCols + off + tj];
          } else {
            const double* rx = d.xe_r + (size_t)x * kXRows;
            for (int a = 0; a < m; ++a) s += J[a * kXCols + off + (t - TB)] * rx[a];
          }
          acc += (AT)s;
        }
        hx[warp][t] = acc;
      }
      // off-diagonal blocks H_ij = J_i^T J_j of the two-keyframe edges whose first
      // keyframe is c (read by the camera half of the Schur product)
      AT* xH = reinterpret_cast<AT*>(d.xe_H);
      for (int u = xa; u < xb; ++u) {
        const int code = d.xk_list[u], x = code >> 1;
        if ((code & 1) || d.xe_j[x] < 0) continue;
        const double* J = d.xe_J + (size_t)x * kXJ;
        const int m = xrows(d.xe_kind[x]);
        for (int t = lane; t < DB * DB; t += 32) {
          const int a = t / DB, b = t - a * DB;
          double s = 0.0;
          for (int r = 0; r < m; ++r) s += J[r * kXCols + a] * J[r * kXCols + DB + b];
          xH[(size_t)x * DB * DB + t] = (AT)s;
        }
      }
    }
    __syncwarp();
    AT* Hcl = reinterpret_cast<AT*>(d.Hcl) + (size_t)c * TB;
    AT* S = reinterpret_cast<AT*>(d.S) + (size_t)c * TB;
    AT* Mi = reinterpret_cast<AT*>(d.Minv) + (size_t)c * TB;
    // H_cc + lambda D_c and S_cc, entry by entry: the slot partials fill the first DC
    // coordinates of the block, the camera-side edges all of it
    for (int t = lane; t < TB; t += 32) {
      int ti, tj;
      tri_ij(DB, t, ti, tj);
      const bool obs = ti < DC && tj < DC;
      const int tc = obs ? tri_idx(DC, ti, tj) : 0;
      AT h = (AT)0;
      if constexpr (Mo::kExtra) h = hx[warp][t];
      if (obs) h += vals[warp][tc];
      if (ti == tj) h += lam * damp_diag(h, sc);
      Hcl[t] = h;
      const AT hc = h;
      if (obs) h -= vals[warp][NPA + tc];
      S[t] = h;
      // preconditioner block: S_cc^-1, or (H_cc + lambda D_c)^-1 for the full system
      const AT hm = sc->full ? hc : h;
      Sf[warp][ti * DB + tj] = hm;
      Sf[warp][tj * DB + ti] = hm;
    }
    __syncwarp();
    warp_spd_inverse<DB>(Sf[warp], Mi, lane);
    __syncwarp();
    AT* g = reinterpret_cast<AT*>(d.g) + DB * (size_t)c;
    AT* bc = reinterpret_cast<AT*>(d.bc) + DB * (size_t)c;
    if (lane < DB) {
      AT bi = (AT)0, si = (AT)0;
      if (lane < DC) {
        bi = vals[warp][TC + lane];
        si = vals[warp][NPA + TC + lane];
      }
      if constexpr (Mo::kExtra) bi += hx[warp][TB + lane];
      const AT gi = sc->full ? -bi : -bi + si;   // full system: the camera rows of -b
      g[lane] = gi;
      bc[lane] = bi;
      reinterpret_cast<AT*>(d.x)[DB * (size_t)c + lane] = (AT)0;
      reinterpret_cast<AT*>(d.xbest)[DB * (size_t)c + lane] = (AT)0;
      reinterpret_cast<AT*>(d.r)[DB * (size_t)c + lane] = gi;
    }
    __syncwarp();
    if (lane < DB) {
      AT zi = (AT)0;
      for (int j = 0; j < DB; ++j) zi += Mi[sym_idx(DB, lane, j)] * g[j];
      reinterpret_cast<AT*>(d.z)[DB * (size_t)c + lane] = zi;
      reinterpret_cast<AT*>(d.p)[DB * (size_t)c + lane] = (AT)0;   // p_{-1}: p_0 = z_0
      const AT gi = g[lane];
      rz_c = gi * zi;
      rr_c = gi * gi;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rz_c += __shfl_down_sync(0xffffffffu, rz_c, o);
    rr_c += __shfl_down_sync(0xffffffffu, rr_c, o);
  }
  if (lane == 0) {
    red[warp][0] = (double)rz_c;
    red[warp][1] = (double)rr_c;
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
  if (sc->full) {   // the point rows, started by k_full_init
    double rzq, rrq;
    __syncthreads();
    sum_partials(d.pt_part, point_blocks(d), rzq, rrq);
    rz += rzq;
    rr += rrq;
  }
  if (threadIdx.x == 0) {
    const double gn = sqrt(rr);
    sc->rz = rz;
    sc->gnorm = gn;
    sc->rnorm = gn;
    sc->rmin = gn;
    sc->sigma = 1.0;
    sc->inv_n = 1.0;
    sc->beta = 0.0;
    sc->inv_n_f = 1.0f;
    sc->beta_f = 0.0f;
    sc->pidx = 0;
    sc->pcg_it = 0;
    sc->pcg_products = 0;
    sc->restart = 0;
    sc->use_best = 0;
    sc->save_best = 0;
    sc->tol_abs = sc->pcg_rel ? sc->pcg_tol * gn : sc->pcg_tol;
    sc->pcg_done = (rr == 0.0 || !(rz > 0.0) || !isfinite(rz)) ? 1 : 0;
    // a nonzero right-hand side with r^T M r not positive: the preconditioner is not
    // positive definite at this damping, so no step can be taken
    sc->pcg_fail = (rr > 0.0 && (!(rz > 0.0) || !isfinite(rz))) ? 1 : 0;
    sc->pcg_breakdown = 0;
    sc->have_best = 0;
    if (!sc->pcg_done) atomicAdd(ls.running, 1);
    sc->ticket = 0u;
  }
}

// ---------------------------------------------------------------- PCG

// y_c = (H_cc + lambda D_c) p_c - sum_slots v (+ the camera-side edges' off-diagonal
// products), four warps per camera (each sums a quarter of the camera's slot
// partials and of its camera-side edges; the quarters are added in a fixed order).  The CTAs of camera block b
// are 4b .. 4b + 3, two cameras each.  The last CTA of the problem reduces p^T y and
// sets alpha = r^T z / p^T y.
constexpr int kApplySplit = 4;
template <class Mo, class AT>
struct ApplyShared {
  double red[kCamPerBlock];
  AT quarter[kCamPerBlock][Mo::DC];
  AT qx[Mo::kExtra ? kCamPerBlock : 1][Mo::DB];
};
// The camera a warp of a camera-half unit works on (CTA-part `part` of camera block cbl:
// two cameras, four warps each), and its slot range, a schedule table the host writes
// before the launches (so a launch may read it before it waits for its predecessor).
__device__ __forceinline__ int unit_camera(int cbl, int part) {
  return cbl * kCamPerBlock + part * (kCamPerBlock / kApplySplit) + (int)(threadIdx.x >> 5) / kApplySplit;
}
__device__ __forceinline__ int2 cam_slot_range(const DevBA& d, int cbl, int part) {
  const int c = unit_camera(cbl, part);
  return c < d.C ? make_int2(d.cam_s_off[c], d.cam_s_off[c + 1]) : make_int2(0, 0);
}
// One unit of the camera half: CTA-part `part` of camera block cbl of the problem bound
// in d, sr the warp's camera's slot range (every thread calls; returns uniformly).
// kFused: the unit stops after writing its p^T y partial; alpha is formed after the
// fused kernel's grid barrier by every CTA of the update (the same partials summed in
// the same order, so the same value).
template <class Mo, class AT, bool kFused = false>
__device__ void cam_apply_body(const LaunchSet& ls, const DevBA& d, int cbl, int part, ApplyShared<Mo, AT>& S,
                               int2 sr) {
  constexpr int DB = Mo::DB, DC = Mo::DC, TB = Dims<Mo>::TB;
  double* red = S.red;
  auto& quarter = S.quarter;
  auto& qx = S.qx;
  Scalars* sc = d.sc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = unit_camera(cbl, part);
  const int q = warp % kApplySplit;                                // quarter of the slots
  const int sa = sr.x, sb = sr.y;
  // The unit's loads are issued before any is used (one round trip): the solve's flags
  // and scalars, the camera's slot partials, and for the camera's first warp the
  // direction's inputs under either choice of restart (z, x and both direction
  // buffers) and, in the fused FP32 kernel (registers to spare), its row of the damped
  // block (the other forms load that row once the slot sums are in).
  constexpr bool kEarlyH = kFused && sizeof(AT) == 4;
  const int active = sc->active, done = sc->pcg_done, restart = sc->restart, pidx = sc->pidx;
  const AT beta_a = sc_beta<AT>(sc), inv_n_a = sc_inv_n<AT>(sc);
  const int full = sc->full, save_best = sc->save_best;
  const bool lead = c < d.C && q == 0 && lane < DB;
  const AT* H = reinterpret_cast<const AT*>(d.Hcl) + (size_t)(c < d.C ? c : 0) * TB;
  AT hrow[kEarlyH ? DB : 1];
  AT zc = (AT)0, xc = (AT)0, pc0 = (AT)0, pc1 = (AT)0;
  if (lead) {
    if constexpr (kEarlyH) {
#pragma unroll
      for (int j = 0; j < DB; ++j) hrow[j] = H[sym_idx(DB, lane, j)];
    }
    const size_t o = DB * (size_t)c + lane;
    zc = reinterpret_cast<const AT*>(d.z)[o];
    xc = reinterpret_cast<const AT*>(d.x)[o];
    pc0 = reinterpret_cast<const AT*>(d.p)[o];
    pc1 = reinterpret_cast<const AT*>(d.p2)[o];
  }
  AT acc[DC];
#pragma unroll
  for (int k = 0; k < DC; ++k) acc[k] = (AT)0;
  if (c < d.C) {   // warp-uniform
    const AT* partV = reinterpret_cast<const AT*>(d.partV);
#pragma unroll 4
    for (int s = sa + q * 32 + lane; s < sb; s += 32 * kApplySplit) {
      const AT* src = partV + (size_t)s * DC;   // camera-major rows
#pragma unroll
      for (int k = 0; k < DC; ++k) acc[k] += src[k];
    }
  }
  if (!active || done) return;
  // the vector the product is taken of: the direction p = (z + beta p_old) / n, or in a
  // restart iteration the current solution x (read as (x + 0 x) / 1, exactly x)
  const AT* z_all = reinterpret_cast<const AT*>(restart ? d.x : d.z);
  const AT* pold_all = restart ? z_all : reinterpret_cast<const AT*>(pidx ? d.p2 : d.p);
  const AT beta = restart ? (AT)0 : beta_a, inv_n = restart ? (AT)1 : inv_n_a;
  AT dot = (AT)0;   // per-warp partial in AT, accumulated across warps in FP64
  AT pi = (AT)0;
  if (c < d.C) {   // warp-uniform
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < DC; ++k) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < DC; ++k) quarter[warp][k] = acc[k];
    }
    if constexpr (Mo::kExtra) {
      // H_co p_o of the two-keyframe edges joining c to another keyframe o, the
      // camera's edges dealt round-robin to its four warps
      const AT* xH = reinterpret_cast<const AT*>(d.xe_H);
      AT ex = (AT)0;
      for (int u = d.xk_off[c] + q; u < d.xk_off[c + 1]; u += kApplySplit) {
        const int code = d.xk_list[u], x = code >> 1, side = code & 1;
        const int o = side ? d.xe_i[x] : d.xe_j[x];
        if (o < 0) continue;   // unary edge: diagonal only
        const AT* H = xH + (size_t)x * DB * DB;
        const AT po = lane < DB ? (z_all[DB * (size_t)o + lane] + beta * pold_all[DB * (size_t)o + lane]) * inv_n : (AT)0;
#pragma unroll
        for (int k = 0; k < DB; ++k) {
          const AT pk = __shfl_sync(0xffffffffu, po, k);
          if (lane < DB) ex += (side ? H[k * DB + lane] : H[lane * DB + k]) * pk;   // H_ij or H_ij^T
        }
      }
      if (lane < DB) qx[warp][lane] = ex;
    }
  }
  __syncthreads();
  if (c < d.C && q == 0) {
    AT sv = (AT)0;
    if (lane < DC) {
      sv = quarter[warp][lane];
      for (int j = 1; j < kApplySplit; ++j) sv += quarter[warp + j][lane];
    }
    // p_k = (z_k + beta_k p_{k-1}) / n_k for this camera (the same values the Schur
    // product gathered), written to the other direction buffer
    AT* pnew = reinterpret_cast<AT*>(pidx ? d.p : d.p2) + DB * (size_t)c;
    const AT zsel = restart ? xc : zc, psel = restart ? xc : (pidx ? pc1 : pc0);
    pi = lane < DB ? (zsel + beta * psel) * inv_n : (AT)0;
    if (lane < DB) {
      if (!restart) pnew[lane] = pi;
      if (save_best) reinterpret_cast<AT*>(d.xbest)[DB * (size_t)c + lane] = xc;
    }
    AT yi = (AT)0;
#pragma unroll
    for (int j = 0; j < DB; ++j) {
      const AT pj = __shfl_sync(0xffffffffu, pi, j);
      if constexpr (kEarlyH) {
        if (lane < DB) yi += hrow[j] * pj;
      } else {
        if (lane < DB) yi += H[sym_idx(DB, lane, j)] * pj;
      }
    }
    if constexpr (Mo::kExtra) {
      if (lane < DB)
        for (int j = 0; j < kApplySplit; ++j) yi += qx[warp + j][lane];
    }
    if (lane < DB) {
      // the Schur complement subtracts the points' coupling; the full system's product
      // adds the edges' coupling terms J_c^T J_p v_p
      if (full) yi += sv;
      else yi -= sv;
      reinterpret_cast<AT*>(d.y)[DB * (size_t)c + lane] = yi;
      dot = pi * yi;
    }
  }
  if (restart) return;   // S x needs no alpha (uniform for the CTA)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
  if (lane == 0) red[warp] = (double)dot;
  __syncthreads();
  const int ctas = d.ncblk * kApplySplit, me = cbl * kApplySplit + part;
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < kCamPerBlock; ++w) a += red[w];
    d.cblk_part[2 * me] = a;
    d.cblk_part[2 * me + 1] = 0.0;
  }
  if constexpr (kFused) return;
  if (!last_cta(&sc->ticket, ctas)) return;
  double pAp = sum_partials_first(d.cblk_part, ctas);
  if (sc->full) pAp += sum_singles(d.md_part, d.NCH);   // the points' p^T H p, per chunk
  if (threadIdx.x == 0) {
    sc->pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) {
      sc->alpha = 0.0;
      sc->pcg_done = 1;
      // p^T S p not positive: S is not positive definite at this damping
      if (sc->pcg_it == 0) sc->pcg_fail = 1;
      else sc->pcg_breakdown = 1;
      atomicSub(ls.running, 1);
    } else {
      sc->alpha = sc->rz / pAp;
    }
    sc->ticket = 0u;
  }
}

template <class Mo, class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_cam_apply(LaunchSet ls) {
  __shared__ ApplyShared<Mo, AT> S;
  __shared__ DevBA d;
  pdl_trigger();
  const int cb = blockIdx.x / kApplySplit, part = blockIdx.x % kApplySplit;
  const int prob_ = ls.nprob == 1 ? 0 : ls.cb_prob[cb];
  const int cbl = ls.nprob == 1 ? cb : cb - ls.cb_base[prob_];
  bind_problem(d, ls.probs + prob_);
  const int2 sr = cam_slot_range(d, cbl, part);
  pdl_wait();
  cam_apply_body<Mo, AT>(ls, d, cbl, part, S, sr);
}

// The update's inputs that the camera half does not write (the fused kernel loads
// them before its grid barrier): the camera's row of M, r, g and x.  (The direction p
// and y = S p are the camera half's outputs.)
template <class Mo, class AT>
struct UpdateIn {
  AT r0, g0, x0, mrow[Mo::DB];
};
template <class Mo, class AT>
__device__ __forceinline__ void pcg_update_load(const DevBA& d, int cbl, UpdateIn<Mo, AT>& in) {
  constexpr int DB = Mo::DB, TB = Dims<Mo>::TB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = cbl * kCamPerBlock + warp;
  in.r0 = in.g0 = in.x0 = (AT)0;
#pragma unroll
  for (int j = 0; j < DB; ++j) in.mrow[j] = (AT)0;
  if (c < d.C && lane < DB) {
    const AT* Mi = reinterpret_cast<const AT*>(d.Minv) + (size_t)c * TB;
    const size_t o = DB * (size_t)c + lane;
    in.r0 = reinterpret_cast<const AT*>(d.r)[o];
    in.g0 = reinterpret_cast<const AT*>(d.g)[o];
    in.x0 = reinterpret_cast<const AT*>(d.x)[o];
#pragma unroll
    for (int j = 0; j < DB; ++j) in.mrow[j] = Mi[sym_idx(DB, lane, j)];
  }
}

// The end of a PCG update, reached by every CTA of the update after writing its
// partial (r^T z, |r|^2): the last one of the problem sums the camera blocks' partials
// (and, in the full-system form, the point blocks' after them), applies the stopping
// rules (tolerance, rejection ratio, iteration cap) and computes beta and the
// normalisation factor.
__device__ inline void pcg_update_finish(const LaunchSet& ls, const DevBA& d, int restart) {
  Scalars* sc = d.sc;
  const int full = sc->full;
  const int npb = full ? update_point_blocks(d.P) : 0;   // the update's point CTAs
  if (!last_cta(&sc->ticket, d.ncblk + npb)) return;
  // the solve's state, read by thread 0 in one batch while the partials are summed (read
  // one at a time between the writes below, they were a chain of dependent round trips)
  double sigma = 0.0, rmin = 0.0, ratio = 0.0, tol_abs = 0.0, rz_old = 0.0;
  int pcg_it = 0, max_it = 0, normalize = 0, restart_every = 0, pidx = 0, pcg_total = 0, pcg_products = 0;
  if (threadIdx.x == 0) {
    sigma = sc->sigma;
    rmin = sc->rmin;
    ratio = sc->ratio;
    tol_abs = sc->tol_abs;
    rz_old = sc->rz;
    pcg_it = sc->pcg_it;
    max_it = sc->max_it;
    normalize = sc->normalize;
    restart_every = sc->restart_every;
    pidx = sc->pidx;
    pcg_total = sc->pcg_total;
    pcg_products = sc->pcg_products;
  }
  double rz, rr;
  sum_partials(d.cblk_part + 2 * kApplySplit * (size_t)d.ncblk, d.ncblk, rz, rr);
  if (full) {
    double rzq, rrq;
    __syncthreads();   // every thread has read the first sums out of the shared tree
    sum_partials(d.pt_part, npb, rzq, rrq);
    rz += rzq;
    rr += rrq;
  }
  if (threadIdx.x == 0) {
    const double n = sqrt(rr);
    if (restart) sigma = 1.0;                // r is now the true residual
    const double rtrue = sigma * n;
    if (!restart) pcg_it += 1;               // a restart is an extra product, not an iteration
    int done = 0, save_best = 0, have_best = 0, use_best = 0, breakdown = 0;
    if (ratio > 0.0) {
      if (rtrue < rmin) {
        rmin = rtrue;
        save_best = 1;
        have_best = 1;
      } else if (rtrue > ratio * rmin) {
        done = 1;
        use_best = 1;
      }
    }
    if (rtrue <= tol_abs || pcg_it >= max_it || !isfinite(rtrue) || !(rz > 0.0)) {
      done = 1;
      if (!isfinite(rtrue)) use_best = 1;
      // r^T M r not positive before the tolerance is met: the preconditioned system is
      // not positive definite at this damping (after at least one step)
      if (!(rz > 0.0) && !(rtrue <= tol_abs)) breakdown = 1;
    }
    const double beta = restart ? 0.0 : rz / rz_old;   // a restart starts the direction from z
    double inv_n, rz_new;
    if (normalize && n > 0.0) {
      inv_n = 1.0 / n;
      sigma *= n;
      rz_new = rz / (n * n);
    } else {
      inv_n = 1.0;
      rz_new = rz;
    }
    sc->sigma = sigma;
    sc->pcg_it = pcg_it;
    sc->pcg_total = pcg_total + 1;
    sc->pcg_products = pcg_products + 1;
    sc->rnorm = rtrue;
    sc->rmin = rmin;
    sc->save_best = save_best;
    if (have_best) sc->have_best = 1;
    if (use_best) sc->use_best = 1;
    if (breakdown) sc->pcg_breakdown = 1;
    sc->beta = beta;
    sc->inv_n = inv_n;
    sc->rz = rz_new;
    sc->beta_f = (float)beta;
    sc->inv_n_f = (float)inv_n;
    if (!restart) sc->pidx = pidx ^ 1;       // a restart wrote no new direction
    sc->restart = (!done && !restart && restart_every > 0 && pcg_it % restart_every == 0) ? 1 : 0;
    sc->pcg_done = done;
    if (done) atomicSub(ls.running, 1);
    sc->ticket = 0u;
  }
}

// One warp per camera: x += sigma alpha p, r -= alpha y, z = M r; the last CTA of
// the problem reduces r^T z and |r|^2, applies the stopping rules (tolerance,
// rejection ratio, iteration cap) and computes beta and the normalisation factor.
// Its partials sit after the camera half's (which the fused form still reads here).
// kFused: alpha = r^T z / p^T y is formed here from the camera half's partials (every
// CTA the same value; camera block 0 records it, or stops a solve whose p^T y is not
// positive, as the camera half's last CTA does in the separate launches).
template <class Mo, class AT, bool kFused = false>
__device__ void pcg_update_body(const LaunchSet& ls, const DevBA& d, int cbl, double (*red)[2],
                                const UpdateIn<Mo, AT>& in) {
  constexpr int DB = Mo::DB;
  Scalars* sc = d.sc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = cbl * kCamPerBlock + warp;
  const bool mine = c < d.C && lane < DB;
  const AT y0 = mine ? reinterpret_cast<const AT*>(d.y)[DB * (size_t)c + lane] : (AT)0;
  const AT p0 = mine ? reinterpret_cast<const AT*>(sc->pidx ? d.p : d.p2)[DB * (size_t)c + lane] : (AT)0;
  if constexpr (kFused) {
    // one thread reads the flags for the CTA: camera block 0 may stop the solve (p^T S p
    // not positive) while other blocks read them, and the CTA's threads must agree
    __shared__ int stop_s;
    if (threadIdx.x == 0) stop_s = !sc->active || sc->pcg_done;
    __syncthreads();
    if (stop_s) return;
  } else if (!sc->active || sc->pcg_done) {
    return;
  }
  // a restart iteration: y = S x at the current solution, and the residual becomes the
  // true one, g - S x (unit scale), with the direction restarted from z = M r
  const int restart = sc->restart;
  // The step's scalars in FP64 by one thread, shared in AT (the FP64 pipe is a small
  // fraction of the FP32 one: no thread repeats the division).
  __shared__ AT coef[3];   // alpha, sigma alpha, 1 / n
  __shared__ int bad_s;
  double pAp = 0.0;
  if constexpr (kFused) {
    if (!restart) pAp = sum_partials_first(d.cblk_part, d.ncblk * kApplySplit);
  }
  if (threadIdx.x == 0) {
    double alpha_d;
    int bad = 0;
    if constexpr (kFused) {
      if (sc->pcg_done) {   // stopped by camera block 0 since the check above
        bad = 1;
        alpha_d = 0.0;
      } else if (!restart) {
        bad = !(pAp > 0.0) || !isfinite(pAp);
        alpha_d = bad ? 0.0 : sc->rz / pAp;
        if (cbl == 0) {
          sc->pAp = pAp;
          sc->alpha = alpha_d;
          if (bad) {
            sc->pcg_done = 1;
            // p^T S p not positive: S is not positive definite at this damping
            if (sc->pcg_it == 0) sc->pcg_fail = 1;
            else sc->pcg_breakdown = 1;
            atomicSub(ls.running, 1);
          }
        }
      } else {
        alpha_d = 0.0;
      }
    } else {
      alpha_d = sc->alpha;
    }
    coef[0] = (AT)alpha_d;
    coef[1] = (AT)(sc->sigma * alpha_d);
    coef[2] = sc_inv_n<AT>(sc);
    bad_s = bad;
  }
  __syncthreads();
  if (bad_s) return;
  AT rz_c = (AT)0, rr_c = (AT)0;   // per-warp partials in AT, accumulated across warps in FP64
  if (c < d.C) {   // warp-uniform
    const AT alpha = coef[0], sa = coef[1], sn = coef[2];
    AT* x = reinterpret_cast<AT*>(d.x) + DB * (size_t)c;
    AT* r = reinterpret_cast<AT*>(d.r) + DB * (size_t)c;
    AT* z = reinterpret_cast<AT*>(d.z) + DB * (size_t)c;
    AT ri = (AT)0;
    if (lane < DB) {
      if (restart) {
        ri = in.g0 - y0;
      } else {
        x[lane] = in.x0 + sa * p0;
        ri = in.r0 * sn - alpha * y0;
      }
      r[lane] = ri;
    }
    AT zi = (AT)0;
#pragma unroll
    for (int j = 0; j < DB; ++j) {
      const AT rj = __shfl_sync(0xffffffffu, ri, j);
      if (lane < DB) zi += in.mrow[j] * rj;
    }
    if (lane < DB) {
      z[lane] = zi;
      rz_c = ri * zi;
      rr_c = ri * ri;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rz_c += __shfl_down_sync(0xffffffffu, rz_c, o);
    rr_c += __shfl_down_sync(0xffffffffu, rr_c, o);
  }
  if (lane == 0) {
    red[warp][0] = (double)rz_c;
    red[warp][1] = (double)rr_c;
  }
  __syncthreads();
  double* upart = d.cblk_part + 2 * kApplySplit * (size_t)d.ncblk;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kCamPerBlock; ++w) { a += red[w][0]; b += red[w][1]; }
    upart[2 * cbl] = a;
    upart[2 * cbl + 1] = b;
  }
  pcg_update_finish(ls, d, restart);
}
template <class Mo, class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_pcg_update(LaunchSet ls) {
  __shared__ double red[kCamPerBlock][2];
  GPO_BIND(cb, cbl)
  UpdateIn<Mo, AT> in;
  pcg_update_load<Mo, AT>(d, cbl, in);
  pcg_update_body<Mo, AT>(ls, d, cbl, red, in);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr unsigned long long kWaitNs = 1000000000ull;   // bounded waits give up after 1 s

// Grid-wide barrier of the persistent camera kernel (every CTA resident; called after a
// CTA barrier): thread 0 arrives with an acquire-release add, the last CTA to arrive
// resets the count and advances the generation with a release add, and the others
// wait for it with acquire loads.  The wait is bounded (kWaitNs of wall time); false if
// it gave up (the caller raises *ls.err).
__device__ __forceinline__ bool grid_sync(int* count, int* gen, int ctas) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned int* ucount = reinterpret_cast<unsigned int*>(count);
    unsigned int* ugen = reinterpret_cast<unsigned int*>(gen);
    const unsigned int g0 = ld_acquire(ugen);
    if (atom_add_acq_rel(ucount, 1u) == (unsigned int)ctas - 1u) {
      atomicExch(ucount, 0u);
      red_add_release(ugen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire(ugen) == g0) {
        if (global_ns() - t0 > kWaitNs) {
          ok = 0;
          break;
        }
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

// The camera half of the Schur product and the PCG update in one persistent launch
// (the production path; profiling times the two separately): each CTA runs one unit
// of the camera half (camera block, quarter), loads its update block's inputs that the
// camera half does not write, and meets the others at a grid barrier; then CTA b
// updates camera block b, every update CTA forming alpha from the camera half's
// partials itself (no ticket between the halves), and the last block of a problem
// applies the stopping rules and sets beta.  The same bodies and sums as k_cam_apply
// and k_pcg_update: bit-identical results.  Launched only when the
// camera half's units fit one wave of resident CTAs (one unit per CTA; the grid is
// then resident when the barrier waits); larger problems keep the two launches, whose
// many concurrent CTAs hide the units' latency better than a persistent loop.
template <class Mo, class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32, 4) k_pcg_camera(LaunchSet ls) {
  __shared__ ApplyShared<Mo, AT> S;
  __shared__ double red[kCamPerBlock][2];
  __shared__ DevBA d;
  pdl_trigger();
  const int G = gridDim.x, units = ls.n_cb * kApplySplit;
  int bound = -1;
  auto bind = [&](int q) {
    if (q != bound) {          // CTA-uniform
      __syncthreads();         // no thread still reads the previous descriptor
      bind_problem(d, ls.probs + q);
      bound = q;
    }
  };
  // the first unit's descriptor and slot ranges (host-written) before the wait
  int2 sr0 = make_int2(0, 0);
  if ((int)blockIdx.x < units) {
    const int cb = blockIdx.x / kApplySplit, q = ls.nprob == 1 ? 0 : ls.cb_prob[cb];
    bind(q);
    sr0 = cam_slot_range(d, ls.nprob == 1 ? cb : cb - ls.cb_base[q], blockIdx.x % kApplySplit);
  }
  pdl_wait();
  if (ls.nprob == 1) {
    // a stopped solve (the launches of a captured group after the stop): every CTA
    // returns before the grid barrier.  The flags change only after the barrier, so
    // every CTA reads the same values.
    __shared__ int stop;
    if (threadIdx.x == 0) {
      const Scalars* sc = ls.probs[0].sc;
      stop = !sc->active || sc->pcg_done;
    }
    __syncthreads();
    if (stop) return;
  }
  for (int u = blockIdx.x; u < units; u += G) {
    const int cb = u / kApplySplit, part = u % kApplySplit;
    const int q = ls.nprob == 1 ? 0 : ls.cb_prob[cb];
    bind(q);
    const int cbl = ls.nprob == 1 ? cb : cb - ls.cb_base[q];
    cam_apply_body<Mo, AT, true>(ls, d, cbl, part, S, u == (int)blockIdx.x ? sr0 : cam_slot_range(d, cbl, part));
    __syncthreads();
  }
  // the grid has one CTA per unit (n_cb * kApplySplit >= n_cb), so CTA b < n_cb updates
  // camera block b; its inputs that the camera half does not write are loaded first
  const int ucb = blockIdx.x;
  int ucbl = 0;
  UpdateIn<Mo, AT> in;
  if (ucb < ls.n_cb) {
    const int q = ls.nprob == 1 ? 0 : ls.cb_prob[ucb];
    bind(q);
    ucbl = ls.nprob == 1 ? ucb : ucb - ls.cb_base[q];
    pcg_update_load<Mo, AT>(d, ucbl, in);
  }
  if (!grid_sync(ls.work + 2, ls.work + 3, G + ls.debug_wait)) {
    if (threadIdx.x == 0) atomicExch(ls.err, 1);
    return;
  }
  if (ucb < ls.n_cb) pcg_update_body<Mo, AT, true>(ls, d, ucbl, red, in);
}

// ---------------------------------------------------------------- back-substitution

// One CTA per chunk: dp = H_pp^-1 (-b_p - sum_e Jp^T Jc dc) (the full-system PCG's
// point rows instead when it solved them) and the chunk's share of the model decrease
// -b_p^T dp - 1/2 sum_e |Jc dc + Jp dp|^2 (FP64 accumulation).
template <class Mo, class JT, bool kDyn = false>
__global__ void __launch_bounds__(kThreads) k_backsub(LaunchSet ls) {
  using AT = typename AccOf<JT>::T;
  using Dm = Dims<Mo>;
  constexpr int M = Mo::M, DC = Mo::DC, DB = Mo::DB, NJ = Mo::NJ, JP0 = Dm::JP0;
  __shared__ double red[kThreads];
  GPO_BIND(ch, kl)
  if (!d.sc->active) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int CH = d.ch_max;
  AT* qv = reinterpret_cast<AT*>(smem);   // [M][CH]
  AT* av = qv + M * CH;                   // [3][CH]
  const ChunkRange cr = chunk_range(d, kl);
  const JT* Jg = reinterpret_cast<const JT*>(d.J);
  const AT* xs = reinterpret_cast<const AT*>(d.sc->use_best ? d.xbest : d.x);
  const AT* Hinv = reinterpret_cast<const AT*>(d.Hinv);
  const AT* bp = reinterpret_cast<const AT*>(d.bp);
  AT* dp = reinterpret_cast<AT*>(d.dp);
  for (int i = threadIdx.x; i < cr.nE; i += kThreads) {
    const int c = __ldg(d.e_cam + cr.e0 + i);
    AT row[NJ];
    row_of<Mo, JT, AT, kDyn>(d, Jg, cr.e0 + i, row);
    AT q[M];
#pragma unroll
    for (int a = 0; a < M; ++a) q[a] = (AT)0;
#pragma unroll
    for (int k = 0; k < DC; ++k) {
      const AT xk = xs[DB * (size_t)c + k];
#pragma unroll
      for (int a = 0; a < M; ++a) q[a] += row[a * DC + k] * xk;
    }
#pragma unroll
    for (int a = 0; a < M; ++a) qv[a * CH + i] = q[a];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      AT s = row[JP0 + k] * q[0];
#pragma unroll
      for (int a = 1; a < M; ++a) s += row[JP0 + 3 * a + k] * q[a];
      av[k * CH + i] = s;
    }
  }
  __syncthreads();
  double md = 0.0;
  for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
    const int pj = cr.p0 + j;
    const int a0 = d.pt_off[pj] - cr.e0, b0 = d.pt_off[pj + 1] - cr.e0;
    AT u[3] = {0, 0, 0};
    for (int i = a0; i < b0; ++i) {
#pragma unroll
      for (int k = 0; k < 3; ++k) u[k] += av[k * CH + i];
    }
    AT hi[6], rhs[3], t[3];
    if (d.sc->full) {   // the full-system PCG solved the point rows itself
      const AT* xq = reinterpret_cast<const AT*>(d.sc->use_best ? d.xqbest : d.xq) + 3 * (size_t)pj;
#pragma unroll
      for (int k = 0; k < 3; ++k) t[k] = xq[k];
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) hi[k] = Hinv[6 * (size_t)pj + k];
#pragma unroll
      for (int k = 0; k < 3; ++k) rhs[k] = -bp[3 * (size_t)pj + k] - u[k];
      mul3(hi, rhs, t);
    }
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
    AT row[NJ];
    row_of<Mo, JT, AT, kDyn>(d, Jg, cr.e0 + i, row);
    double sq = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const double ja = (double)(qv[a * CH + i] + row[JP0 + 3 * a] * t0 + row[JP0 + 3 * a + 1] * t1 +
                                 row[JP0 + 3 * a + 2] * t2);
      sq += ja * ja;
    }
    md -= 0.5 * sq;
  }
  const double s = block_sum(md, red);
  if (threadIdx.x == 0) d.md_part[kl] = s;
}

// ---------------------------------------------------------------- retraction (FP64)

template <class Mo, class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_retract_cams(LaunchSet ls) {
  constexpr int SS = Mo::SS, DB = Mo::DB;
  GPO_BIND(cb, cbl)
  if (!d.sc->active) return;
  const int c = cbl * kCamPerBlock + (threadIdx.x >> 5);
  if (c >= d.C || (threadIdx.x & 31) != 0) return;
  const double* cur = d.cam + SS * (size_t)c;
  double* nxt = d.cam_cand + SS * (size_t)c;
  double* rb = d.camrb_cand + 16 * (size_t)c;
  float* rbf = d.camrbf_cand + 16 * (size_t)c;
  if (d.cam_fixed[c]) {
    for (int i = 0; i < SS; ++i) nxt[i] = cur[i];
    for (int i = 0; i < 16; ++i) rb[i] = d.camrb[16 * (size_t)c + i];
    for (int i = 0; i < 16; ++i) rbf[i] = d.camrbf[16 * (size_t)c + i];
    return;
  }
  const AT* xs = reinterpret_cast<const AT*>(d.sc->use_best ? d.xbest : d.x) + DB * (size_t)c;
  double dl[DB];
  for (int i = 0; i < DB; ++i) dl[i] = (double)xs[i];
  double cu[SS], nx[SS];
  for (int i = 0; i < SS; ++i) cu[i] = cur[i];
  Mo::retract(cu, dl, nx);
  for (int i = 0; i < SS; ++i) nxt[i] = nx[i];
  double r16[16];
  Mo::render(d, nx, r16);
  for (int i = 0; i < 16; ++i) rb[i] = r16[i];
  for (int i = 0; i < 16; ++i) rbf[i] = (float)r16[i];
}

template <class Mo, class AT>
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

template <class Mo, class AT>
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
  if constexpr (Mo::kExtra) {
    for (int x = threadIdx.x; x < d.NX; x += kThreads) {
      fc += d.xe_cost[x];
      md += d.xe_md[x];
    }
  }
  const AT* xs = reinterpret_cast<const AT*>(sc->use_best ? d.xbest : d.x);
  const AT* bc = reinterpret_cast<const AT*>(d.bc);
  for (int i = threadIdx.x; i < Mo::DB * d.C; i += kThreads) md -= (double)bc[i] * (double)xs[i];
  const double Fc = block_sum(fc, red);
  const double L = block_sum(md, red);
  if (threadIdx.x != 0) return;
  const double F = sc->cost;
  // a linear solve that broke down before its first step (the damped system is not
  // positive definite in the working precision), or whose best iterate is the zero
  // start, failed: the step is rejected and the damping grows (as a factorisation that
  // finds the damped system indefinite rejects the step in the oracle).  A solve that
  // broke down after a step returns a descent step, judged as any other, but the
  // damping that brought the system to the edge of definiteness is not lowered.
  const bool failed = sc->pcg_fail || (sc->use_best && !sc->have_best);
  const bool hold = sc->pcg_breakdown != 0;
  const bool acc = !failed && L > 0.0 && isfinite(Fc) && Fc < F;
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
    h.pcg_products = sc->pcg_products;
    h.pcg_failed = failed ? 1 : (hold ? 2 : 0);
  }
  double lam = sc->lambda, nu = sc->nu;
  if (acc) {
    const double t = 2.0 * rho - 1.0;
    if (!hold) lam *= fmax(1.0 / 3.0, 1.0 - t * t * t);
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

template <class Mo>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_commit_cams(LaunchSet ls) {
  GPO_BIND(cb, cbl)
  if (!d.sc->active || !d.sc->accepted) return;
  const int lane = threadIdx.x & 31;
  const int c = cbl * kCamPerBlock + (threadIdx.x >> 5);
  if (c >= d.C) return;
  if (lane < Mo::SS) d.cam[Mo::SS * (size_t)c + lane] = d.cam_cand[Mo::SS * (size_t)c + lane];
  if (lane < 16) d.camrb[16 * (size_t)c + lane] = d.camrb_cand[16 * (size_t)c + lane];
  if (lane < 16) d.camrbf[16 * (size_t)c + lane] = d.camrbf_cand[16 * (size_t)c + lane];
}

template <class Mo>
__global__ void __launch_bounds__(256) k_commit_pts(LaunchSet ls) {
  GPO_BIND(pb, pbl)
  if (!d.sc->active || !d.sc->accepted) return;
  const int p = pbl * 256 + threadIdx.x;
  if (p >= d.P) return;
  for (int k = 0; k < 3; ++k) d.pt[3 * (size_t)p + k] = d.pt_cand[3 * (size_t)p + k];
}

// ---------------------------------------------------------------- launchers

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

// Raises a kernel's dynamic shared-memory limit once per (device, kernel, size).
static void set_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static const void* keys[256];
  static int devs[256];
  static size_t vals[256];
  static int n = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < n; ++i)
    if (keys[i] == kernel && devs[i] == dev) {
      if (vals[i] >= bytes) return;
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      vals[i] = bytes;
      return;
    }
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (n < 256) { keys[n] = kernel; devs[n] = dev; vals[n] = bytes; ++n; }
}

}  // namespace gpo

#include "schur_full.cuh"
#include "autodiff.cuh"

namespace gpo {

// Shared-memory sizes and launchers of one model.
template <class Mo>
struct Launch {
  using Dm = Dims<Mo>;
  static size_t sJ(Prec pr) { return pr == Prec::F64 ? 8 : (pr == Prec::F32 ? 4 : 2); }
  static size_t sA(Prec pr) { return pr == Prec::F64 ? 8 : 4; }
  static size_t lin_rsy(Prec pr) {
    return pr == Prec::F64 ? LinRec<Mo, double>::RSY * 8
                           : (pr == Prec::F32 ? LinRec<Mo, float>::RSY * 4 : LinRec<Mo, __nv_bfloat16>::RSY * 2);
  }
  static size_t lin_smem(Prec pr, int ch) {
    return (LinRec<Mo, float>::RSG * sA(pr) + lin_rsy(pr) + 2) * (size_t)ch;
  }
  // np = most points of a chunk (the point records); np = ch bounds any chunk
  static size_t schur_smem(Prec pr, int ch, int np) {
    const size_t rsy = pr == Prec::F64 ? SchurRec<Mo, double>::RSY : SchurRec<Mo, float>::RSY;
    return ((rsy + SchurRec<Mo, float>::RSG) * sA(pr) + 2) * (size_t)ch + 9 * sA(pr) * (size_t)np;
  }
  static size_t spmv_smem(Prec pr, const LaunchSet& ls) {
    return sA(pr) * ((Dm::VW + 3) * (size_t)(ls.ch_max + 1) + Mo::DC * (size_t)ls.ns_max + 6 * (size_t)ls.np_max) +
           4 * (size_t)(ls.np_max + 2 * ls.ns_max + 2);
  }
  static size_t backsub_smem(Prec pr, int ch) { return (Mo::M + 3) * sA(pr) * (size_t)ch; }
  static size_t full_smem(Prec pr, const LaunchSet& ls) {
    return sA(pr) * ((Mo::DC + 3) * (size_t)(ls.ch_max + 1) + Mo::DC * (size_t)ls.ns_max + 3 * (size_t)ls.np_max) +
           4 * (size_t)(ls.np_max + 2 * ls.ns_max + 2);
  }
  static int full_init(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (ls.n_pb == 0) return 0;
    if (pr == Prec::F64) launch_pdl(k_full_init<Mo, double>, ls.n_pb, 256, 0, st, ls);
    else launch_pdl(k_full_init<Mo, float>, ls.n_pb, 256, 0, st, ls);
    return 1;
  }
  template <class JT>
  static void full_spmv_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const size_t sm = full_smem(pr, ls);
    set_smem(reinterpret_cast<const void*>(k_full_spmv<Mo, JT>), sm);
    launch_pdl(k_full_spmv<Mo, JT>, ls.n_ch, kThreads, sm, st, ls);
  }
  static int full_spmv(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (ls.n_ch == 0) return 0;
    if (pr == Prec::F64) full_spmv_t<double>(ls, pr, st);
    else if (pr == Prec::F32) full_spmv_t<float>(ls, pr, st);
    else full_spmv_t<__nv_bfloat16>(ls, pr, st);
    return 1;
  }
  static int autodiff(const LaunchSet& ls, int n_edges, double* r, double* J, cudaStream_t st) {
    if (n_edges <= 0) return 0;
    launch_pdl(k_autodiff<Mo>, (n_edges + 255) / 256, 256, 0, st, ls, r, J);
    return 1;
  }
  static int full_update(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const int n = ls.n_cb + (ls.n_pb > 0 ? update_point_blocks(ls.n_pb * 256) : 0);
    if (n == 0) return 0;
    if (pr == Prec::F64) launch_pdl(k_full_update<Mo, double>, n, kCamPerBlock * 32, 0, st, ls);
    else launch_pdl(k_full_update<Mo, float>, n, kCamPerBlock * 32, 0, st, ls);
    return 1;
  }
  static int max_supported_ch(Prec pr) {
    // largest chunk whose linearisation tile fits the 227 KB opt-in shared memory
    const size_t limit = 227 * 1024;
    int ch = 64;
    while (lin_smem(pr, ch * 2) <= limit && schur_smem(pr, ch * 2, ch * 2) <= limit) ch *= 2;
    return ch;
  }

  static int cam_prepare(const LaunchSet& ls, bool candidate, cudaStream_t st) {
    if (ls.n_cb == 0) return 0;
    launch_pdl(k_cam_prepare<Mo>, ls.n_cb, kCamPerBlock * 32, 0, st, ls, candidate ? 1 : 0);
    return 1;
  }
  static int cost(const LaunchSet& ls, bool candidate, cudaStream_t st) {
    if (ls.n_ch == 0) return 0;
    launch_pdl(k_cost<Mo>, ls.n_ch, kThreads, 0, st, ls, candidate ? 1 : 0);
    return 1;
  }
  static int cost_init(const LaunchSet& ls, cudaStream_t st) {
    launch_pdl(k_cost_init<Mo>, ls.nprob, kThreads, 0, st, ls);
    return 1;
  }
  template <class JT>
  static void lin_t(const LaunchSet& ls, Prec pr, bool force, cudaStream_t st) {
    const size_t sm = lin_smem(pr, ls.ch_max);
    set_smem(reinterpret_cast<const void*>(k_linearize<Mo, JT>), sm);
    launch_pdl(k_linearize<Mo, JT>, ls.n_ch, kThreads, sm, st, ls, force ? 1 : 0);
  }
  static int linearize(const LaunchSet& ls, Prec pr, bool force, cudaStream_t st) {
    if (ls.n_ch == 0) return 0;
    if (pr == Prec::F64) lin_t<double>(ls, pr, force, st);
    else if (pr == Prec::F32) lin_t<float>(ls, pr, force, st);
    else lin_t<__nv_bfloat16>(ls, pr, force, st);
    return 1;
  }
  // Dynamic Jacobians (spmv_variant 4) keep no rows: the per-edge kernels evaluate them.
  static bool dyn_rows(const LaunchSet& ls) { return ls.spmv_variant == 4; }
  template <class JT, bool kDyn>
  static void schur_k(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const size_t sm = schur_smem(pr, ls.ch_max, ls.np_max);
    set_smem(reinterpret_cast<const void*>(k_schur_prepare<Mo, JT, kDyn>), sm);
    launch_pdl(k_schur_prepare<Mo, JT, kDyn>, ls.n_ch, kThreads, sm, st, ls);
  }
  template <class JT>
  static void schur_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (dyn_rows(ls)) schur_k<JT, true>(ls, pr, st);
    else schur_k<JT, false>(ls, pr, st);
  }
  static int schur_prepare(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (ls.n_ch == 0) return 0;
    if (pr == Prec::F64) schur_t<double>(ls, pr, st);
    else if (pr == Prec::F32) schur_t<float>(ls, pr, st);
    else schur_t<__nv_bfloat16>(ls, pr, st);
    return 1;
  }
  static int cam_finalize(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (ls.n_cb == 0) return 0;
    if (pr == Prec::F64) launch_pdl(k_cam_finalize<Mo, double>, ls.n_cb, kCamPerBlock * 32, 0, st, ls);
    else launch_pdl(k_cam_finalize<Mo, float>, ls.n_cb, kCamPerBlock * 32, 0, st, ls);
    return 1;
  }
  template <class JT, int EPT>
  static void spmv_e(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const size_t sm = spmv_smem(pr, ls);
    set_smem(reinterpret_cast<const void*>(k_spmv<Mo, JT, EPT>), sm);
    launch_pdl(k_spmv<Mo, JT, EPT>, ls.n_ch, kThreads, sm, st, ls);
  }
  template <class JT>
  static void spmv_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const int ept = (ls.ch_max + kThreads - 1) / kThreads;
    if (ept <= 1) spmv_e<JT, 1>(ls, pr, st);
    else if (ept <= 2) spmv_e<JT, 2>(ls, pr, st);
    else if (ept <= 4) spmv_e<JT, 4>(ls, pr, st);
    else spmv_e<JT, 8>(ls, pr, st);
  }
  // Dynamic Jacobians: chunks of at most 512 edges (two per thread), else the classic
  // stored-row product runs.
  static bool dyn_ok(const LaunchSet& ls) { return ls.spmv_variant == 4 && ls.ch_max <= 2 * kThreads; }
  template <class AT, int EPT>
  static void dyn_e(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const size_t sm = spmv_smem(pr, ls);
    set_smem(reinterpret_cast<const void*>(k_spmv_dyn<Mo, AT, EPT>), sm);
    launch_pdl(k_spmv_dyn<Mo, AT, EPT>, ls.n_ch, kThreads, sm, st, ls);
  }
  template <class AT>
  static void dyn_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (ls.ch_max <= kThreads) dyn_e<AT, 1>(ls, pr, st);
    else dyn_e<AT, 2>(ls, pr, st);
  }
  static size_t ws_smem(Prec pr, const LaunchSet& ls) {
    const StageLayout L = stage_layout<Mo>(sJ(pr), sA(pr), ls.ch_max, ls.np_max, ls.ns_max);
    return kStages * (size_t)L.size + sA(pr) * (Dm::VW + 3) * (size_t)(ls.ch_max + 1);
  }
  // The staged kernel packs in-chunk positions in 10 bits and needs its stages to fit
  // the opt-in shared memory.
  static bool ws_ok(Prec pr, const LaunchSet& ls) {
    return ls.spmv_variant == 1 && ls.ch_max <= 1024 && ws_smem(pr, ls) <= 220 * 1024;
  }
  template <class JT>
  static void ws_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const size_t sm = ws_smem(pr, ls);
    set_smem(reinterpret_cast<const void*>(k_spmv_ws<Mo, JT>), sm);
    static int n_sm = 0;
    if (!n_sm) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      if (n_sm <= 0) n_sm = 1;
    }
    static size_t occ_sm = 0;   // occupancy for the last shared-memory size asked
    static int occ = 0;
    if (sm != occ_sm) {
      occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_ws<Mo, JT>, kWsThreads, sm);
      occ_sm = sm;
    }
    const int grid = std::max(1, std::min(ls.n_ch, n_sm * std::max(occ, 1)));
    launch_pdl(k_spmv_ws<Mo, JT>, grid, kWsThreads, sm, st, ls);
  }
  static size_t pp_smem(Prec pr, const LaunchSet& ls) {
    return pipe_layout<Mo>(sA(pr), ls.ch_max, ls.np_max, ls.ns_max).size;
  }
  // The pipelined kernel reads packed edge words (chunks of at most 1024 edges).  It is
  // the automatic choice for BF16 and FP32 storage (measured faster there; FP64 keeps
  // the classic kernel).
  static bool pp_ok(Prec pr, const LaunchSet& ls) {
    const bool want = ls.spmv_variant == 3 || (ls.spmv_variant == 0 && pr != Prec::F64);
    return want && ls.ch_max <= 1024 && pp_smem(pr, ls) <= 220 * 1024;
  }
  template <class JT, int EPT, int kCH = 0>
  static void pp_e(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const size_t sm = pp_smem(pr, ls);
    set_smem(reinterpret_cast<const void*>(k_spmv_pp<Mo, JT, EPT, kCH>), sm);
    static int n_sm = 0;
    if (!n_sm) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      if (n_sm <= 0) n_sm = 1;
    }
    static size_t occ_sm = 0;   // occupancy for the last shared-memory size asked
    static int occ = 0;
    if (sm != occ_sm) {
      occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_pp<Mo, JT, EPT, kCH>, kThreads, sm);
      occ_sm = sm;
    }
    const int grid = std::max(1, std::min(ls.n_ch, n_sm * std::max(occ, 1)));
    launch_pdl(k_spmv_pp<Mo, JT, EPT, kCH>, grid, kThreads, sm, st, ls);
  }
  // the default chunk bound (512 edges) has its own instantiation (compile-time strides)
  template <class JT>
  static void pp_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const int ept = (ls.ch_max + kThreads - 1) / kThreads;
    if (ls.ch_max == 2 * kThreads) pp_e<JT, 2, 2 * kThreads>(ls, pr, st);
    else if (ept <= 1) pp_e<JT, 1>(ls, pr, st);
    else if (ept <= 2) pp_e<JT, 2>(ls, pr, st);
    else pp_e<JT, 4>(ls, pr, st);
  }
  static size_t wg_smem(Prec pr, const LaunchSet& ls) {
    return wg_layout<Mo>(sA(pr), ls.ch_max, ls.ns_max).size;
  }
  // The warp-group kernel (spmv_variant 5) reads packed edge words (chunks of at most
  // 1024 edges) and keeps the rows in registers (BF16 or FP32 storage).
  static bool wg_ok(Prec pr, const LaunchSet& ls) {
    return ls.spmv_variant == 5 && pr != Prec::F64 && ls.ch_max <= 1024 && wg_smem(pr, ls) <= 200 * 1024;
  }
  template <class JT>
  static void wg_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const size_t sm = wg_smem(pr, ls);
    set_smem(reinterpret_cast<const void*>(k_spmv_wg<Mo, JT>), sm);
    struct Occ {
      std::atomic<int> n_sm{0}, occ{0};
      std::atomic<size_t> occ_sm{0};
    };
    static Occ cache[kMaxDevices];
    int dev = 0;
    cudaGetDevice(&dev);
    Occ& o = cache[dev >= 0 && dev < kMaxDevices ? dev : 0];
    if (!o.n_sm.load()) {
      int n = 0;
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
      o.n_sm.store(std::max(n, 1));
    }
    if (o.occ_sm.load() != sm) {
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_wg<Mo, JT>, kThreads, sm);
      o.occ.store(std::max(occ, 1));
      o.occ_sm.store(sm);
    }
    const int grid = std::max(1, std::min(ls.n_ch, o.n_sm.load() * o.occ.load()));
    launch_pdl(k_spmv_wg<Mo, JT>, grid, kThreads, sm, st, ls);
  }
  // The Schur-product kernel pcg_spmv dispatches for this launch set (spmv_variant
  // numbering: 1 staged, 2 classic, 3 pipelined, 4 dynamic, 5 warp groups).
  static size_t wgs_smem(Prec pr, const LaunchSet& ls) {
    const WgsLayout L = wgs_layout<Mo>(sJ(pr), sA(pr), ls.ch_max, ls.np_max, ls.ns_max);
    return kWgsStages * (size_t)L.size + sA(pr) * Dm::VW * (size_t)(ls.ch_max + 1);
  }
  // The staged warp-group kernel (spmv_variant 6): as 5, fed through shared-memory stages.
  static bool wgs_ok(Prec pr, const LaunchSet& ls) {
    return ls.spmv_variant == 6 && pr != Prec::F64 && ls.ch_max <= 1024 && wgs_smem(pr, ls) <= 220 * 1024;
  }
  template <class JT>
  static void wgs_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const size_t sm = wgs_smem(pr, ls);
    set_smem(reinterpret_cast<const void*>(k_spmv_wgs<Mo, JT>), sm);
    struct Occ {
      std::atomic<int> n_sm{0}, occ{0};
      std::atomic<size_t> occ_sm{0};
    };
    static Occ cache[kMaxDevices];
    int dev = 0;
    cudaGetDevice(&dev);
    Occ& o = cache[dev >= 0 && dev < kMaxDevices ? dev : 0];
    if (!o.n_sm.load()) {
      int n = 0;
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
      o.n_sm.store(std::max(n, 1));
    }
    if (o.occ_sm.load() != sm) {
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_wgs<Mo, JT>, kWsThreads, sm);
      o.occ.store(std::max(occ, 1));
      o.occ_sm.store(sm);
    }
    const int grid = std::max(1, std::min(ls.n_ch, o.n_sm.load() * o.occ.load()));
    launch_pdl(k_spmv_wgs<Mo, JT>, grid, kWsThreads, sm, st, ls);
  }
  static int spmv_kind(const LaunchSet& ls, Prec pr) {
    if (wgs_ok(pr, ls)) return 6;
    if (wg_ok(pr, ls)) return 5;
    if (dyn_ok(ls)) return 4;
    if (pp_ok(pr, ls)) return 3;
    if (ws_ok(pr, ls)) return 1;
    return 2;
  }
  static int pcg_spmv(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (ls.n_ch == 0) return 0;
    if (wgs_ok(pr, ls)) {
      if (pr == Prec::F32) wgs_t<float>(ls, pr, st);
      else wgs_t<__nv_bfloat16>(ls, pr, st);
      return 1;
    }
    if (wg_ok(pr, ls)) {
      if (pr == Prec::F32) wg_t<float>(ls, pr, st);
      else wg_t<__nv_bfloat16>(ls, pr, st);
      return 1;
    }
    if (dyn_ok(ls)) {
      if (pr == Prec::F64) dyn_t<double>(ls, pr, st);
      else dyn_t<float>(ls, pr, st);
      return 1;
    }
    if (pp_ok(pr, ls)) {
      if (pr == Prec::F64) pp_t<double>(ls, pr, st);
      else if (pr == Prec::F32) pp_t<float>(ls, pr, st);
      else pp_t<__nv_bfloat16>(ls, pr, st);
      return 1;
    }
    if (ws_ok(pr, ls)) {
      if (pr == Prec::F64) ws_t<double>(ls, pr, st);
      else if (pr == Prec::F32) ws_t<float>(ls, pr, st);
      else ws_t<__nv_bfloat16>(ls, pr, st);
      return 1;
    }
    if (pr == Prec::F64) spmv_t<double>(ls, pr, st);
    else if (pr == Prec::F32) spmv_t<float>(ls, pr, st);
    else spmv_t<__nv_bfloat16>(ls, pr, st);
    return 1;
  }
  static int cam_apply(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (ls.n_cb == 0) return 0;
    if (pr == Prec::F64) launch_pdl(k_cam_apply<Mo, double>, ls.n_cb * kApplySplit, kCamPerBlock * 32, 0, st, ls);
    else launch_pdl(k_cam_apply<Mo, float>, ls.n_cb * kApplySplit, kCamPerBlock * 32, 0, st, ls);
    return 1;
  }
  // Per device: the fused camera kernel's resident-CTA capacity (per accumulation type)
  // and the launch form the driver accepted on the first use (0 unknown, 1 cooperative
  // with programmatic serialization, 2 cooperative only, -1 neither: two launches).
  struct CoopState {
    std::atomic<int> cap[2];
    std::atomic<int> mode;
  };
  static CoopState& coop_state(int dev) {
    static CoopState st[kMaxDevices];
    return st[dev >= 0 && dev < kMaxDevices ? dev : 0];
  }
  template <class AT>
  static int pcg_camera_cap(int dev) {
    std::atomic<int>& cap = coop_state(dev).cap[std::is_same<AT, double>::value ? 1 : 0];
    int c = cap.load(std::memory_order_relaxed);
    if (!c) {
      int n_sm = 0, occ = 0;
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg_camera<Mo, AT>, kCamPerBlock * 32, 0);
      c = std::max(1, n_sm) * std::max(1, occ);
      cap.store(c, std::memory_order_relaxed);
    }
    return c;
  }
  // A cooperative launch: the driver starts the grid only if every CTA can be resident
  // at once, which the kernel's grid barrier relies on.
  template <class AT>
  static cudaError_t launch_coop(int grid, cudaStream_t st, bool pdl, const LaunchSet& ls) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)(kCamPerBlock * 32));
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_pcg_camera<Mo, AT>, ls);
  }
  // Launches the fused camera kernel if the camera half's units fit one resident wave
  // (returns 1); otherwise, or if the driver refuses the cooperative launch, launches
  // nothing and returns 0 (the caller launches cam_apply and pcg_update).  The first
  // call on a device tries cooperative launch with programmatic serialization, then
  // without, and keeps the form that was accepted.
  template <class AT>
  static int pcg_camera_t(const LaunchSet& ls, cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int units = ls.n_cb * kApplySplit;
    if (units > pcg_camera_cap<AT>(dev)) return 0;
    std::atomic<int>& mode = coop_state(dev).mode;
    int m = mode.load(std::memory_order_relaxed);
    if (m < 0) return 0;
    if (m == 0) {
      if (launch_coop<AT>(units, st, true, ls) == cudaSuccess) {
        mode.store(1, std::memory_order_relaxed);
        return 1;
      }
      cudaGetLastError();
      if (launch_coop<AT>(units, st, false, ls) == cudaSuccess) {
        mode.store(2, std::memory_order_relaxed);
        return 1;
      }
      cudaGetLastError();
      mode.store(-1, std::memory_order_relaxed);
      return 0;
    }
    if (launch_coop<AT>(units, st, m == 1, ls) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return 1;
  }
  static int pcg_camera(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (ls.n_cb == 0) return 0;
    return pr == Prec::F64 ? pcg_camera_t<double>(ls, st) : pcg_camera_t<float>(ls, st);
  }
  static int pcg_update(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (ls.n_cb == 0) return 0;
    if (pr == Prec::F64) launch_pdl(k_pcg_update<Mo, double>, ls.n_cb, kCamPerBlock * 32, 0, st, ls);
    else launch_pdl(k_pcg_update<Mo, float>, ls.n_cb, kCamPerBlock * 32, 0, st, ls);
    return 1;
  }
  template <class JT, bool kDyn>
  static void backsub_k(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    const size_t sm = backsub_smem(pr, ls.ch_max);
    set_smem(reinterpret_cast<const void*>(k_backsub<Mo, JT, kDyn>), sm);
    launch_pdl(k_backsub<Mo, JT, kDyn>, ls.n_ch, kThreads, sm, st, ls);
  }
  template <class JT>
  static void backsub_t(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (dyn_rows(ls)) backsub_k<JT, true>(ls, pr, st);
    else backsub_k<JT, false>(ls, pr, st);
  }
  static int backsub(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (ls.n_ch == 0) return 0;
    if (pr == Prec::F64) backsub_t<double>(ls, pr, st);
    else if (pr == Prec::F32) backsub_t<float>(ls, pr, st);
    else backsub_t<__nv_bfloat16>(ls, pr, st);
    return 1;
  }
  static int retract(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    int n = 0;
    if (pr == Prec::F64) {
      if (ls.n_cb) { launch_pdl(k_retract_cams<Mo, double>, ls.n_cb, kCamPerBlock * 32, 0, st, ls); ++n; }
      if (ls.n_pb) { launch_pdl(k_retract_pts<Mo, double>, ls.n_pb, 256, 0, st, ls); ++n; }
    } else {
      if (ls.n_cb) { launch_pdl(k_retract_cams<Mo, float>, ls.n_cb, kCamPerBlock * 32, 0, st, ls); ++n; }
      if (ls.n_pb) { launch_pdl(k_retract_pts<Mo, float>, ls.n_pb, 256, 0, st, ls); ++n; }
    }
    return n;
  }
  static int decide(const LaunchSet& ls, Prec pr, cudaStream_t st) {
    if (pr == Prec::F64) launch_pdl(k_decide<Mo, double>, ls.nprob, kThreads, 0, st, ls);
    else launch_pdl(k_decide<Mo, float>, ls.nprob, kThreads, 0, st, ls);
    return 1;
  }
  static int commit(const LaunchSet& ls, cudaStream_t st) {
    int n = 0;
    if (ls.n_cb) { launch_pdl(k_commit_cams<Mo>, ls.n_cb, kCamPerBlock * 32, 0, st, ls); ++n; }
    if (ls.n_pb) { launch_pdl(k_commit_pts<Mo>, ls.n_pb, 256, 0, st, ls); ++n; }
    return n;
  }
};

template <class Mo>
KernelSet make_kernel_set(ModelKind kind) {
  using L = Launch<Mo>;
  KernelSet k{};
  k.model = kind;
  k.SS = Mo::SS; k.DB = Mo::DB; k.DC = Mo::DC; k.M = Mo::M; k.NJ = Mo::NJ; k.NPA = Dims<Mo>::NPA;
  k.cam_prepare = &L::cam_prepare;
  k.cost = &L::cost;
  k.cost_init = &L::cost_init;
  k.linearize = &L::linearize;
  k.schur_prepare = &L::schur_prepare;
  k.cam_finalize = &L::cam_finalize;
  k.pcg_spmv = &L::pcg_spmv;
  k.cam_apply = &L::cam_apply;
  k.pcg_update = &L::pcg_update;
  k.pcg_camera = &L::pcg_camera;
  k.full_init = &L::full_init;
  k.full_spmv = &L::full_spmv;
  k.full_update = &L::full_update;
  k.autodiff = &L::autodiff;
  k.backsub = &L::backsub;
  k.retract = &L::retract;
  k.decide = &L::decide;
  k.commit = &L::commit;
  k.max_supported_ch = &L::max_supported_ch;
  k.spmv_kind = &L::spmv_kind;
  return k;
}

}  // namespace gpo
