// The PCG's matrix-free Schur product in warp groups (k_spmv_wg): each chunk of
// point-major edges is cut into warp groups of whole points (at most kGroupEdges edges,
// two per lane; a point with more edges is a group of its own), and one warp owns a
// group from its Jacobian rows to its camera terms:
//   * the group's rows are read from HBM once into registers (packed storage values)
//     and stay there for both halves of the product;
//   * a_e = Jp^T (Jc x_c(e)) per edge, then the point sums u_p = sum_{e in p} a_e by a
//     segmented scan across the warp's lanes (points are runs of consecutive edges),
//     t_p = H_pp^-1 u_p at each run's last lane, broadcast back over the run;
//   * v_e = Jc^T (Jp t_p) per edge, written to the edge's slot-sorted position of the
//     chunk's shared-memory scratch.
// Only the camera-side sums cross warps: after one barrier per chunk, fixed-order
// per-slot sums over contiguous positions give the slot partials (as in the other
// Schur-product kernels), so the product is deterministic and needs no atomics.  The
// scratch and the slot cameras' search direction are double-buffered, so the next
// chunk's warps start while this chunk's slot sums finish.  Persistent CTAs take
// chunks from a shared counter (as the pipelined kernel), prefetch the next chunk's
// rows into L2 and gather its search direction before the barrier.
// Sec. IV-E (implicit PCG on products of the stored Jacobians).
#pragma once

#include "schur_spmv.cuh"

namespace gpo {

constexpr int kWarps = kThreads / 32;

// Dynamic shared memory of k_spmv_wg: two scratch buffers [VW][ch_max + 1] and two
// buffers of the slot cameras' search direction [ns_max][DC].
struct WgLayout {
  uint32_t vv[2], xs[2], size;
};
template <class Mo>
__host__ __device__ inline WgLayout wg_layout(size_t sA, int ch_max, int ns_max) {
  auto al = [](size_t v) { return (uint32_t)((v + 15u) & ~(size_t)15u); };
  const int vw = Mo::DC > 3 ? Mo::DC : 3;
  const uint32_t vvb = al(vw * (size_t)(ch_max + 1) * sA);
  const uint32_t xsb = al((size_t)ns_max * Mo::DC * sA);
  WgLayout L;
  L.vv[0] = 0;
  L.vv[1] = vvb;
  L.xs[0] = 2 * vvb;
  L.xs[1] = 2 * vvb + xsb;
  L.size = 2 * vvb + 2 * xsb;
  return L;
}

// a = Jp^T (Jc x) of one edge from its packed row.
template <class Mo, class JT, class AT>
__device__ __forceinline__ void wg_point_term(const uint4 (&w)[JTiles<JT, Mo::NJ>::Q], const AT* xc, AT (&a)[3]) {
  constexpr int M = Mo::M, DC = Mo::DC, NJ = Mo::NJ, JP0 = Dims<Mo>::JP0;
  AT row[NJ];
  load_row<NJ>(reinterpret_cast<const JT*>(w), row);
  AT q[M];
#pragma unroll
  for (int r = 0; r < M; ++r) q[r] = (AT)0;
#pragma unroll
  for (int k = 0; k < DC; ++k) {
    const AT xk = xc[k];
#pragma unroll
    for (int r = 0; r < M; ++r) q[r] += row[r * DC + k] * xk;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    AT s = row[JP0 + k] * q[0];
#pragma unroll
    for (int r = 1; r < M; ++r) s += row[JP0 + 3 * r + k] * q[r];
    a[k] = s;
  }
}

// v = Jc^T (Jp t) of one edge, written to column `pos` of the scratch [DC][LD].
template <class Mo, class JT, class AT>
__device__ __forceinline__ void wg_camera_term(const uint4 (&w)[JTiles<JT, Mo::NJ>::Q], const AT (&t)[3], AT* vv,
                                               int LD, int pos) {
  constexpr int M = Mo::M, DC = Mo::DC, NJ = Mo::NJ, JP0 = Dims<Mo>::JP0;
  AT row[NJ];
  load_row<NJ>(reinterpret_cast<const JT*>(w), row);
  AT s[M];
#pragma unroll
  for (int r = 0; r < M; ++r) s[r] = row[JP0 + 3 * r] * t[0] + row[JP0 + 3 * r + 1] * t[1] + row[JP0 + 3 * r + 2] * t[2];
#pragma unroll
  for (int k = 0; k < DC; ++k) {
    AT v = row[k] * s[0];
#pragma unroll
    for (int r = 1; r < M; ++r) v += row[r * DC + k] * s[r];
    vv[k * LD + pos] = v;
  }
}

// t = H_pp^-1 u for point p (the damped inverse in the point's record).
template <class AT>
__device__ __forceinline__ void wg_point_solve(const DevBA& d, int p, const AT (&u)[3], AT (&t)[3]) {
  constexpr size_t PRB = (6 * sizeof(AT) + 8 + 15) & ~(size_t)15;
  const AT* h = reinterpret_cast<const AT*>(static_cast<const unsigned char*>(d.pt_rec) + (size_t)p * PRB);
  AT hv[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) hv[k] = __ldg(h + k);
  mul3(hv, u, t);
}

template <class Mo, class JT>
__device__ __forceinline__ void wg_load_row(const DevBA& d, size_t e, uint4 (&w)[JTiles<JT, Mo::NJ>::Q]) {
  using T = JTiles<JT, Mo::NJ>;
  const uint4* J4 = reinterpret_cast<const uint4*>(d.J);
#pragma unroll
  for (int q = 0; q < T::Q; ++q) w[q] = __ldg(J4 + T::piece(e, q));
}

// One warp group of at most kGroupEdges edges: local edges [gb, ge) of chunk c.
template <class Mo, class JT>
__device__ __forceinline__ void wg_group(const DevBA& d, const PipeChunk& c, int gb, int ge, const float* xs,
                                         float* vv, int LD) {
  using AT = float;
  constexpr int DC = Mo::DC, Q = JTiles<JT, Mo::NJ>::Q;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, n = ge - gb;
  const bool v0 = lane < n, v1 = lane + 32 < n;
  const size_t e0 = (size_t)c.e0 + gb + lane, e1 = e0 + 32;
  const uint32_t m0 = v0 ? __ldg(d.e_meta + e0) : 0u, m1 = v1 ? __ldg(d.e_meta + e1) : 0u;
  uint4 w0[Q], w1[Q];
  if (v0) wg_load_row<Mo, JT>(d, e0, w0);
  if (v1) wg_load_row<Mo, JT>(d, e1, w1);
  // pass 1: a_e = Jp^T (Jc x_c)
  AT a0[3] = {0, 0, 0}, a1[3] = {0, 0, 0};
  if (v0) wg_point_term<Mo, JT, AT>(w0, xs + DC * (int)((m0 >> 10) & 1023u), a0);
  if (v1) wg_point_term<Mo, JT, AT>(w1, xs + DC * (int)((m1 >> 10) & 1023u), a1);
  // run keys: the edge's local point; lanes without an edge get keys of their own
  const int k0 = v0 ? (int)(m0 >> 20) : -1 - lane, k1 = v1 ? (int)(m1 >> 20) : -33 - lane;
  // longest run within a half (lanes from the run's first lane) bounds the scan steps
  const int up0 = __shfl_up_sync(FULL, k0, 1), up1 = __shfl_up_sync(FULL, k1, 1);
  const unsigned H0 = __ballot_sync(FULL, lane == 0 || up0 != k0);
  const unsigned H1 = __ballot_sync(FULL, lane == 0 || up1 != k1);
  const unsigned below = 0xffffffffu >> (31 - lane);
  const int run0 = lane - (31 - __clz(H0 & below)), run1 = lane - (31 - __clz(H1 & below));
  const int maxrun = (int)__reduce_max_sync(FULL, (unsigned)max(run0, run1));
  // inclusive segmented scan of each half: after the step of distance dd every lane
  // holds the sum over min(2 dd, its run so far) edges ending at itself
  for (int dd = 1; dd <= maxrun; dd <<= 1) {
    const int u0 = __shfl_up_sync(FULL, k0, dd), u1 = __shfl_up_sync(FULL, k1, dd);
    const bool t0 = lane >= dd && u0 == k0, t1 = lane >= dd && u1 == k1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const AT x0 = __shfl_up_sync(FULL, a0[k], dd), x1 = __shfl_up_sync(FULL, a1[k], dd);
      if (t0) a0[k] += x0;
      if (t1) a1[k] += x1;
    }
  }
  // the run that ends half 0 continues at the start of half 1: add its half-0 sum
  const int k31 = __shfl_sync(FULL, k0, 31);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const AT cy = __shfl_sync(FULL, a0[k], 31);
    if (k1 == k31) a1[k] += cy;
  }
  // each run's last edge solves its point: t_p = H_pp^-1 u_p
  const int dn0 = __shfl_down_sync(FULL, k0, 1), dn1 = __shfl_down_sync(FULL, k1, 1);
  const int first1 = __shfl_sync(FULL, k1, 0);
  const bool tail0 = v0 && (lane == 31 ? first1 : dn0) != k0;
  const bool tail1 = v1 && (lane == 31 || dn1 != k1);
  AT t0[3] = {0, 0, 0}, t1[3] = {0, 0, 0};
  if (tail0) wg_point_solve<AT>(d, c.p0 + k0, a0, t0);
  if (tail1) wg_point_solve<AT>(d, c.p0 + k1, a1, t1);
  // broadcast t_p over the run from its last lane (a half-0 run without its last edge
  // in half 0 ends at the first tail of half 1)
  const unsigned T0 = __ballot_sync(FULL, tail0), T1 = __ballot_sync(FULL, tail1);
  const unsigned at0 = T0 & (0xffffffffu << lane), at1 = T1 & (0xffffffffu << lane);
  const int s0 = at0 ? __ffs(at0) - 1 : 0, s0x = T1 ? __ffs(T1) - 1 : 0, s1 = at1 ? __ffs(at1) - 1 : 0;
  AT p0[3], p1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const AT x = __shfl_sync(FULL, t0[k], s0), y = __shfl_sync(FULL, t1[k], s0x), z = __shfl_sync(FULL, t1[k], s1);
    p0[k] = at0 ? x : y;
    p1[k] = z;
  }
  // pass 3: v_e = Jc^T (Jp t_p) to the slot-sorted position
  if (v0) wg_camera_term<Mo, JT, AT>(w0, p0, vv, LD, (int)(m0 & 1023u));
  if (v1) wg_camera_term<Mo, JT, AT>(w1, p1, vv, LD, (int)(m1 & 1023u));
}

// A warp group of one point with more than kGroupEdges edges: the warp strides over
// its edges twice (rows re-read), with a butterfly sum for u_p in between.
template <class Mo, class JT>
__device__ __noinline__ void wg_long_point(const DevBA& d, const PipeChunk& c, int gb, int ge, const float* xs,
                                           float* vv, int LD) {
  using AT = float;
  constexpr int DC = Mo::DC, Q = JTiles<JT, Mo::NJ>::Q;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  AT u[3] = {0, 0, 0};
  for (int i = gb + lane; i < ge; i += 32) {
    const size_t e = (size_t)c.e0 + i;
    const uint32_t m = __ldg(d.e_meta + e);
    uint4 w[Q];
    wg_load_row<Mo, JT>(d, e, w);
    AT a[3];
    wg_point_term<Mo, JT, AT>(w, xs + DC * (int)((m >> 10) & 1023u), a);
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] += a[k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] += __shfl_xor_sync(FULL, u[k], o);
  }
  AT t[3];
  wg_point_solve<AT>(d, c.p0 + (int)(__ldg(d.e_meta + (size_t)c.e0 + gb) >> 20), u, t);
  for (int i = gb + lane; i < ge; i += 32) {
    const size_t e = (size_t)c.e0 + i;
    const uint32_t m = __ldg(d.e_meta + e);
    uint4 w[Q];
    wg_load_row<Mo, JT>(d, e, w);
    wg_camera_term<Mo, JT, AT>(w, t, vv, LD, (int)(m & 1023u));
  }
}

// Resident CTAs per SM the register budget targets.
template <class JT> struct WgOcc { static constexpr int value = sizeof(JT) == 2 ? 3 : 2; };

// The warp-group Schur product: persistent CTAs; chunk n's warps, the next chunk's
// search-direction gather, one barrier, chunk n's slot sums.  Requires chunks of at
// most 1024 edges (packed positions) and storage in BF16 or FP32.  The last CTA to
// finish puts the chunk counters back to 0.
template <class Mo, class JT>
__global__ void __launch_bounds__(kThreads, WgOcc<JT>::value) k_spmv_wg(LaunchSet ls) {
  using AT = float;
  constexpr int DC = Mo::DC, DB = Mo::DB, NJ = Mo::NJ;
  constexpr int kWords = (int)(sizeof(DevBA) / 4);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevBA d;
  __shared__ PipeChunk ck[4];
  pdl_trigger();
  const int LD = ls.ch_max + 1;
  const WgLayout WL = wg_layout<Mo>(sizeof(AT), ls.ch_max, ls.ns_max);
  const int warp = threadIdx.x >> 5;
  int bound_q = -1;
  pdl_wait();

  auto grab = [&]() -> int {
    for (;;) {
      const int k = atomicAdd(ls.work, 1);
      if (k >= ls.n_ch) return -1;
      if (ls.nprob == 1) return k;
      const Scalars* sc = ls.probs[ls.ch_prob[k]].sc;
      if (sc->active && !sc->pcg_done) return k;
    }
  };
  auto finish = [&]() {
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(ls.work + 1, 1) == (int)gridDim.x - 1) {
        ls.work[0] = 0;
        ls.work[1] = 0;
      }
    }
  };
  auto plan = [&](int k) -> PipeChunk {
    PipeChunk c;
    c.k = k;
    if (k < 0) return c;
    const int q = ls.nprob == 1 ? 0 : ls.ch_prob[k];
    const int kl = ls.nprob == 1 ? k : k - ls.ch_base[q];
    const DevBA* P = q == bound_q ? &d : ls.probs + q;
    c.q = q;
    c.kl = kl;
    c.e0 = P->ch_e0[kl];
    c.nE = P->ch_e0[kl + 1] - c.e0;
    c.p0 = P->ch_p0[kl];
    c.nP = P->ch_p0[kl + 1] - c.p0;
    c.s0 = P->ch_s0[kl];
    c.nS = P->ch_s0[kl + 1] - c.s0;
    return c;
  };
  // the slot cameras' search direction p = (z + beta p_old) / n of chunk c (the
  // current solution x in a restart iteration)
  auto gather = [&](const PipeChunk& c, AT* xs) {
    if (c.k < 0) return;
    const DevBA* P = c.q == bound_q ? &d : ls.probs + c.q;
    const Scalars* sc = P->sc;
    const int restart = sc->restart;
    const AT* zv = reinterpret_cast<const AT*>(restart ? P->x : P->z);
    const AT* pold = restart ? zv : reinterpret_cast<const AT*>(sc->pidx ? P->p2 : P->p);
    const AT beta = restart ? (AT)0 : (AT)sc->beta, inv_n = restart ? (AT)1 : (AT)sc->inv_n;
    const int4* sr = P->slot_rec + c.s0;
    for (int w = threadIdx.x; w < c.nS * DC; w += kThreads) {
      const int sl = w / DC, k = w - sl * DC;
      const size_t o = DB * (size_t)__ldg(&sr[sl].z) + k;
      xs[w] = (zv[o] + beta * pold[o]) * inv_n;
    }
  };

  if (ls.nprob == 1) {
    const Scalars* sc = ls.probs[0].sc;
    if (!sc->active || sc->pcg_done) return;
  }
  if (threadIdx.x == 0) {
    const int k0 = grab();
    ck[0] = plan(k0);
    ck[1] = plan(k0 < 0 ? -1 : grab());
  }
  __syncthreads();
  if (ck[0].k < 0) {
    finish();
    return;
  }
  gather(ck[0], reinterpret_cast<AT*>(smem + WL.xs[0]));
  for (int n = 0;; ++n) {
    const int b = n & 1;
    const PipeChunk c = ck[n & 3];
    if (c.k < 0) break;
    const PipeChunk cn = ck[(n + 1) & 3];
    if (c.q != bound_q) {        // CTA-uniform: bind the chunk's problem
      __syncthreads();           // every thread is past the previous use of d (and the gather)
      for (int i = threadIdx.x; i < kWords; i += kThreads)
        reinterpret_cast<int*>(&d)[i] = reinterpret_cast<const int*>(ls.probs + c.q)[i];
      bound_q = c.q;
      __syncthreads();
    } else if (n == 0) {
      __syncthreads();           // the first chunk's direction gather
    }
    // one thread plans the chunk after next; another prefetches the next chunk's rows
    if (threadIdx.x == kThreads - 32) ck[(n + 2) & 3] = plan(cn.k < 0 ? -1 : grab());
    if (threadIdx.x == kThreads - 64 && cn.k >= 0 && cn.nE > 0) {
      const DevBA* P = cn.q == bound_q ? &d : ls.probs + cn.q;
      const size_t t0 = (size_t)cn.e0 >> 5, t1 = (size_t)(cn.e0 + cn.nE - 1) >> 5;
      prefetch_l2(static_cast<const JT*>(P->J) + t0 * kJTile * NJ, (uint32_t)((t1 - t0 + 1) * kJTile * NJ * sizeof(JT)));
    }
    AT* vv = reinterpret_cast<AT*>(smem + WL.vv[b]);
    const AT* xs = reinterpret_cast<const AT*>(smem + WL.xs[b]);
    // the warps' groups
    const uint16_t* gr = d.ch_grp + (size_t)c.kl * kMaxGroups;
    for (int g = warp; g < kMaxGroups; g += kWarps) {
      const int gb = g == 0 ? 0 : (int)__ldg(gr + g - 1), ge = (int)__ldg(gr + g);
      if (gb >= ge) break;       // warp-uniform; empty groups are at the end
      if (ge - gb <= kGroupEdges) wg_group<Mo, JT>(d, c, gb, ge, xs, vv, LD);
      else wg_long_point<Mo, JT>(d, c, gb, ge, xs, vv, LD);
    }
    // the next chunk's search direction (its buffer was last read by the previous chunk)
    gather(cn, reinterpret_cast<AT*>(smem + WL.xs[b ^ 1]));
    __syncthreads();             // this chunk's terms and the next chunk's direction are in place
    // per-slot sums over contiguous positions
    AT* partV = reinterpret_cast<AT*>(d.partV);
    const int4* sr = d.slot_rec + c.s0;
    for (int w = threadIdx.x; w < c.nS * DC; w += kThreads) {
      const int sl = w / DC, comp = w - sl * DC;
      const int4 r4 = __ldg(sr + sl);
      partV[(size_t)r4.w * DC + comp] = seg_sum(vv + comp * LD, r4.x, r4.y);
    }
  }
  finish();
}

}  // namespace gpo
