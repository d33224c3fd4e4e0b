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
  AT row[Mo::NJ];
  load_row<Mo::NJ>(reinterpret_cast<const JT*>(w), row);
  edge_point_term<Mo>(row, xc, a);
}

// v = Jc^T (Jp t) of one edge, written to column `pos` of the scratch [DC][LD].
template <class Mo, class JT, class AT>
__device__ __forceinline__ void wg_camera_term(const uint4 (&w)[JTiles<JT, Mo::NJ>::Q], const AT (&t)[3], AT* vv,
                                               int LD, int pos) {
  AT row[Mo::NJ];
  load_row<Mo::NJ>(reinterpret_cast<const JT*>(w), row);
  AT v[Mo::DC];
  edge_camera_term<Mo>(row, t[0], t[1], t[2], v);
#pragma unroll
  for (int k = 0; k < Mo::DC; ++k) vv[k * LD + pos] = v[k];
}

// Rows of a chunk: the 16-byte pieces of its 32-edge tiles, starting at the tile that
// holds the chunk's first edge (jskew = that edge's position in its tile), in global
// memory or in a shared-memory stage.
template <class Mo, class JT>
__device__ __forceinline__ void wg_load_row(const uint4* J4, int i, uint4 (&w)[JTiles<JT, Mo::NJ>::Q]) {
  using T = JTiles<JT, Mo::NJ>;
#pragma unroll
  for (int q = 0; q < T::Q; ++q) w[q] = J4[T::piece((size_t)i, q)];
}

// t = H_pp^-1 u from a point record (the damped inverse first).
template <class AT>
__device__ __forceinline__ void wg_solve_rec(const unsigned char* rec, const AT (&u)[3], AT (&t)[3]) {
  const AT* h = reinterpret_cast<const AT*>(rec);
  AT hv[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) hv[k] = h[k];
  mul3(hv, u, t);
}

// The inputs of one chunk as the warp phase reads them: J4 its rows (tile-relative,
// local edge i at tile position i + jskew), meta its packed per-edge positions, prec
// its point records (local point order), xs its slot cameras' search direction.
struct WgChunk {
  const uint4* J4;
  int jskew;
  const uint32_t* meta;
  const unsigned char* prec;
  const float* xs;
};

// One warp group of at most kGroupEdges edges: local edges [gb, ge) of the chunk.
template <class Mo, class JT>
__device__ __forceinline__ void wg_group(const WgChunk& in, int gb, int ge, float* vv, int LD) {
  using AT = float;
  constexpr int DC = Mo::DC, Q = JTiles<JT, Mo::NJ>::Q;
  constexpr size_t PRB = (6 * sizeof(AT) + 8 + 15) & ~(size_t)15;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, n = ge - gb;
  const bool v0 = lane < n, v1 = lane + 32 < n;
  const int i0 = gb + lane, i1 = i0 + 32;
  const uint32_t m0 = v0 ? in.meta[i0] : 0u, m1 = v1 ? in.meta[i1] : 0u;
  uint4 w0[Q], w1[Q];
  if (v0) wg_load_row<Mo, JT>(in.J4, i0 + in.jskew, w0);
  if (v1) wg_load_row<Mo, JT>(in.J4, i1 + in.jskew, w1);
  // pass 1: a_e = Jp^T (Jc x_c)
  AT a0[3] = {0, 0, 0}, a1[3] = {0, 0, 0};
  if (v0) wg_point_term<Mo, JT, AT>(w0, in.xs + DC * (int)((m0 >> 10) & 1023u), a0);
  if (v1) wg_point_term<Mo, JT, AT>(w1, in.xs + DC * (int)((m1 >> 10) & 1023u), a1);
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
  if (tail0) wg_solve_rec<AT>(in.prec + (size_t)k0 * PRB, a0, t0);
  if (tail1) wg_solve_rec<AT>(in.prec + (size_t)k1 * PRB, a1, t1);
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
__device__ __noinline__ void wg_long_point(const WgChunk& in, int gb, int ge, float* vv, int LD) {
  using AT = float;
  constexpr int DC = Mo::DC, Q = JTiles<JT, Mo::NJ>::Q;
  constexpr size_t PRB = (6 * sizeof(AT) + 8 + 15) & ~(size_t)15;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  AT u[3] = {0, 0, 0};
  for (int i = gb + lane; i < ge; i += 32) {
    const uint32_t m = in.meta[i];
    uint4 w[Q];
    wg_load_row<Mo, JT>(in.J4, i + in.jskew, w);
    AT a[3];
    wg_point_term<Mo, JT, AT>(w, in.xs + DC * (int)((m >> 10) & 1023u), a);
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] += a[k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] += __shfl_xor_sync(FULL, u[k], o);
  }
  AT t[3];
  wg_solve_rec<AT>(in.prec + (size_t)(in.meta[gb] >> 20) * PRB, u, t);
  for (int i = gb + lane; i < ge; i += 32) {
    const uint32_t m = in.meta[i];
    uint4 w[Q];
    wg_load_row<Mo, JT>(in.J4, i + in.jskew, w);
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
    const AT beta = restart ? (AT)0 : sc_beta<AT>(sc), inv_n = restart ? (AT)1 : sc_inv_n<AT>(sc);
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
    constexpr size_t PRB = (6 * sizeof(AT) + 8 + 15) & ~(size_t)15;
    const WgChunk in{reinterpret_cast<const uint4*>(d.J) + (size_t)(c.e0 >> 5) * (kJTile * NJ * sizeof(JT) / 16),
                     c.e0 & (kJTile - 1), d.e_meta + c.e0,
                     static_cast<const unsigned char*>(d.pt_rec) + (size_t)c.p0 * PRB, xs};
    const uint16_t* gr = d.ch_grp + (size_t)c.kl * kMaxGroups;
    for (int g = warp; g < kMaxGroups; g += kWarps) {
      const int gb = g == 0 ? 0 : (int)__ldg(gr + g - 1), ge = (int)__ldg(gr + g);
      if (gb >= ge) break;       // warp-uniform; empty groups are at the end
      if (ge - gb <= kGroupEdges) wg_group<Mo, JT>(in, gb, ge, vv, LD);
      else wg_long_point<Mo, JT>(in, gb, ge, vv, LD);
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

// ---------------------------------------------------------------- staged form

// Byte layout of one stage of the staged warp-group product (16-byte aligned offsets):
// the chunk's row tiles, a 16-byte-aligned run of its packed positions, its point
// records, slot records, group table and the slot cameras' search direction.
struct WgsLayout {
  uint32_t j, meta, pt, slot, grp, xs, size;
};
template <class Mo>
__host__ __device__ inline WgsLayout wgs_layout(size_t sJ, size_t sA, int ch_max, int np_max, int ns_max) {
  auto al = [](size_t v) { return (uint32_t)((v + 15u) & ~(size_t)15u); };
  const size_t prb = (6 * sA + 8 + 15) & ~(size_t)15;
  WgsLayout L;
  L.j = 0;   // whole 32-edge tiles covering the chunk (a chunk may start inside a tile)
  L.meta = al((size_t)(ch_max / kJTile + 2) * kJTile * Mo::NJ * sJ);
  L.pt = L.meta + al((size_t)ch_max * 4 + 16);
  L.slot = L.pt + al((size_t)np_max * prb);
  L.grp = L.slot + al((size_t)ns_max * 16);
  L.xs = L.grp + al(kMaxGroups * 2);
  L.size = L.xs + al((size_t)ns_max * Mo::DC * sA);
  return L;
}
constexpr int kWgsStages = 2;

// The warp-group product fed through shared memory.  One producer warp walks the
// chunks blockIdx.x, + gridDim.x, ... (skipping problems whose PCG has stopped) and,
// up to kWgsStages chunks ahead, streams each chunk's inputs into a stage with 1-D bulk
// copies completing on the stage's "full" mbarrier -- row tiles, packed positions,
// point records, slot records, the group table -- and gathers the slot cameras'
// search direction into it.  The eight consumer warps run their warp groups entirely
// from the stage (rows, positions and point inverses at shared-memory latency), meet
// at a named barrier, form the slot sums, meet again and release the stage on its
// "empty" mbarrier.  So every chunk's HBM reads are in flight while the previous
// chunk is computed.  The sums are those of k_spmv_wg.  Every wait is bounded: a wait
// that gives up raises *ls.err, and the producer lets its copies in flight land
// (bounded again) before the CTA exits.
template <class Mo, class JT>
__global__ void __launch_bounds__(kWsThreads) k_spmv_wgs(LaunchSet ls) {
  using AT = float;
  constexpr int DC = Mo::DC, DB = Mo::DB, NJ = Mo::NJ;
  constexpr uint32_t RB = NJ * sizeof(JT);
  constexpr uint32_t PRB = (6 * sizeof(AT) + 8 + 15) & ~15u;
  constexpr int S = kWgsStages;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[S], empty[S];
  __shared__ StageInfo info[S];
  __shared__ int s_fail;
  pdl_trigger();
  const WgsLayout SL = wgs_layout<Mo>(sizeof(JT), sizeof(AT), ls.ch_max, ls.np_max, ls.ns_max);
  const int LD = ls.ch_max + 1;
  AT* vv = reinterpret_cast<AT*>(smem + S * SL.size);   // [DC][LD] consumer scratch
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(smem_u32(&full[st]), 2);    // the producer's expect_tx arrival + its gather arrival
      mbar_init(smem_u32(&empty[st]), 1);   // one consumer arrival
    }
    mbar_fence_init();
    s_fail = 0;
  }
  pdl_wait();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == kWarps) {
    // ================================================================ producer warp
    auto next_live = [&](int k) -> int {
      while (k < ls.n_ch) {
        const int q = ls.nprob == 1 ? 0 : ls.ch_prob[k];
        const Scalars* sc = ls.probs[q].sc;
        if (sc->active && !sc->pcg_done) return k;
        const int nxt = q + 1 < ls.nprob ? ls.ch_base[q + 1] : ls.n_ch;
        k += ((nxt - k) + G - 1) / G * G;
      }
      return -1;
    };
    int last_use[S];
#pragma unroll
    for (int st = 0; st < S; ++st) last_use[st] = -1;
    int k = __shfl_sync(0xffffffffu, lane == 0 ? next_live(blockIdx.x) : 0, 0);
    int cq = -1;
    const DevBA* P = nullptr;
    const AT* zv = nullptr;
    const AT* pold = nullptr;
    AT beta = (AT)0, inv_n = (AT)1;
    for (int n = 0;; ++n) {
      const int st = n % S, use = n / S;
      if (use > 0 && !mbar_wait(smem_u32(&empty[st]), (uint32_t)(use - 1) & 1u)) {
        if (lane == 0) s_fail = 1;
        break;
      }
      const uint32_t fb = smem_u32(&full[st]);
      last_use[st] = use;
      if (k < 0) {   // end of work: an empty stage with no transfer
        if (lane == 0) {
          info[st].k = -1;
          mbar_arrive(fb, 2);
        }
        break;
      }
      const int q = ls.nprob == 1 ? 0 : ls.ch_prob[k];
      if (q != cq) {
        cq = q;
        P = ls.probs + q;
        const Scalars* sc = P->sc;
        const int restart = sc->restart;   // a restart's product is taken of x
        zv = reinterpret_cast<const AT*>(restart ? P->x : P->z);
        pold = restart ? zv : reinterpret_cast<const AT*>(sc->pidx ? P->p2 : P->p);
        beta = restart ? (AT)0 : sc_beta<AT>(sc);
        inv_n = restart ? (AT)1 : sc_inv_n<AT>(sc);
      }
      const int kl = ls.nprob == 1 ? k : k - ls.ch_base[q];
      const int e0 = P->ch_e0[kl], e1 = P->ch_e0[kl + 1];
      const int p0 = P->ch_p0[kl], p1 = P->ch_p0[kl + 1];
      const int s0 = P->ch_s0[kl], s1 = P->ch_s0[kl + 1];
      unsigned char* base = smem + st * SL.size;
      if (lane == 0) {
        const uint32_t bJ = e1 > e0 ? (uint32_t)(((e1 - 1) >> 5) - (e0 >> 5) + 1) * kJTile * RB : 0u;
        const uintptr_t ms = reinterpret_cast<uintptr_t>(P->e_meta + e0);
        const uintptr_t ma = ms & ~(uintptr_t)15;
        const uint32_t skew = (uint32_t)(ms - ma);
        const uint32_t bM = e1 > e0 ? (skew + 4u * (uint32_t)(e1 - e0) + 15u) & ~15u : 0u;
        const uint32_t bP = (uint32_t)(p1 - p0) * PRB;
        const uint32_t bS = (uint32_t)(s1 - s0) * 16u;
        const uint32_t bG = kMaxGroups * 2;
        info[st] = StageInfo{k, q, e1 - e0, p1 - p0, s1 - s0, (int)(skew / 4), e0 & (kJTile - 1)};
        fence_proxy_async();
        mbar_expect_tx(fb, bJ + bM + bP + bS + bG);
        if (bJ) bulk_g2s(smem_u32(base + SL.j), static_cast<const JT*>(P->J) + (size_t)(e0 >> 5) * kJTile * NJ, bJ, fb);
        if (bM) bulk_g2s(smem_u32(base + SL.meta), reinterpret_cast<const void*>(ma), bM, fb);
        if (bP) bulk_g2s(smem_u32(base + SL.pt), static_cast<const unsigned char*>(P->pt_rec) + (size_t)p0 * PRB, bP, fb);
        if (bS) bulk_g2s(smem_u32(base + SL.slot), P->slot_rec + s0, bS, fb);
        bulk_g2s(smem_u32(base + SL.grp), P->ch_grp + (size_t)kl * kMaxGroups, bG, fb);
      }
      // the slot cameras' search-direction values, gathered by the whole warp
      AT* xs = reinterpret_cast<AT*>(base + SL.xs);
      for (int w = lane; w < (s1 - s0) * DC; w += 32) {
        const int sl = w / DC, kk = w - sl * DC;
        const size_t o = DB * (size_t)__ldg(&P->slot_rec[s0 + sl].z) + kk;
        xs[w] = (zv[o] + beta * pold[o]) * inv_n;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(fb, 1);
      k = __shfl_sync(0xffffffffu, lane == 0 ? next_live(k + G) : 0, 0);
    }
    // let every copy issued into a stage land before the CTA can exit (already true
    // unless a wait gave up); bounded
    if (lane == 0) {
#pragma unroll
      for (int st = 0; st < S; ++st)
        if (last_use[st] >= 0) mbar_wait(smem_u32(&full[st]), (uint32_t)last_use[st] & 1u);
      if (s_fail) atomicExch(ls.err, 1);
    }
  } else {
    // ================================================================ consumer warps
    for (int n = 0;; ++n) {
      const int st = n % S;
      const bool ok = mbar_wait(smem_u32(&full[st]), (uint32_t)(n / S) & 1u);
      if (consumer_any(!ok)) {
        if (threadIdx.x == 0) s_fail = 1;
        break;
      }
      const StageInfo in = info[st];
      if (in.k < 0) break;
      const unsigned char* stg = smem + st * SL.size;
      const WgChunk ch{reinterpret_cast<const uint4*>(stg + SL.j), in.jskew,
                       reinterpret_cast<const uint32_t*>(stg + SL.meta) + in.skew, stg + SL.pt,
                       reinterpret_cast<const AT*>(stg + SL.xs)};
      const uint16_t* gr = reinterpret_cast<const uint16_t*>(stg + SL.grp);
      for (int g = warp; g < kMaxGroups; g += kWarps) {
        const int gb = g == 0 ? 0 : (int)gr[g - 1], ge = (int)gr[g];
        if (gb >= ge) break;       // warp-uniform; empty groups are at the end
        if (ge - gb <= kGroupEdges) wg_group<Mo, JT>(ch, gb, ge, vv, LD);
        else wg_long_point<Mo, JT>(ch, gb, ge, vv, LD);
      }
      consumer_sync();             // the chunk's camera terms are in place
      AT* partV = reinterpret_cast<AT*>(ls.probs[in.q].partV);
      const int4* srec = reinterpret_cast<const int4*>(stg + SL.slot);
      for (int w = threadIdx.x; w < in.nS * DC; w += kThreads) {
        const int sl = w / DC, comp = w - sl * DC;
        const int4 r4 = srec[sl];
        partV[(size_t)r4.w * DC + comp] = seg_sum(vv + comp * LD, r4.x, r4.y);
      }
      consumer_sync();             // scratch and stage free
      if (threadIdx.x == 0) mbar_arrive(smem_u32(&empty[st]), 1);
    }
  }
}

}  // namespace gpo
