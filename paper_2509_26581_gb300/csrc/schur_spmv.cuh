// The PCG's matrix-free Schur product (the hot loop), in two forms that compute the
// same sums in the same order: k_spmv, one CTA per chunk of point-major edges, and
// k_spmv_ws, a warp-specialised persistent kernel streaming chunks through shared
// memory with bulk copies.  Sec. IV-E (implicit PCG on products of the stored
// Jacobians), Sec. IV-E last paragraph (no sparse-matrix format).
#pragma once
#include <algorithm>

#include "schur_common.cuh"

namespace gpo {

// ---------------------------------------------------------------- PCG

// Matrix-free Schur product, one CTA per chunk (the hot loop).  With t_p =
// H_pp^-1 sum_e Jp_e^T Jc_e x_c(e), each edge contributes v_e = Jc_e^T Jp_e t_p(e) to
// its camera.  The CTA first issues its index loads, stages the camera vector of
// each slot once (instead of once per edge), the point inverses, point offsets and
// slot ranges, then runs barrier-separated passes in shared memory: per-edge point
// terms, point sums, per-edge camera terms scattered to slot-sorted positions, and
// contiguous per-slot sums.  Each chunk's Jacobian rows are read twice, the second
// time mostly from L1/L2.
template <class Mo, class JT, int EPT>
__global__ void __launch_bounds__(kThreads) k_spmv(LaunchSet ls) {
  using AT = typename AccOf<JT>::T;
  using Dm = Dims<Mo>;
  constexpr int DC = Mo::DC, DB = Mo::DB, NJ = Mo::NJ, VW = Dm::VW;
  GPO_BIND(ch, kl)
  // the chunk's ranges and the solve's scalars are loaded together, ahead of the
  // early exit, so that the index loads below start one round trip sooner
  const Scalars* sc = d.sc;
  const ChunkRange cr = chunk_range(d, kl);
  const int act = sc->active, done = sc->pcg_done, pidx = sc->pidx, restart = sc->restart;
  const AT beta_a = sc_beta<AT>(sc), inv_n_a = sc_inv_n<AT>(sc);
  if (!act || done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int CH = d.ch_max, LD = CH + 1;
  AT* vv = reinterpret_cast<AT*>(smem);        // [VW][LD]; rows 0..2 hold a_e in pass 1
  AT* tp = vv + VW * LD;                       // [3][LD] point solutions
  AT* xs = tp + 3 * LD;                        // [ls.ns_max][DC] slot camera vectors
  AT* hv = xs + DC * ls.ns_max;                // [ls.np_max][6] point inverses
  int* po = reinterpret_cast<int*>(hv + 6 * ls.np_max);   // [np + 1] local point offsets
  int* so = po + ls.np_max + 1;                           // [ns + 1] local slot offsets
  int* sp = so + ls.ns_max + 1;                           // [ns] camera-major slot rows
  const JT* Jg = reinterpret_cast<const JT*>(d.J);

  // per-edge positions: one packed word per edge when chunks fit 10-bit positions
  int pos[EPT], slot[EPT], ptl[EPT];
  const bool packed = ls.ch_max <= 1024;
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const int i = threadIdx.x + m * kThreads;
    if (i < cr.nE) {
      if (packed) {
        const uint32_t w = __ldg(d.e_meta + cr.e0 + i);
        pos[m] = (int)(w & 1023u);
        slot[m] = (int)((w >> 10) & 1023u);
        ptl[m] = (int)(w >> 20);
      } else {
        pos[m] = __ldg(d.e_pos + cr.e0 + i);
        slot[m] = __ldg(d.e_slot + cr.e0 + i);
        ptl[m] = __ldg(d.e_pt + cr.e0 + i) - cr.p0;
      }
    }
  }
  // one thread per slot: its record (edge range, camera, partial row) and the search
  // direction p_k = (z_k + beta_k p_{k-1}) / n_k of its camera
  // the direction p = (z + beta p_old) / n, or in a restart iteration the solution x
  const AT* zv = reinterpret_cast<const AT*>(restart ? d.x : d.z);
  const AT* pold = restart ? zv : reinterpret_cast<const AT*>(pidx ? d.p2 : d.p);
  const AT beta = restart ? (AT)0 : beta_a, inv_n = restart ? (AT)1 : inv_n_a;
  for (int t = threadIdx.x; t < cr.nS; t += kThreads) {
    const int4 r4 = __ldg(d.slot_rec + cr.s0 + t);
    so[t] = r4.x;
    so[t + 1] = r4.y;
    sp[t] = r4.w;
    const size_t o = DB * (size_t)r4.z;
#pragma unroll
    for (int k = 0; k < DC; ++k) xs[DC * t + k] = (zv[o + k] + beta * pold[o + k]) * inv_n;
  }
  // one thread per point: its record (H_pp^-1 and edge range)
  constexpr size_t PRB = (6 * sizeof(AT) + 8 + 15) & ~(size_t)15;
  const unsigned char* prec = static_cast<const unsigned char*>(d.pt_rec) + (size_t)cr.p0 * PRB;
  for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
    const AT* h = reinterpret_cast<const AT*>(prec + (size_t)j * PRB);
    const int* se = reinterpret_cast<const int*>(prec + (size_t)j * PRB + 6 * sizeof(AT));
#pragma unroll
    for (int k = 0; k < 6; ++k) hv[6 * j + k] = h[k];
    po[j] = se[0];
    po[j + 1] = se[1];
  }
  if (threadIdx.x == 0 && cr.nP == 0) po[0] = 0;
  if (threadIdx.x == 0 && cr.nS == 0) so[0] = 0;
  __syncthreads();

  // ---- pass 1: a_e = Jp^T (Jc x_c)
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const int i = threadIdx.x + m * kThreads;
    if (i >= cr.nE) break;
    AT row[NJ];
    load_row_t<NJ>(Jg, (size_t)(cr.e0 + i), row);
    AT a[3];
    edge_point_term<Mo>(row, xs + DC * slot[m], a);
#pragma unroll
    for (int k = 0; k < 3; ++k) vv[k * LD + i] = a[k];
  }
  __syncthreads();
  // ---- pass 2: t_p = H_pp^-1 sum_e a_e
  for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
    AT u[3];
    point_sum<JT>(vv, LD, po[j], po[j + 1], u);
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
    AT row[NJ];
    load_row_t<NJ>(Jg, (size_t)(cr.e0 + i), row);
    const int pl = ptl[m];
    AT v[DC];
    edge_camera_term<Mo>(row, tp[pl], tp[LD + pl], tp[2 * LD + pl], v);
#pragma unroll
    for (int k = 0; k < DC; ++k) vv[k * LD + pos[m]] = v[k];
  }
  __syncthreads();
  // ---- pass 4: per-slot sums over contiguous positions
  AT* partV = reinterpret_cast<AT*>(d.partV);
  for (int w = threadIdx.x; w < cr.nS * DC; w += kThreads) {
    const int sl = w / DC, comp = w - sl * DC;
    partV[(size_t)sp[sl] * DC + comp] = seg_sum(vv + comp * LD, so[sl], so[sl + 1]);
  }
}

// ---------------------------------------------------------------- Schur product, bulk-copy pipeline

// Async-proxy helpers (sm_90+): mbarrier with transaction counts and 1-D bulk copies
// from global to shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
constexpr unsigned kSpinLimit = 1u << 22;   // bounded waits: well under a second of polling
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (unsigned n = 0; n < kSpinLimit; ++n)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

constexpr int kStages = 3;                    // chunks in flight per CTA
constexpr int kWsThreads = kThreads + 32;     // eight consumer warps and one producer warp

// Named barrier of the consumer warps (the producer warp does not take part), and its
// OR-reduction form.
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory"); }
__device__ __forceinline__ bool consumer_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kThreads)
      : "memory");
  return r != 0;
}

// Byte layout of one pipeline stage in shared memory (all offsets 16-byte aligned).
struct StageLayout {
  uint32_t j, meta, pt, slot, xs, size;
};
template <class Mo>
__host__ __device__ inline StageLayout stage_layout(size_t sJ, size_t sA, int ch_max, int np_max, int ns_max) {
  auto al = [](uint32_t v) { return (v + 15u) & ~15u; };
  StageLayout L;
  const uint32_t prb = (uint32_t)((6 * sA + 8 + 15) & ~(size_t)15);
  L.j = 0;   // whole 32-edge tiles covering the chunk (a chunk may start inside a tile)
  L.meta = al((uint32_t)((ch_max / kJTile + 2) * kJTile * Mo::NJ * sJ));
  L.pt = L.meta + al((uint32_t)(ch_max * 4 + 16));
  L.slot = L.pt + al((uint32_t)(np_max * prb));
  L.xs = L.slot + al((uint32_t)(ns_max * 16));
  L.size = L.xs + al((uint32_t)(ns_max * Mo::DC * sA));
  return L;
}

struct StageInfo {
  int k, q, nE, nP, nS, skew;   // chunk (-1: no more chunks), problem, sizes, meta skew
  int jskew;                    // position of the chunk's first row in its first tile
};

// Warp-specialised persistent Schur product.  One producer warp walks the chunks
// blockIdx.x, + gridDim.x, ... of the launch set (skipping problems whose PCG has
// stopped) and, kStages chunks ahead of the consumers, streams each chunk's inputs
// -- Jacobian rows, packed per-edge positions, point records (H_pp^-1 and edge range)
// and slot records (edge range, camera, partial row) -- into a shared-memory stage
// with 1-D bulk copies completing on the stage's "full" mbarrier, and gathers the
// slot cameras' search-direction values p = (z + beta p_old) / n into the stage
// itself.  Eight consumer warps run the passes of k_spmv on the stage (named barriers
// among themselves) and release it on its "empty" mbarrier.  Results are bit-identical
// to k_spmv.  Every wait is bounded: a wait that gives up raises *ls.err, and the
// producer lets its copies in flight land (bounded again) before the CTA exits.
template <class Mo, class JT>
__global__ void __launch_bounds__(kWsThreads) k_spmv_ws(LaunchSet ls) {
  using AT = typename AccOf<JT>::T;
  using Dm = Dims<Mo>;
  constexpr int DC = Mo::DC, DB = Mo::DB, NJ = Mo::NJ, VW = Dm::VW;
  constexpr uint32_t RB = NJ * sizeof(JT);
  constexpr uint32_t PRB = (6 * sizeof(AT) + 8 + 15) & ~15u;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ StageInfo info[kStages];
  __shared__ int s_fail;
  pdl_trigger();
  const StageLayout SL = stage_layout<Mo>(sizeof(JT), sizeof(AT), ls.ch_max, ls.np_max, ls.ns_max);
  const int LD = ls.ch_max + 1;
  AT* vv = reinterpret_cast<AT*>(smem + kStages * SL.size);   // [VW][LD] consumer scratch
  AT* tp = vv + VW * LD;                                        // [3][LD]
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(smem_u32(&full[st]), 2);    // the producer's expect_tx arrival + its gather arrival
      mbar_init(smem_u32(&empty[st]), 1);   // one consumer arrival
    }
    mbar_fence_init();
    s_fail = 0;
  }
  pdl_wait();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == kThreads / 32) {
    // ================================================================ producer warp
    // next chunk k' >= k of this CTA whose problem still iterates, or -1
    auto next_live = [&](int k) -> int {
      while (k < ls.n_ch) {
        const int q = ls.ch_prob[k];
        const Scalars* sc = ls.probs[q].sc;
        if (sc->active && !sc->pcg_done) return k;
        const int nxt = q + 1 < ls.nprob ? ls.ch_base[q + 1] : ls.n_ch;
        k += ((nxt - k) + G - 1) / G * G;
      }
      return -1;
    };
    int last_use[kStages];
#pragma unroll
    for (int st = 0; st < kStages; ++st) last_use[st] = -1;
    int k = __shfl_sync(0xffffffffu, lane == 0 ? next_live(blockIdx.x) : 0, 0);
    int cq = -1;
    const DevBA* P = nullptr;
    const AT* zv = nullptr;
    const AT* pold = nullptr;
    AT beta = (AT)0, inv_n = (AT)1;
    for (int n = 0;; ++n) {
      const int st = n % kStages, use = n / kStages;
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
      const int q = ls.ch_prob[k];
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
      const int kl = k - ls.ch_base[q];
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
        info[st] = StageInfo{k, q, e1 - e0, p1 - p0, s1 - s0, (int)(skew / 4), e0 & (kJTile - 1)};
        fence_proxy_async();
        mbar_expect_tx(fb, bJ + bM + bP + bS);
        if (bJ) bulk_g2s(smem_u32(base + SL.j), static_cast<const JT*>(P->J) + (size_t)(e0 >> 5) * kJTile * NJ, bJ, fb);
        if (bM) bulk_g2s(smem_u32(base + SL.meta), reinterpret_cast<const void*>(ma), bM, fb);
        if (bP) bulk_g2s(smem_u32(base + SL.pt), static_cast<const unsigned char*>(P->pt_rec) + (size_t)p0 * PRB, bP, fb);
        if (bS) bulk_g2s(smem_u32(base + SL.slot), P->slot_rec + s0, bS, fb);
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
      for (int st = 0; st < kStages; ++st)
        if (last_use[st] >= 0) mbar_wait(smem_u32(&full[st]), (uint32_t)last_use[st] & 1u);
      if (s_fail) atomicExch(ls.err, 1);
    }
  } else {
    // ================================================================ consumer warps
    for (int n = 0;; ++n) {
      const int st = n % kStages;
      const bool ok = mbar_wait(smem_u32(&full[st]), (uint32_t)(n / kStages) & 1u);
      if (consumer_any(!ok)) {
        if (threadIdx.x == 0) s_fail = 1;
        break;
      }
      const StageInfo in = info[st];
      if (in.k < 0) break;
      const unsigned char* stg = smem + st * SL.size;
      const JT* Js = reinterpret_cast<const JT*>(stg + SL.j);
      const uint32_t* meta = reinterpret_cast<const uint32_t*>(stg + SL.meta) + in.skew;
      const unsigned char* prec = stg + SL.pt;
      const int4* srec = reinterpret_cast<const int4*>(stg + SL.slot);
      const AT* xs = reinterpret_cast<const AT*>(stg + SL.xs);
      // ---- pass 1: a_e = Jp^T (Jc x_c)
      for (int i = threadIdx.x; i < in.nE; i += kThreads) {
        AT row[NJ];
        load_row_t<NJ>(Js, (size_t)(i + in.jskew), row);
        AT a[3];
        edge_point_term<Mo>(row, xs + DC * (int)((meta[i] >> 10) & 1023u), a);
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) vv[kk * LD + i] = a[kk];
      }
      consumer_sync();
      // ---- pass 2: t_p = H_pp^-1 sum_e a_e
      for (int j = threadIdx.x; j < in.nP; j += kThreads) {
        const unsigned char* pr = prec + (size_t)j * PRB;
        const AT* hv = reinterpret_cast<const AT*>(pr);
        const int* se = reinterpret_cast<const int*>(pr + 6 * sizeof(AT));
        AT u[3];
        point_sum<JT>(vv, LD, se[0], se[1], u);
        AT t[3];
        mul3(hv, u, t);
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) tp[kk * LD + j] = t[kk];
      }
      consumer_sync();
      // ---- pass 3: v_e = Jc^T (Jp t_p), scattered to the edge's slot-sorted position
      for (int i = threadIdx.x; i < in.nE; i += kThreads) {
        AT row[NJ];
        load_row_t<NJ>(Js, (size_t)(i + in.jskew), row);
        const uint32_t m = meta[i];
        const int pl = (int)(m >> 20), pos = (int)(m & 1023u);
        AT v[DC];
        edge_camera_term<Mo>(row, tp[pl], tp[LD + pl], tp[2 * LD + pl], v);
#pragma unroll
        for (int kk = 0; kk < DC; ++kk) vv[kk * LD + pos] = v[kk];
      }
      consumer_sync();
      // ---- pass 4: per-slot sums over contiguous positions
      AT* partV = reinterpret_cast<AT*>(ls.probs[in.q].partV);
      for (int w = threadIdx.x; w < in.nS * DC; w += kThreads) {
        const int sl = w / DC, comp = w - sl * DC;
        const int4 r4 = srec[sl];
        partV[(size_t)r4.w * DC + comp] = seg_sum(vv + comp * LD, r4.x, r4.y);
      }
      consumer_sync();
      if (threadIdx.x == 0) mbar_arrive(smem_u32(&empty[st]), 1);
    }
  }
}


// ---------------------------------------------------------------- Schur product, pipelined persistent form

// Asynchronous global-to-shared copies of 4 and 16 bytes (the per-thread form; a
// group is committed per chunk and waited for one chunk later).
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Shared memory of the pipelined kernel: the passes' scratch (per-edge terms [VW][LD],
// point solutions [3][np_max + 1]), the slot cameras' search direction, two buffers of
// one chunk's index copies (packed edge words, slot records), and one buffer of point
// records (refilled for the next chunk once pass 2 has read it: a second buffer would
// leave less of the SM's memory to L1).
struct PipeLayout {
  uint32_t tp, xs, buf;          // offsets
  uint32_t meta, srec, prec;     // offsets inside a buffer
  uint32_t bsize, size;
};
template <class Mo>
__host__ __device__ inline PipeLayout pipe_layout(size_t sA, int ch_max, int np_max, int ns_max) {
  auto al = [](uint32_t v) { return (v + 15u) & ~15u; };
  const uint32_t prb = (uint32_t)((6 * sA + 8 + 15) & ~(size_t)15);
  const int vw = Mo::DC > 3 ? Mo::DC : 3;
  PipeLayout L;
  L.tp = al((uint32_t)(vw * (size_t)(ch_max + 1) * sA));
  L.xs = L.tp + al((uint32_t)(3 * (size_t)(np_max + 1) * sA));
  L.buf = L.xs + al((uint32_t)(ns_max * Mo::DC * sA));
  L.meta = 0;
  L.srec = al((uint32_t)ch_max * 4u);
  L.bsize = L.srec + al((uint32_t)ns_max * 16u);
  L.prec = L.buf + 2 * L.bsize;                // one buffer of point records
  L.size = L.prec + al((uint32_t)np_max * prb);
  return L;
}

struct PipeChunk {
  int k, q, kl, e0, nE, p0, nP, s0, nS;   // k < 0: no more chunks
};

// The classic Schur product's passes as a persistent kernel.  CTAs take chunks from a
// shared counter (skipping problems whose PCG has stopped), so a CTA that starts late
// -- the launch overlaps its predecessor's tail -- simply takes fewer; which CTA sums
// a chunk does not change any result.  While a chunk's passes run, every thread has
// already issued its share of the next chunk's index copies (packed edge words, slot
// records) into the other of two shared-memory buffers and, once pass 2 is done, of its
// point records, the next chunk's Jacobian tiles are being prefetched into L2, the
// chunk after that is being taken, and the next chunk's search-direction gather
// overlaps pass 3.  The sums and
// their order are those of k_spmv (bit-identical results).  The last CTA to finish
// puts the counters back to 0.  Requires chunks of at most 1024 edges.
//
// PipeOcc: resident CTAs per SM the register budget targets.  BF16 rows are re-read
// from L2 anyway, so more CTAs win; FP32 rows are twice as long and their second read
// hits L1 only while fewer CTAs share it; FP64 is limited by shared memory.
//
// kCH: the launch's chunk bound (ls.ch_max) when known at compile time (0: read at run
// time), so that the per-edge terms' row stride in shared memory is an immediate offset.
template <class JT> struct PipeOcc { static constexpr int value = sizeof(JT) == 2 ? 5 : (sizeof(JT) == 4 ? 4 : 2); };
template <class Mo, class JT, int EPT, int kCH = 0>
__global__ void __launch_bounds__(kThreads, PipeOcc<JT>::value) k_spmv_pp(LaunchSet ls) {
  using AT = typename AccOf<JT>::T;
  using Dm = Dims<Mo>;
  constexpr int DC = Mo::DC, DB = Mo::DB, NJ = Mo::NJ;
  constexpr size_t PRB = (6 * sizeof(AT) + 8 + 15) & ~(size_t)15;
  constexpr int kWords = (int)(sizeof(DevBA) / 4);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevBA d;
  __shared__ PipeChunk ck[3];
  pdl_trigger();
  const int CH = kCH ? kCH : ls.ch_max, LD = CH + 1, LP = ls.np_max + 1;
  const PipeLayout PL = pipe_layout<Mo>(sizeof(AT), CH, ls.np_max, ls.ns_max);
  AT* vv = reinterpret_cast<AT*>(smem);                 // [VW][LD]; rows 0..2 hold a_e in pass 1
  AT* tp = reinterpret_cast<AT*>(smem + PL.tp);         // [3][LP] point solutions
  AT* xs = reinterpret_cast<AT*>(smem + PL.xs);         // [ns_max][DC] slot cameras' direction
  unsigned char* bufs = smem + PL.buf;
  int bound_q = -1;              // problem whose descriptor is in d
  pdl_wait();

  // The next chunk from the shared counter whose problem still iterates (-1: none
  // left).  The problems' scalars do not change during the launch; a one-problem
  // launch checks them once, a batch skips a stopped problem's remaining chunks.
  auto grab = [&]() -> int {
    for (;;) {
      const int k = atomicAdd(ls.work, 1);
      if (k >= ls.n_ch) return -1;
      if (ls.nprob == 1) return k;
      const int q = ls.ch_prob[k];
      const Scalars* sc = ls.probs[q].sc;
      if (sc->active && !sc->pcg_done) return k;
    }
  };
  // a CTA that has taken its last chunk; the last one resets the counters
  auto finish = [&]() {
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(ls.work + 1, 1) == (int)gridDim.x - 1) {
        ls.work[0] = 0;
        ls.work[1] = 0;
      }
    }
  };
  // a chunk's problem and ranges (thread 0)
  auto plan = [&](int k) -> PipeChunk {
    PipeChunk c;
    c.k = k;
    if (k < 0) return c;
    const int q = ls.nprob == 1 ? 0 : ls.ch_prob[k];
    const int kl = ls.nprob == 1 ? k : k - ls.ch_base[q];
    const DevBA* P = q == bound_q ? &d : ls.probs + q;
    const int* ce = P->ch_e0;
    const int* cp = P->ch_p0;
    const int* cs = P->ch_s0;
    c.q = q; c.kl = kl;
    c.e0 = ce[kl]; c.nE = ce[kl + 1] - c.e0;
    c.p0 = cp[kl]; c.nP = cp[kl + 1] - c.p0;
    c.s0 = cs[kl]; c.nS = cs[kl + 1] - c.s0;
    return c;
  };
  // every thread's share of a chunk's index copies, and the L2 prefetch of its tiles
  auto issue = [&](const PipeChunk& c, int b, int bound) {
    if (c.k < 0) return;
    const DevBA* P = c.q == bound ? &d : ls.probs + c.q;
    unsigned char* B = bufs + b * PL.bsize;
    const uint32_t* meta = P->e_meta + c.e0;
    for (int i = threadIdx.x; i < c.nE; i += kThreads) cp_async4(B + PL.meta + 4 * i, meta + i);
    const int4* sr = P->slot_rec + c.s0;
    for (int t = threadIdx.x; t < c.nS; t += kThreads) cp_async16(B + PL.srec + 16 * t, sr + t);
    if (threadIdx.x == 0 && c.nE > 0) {
      const size_t t0 = (size_t)c.e0 >> 5, t1 = (size_t)(c.e0 + c.nE - 1) >> 5;
      prefetch_l2(static_cast<const JT*>(P->J) + t0 * kJTile * NJ,
                  (uint32_t)((t1 - t0 + 1) * kJTile * NJ * sizeof(JT)));
    }
  };

  // a chunk's point records into the one point-record buffer
  auto issue_prec = [&](const PipeChunk& c, int bound) {
    if (c.k < 0) return;
    const DevBA* P = c.q == bound ? &d : ls.probs + c.q;
    const unsigned char* pr = static_cast<const unsigned char*>(P->pt_rec) + (size_t)c.p0 * PRB;
    const int pieces = (int)(c.nP * (PRB / 16));
    for (int u = threadIdx.x; u < pieces; u += kThreads) cp_async16(smem + PL.prec + 16 * u, pr + 16 * u);
  };
  // the slot cameras' search direction p = (z + beta p_old) / n of a chunk whose slot
  // records are in buffer b
  auto gather = [&](const PipeChunk& c, int b) {
    if (c.k < 0) return;
    const DevBA* P = c.q == bound_q ? &d : ls.probs + c.q;
    const int4* srec = reinterpret_cast<const int4*>(bufs + b * PL.bsize + PL.srec);
    const Scalars* sc = P->sc;
    const int restart = sc->restart;     // a restart's product is taken of x
    const AT* zv = reinterpret_cast<const AT*>(restart ? P->x : P->z);
    const AT* pold = restart ? zv : reinterpret_cast<const AT*>(sc->pidx ? P->p2 : P->p);
    const AT beta = restart ? (AT)0 : sc_beta<AT>(sc), inv_n = restart ? (AT)1 : sc_inv_n<AT>(sc);
    for (int w = threadIdx.x; w < c.nS * DC; w += kThreads) {
      const int sl = w / DC, k = w - sl * DC;
      const size_t o = DB * (size_t)srec[sl].z + k;
      xs[w] = (zv[o] + beta * pold[o]) * inv_n;
    }
  };

  if (ls.nprob == 1) {          // a one-problem launch stops at once if its PCG has
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
  issue(ck[0], 0, -1);
  issue_prec(ck[0], -1);
  cp_async_commit();
  for (int n = 0;; ++n) {
    const int b = n & 1;
    const PipeChunk c = ck[n % 3];
    if (c.k < 0) break;
    const PipeChunk cn = ck[(n + 1) % 3];
    if (c.q != bound_q) {        // CTA-uniform: bind the chunk's problem
      __syncthreads();           // every thread is past the previous use of d
      for (int i = threadIdx.x; i < kWords; i += kThreads)
        reinterpret_cast<int*>(&d)[i] = reinterpret_cast<const int*>(ls.probs + c.q)[i];
      bound_q = c.q;
      __syncthreads();
    }
    issue(cn, b ^ 1, bound_q);
    cp_async_commit();
    // Buffer b: the first chunk's copies are waited for here; a later chunk's landed
    // at the end of the previous chunk's pass 1 (wait_all, then the barrier before its
    // pass 2), and its search direction was gathered in the previous pass 3 -- no
    // barrier needed.  The chunk's point records are waited for at the end of pass 1.
    if (n == 0) {
      cp_async_wait_prev();
      __syncthreads();
    }

    unsigned char* B = bufs + b * PL.bsize;
    const uint32_t* meta = reinterpret_cast<const uint32_t*>(B + PL.meta);
    const int4* srec = reinterpret_cast<const int4*>(B + PL.srec);
    const unsigned char* prec = smem + PL.prec;
    if (n == 0) gather(c, b);    // later chunks' directions were gathered one chunk ahead
    int pos[EPT], slot[EPT], ptl[EPT];
#pragma unroll
    for (int m = 0; m < EPT; ++m) {
      const int i = threadIdx.x + m * kThreads;
      if (i < c.nE) {
        const uint32_t w = meta[i];
        pos[m] = (int)(w & 1023u);
        slot[m] = (int)((w >> 10) & 1023u);
        ptl[m] = (int)(w >> 20);
      }
    }
    if (n == 0) __syncthreads();   // the first chunk's direction gather
    const JT* Jg = reinterpret_cast<const JT*>(d.J);
    // ---- pass 1: a_e = Jp^T (Jc x_c)
#pragma unroll
    for (int m = 0; m < EPT; ++m) {
      const int i = threadIdx.x + m * kThreads;
      if (i >= c.nE) break;
      AT row[NJ];
      load_row_t<NJ>(Jg, (size_t)(c.e0 + i), row);
      AT a[3];
      edge_point_term<Mo>(row, xs + DC * slot[m], a);
#pragma unroll
      for (int k = 0; k < 3; ++k) vv[k * LD + i] = a[k];
    }
    cp_async_wait_all();         // this chunk's point records, the next chunk's indices
    __syncthreads();
    // ---- pass 2: t_p = H_pp^-1 sum_e a_e; meanwhile the last warp's first thread
    // locates the chunk after next (its loads overlap the pass)
    if (threadIdx.x == kThreads - 32) ck[(n + 2) % 3] = plan(cn.k < 0 ? -1 : grab());
    for (int j = threadIdx.x; j < c.nP; j += kThreads) {
      const AT* hv = reinterpret_cast<const AT*>(prec + (size_t)j * PRB);
      const int* se = reinterpret_cast<const int*>(prec + (size_t)j * PRB + 6 * sizeof(AT));
      AT u[3];
      point_sum<JT>(vv, LD, se[0], se[1], u);
      AT t[3];
      mul3(hv, u, t);
#pragma unroll
      for (int k = 0; k < 3; ++k) tp[k * LP + j] = t[k];
    }
    __syncthreads();
    issue_prec(cn, bound_q);     // pass 2 was the last reader of the point records
    cp_async_commit();
    // the next chunk's search direction (its slot records have landed; this chunk's
    // pass 1 was the last reader of xs), overlapping pass 3
    gather(cn, b ^ 1);
    // ---- pass 3: v_e = Jc^T (Jp t_p), scattered to the edge's slot-sorted position
#pragma unroll
    for (int m = 0; m < EPT; ++m) {
      const int i = threadIdx.x + m * kThreads;
      if (i >= c.nE) break;
      AT row[NJ];
      load_row_t<NJ>(Jg, (size_t)(c.e0 + i), row);
      const int pl = ptl[m];
      AT v[DC];
      edge_camera_term<Mo>(row, tp[pl], tp[LP + pl], tp[2 * LP + pl], v);
#pragma unroll
      for (int k = 0; k < DC; ++k) vv[k * LD + pos[m]] = v[k];
    }
    __syncthreads();
    // ---- pass 4: per-slot sums over contiguous positions
    AT* partV = reinterpret_cast<AT*>(d.partV);
    for (int w = threadIdx.x; w < c.nS * DC; w += kThreads) {
      const int sl = w / DC, comp = w - sl * DC;
      const int4 r4 = srec[sl];
      partV[(size_t)r4.w * DC + comp] = seg_sum(vv + comp * LD, r4.x, r4.y);
    }
    __syncthreads();             // vv, xs and buffer b are free again
  }
  cp_async_wait_all();           // no copy may still be landing when the CTA exits
  finish();
}

}  // namespace gpo
