// Schur product with dynamic Jacobians (Sec. IV-D: Jacobians may be recomputed where
// they are used instead of being stored).  The same passes and sums as the classic
// one-CTA-per-chunk product, but each edge's whitened, IRLS-weighted rows are evaluated
// from the current state (render block, point, measurement) in the accumulation type,
// once per product, and kept in registers between the two passes that use them.  With
// FP64 accumulation the rows equal the stored ones bit for bit, so the product is
// bit-identical to the stored-row product; with FP32 accumulation it uses the unrounded
// FP32 rows where the stored path reads BF16 or FP32 copies.
#pragma once

#include "schur_common.cuh"

namespace gpo {

// The row of edge e in the stored layout (camera rows M x DC, then point rows M x 3),
// with the fixed-vertex columns zeroed, as k_linearize forms it.
template <class Mo, class AT>
__device__ __forceinline__ void dyn_row(const DevBA& d, int e, AT (&row)[Dims<Mo>::NJU]) {
  constexpr int M = Mo::M, DC = Mo::DC, JP0 = Dims<Mo>::JP0;
  const int c = __ldg(d.e_cam + e), p = __ldg(d.e_pt + e);
  double rb[16];
  load_rb(d.camrb + 16 * (size_t)c, rb);
  const double X[3] = {d.pt[3 * (size_t)p], d.pt[3 * (size_t)p + 1], d.pt[3 * (size_t)p + 2]};
  AT r[M], sw;
  AT Jc[M][DC], Jp[M][3];
  Mo::template eval<AT>(d, e, rb, d.camrbf + 16 * (size_t)c, X, r, sw, Jc, Jp);
  const bool cf = d.cam_fixed[c] != 0, pf = d.pt_fixed[p] != 0;
#pragma unroll
  for (int a = 0; a < M; ++a) {
#pragma unroll
    for (int k = 0; k < DC; ++k) row[a * DC + k] = cf ? (AT)0 : Jc[a][k];
#pragma unroll
    for (int k = 0; k < 3; ++k) row[JP0 + 3 * a + k] = pf ? (AT)0 : Jp[a][k];
  }
}

// The row of edge e for the per-edge kernels: read from storage, or (kDyn: dynamic
// Jacobians, no rows stored) evaluated from the current state in the accumulation type.
template <class Mo, class JT, class AT, bool kDyn>
__device__ __forceinline__ void row_of(const DevBA& d, const JT* J, int e, AT (&row)[Mo::NJ]) {
  if constexpr (kDyn) {
    constexpr int NJU = Dims<Mo>::NJU;
    AT r[NJU];
    dyn_row<Mo, AT>(d, e, r);
#pragma unroll
    for (int k = 0; k < NJU; ++k) row[k] = r[k];
#pragma unroll
    for (int k = NJU; k < Mo::NJ; ++k) row[k] = (AT)0;
  } else {
    load_row_t<Mo::NJ>(J, (size_t)e, row);
  }
}

template <class Mo, class AT, int EPT>
__global__ void __launch_bounds__(kThreads) k_spmv_dyn(LaunchSet ls) {
  constexpr int DC = Mo::DC, DB = Mo::DB, NJU = Dims<Mo>::NJU, VW = Dims<Mo>::VW;
  GPO_BIND(ch, kl)
  const Scalars* sc = d.sc;
  const ChunkRange cr = chunk_range(d, kl);
  const int act = sc->active, done = sc->pcg_done, pidx = sc->pidx, restart = sc->restart;
  const AT beta_a = sc_beta<AT>(sc), inv_n_a = sc_inv_n<AT>(sc);
  if (!act || done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int CH = d.ch_max, LD = CH + 1;
  AT* vv = reinterpret_cast<AT*>(smem);        // [VW][LD]
  AT* tp = vv + VW * LD;                       // [3][LD] point solutions
  AT* xs = tp + 3 * LD;                        // [ls.ns_max][DC] slot camera vectors
  AT* hv = xs + DC * ls.ns_max;                // [ls.np_max][6] point inverses
  int* po = reinterpret_cast<int*>(hv + 6 * ls.np_max);
  int* so = po + ls.np_max + 1;
  int* sp = so + ls.ns_max + 1;

  // chunks of at most 1024 edges (the only ones this kernel is launched for): one packed
  // word of positions per edge
  int pos[EPT], slot[EPT], ptl[EPT];
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const int i = threadIdx.x + m * kThreads;
    if (i < cr.nE) {
      const uint32_t w = __ldg(d.e_meta + cr.e0 + i);
      pos[m] = (int)(w & 1023u);
      slot[m] = (int)((w >> 10) & 1023u);
      ptl[m] = (int)(w >> 20);
    }
  }
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

  // the rows, evaluated while the records above land
  AT row[EPT][NJU];
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const int i = threadIdx.x + m * kThreads;
    if (i < cr.nE) dyn_row<Mo, AT>(d, cr.e0 + i, row[m]);
  }
  __syncthreads();

  // ---- pass 1: a_e = Jp^T (Jc x_c)
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const int i = threadIdx.x + m * kThreads;
    if (i >= cr.nE) break;
    AT a[3];
    edge_point_term<Mo>(row[m], xs + DC * slot[m], a);
#pragma unroll
    for (int k = 0; k < 3; ++k) vv[k * LD + i] = a[k];
  }
  __syncthreads();
  // ---- pass 2: t_p = H_pp^-1 sum_e a_e
  for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
    AT u[3];
    point_sum<AT>(vv, LD, po[j], po[j + 1], u);
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
    const int pl = ptl[m];
    AT v[DC];
    edge_camera_term<Mo>(row[m], tp[pl], tp[LD + pl], tp[2 * LD + pl], v);
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

}  // namespace gpo
