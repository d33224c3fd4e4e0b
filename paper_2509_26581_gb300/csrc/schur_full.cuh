// PCG on the full damped system (cameras and points together): the paper's own form
// of the solve (Sec. IV-E: an implicit block-Jacobi PCG on the normal equations of all
// vertices, products formed from the stored per-edge Jacobians), beside the camera
// Schur complement that is the default.  Both solve (H + lambda D) dx = -b, so an
// exact solve of either gives the same LM step.
//
// The camera rows reuse the Schur path's camera kernels (k_cam_finalize with the
// camera block (H_cc + lambda D_c)^-1 as preconditioner and -b_c as right-hand side,
// k_cam_apply adding instead of subtracting the edges' camera terms, pcg_update_body);
// the point rows live in [P][3] vectors of the accumulation type, with the point
// blocks (H_pp + lambda D_p)^-1 of k_schur_prepare as preconditioner.  One-problem
// launches only.
#pragma once

#include "schur_common.cuh"

namespace gpo {

// Start of a full-system solve, point rows (one thread per point): r = g = -b_p,
// z = (H_pp + lambda D_p)^-1 r, x = 0, p_{-1} = 0, and each block's (r^T z, |r|^2)
// for k_cam_finalize's last CTA, which adds them to the camera rows'.
template <class Mo, class AT>
__global__ void __launch_bounds__(256) k_full_init(LaunchSet ls) {
  __shared__ double red[kThreads];
  GPO_BIND(pb, pbl)
  if (!d.sc->active || !d.sc->full) return;
  const int p = pbl * 256 + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (p < d.P) {
    const AT* bp = reinterpret_cast<const AT*>(d.bp) + 3 * (size_t)p;
    const AT* Hi = reinterpret_cast<const AT*>(d.Hinv) + 6 * (size_t)p;
    AT h[6], r[3], z[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = Hi[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = -bp[k];
    mul3(h, r, z);
    AT rz_a = (AT)0, rr_a = (AT)0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const size_t o = 3 * (size_t)p + k;
      reinterpret_cast<AT*>(d.rq)[o] = r[k];
      reinterpret_cast<AT*>(d.zq)[o] = z[k];
      reinterpret_cast<AT*>(d.xq)[o] = (AT)0;
      reinterpret_cast<AT*>(d.xqbest)[o] = (AT)0;
      reinterpret_cast<AT*>(d.pq)[o] = (AT)0;
      rz_a += r[k] * z[k];
      rr_a += r[k] * r[k];
    }
    rz = (double)rz_a;
    rr = (double)rr_a;
  }
  const double a = block_sum(rz, red);
  __syncthreads();
  const double b = block_sum(rr, red);
  if (threadIdx.x == 0) {
    d.pt_part[2 * pbl] = a;
    d.pt_part[2 * pbl + 1] = b;
  }
}

// Product with the whole damped system, y = (H + lambda D) v, one CTA per chunk of
// point-major edges.  The diagonal blocks are applied whole ((H_pp + lambda D_p) v_p
// here, (H_cc + lambda D_c) v_c in k_cam_apply), so each edge adds only its coupling
// terms: J_p^T (J_c v_c) to its point (summed over the point's edges, which all lie in
// the chunk: the point rows of y, written here) and J_c^T (J_p v_p) to its camera
// (summed per chunk slot into the same partial rows as the Schur product).  The chunk's share of v^T y over
// its points goes to md_part[chunk] for the camera half's alpha.  v is the direction
// p = (z + beta p_old) / n (or x in a restart iteration), formed here for the points
// (and written to the other direction buffer) and, as in the Schur product, for each
// slot camera.  Each Jacobian row is read once.
template <class Mo, class JT>
__global__ void __launch_bounds__(kThreads) k_full_spmv(LaunchSet ls) {
  using AT = typename AccOf<JT>::T;
  using Dm = Dims<Mo>;
  constexpr int M = Mo::M, DC = Mo::DC, DB = Mo::DB, NJ = Mo::NJ, JP0 = Dm::JP0;
  __shared__ double red[kThreads];
  GPO_BIND(ch, kl)
  const Scalars* sc = d.sc;
  const ChunkRange cr = chunk_range(d, kl);
  const int act = sc->active, done = sc->pcg_done, pidx = sc->pidx, restart = sc->restart;
  const int save_best = sc->save_best;
  const AT beta_a = sc_beta<AT>(sc), inv_n_a = sc_inv_n<AT>(sc);
  const double lam_d = sc->lambda;
  if (!act || done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int CH = d.ch_max, LD = CH + 1;
  AT* vv = reinterpret_cast<AT*>(smem);        // [DC][LD] camera terms, slot-sorted positions
  AT* tv = vv + DC * LD;                       // [3][LD] point terms, edge order
  AT* xs = tv + 3 * LD;                        // [ns_max][DC] slot camera directions
  AT* vp = xs + DC * ls.ns_max;                // [np_max][3] point directions
  int* po = reinterpret_cast<int*>(vp + 3 * ls.np_max);   // [np + 1] local point offsets
  int* so = po + ls.np_max + 1;                           // [ns + 1] local slot offsets
  int* sp = so + ls.ns_max + 1;                           // [ns] camera-major slot rows
  const JT* Jg = reinterpret_cast<const JT*>(d.J);
  const AT beta = restart ? (AT)0 : beta_a, inv_n = restart ? (AT)1 : inv_n_a;
  // the packed positions of this thread's edges (up to four: chunks of at most 1,024
  // edges) are loaded ahead of the gathers, so their latency overlaps them
  const bool packed = ls.ch_max <= 1024;
  uint32_t mw[4] = {0u, 0u, 0u, 0u};
  if (packed) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = threadIdx.x + m * kThreads;
      if (i < cr.nE) mw[m] = __ldg(d.e_meta + cr.e0 + i);
    }
  }
  // slot cameras: record and direction (the Schur product's gather)
  {
    const AT* zv = reinterpret_cast<const AT*>(restart ? d.x : d.z);
    const AT* pold = restart ? zv : reinterpret_cast<const AT*>(pidx ? d.p2 : d.p);
    for (int t = threadIdx.x; t < cr.nS; t += kThreads) {
      const int4 r4 = __ldg(d.slot_rec + cr.s0 + t);
      so[t] = r4.x;
      so[t + 1] = r4.y;
      sp[t] = r4.w;
      const size_t o = DB * (size_t)r4.z;
#pragma unroll
      for (int k = 0; k < DC; ++k) xs[DC * t + k] = (zv[o + k] + beta * pold[o + k]) * inv_n;
    }
  }
  // chunk points: edge range and direction (written for the update)
  {
    constexpr size_t PRB = (6 * sizeof(AT) + 8 + 15) & ~(size_t)15;
    const unsigned char* prec = static_cast<const unsigned char*>(d.pt_rec) + (size_t)cr.p0 * PRB;
    const AT* zq = reinterpret_cast<const AT*>(restart ? d.xq : d.zq);
    const AT* pold = restart ? zq : reinterpret_cast<const AT*>(pidx ? d.pq2 : d.pq);
    AT* pnew = reinterpret_cast<AT*>(pidx ? d.pq : d.pq2);
    for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
      const int* se = reinterpret_cast<const int*>(prec + (size_t)j * PRB + 6 * sizeof(AT));
      po[j] = se[0];
      po[j + 1] = se[1];
      const size_t o = 3 * (size_t)(cr.p0 + j);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const AT v = (zq[o + k] + beta * pold[o + k]) * inv_n;
        vp[3 * j + k] = v;
        if (!restart) pnew[o + k] = v;
        if (save_best) reinterpret_cast<AT*>(d.xqbest)[o + k] = reinterpret_cast<const AT*>(d.xq)[o + k];
      }
    }
  }
  if (threadIdx.x == 0 && cr.nP == 0) po[0] = 0;
  if (threadIdx.x == 0 && cr.nS == 0) so[0] = 0;
  __syncthreads();

  // ---- per edge: the point term J_p^T (J_c v_c) (edge order) and the camera term
  // J_c^T (J_p v_p) (slot-sorted position)
  auto edge = [&](int i, int pos, int slot, int ptl) {
    AT row[NJ];
    load_row_t<NJ>(Jg, (size_t)(cr.e0 + i), row);
    const AT* xc = xs + DC * slot;
    const AT* xp = vp + 3 * ptl;
    AT qc[M], qp[M];   // J_c v_c and J_p v_p
#pragma unroll
    for (int a = 0; a < M; ++a) {
      qp[a] = row[JP0 + 3 * a] * xp[0] + row[JP0 + 3 * a + 1] * xp[1] + row[JP0 + 3 * a + 2] * xp[2];
      qc[a] = (AT)0;
    }
#pragma unroll
    for (int k = 0; k < DC; ++k) {
      const AT xk = xc[k];
#pragma unroll
      for (int a = 0; a < M; ++a) qc[a] += row[a * DC + k] * xk;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      AT t = row[JP0 + k] * qc[0];
#pragma unroll
      for (int a = 1; a < M; ++a) t += row[JP0 + 3 * a + k] * qc[a];
      tv[k * LD + i] = t;
    }
#pragma unroll
    for (int k = 0; k < DC; ++k) {
      AT v = row[k] * qp[0];
#pragma unroll
      for (int a = 1; a < M; ++a) v += row[a * DC + k] * qp[a];
      vv[k * LD + pos] = v;
    }
  };
  if (packed) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = threadIdx.x + m * kThreads;
      if (i >= cr.nE) break;
      edge(i, (int)(mw[m] & 1023u), (int)((mw[m] >> 10) & 1023u), (int)(mw[m] >> 20));
    }
  } else {
    for (int i = threadIdx.x; i < cr.nE; i += kThreads)
      edge(i, __ldg(d.e_pos + cr.e0 + i), __ldg(d.e_slot + cr.e0 + i), __ldg(d.e_pt + cr.e0 + i) - cr.p0);
  }
  __syncthreads();
  // ---- point rows: y_p = (H_pp + lambda D_p) v_p + sum_e J_p^T J_c v_c
  const AT lam = (AT)lam_d;
  const AT* Hpp = reinterpret_cast<const AT*>(d.Hpp);
  AT* yq = reinterpret_cast<AT*>(d.yq);
  double dot = 0.0;
  for (int j = threadIdx.x; j < cr.nP; j += kThreads) {
    const int pj = cr.p0 + j;
    AT u[3];
    point_sum<JT>(tv, LD, po[j], po[j + 1], u);
    AT h[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = Hpp[6 * (size_t)pj + k];
    h[0] += lam * damp_diag(h[0], sc);
    h[3] += lam * damp_diag(h[3], sc);
    h[5] += lam * damp_diag(h[5], sc);
    AT hv[3];
    mul3(h, vp + 3 * j, hv);
    AT da = (AT)0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const AT y = hv[k] + u[k];
      yq[3 * (size_t)pj + k] = y;
      da += vp[3 * j + k] * y;
    }
    dot += (double)da;
  }
  // ---- camera terms: per-slot sums over contiguous positions
  AT* partV = reinterpret_cast<AT*>(d.partV);
  for (int w = threadIdx.x; w < cr.nS * DC; w += kThreads) {
    const int sl = w / DC, comp = w - sl * DC;
    partV[(size_t)sp[sl] * DC + comp] = seg_sum(vv + comp * LD, so[sl], so[sl + 1]);
  }
  const double s = block_sum(dot, red);
  if (threadIdx.x == 0) d.md_part[kl] = s;
}

// Update of a full-system PCG iteration: CTAs 0 .. ncblk-1 are the camera blocks
// (pcg_update_body: x, r, z = M r over the camera rows), the rest point blocks of
// kUpdatePoints points, eight per thread (x += sigma alpha p, r <- r / n - alpha y, or
// the true residual g - y in a restart iteration, z = (H_pp + lambda D_p)^-1 r); large
// point blocks keep the last-CTA ticket and the final sum short.  Every CTA writes its (r^T z,
// |r|^2); the last one of the grid sums camera then point partials and applies the
// stopping rules (pcg_update_finish).
template <class Mo, class AT>
__global__ void __launch_bounds__(kCamPerBlock * 32) k_full_update(LaunchSet ls) {
  static_assert(kCamPerBlock * 32 == 256, "point blocks are 256 threads");
  __shared__ double red[kCamPerBlock][2];
  __shared__ double redp[kThreads];
  __shared__ DevBA d;
  pdl_trigger();
  bind_problem(d, ls.probs);
  pdl_wait();
  const int b = blockIdx.x;
  if (b < d.ncblk) {
    UpdateIn<Mo, AT> in;
    pcg_update_load<Mo, AT>(d, b, in);
    pcg_update_body<Mo, AT>(ls, d, b, red, in);
    return;
  }
  Scalars* sc = d.sc;
  if (!sc->active || sc->pcg_done) return;
  const int pbl = b - d.ncblk;
  const int restart = sc->restart;
  double rz = 0.0, rr = 0.0;
  for (int p = pbl * kUpdatePoints + threadIdx.x; p < min(d.P, (pbl + 1) * kUpdatePoints); p += kThreads) {
    const AT alpha = (AT)sc->alpha, sa = (AT)(sc->sigma * sc->alpha), sn = sc_inv_n<AT>(sc);
    const size_t o = 3 * (size_t)p;
    AT* x = reinterpret_cast<AT*>(d.xq) + o;
    AT* r = reinterpret_cast<AT*>(d.rq) + o;
    AT* z = reinterpret_cast<AT*>(d.zq) + o;
    const AT* y = reinterpret_cast<const AT*>(d.yq) + o;
    const AT* pv = reinterpret_cast<const AT*>(sc->pidx ? d.pq : d.pq2) + o;
    const AT* bp = reinterpret_cast<const AT*>(d.bp) + o;
    const AT* Hi = reinterpret_cast<const AT*>(d.Hinv) + 6 * (size_t)p;
    AT h[6], ri[3], zi[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = Hi[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (restart) {
        ri[k] = -bp[k] - y[k];
      } else {
        x[k] = x[k] + sa * pv[k];
        ri[k] = r[k] * sn - alpha * y[k];
      }
      r[k] = ri[k];
    }
    mul3(h, ri, zi);
    AT rz_a = (AT)0, rr_a = (AT)0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      z[k] = zi[k];
      rz_a += ri[k] * zi[k];
      rr_a += ri[k] * ri[k];
    }
    rz += (double)rz_a;
    rr += (double)rr_a;
  }
  const double a = block_sum(rz, redp);
  const double c = block_sum(rr, redp);
  if (threadIdx.x == 0) {
    d.pt_part[2 * pbl] = a;
    d.pt_part[2 * pbl + 1] = c;
  }
  pcg_update_finish(ls, d, restart);
}

}  // namespace gpo
