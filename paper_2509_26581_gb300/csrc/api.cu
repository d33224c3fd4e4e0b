// C ABI of libgpo: graph construction, topology finalisation and memory planning,
// the Levenberg-Marquardt driver and the diagnostic entry points.
//
// Construction follows the paper's problem statement (Listings 3-5: descriptors
// with reserve / add_vertex / add_factor, set_fixed / set_active, then
// levenberg_marquardt(graph, options)); see include/gpo.h for the contract.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "graph.h"

namespace {
thread_local std::string g_create_err;
}

gpo_status gpo_host::fail(gpo_graph* g, gpo_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (g) g->err = buf;
  else g_create_err = buf;
  return st;
}

using gpo_host::fail;

namespace {

int tangent_dim(int kind) { return kind == GPO_V_BA_CAMERA9 ? 9 : (kind == GPO_V_NAV15 ? 15 : 3); }
int state_dim(int kind) { return kind == GPO_V_BA_CAMERA9 ? 9 : (kind == GPO_V_NAV15 ? 16 : 3); }
bool is_camera(int kind) { return kind == GPO_V_BA_CAMERA9 || kind == GPO_V_NAV15; }
int tri(int n) { return n * (n + 1) / 2; }

// Upper-triangular U with Omega = U^T U (U = L^T of the Cholesky factor L of Omega),
// row-major m x m.  False if Omega is not symmetric positive definite.
bool sqrt_info(const double* Om, int m, double* U) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(Om[i * m + j] - Om[j * m + i]) > 1e-12 * (std::fabs(Om[i * m + i]) + std::fabs(Om[j * m + j])))
        return false;
  double L[81] = {};
  for (int j = 0; j < m; ++j) {
    double s = Om[j * m + j];
    for (int k = 0; k < j; ++k) s -= L[j * m + k] * L[j * m + k];
    if (!(s > 0.0) || !std::isfinite(s)) return false;
    L[j * m + j] = std::sqrt(s);
    for (int i = j + 1; i < m; ++i) {
      double t = Om[i * m + j];
      for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
      L[i * m + j] = t / L[j * m + j];
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) U[i * m + j] = L[j * m + i];
  return true;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device memory plan: requests are laid out in one arena (256-byte aligned).  Requests
// with a host source (`up`) come first, so the arena's prefix is one host image that a
// single copy uploads.
struct Plan {
  struct Req { void** ptr; size_t bytes; const void* src; size_t src_bytes; };
  std::vector<Req> reqs;
  template <class T> void add(T** p, size_t count) {
    reqs.push_back({reinterpret_cast<void**>(p), count * sizeof(T), nullptr, 0});
  }
  void add_raw(void** p, size_t bytes) { reqs.push_back({p, bytes, nullptr, 0}); }
  // an array uploaded from `src` (count elements); the allocation may be larger
  template <class T> void up(T** p, size_t count, const std::vector<T>& src) {
    reqs.push_back({reinterpret_cast<void**>(p), std::max(count, src.size()) * sizeof(T), src.data(),
                    src.size() * sizeof(T)});
  }
  size_t total() const {
    size_t t = 0;
    for (auto& r : reqs) t = align_up(t, 256) + align_up(r.bytes, 256);
    return t;
  }
  // bytes of the uploaded prefix and its host image
  size_t image(std::vector<char>& out) const {
    size_t t = 0, end = 0;
    for (auto& r : reqs) {
      t = align_up(t, 256);
      if (r.src) end = t + r.src_bytes;
      t += align_up(r.bytes, 256);
    }
    out.assign(end, 0);
    t = 0;
    for (auto& r : reqs) {
      t = align_up(t, 256);
      if (r.src && r.src_bytes) std::memcpy(out.data() + t, r.src, r.src_bytes);
      t += align_up(r.bytes, 256);
    }
    return end;
  }
  void assign(char* base) const {
    size_t t = 0;
    for (auto& r : reqs) {
      t = align_up(t, 256);
      *r.ptr = base + t;
      t += align_up(r.bytes, 256);
    }
  }
};

size_t at_size(Prec p) { return p == Prec::F64 ? 8 : 4; }
size_t jt_size(Prec p) { return p == Prec::F64 ? 8 : (p == Prec::F32 ? 4 : 2); }

template <class T>
cudaError_t up(T* dst, const std::vector<T>& src, cudaStream_t st) {
  if (src.empty()) return cudaSuccess;
  return cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

// The row copies between a caller's buffer and the graph's rows (through idx: the
// graph's row of caller row i) take one value per thread over the flattened rows, so
// that a warp's accesses to the caller's buffer -- often page-locked host memory read
// or written in place over the host link -- form one contiguous 256-byte span.  (Two
// values per thread as 16-byte accesses measured no faster.)
// dst rows (through idx) = src rows; *changed = 1 if any value's bits differ (one store
// per CTA at most)
__global__ void k_assign_rows(double* dst, const double* src, const int32_t* idx, int n, int w, int* changed) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  int diff = 0;
  if (e < (size_t)n * w) {
    const int i = (int)(e / (size_t)w), k = (int)(e - (size_t)i * w);
    const int t = idx ? idx[i] : i;
    const double v = src[e];
    double* p = dst + (size_t)t * w + k;
    diff = __double_as_longlong(*p) != __double_as_longlong(v);
    *p = v;
  }
  if (__syncthreads_or(diff) && threadIdx.x == 0) *changed = 1;
}
// dst rows = src rows through idx (the caller's row i is the graph's row idx[i])
__global__ void k_gather_rows(double* dst, const double* src, const int32_t* idx, int n, int w) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * w) return;
  const int i = (int)(e / (size_t)w), k = (int)(e - (size_t)i * w);
  const int t = idx ? idx[i] : i;
  dst[e] = src[(size_t)t * w + k];
}

}  // namespace

void gpo_host::drop_pcg_graph(gpo_graph* g) {
  if (g->pcg_exec) cudaGraphExecDestroy(g->pcg_exec);
  g->pcg_exec = nullptr;
}

void gpo_host::release_device(gpo_graph* g) {
  drop_pcg_graph(g);
  for (void* b : {g->arena, g->full_buf}) {
    if (!b) continue;
    if (g->desc.alloc && g->desc.free) g->desc.free(b, g->desc.alloc_ctx);
    else cudaFree(b);
  }
  g->full_buf = nullptr;
  g->full_bytes = 0;
  g->arena = nullptr;
  g->arena_bytes = 0;
  g->finalized = false;
  g->state_same = false;
}

// ============================================================== topology

// Host-side preparation of a graph's device image: sorted topology, chunks, slots,
// per-edge data in sorted order, the memory plan and the host sources of the uploaded
// prefix of the arena.  Built once (a server plans at submit and uploads at admission)
// and dropped after the upload or when the topology changes.
struct Prepared {
  DevBA d{};
  int ch = 0, NCH = 0, npb = 0;
  size_t jpos = 0, bytes = 0;
  std::vector<int64_t> sorted_edge;
  std::vector<int32_t> pt_new2old, pt_old2new, x_sorted;
  // sources of the uploaded arrays
  std::vector<int32_t> e_cam_s, e_pt_s, pt_off, ch_e0, ch_p0, ch_s0, slot_e0, slot_cam, cam_s_off, cam_s_list,
      slot_pos, slot_rec, xi_s, xj_s, xk_s, xo_off, xk_off, xk_list, zeros_ch, zeros_cb, zeros_pb, zeros_small;
  std::vector<uint16_t> e_pos, e_slot, ch_sorted, ch_grp;
  std::vector<uint32_t> e_meta;
  std::vector<uint8_t> cam_fixed, pt_fixed_s;
  std::vector<double> obs_s, delta_s, info_s, xrec_s, cams, pts, xzeros;
  std::vector<Scalars> sc0;
  // device pointers assigned by the plan
  int *e_cam_d = nullptr, *e_pt_d = nullptr, *pt_off_d = nullptr, *ch_e0_d = nullptr, *ch_p0_d = nullptr,
      *ch_s0_d = nullptr, *slot_e0_d = nullptr, *slot_cam_d = nullptr, *cam_s_off_d = nullptr,
      *cam_s_list_d = nullptr, *slot_pos_d = nullptr, *slot_rec_d = nullptr, *xe_i_d = nullptr, *xe_j_d = nullptr,
      *xe_kind_d = nullptr, *xo_off_d = nullptr, *xk_off_d = nullptr, *xk_list_d = nullptr, *ch_prob_d = nullptr,
      *cb_prob_d = nullptr, *pb_prob_d = nullptr, *base_d = nullptr, *running_d = nullptr,
      *old2new_d = nullptr;
  uint16_t *e_pos_d = nullptr, *e_slot_d = nullptr, *ch_sorted_d = nullptr, *ch_grp_d = nullptr;
  uint32_t* e_meta_d = nullptr;
  uint8_t *cam_fixed_d = nullptr, *pt_fixed_d = nullptr;
  double *obs_d = nullptr, *delta_d = nullptr, *info_d = nullptr, *xe_rec_d = nullptr;
  DevBA* desc_d = nullptr;
  Plan pl;
};

void PrepDeleter::operator()(Prepared* p) const { delete p; }

static gpo_status prepare(gpo_graph* g) {
  const gpo::KernelSet& ks = gpo_host::kernels_of(g);
  const int SS = ks.SS, DB = ks.DB, M = ks.M, NJ = ks.NJ, NPA = ks.NPA, DC = ks.DC;
  const int TB = tri(DB), NQ = tri(M);
  const int C = (int)g->cam_fixed.size();
  const int P = (int)g->pt_fixed.size();
  const int64_t Eall = (int64_t)g->e_cam.size();
  if (Eall > INT32_MAX / 2) return fail(g, GPO_ERR_UNSUPPORTED, "too many edges (%lld)", (long long)Eall);
  if (ks.model == gpo::ModelKind::STEREO && Eall > 0 && !g->camk_set)
    return fail(g, GPO_ERR_STATE, "stereo edges need the rig: call gpo_set_stereo_camera first");
  std::unique_ptr<Prepared> pp(new (std::nothrow) Prepared());
  if (!pp) return fail(g, GPO_ERR_OOM, "host allocation failed");
  Prepared& R = *pp;

  // point order: by the smallest camera index among the point's active edges
  // (points without active edges last), ties by point index.  Consecutive points
  // then share cameras, which keeps the per-chunk camera slot count small.
  std::vector<int32_t> key(P, C);
  std::vector<int32_t> deg(P, 0);
  for (int64_t e = 0; e < Eall; ++e)
    if (g->e_active[e]) {
      const int p = g->e_pt[e];
      key[p] = std::min(key[p], g->e_cam[e]);
      deg[p]++;
    }
  std::vector<int32_t> cnt(C + 2, 0);
  for (int p = 0; p < P; ++p) cnt[key[p] + 1]++;
  for (int k = 0; k <= C; ++k) cnt[k + 1] += cnt[k];
  R.pt_new2old.assign(P, 0);
  R.pt_old2new.assign(P, 0);
  for (int p = 0; p < P; ++p) {
    const int np = cnt[key[p]]++;
    R.pt_new2old[np] = p;
    R.pt_old2new[p] = np;
  }
  // edges: point-major (new point order), then edge id
  R.pt_off.assign(P + 1, 0);
  for (int p = 0; p < P; ++p) R.pt_off[R.pt_old2new[p] + 1] = deg[p];
  for (int p = 0; p < P; ++p) R.pt_off[p + 1] += R.pt_off[p];
  const int E = R.pt_off[P];
  int maxdeg = 0;
  for (int p = 0; p < P; ++p) maxdeg = std::max(maxdeg, deg[p]);
  R.sorted_edge.assign(E, 0);
  {
    std::vector<int32_t> fill(R.pt_off.begin(), R.pt_off.end() - 1);
    for (int64_t e = 0; e < Eall; ++e)
      if (g->e_active[e]) R.sorted_edge[fill[R.pt_old2new[g->e_pt[e]]]++] = e;
  }
  // chunk size
  int ch = g->desc.chunk_edges > 0 ? g->desc.chunk_edges : gpo::default_ch_max(g->prec);
  if (ch < 32) ch = 32;
  ch = std::min(ch, ks.max_supported_ch(g->prec));   // a larger request is a hint only
  while (ch < maxdeg) ch *= 2;
  if (ch > ks.max_supported_ch(g->prec))
    return fail(g, GPO_ERR_UNSUPPORTED,
                "a point has %d observations; this precision supports at most %d per point", maxdeg,
                ks.max_supported_ch(g->prec));
  R.ch = ch;
  const bool dyn = g->desc.spmv_variant == 4;   // dynamic Jacobians: no stored rows
  if (dyn && ch > 2 * gpo::kThreads)
    return fail(g, GPO_ERR_UNSUPPORTED,
                "dynamic Jacobians need chunks of at most %d edges (a point has %d observations)",
                2 * gpo::kThreads, maxdeg);
  // Chunks of whole points, at most ch edges and ch points each, cut into warp groups:
  // runs of whole points of at most kGroupEdges edges (a point with more edges is a group
  // of its own), at most ch / kGroupEdges groups (and kMaxGroups) per chunk, so that
  // every warp of a chunk kernel can own one group.  ch_grp[k][g] is the local edge
  // offset where group g of chunk k ends (groups after the last end at the chunk's end).
  R.ch_e0.assign(1, 0);
  R.ch_p0.assign(1, 0);
  {
    const int GE = gpo::kGroupEdges;
    const int GPC = std::max(1, std::min(gpo::kMaxGroups, ch / GE));
    uint16_t cur[gpo::kMaxGroups];
    int ne = 0, np = 0, ng = 0, ge = 0;
    auto close_chunk = [&](int p_end) {
      if (ng > 0) cur[ng - 1] = (uint16_t)ne;
      for (int q = ng; q < gpo::kMaxGroups; ++q) cur[q] = (uint16_t)ne;
      R.ch_grp.insert(R.ch_grp.end(), cur, cur + gpo::kMaxGroups);
      R.ch_e0.push_back(R.pt_off[p_end]);
      R.ch_p0.push_back(p_end);
    };
    for (int p = 0; p < P; ++p) {
      const int L = R.pt_off[p + 1] - R.pt_off[p];
      bool fits = ng > 0 && L <= GE && ge + L <= GE;
      if (np > 0 && (ne + L > ch || np + 1 > ch || (!fits && ng + 1 > GPC))) {
        close_chunk(p);
        ne = np = ng = ge = 0;
        fits = false;
      }
      if (!fits) {
        if (ng > 0) cur[ng - 1] = (uint16_t)ne;
        ++ng;
        ge = 0;
      }
      ge += L;
      ne += L;
      np += 1;
    }
    if (np > 0) close_chunk(P);
  }
  const int NCH = (int)R.ch_e0.size() - 1;
  R.NCH = NCH;
  // slots: distinct cameras per chunk in ascending order; the chunk's edges bucketed by
  // slot, stable in edge order
  R.e_cam_s.resize(E);
  R.e_pt_s.resize(E);
  for (int i = 0; i < E; ++i) {
    const int64_t e = R.sorted_edge[i];
    R.e_cam_s[i] = g->e_cam[e];
    R.e_pt_s[i] = R.pt_old2new[g->e_pt[e]];
  }
  R.e_pos.resize(E);
  R.e_slot.resize(E);
  R.ch_sorted.resize(E);
  R.ch_s0.assign(1, 0);
  {
    std::vector<int32_t> cam2slot(std::max(C, 1), -1), cams, fill;
    for (int k = 0; k < NCH; ++k) {
      const int e0 = R.ch_e0[k], n = R.ch_e0[k + 1] - e0;
      cams.clear();
      for (int i = 0; i < n; ++i) {
        const int c = R.e_cam_s[e0 + i];
        if (cam2slot[c] == -1) {
          cam2slot[c] = -2;
          cams.push_back(c);
        }
      }
      std::sort(cams.begin(), cams.end());
      const int ns = (int)cams.size();
      fill.assign(ns + 1, 0);
      for (int s2 = 0; s2 < ns; ++s2) cam2slot[cams[s2]] = s2;
      for (int i = 0; i < n; ++i) fill[cam2slot[R.e_cam_s[e0 + i]] + 1]++;
      for (int s2 = 0; s2 < ns; ++s2) fill[s2 + 1] += fill[s2];
      for (int s2 = 0; s2 < ns; ++s2) {
        R.slot_e0.push_back(e0 + fill[s2]);
        R.slot_cam.push_back(cams[s2]);
      }
      for (int i = 0; i < n; ++i) {
        const int sl = cam2slot[R.e_cam_s[e0 + i]];
        const int q = fill[sl]++;
        R.e_pos[e0 + i] = (uint16_t)q;
        R.e_slot[e0 + i] = (uint16_t)sl;
        R.ch_sorted[e0 + q] = (uint16_t)i;
      }
      for (int c : cams) cam2slot[c] = -1;
      R.ch_s0.push_back((int)R.slot_cam.size());
    }
    R.slot_e0.push_back(E);
  }
  const int NS = (int)R.slot_cam.size();
  int ns_max = 1, np_max = 1;
  for (int k = 0; k < NCH; ++k) {
    ns_max = std::max(ns_max, R.ch_s0[k + 1] - R.ch_s0[k]);
    np_max = std::max(np_max, R.ch_p0[k + 1] - R.ch_p0[k]);
  }
  R.jpos = (size_t)std::max<int64_t>((E + gpo::kJTile - 1) / gpo::kJTile, 1) * gpo::kJTile * NJ;   // whole tiles
  // per camera: its slots in chunk order
  R.cam_s_off.assign(C + 1, 0);
  R.cam_s_list.resize(NS);
  R.slot_pos.assign(std::max(NS, 1), 0);
  for (int s2 = 0; s2 < NS; ++s2) R.cam_s_off[R.slot_cam[s2] + 1]++;
  for (int c = 0; c < C; ++c) R.cam_s_off[c + 1] += R.cam_s_off[c];
  {
    std::vector<int32_t> fill(R.cam_s_off.begin(), R.cam_s_off.end() - 1);
    for (int s2 = 0; s2 < NS; ++s2) {
      R.slot_pos[s2] = fill[R.slot_cam[s2]];
      R.cam_s_list[fill[R.slot_cam[s2]]++] = s2;
    }
  }
  // per-edge data in sorted order
  R.obs_s.resize((size_t)M * E);
  R.delta_s.resize(E);
  for (int i = 0; i < E; ++i) {
    const int64_t e = R.sorted_edge[i];
    for (int k = 0; k < M; ++k) R.obs_s[(size_t)M * i + k] = g->e_obs[(size_t)M * e + k];
    R.delta_s[i] = g->e_delta[e];
  }
  if (g->any_info) {
    R.info_s.resize((size_t)NQ * E);
    for (int i = 0; i < E; ++i)
      for (int k = 0; k < NQ; ++k) R.info_s[(size_t)NQ * i + k] = g->e_sqinfo[(size_t)NQ * R.sorted_edge[i] + k];
  }
  R.pt_fixed_s.resize(P);
  for (int p = 0; p < P; ++p) R.pt_fixed_s[R.pt_old2new[p]] = g->pt_fixed[p];
  R.cam_fixed = g->cam_fixed;
  // staged Schur-product inputs: packed per-edge positions and per-slot records
  R.e_meta.assign((size_t)E + 4, 0u);
  R.slot_rec.assign(4 * (size_t)std::max(NS, 1), 0);
  for (int k = 0; k < NCH; ++k) {
    for (int i = R.ch_e0[k]; i < R.ch_e0[k + 1] && ch <= 1024; ++i)
      R.e_meta[i] = (uint32_t)R.e_pos[i] | ((uint32_t)R.e_slot[i] << 10) | ((uint32_t)(R.e_pt_s[i] - R.ch_p0[k]) << 20);
    for (int s2 = R.ch_s0[k]; s2 < R.ch_s0[k + 1]; ++s2) {
      R.slot_rec[4 * (size_t)s2] = R.slot_e0[s2] - R.ch_e0[k];
      R.slot_rec[4 * (size_t)s2 + 1] = R.slot_e0[s2 + 1] - R.ch_e0[k];
      R.slot_rec[4 * (size_t)s2 + 2] = R.slot_cam[s2];
      R.slot_rec[4 * (size_t)s2 + 3] = R.slot_pos[s2];
    }
  }
  // camera-side edges: active ones, sorted by (first camera, index)
  for (size_t x = 0; x < g->x_kind.size(); ++x)
    if (g->x_active[x]) R.x_sorted.push_back((int32_t)x);
  std::stable_sort(R.x_sorted.begin(), R.x_sorted.end(), [&](int32_t a, int32_t b) { return g->x_i[a] < g->x_i[b]; });
  const int NX = (int)R.x_sorted.size();
  R.xi_s.resize(NX);
  R.xj_s.resize(NX);
  R.xk_s.resize(NX);
  R.xo_off.assign(C + 1, 0);
  R.xk_off.assign(C + 1, 0);
  R.xk_list.resize(2 * (size_t)NX);
  R.xrec_s.resize((size_t)NX * gpo::kXRec);
  for (int t = 0; t < NX; ++t) {
    const int x = R.x_sorted[t];
    R.xi_s[t] = g->x_i[x];
    R.xj_s[t] = g->x_j[x];
    R.xk_s[t] = g->x_kind[x];
    std::memcpy(&R.xrec_s[(size_t)t * gpo::kXRec], &g->x_rec[(size_t)x * gpo::kXRec], gpo::kXRec * sizeof(double));
    R.xo_off[R.xi_s[t] + 1]++;
    R.xk_off[R.xi_s[t] + 1]++;
    if (R.xj_s[t] >= 0) R.xk_off[R.xj_s[t] + 1]++;
  }
  for (int c = 0; c < C; ++c) {
    R.xo_off[c + 1] += R.xo_off[c];
    R.xk_off[c + 1] += R.xk_off[c];
  }
  {
    std::vector<int32_t> fill(R.xk_off.begin(), R.xk_off.end() - 1);
    for (int t = 0; t < NX; ++t) {
      R.xk_list[fill[R.xi_s[t]]++] = 2 * t;
      if (R.xj_s[t] >= 0) R.xk_list[fill[R.xj_s[t]]++] = 2 * t + 1;
    }
  }
  // FP64 state in device order
  R.cams = g->cam_state;
  R.pts.resize(3 * (size_t)P);
  for (int p = 0; p < P; ++p)
    for (int k = 0; k < 3; ++k) R.pts[3 * (size_t)R.pt_old2new[p] + k] = g->pt_state[3 * (size_t)p + k];

  // ---- memory plan (uploaded arrays first)
  const Prec pr = g->prec;
  const size_t sA = at_size(pr), sJ = jt_size(pr);
  DevBA& d = R.d;
  d.C = C; d.P = P; d.E = E; d.NCH = NCH; d.NS = NS; d.NX = NX; d.ch_max = ch;
  d.model = (int)ks.model;
  std::memcpy(d.camk, g->camk, sizeof(d.camk));
  d.ns_max = ns_max; d.np_max = np_max;
  d.ncblk = std::max(1, (C + gpo::kCamPerBlock - 1) / gpo::kCamPerBlock);
  R.npb = std::max(1, (P + 255) / 256);
  R.zeros_ch.assign(std::max(NCH, 1), 0);
  R.zeros_cb.assign(d.ncblk, 0);
  R.zeros_pb.assign(R.npb, 0);
  R.zeros_small.assign(8, 0);
  R.xzeros.assign(std::max(NX, 1), 0.0);
  R.sc0.assign(1, Scalars{});
  Plan& pl = R.pl;
  pl.up(&R.e_cam_d, E, R.e_cam_s); pl.up(&R.e_pt_d, E, R.e_pt_s); pl.up(&R.obs_d, (size_t)M * E, R.obs_s);
  pl.up(&R.delta_d, E, R.delta_s);
  if (g->any_info) pl.up(&R.info_d, (size_t)NQ * E, R.info_s);
  pl.up(&R.pt_off_d, P + 1, R.pt_off); pl.up(&R.ch_e0_d, NCH + 1, R.ch_e0); pl.up(&R.ch_p0_d, NCH + 1, R.ch_p0);
  pl.up(&R.ch_s0_d, NCH + 1, R.ch_s0); pl.up(&R.e_pos_d, E, R.e_pos); pl.up(&R.e_slot_d, E, R.e_slot);
  pl.up(&R.ch_sorted_d, E, R.ch_sorted); pl.up(&R.slot_e0_d, NS + 1, R.slot_e0);
  pl.up(&R.ch_grp_d, (size_t)std::max(NCH, 1) * gpo::kMaxGroups, R.ch_grp);
  pl.up(&R.slot_cam_d, std::max(NS, 1), R.slot_cam);
  pl.up(&R.e_meta_d, (size_t)E + 4, R.e_meta); pl.up(&R.slot_rec_d, 4 * (size_t)std::max(NS, 1), R.slot_rec);
  pl.up(&R.cam_s_off_d, C + 1, R.cam_s_off); pl.up(&R.cam_s_list_d, std::max(NS, 1), R.cam_s_list);
  pl.up(&R.slot_pos_d, std::max(NS, 1), R.slot_pos);
  pl.up(&R.cam_fixed_d, std::max(C, 1), R.cam_fixed); pl.up(&R.pt_fixed_d, std::max(P, 1), R.pt_fixed_s);
  pl.up(&R.xe_i_d, std::max(NX, 1), R.xi_s); pl.up(&R.xe_j_d, std::max(NX, 1), R.xj_s);
  pl.up(&R.xe_kind_d, std::max(NX, 1), R.xk_s);
  pl.up(&R.xe_rec_d, (size_t)std::max(NX, 1) * gpo::kXRec, R.xrec_s);
  pl.up(&R.xo_off_d, C + 1, R.xo_off); pl.up(&R.xk_off_d, C + 1, R.xk_off);
  pl.up(&R.xk_list_d, std::max(2 * NX, 1), R.xk_list);
  pl.up(&d.xe_cost, std::max(NX, 1), R.xzeros); pl.up(&d.xe_md, std::max(NX, 1), R.xzeros);
  pl.up(&d.cam, (size_t)SS * C, R.cams);
  pl.up(&d.pt, 3 * (size_t)P, R.pts);
  pl.up(&d.sc, 1, R.sc0);
  pl.up(&R.ch_prob_d, std::max(NCH, 1), R.zeros_ch); pl.up(&R.cb_prob_d, d.ncblk, R.zeros_cb);
  pl.up(&R.pb_prob_d, R.npb, R.zeros_pb);
  pl.up(&R.base_d, 1, R.zeros_small); pl.up(&R.running_d, 8, R.zeros_small);
  pl.up(&R.old2new_d, std::max(P, 1), R.pt_old2new);   // point id -> sorted row (state copies)
  // device-only arrays
  pl.add(&d.xe_J, (size_t)std::max(NX, 1) * gpo::kXJ); pl.add(&d.xe_r, (size_t)std::max(NX, 1) * gpo::kXRows);
  pl.add_raw(&d.xe_H, (size_t)std::max(NX, 1) * DB * DB * sA);
  pl.add(&d.cam_cand, (size_t)SS * C);
  pl.add(&d.camrb, 16 * (size_t)C); pl.add(&d.camrb_cand, 16 * (size_t)C);
  pl.add(&d.camrbf, 16 * (size_t)C); pl.add(&d.camrbf_cand, 16 * (size_t)C);
  pl.add(&d.pt_cand, 3 * (size_t)P);
  if (!dyn) pl.add_raw(&d.J, std::max<size_t>(R.jpos, 8) * sJ);   // dynamic Jacobians: none
  pl.add_raw(&d.Hpp, 6 * (size_t)P * sA); pl.add_raw(&d.bp, 3 * (size_t)P * sA);
  pl.add_raw(&d.Hinv, 6 * (size_t)P * sA); pl.add_raw(&d.dp, 3 * (size_t)P * sA);
  pl.add_raw(&d.pt_rec, (size_t)std::max(P, 1) * (pr == Prec::F64 ? 64 : 32));
  pl.add_raw(&d.partA, (size_t)NPA * NS * sA); pl.add_raw(&d.partB, (size_t)NPA * NS * sA);
  pl.add_raw(&d.partV, (size_t)DC * NS * sA);
  pl.add_raw(&d.Hcl, (size_t)TB * C * sA); pl.add_raw(&d.bc, (size_t)DB * C * sA);
  pl.add_raw(&d.S, (size_t)TB * C * sA); pl.add_raw(&d.Minv, (size_t)TB * C * sA);
  pl.add_raw(&d.g, (size_t)DB * C * sA);
  pl.add_raw(&d.x, (size_t)DB * C * sA); pl.add_raw(&d.r, (size_t)DB * C * sA);
  pl.add_raw(&d.z, (size_t)DB * C * sA); pl.add_raw(&d.p, (size_t)DB * C * sA);
  pl.add_raw(&d.y, (size_t)DB * C * sA); pl.add_raw(&d.xbest, (size_t)DB * C * sA);
  pl.add_raw(&d.p2, (size_t)DB * C * sA);
  pl.add(&d.cost_part, std::max(NCH, 1)); pl.add(&d.md_part, std::max(NCH, 1));
  pl.add(&d.cblk_part, 2 * 5 * (size_t)d.ncblk);   // four camera-half CTAs per camera block, then the update's
  pl.add(&d.hist, gpo::kMaxHistory);
  pl.add(&R.desc_d, 1);
  R.bytes = pl.total();
  g->prep.reset(pp.release());
  return GPO_OK;
}

// Plans the graph (sorted topology, chunks, slots, memory plan; kept until the upload)
// and, unless plan_bytes is given, in which case only the planned size is returned,
// allocates the arena and uploads everything with one copy (no wait: the copy
// from pageable host memory is staged before the call returns).
gpo_status gpo_host::finalize(gpo_graph* g, size_t* plan_bytes) {
  if (g->finalized) {
    if (plan_bytes) *plan_bytes = g->arena_bytes;
    return GPO_OK;
  }
  if (!g->prep) {
    gpo_status s = prepare(g);
    if (s != GPO_OK) return s;
  }
  Prepared& R = *g->prep;
  const size_t bytes = R.bytes;
  if (plan_bytes) {
    *plan_bytes = bytes;
    return GPO_OK;
  }
  if (gpo_status s = ensure_stream(g); s != GPO_OK) return s;
  if (g->desc.memory_budget && bytes > g->desc.memory_budget)
    return fail(g, GPO_ERR_OOM, "graph needs %zu bytes of device memory, budget is %zu", bytes,
                (size_t)g->desc.memory_budget);
  void* base = nullptr;
  if (g->desc.alloc && g->desc.free) {
    base = g->desc.alloc(bytes, g->desc.alloc_ctx);
    if (!base) return fail(g, GPO_ERR_OOM, "allocator hook returned NULL for %zu bytes", bytes);
  } else {
    const cudaError_t e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(g, GPO_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
  }
  g->arena = base;
  g->arena_bytes = bytes;
  R.pl.assign(static_cast<char*>(base));
  DevBA& d = R.d;
  d.e_cam = R.e_cam_d; d.e_pt = R.e_pt_d; d.obs = R.obs_d; d.e_delta = R.delta_d; d.e_sqinfo = R.info_d;
  d.pt_off = R.pt_off_d; d.ch_e0 = R.ch_e0_d; d.ch_p0 = R.ch_p0_d; d.ch_s0 = R.ch_s0_d;
  d.e_pos = R.e_pos_d; d.e_slot = R.e_slot_d; d.ch_sorted = R.ch_sorted_d; d.slot_e0 = R.slot_e0_d;
  d.slot_cam = R.slot_cam_d; d.cam_s_off = R.cam_s_off_d; d.cam_s_list = R.cam_s_list_d; d.slot_pos = R.slot_pos_d;
  d.cam_fixed = R.cam_fixed_d; d.pt_fixed = R.pt_fixed_d;
  d.xe_i = R.xe_i_d; d.xe_j = R.xe_j_d; d.xe_kind = R.xe_kind_d; d.xe_rec = R.xe_rec_d;
  d.xo_off = R.xo_off_d; d.xk_off = R.xk_off_d; d.xk_list = R.xk_list_d;
  d.e_meta = R.e_meta_d; d.slot_rec = reinterpret_cast<const int4*>(R.slot_rec_d);
  d.ch_grp = R.ch_grp_d;
  d.dbg_r = nullptr;
  const cudaStream_t st = g->stream;
  {
    std::vector<char> img;
    const size_t n = R.pl.image(img);
    if (n) GPO_CUDA(g, cudaMemcpyAsync(base, img.data(), n, cudaMemcpyHostToDevice, st));
  }
  if (d.J) GPO_CUDA(g, cudaMemsetAsync(d.J, 0, std::max<size_t>(R.jpos, 8) * jt_size(g->prec), st));
  GPO_CUDA(g, cudaMemsetAsync(d.dp, 0, 3 * (size_t)d.P * at_size(g->prec), st));
  GPO_CUDA(g, cudaMemcpyAsync(R.desc_d, &d, sizeof(DevBA), cudaMemcpyHostToDevice, st));
  gpo::LaunchSet ls{};
  ls.probs = R.desc_d;
  ls.ch_prob = R.ch_prob_d; ls.ch_base = R.base_d;
  ls.cb_prob = R.cb_prob_d; ls.cb_base = R.base_d;
  ls.pb_prob = R.pb_prob_d; ls.pb_base = R.base_d;
  ls.running = R.running_d;
  ls.err = R.running_d + 1;
  ls.work = R.running_d + 2;
  ls.spmv_variant = g->desc.spmv_variant;
  ls.nprob = 1; ls.n_ch = R.NCH; ls.n_cb = d.C > 0 ? d.ncblk : 0; ls.n_pb = d.P > 0 ? R.npb : 0;
  ls.ch_max = R.ch;
  ls.ns_max = d.ns_max;
  ls.np_max = d.np_max;
  g->ls = ls;
  g->ks = &gpo_host::kernels_of(g);
  g->dev_desc = R.desc_d;
  g->ch_max = R.ch;
  g->j_elems = R.jpos;
  g->h_ch_e0 = std::move(R.ch_e0);
  g->sorted_edge = std::move(R.sorted_edge);
  g->pt_new2old = std::move(R.pt_new2old);
  g->pt_old2new = std::move(R.pt_old2new);
  g->pt_old2new_d = R.old2new_d;
  g->x_sorted = std::move(R.x_sorted);
  g->dev = d;
  g->finalized = true;
  g->prep.reset();
  g->state_same = false;
  GPO_CUDA(g, cudaGetLastError());
  return GPO_OK;
}

// ============================================================== profiling

static cudaEvent_t prof_event(gpo_graph* g) {
  Profiler& p = g->prof;
  if (p.pool_used == p.pool.size()) {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    p.pool.push_back(e);
  }
  return p.pool[p.pool_used++];
}

// Launches through f (which returns the number of kernels it launched), counting
// launches and, if profiling is on, bracketing them with events.
template <class F>
static void run(gpo_graph* g, int kind, F&& f) {
  Profiler& p = g->prof;
  if (p.on) {
    cudaEvent_t a = prof_event(g), b = prof_event(g);
    cudaEventRecord(a, g->stream);
    p.launches[kind] += f();
    cudaEventRecord(b, g->stream);
    p.marks.push_back({kind, g->cur_lm_iter, g->cur_pcg_k, a, b});
  } else {
    p.launches[kind] += f();
  }
}

// Resolves the recorded events (after a stream sync).  A Schur-product launch is
// active when its PCG iteration ran (iteration index <= that LM iteration's PCG
// count); later launches of the look-ahead group return at once.  A linearisation is
// active when the LM iteration before it accepted its step.
void gpo_host::prof_resolve(gpo_graph* g) {
  Profiler& p = g->prof;
  for (const auto& m : p.marks) {
    float el = 0.f;
    cudaEventElapsedTime(&el, m.a, m.b);
    p.timed[m.kind]++;
    p.ms[m.kind] += el;
    bool act = true;
    if (m.kind == KK_SPMV && m.lm_iter >= 0 && m.lm_iter < (int)g->hist.size())
      act = m.pcg_k <= g->hist[m.lm_iter].pcg_products;
    // the linearisation returns at once after a rejected step (the state is unchanged)
    if (m.kind == KK_LINEARIZE && m.lm_iter >= 1 && m.lm_iter - 1 < (int)g->hist.size())
      act = g->hist[m.lm_iter - 1].accepted != 0;
    if (act) {
      p.active[m.kind]++;
      p.active_ms[m.kind] += el;
    }
  }
  p.marks.clear();
  p.pool_used = 0;
}

// ============================================================== LM driver

void gpo_host::fill_scalars(gpo_graph* g, const gpo_lm_params& p, double lambda, Scalars& s) {
  std::memset(&s, 0, sizeof(s));
  s.lambda = lambda;
  s.nu = (p.initial_nu >= 2.0 && std::isfinite(p.initial_nu)) ? p.initial_nu : 2.0;
  s.lambda_min = p.lambda_min;
  s.lambda_max = p.lambda_max;
  s.diag_min = p.diag_min;
  s.diag_max = p.diag_max;
  s.damping_mode = p.damping_mode;
  s.need_lin = 1;
  s.ratio = (p.pcg_rejection_ratio > 0.0 && std::isfinite(p.pcg_rejection_ratio)) ? p.pcg_rejection_ratio : 0.0;
  s.pcg_tol = p.pcg_tol;
  s.pcg_rel = p.pcg_tol_relative ? 1 : 0;
  s.max_it = std::max(1, p.pcg_max_iters);
  s.normalize = p.pcg_normalize < 0 ? (g->prec != Prec::F64 ? 1 : 0) : (p.pcg_normalize ? 1 : 0);
  s.restart_every = p.pcg_restart_every <= 0 ? 0 : std::max(4, p.pcg_restart_every);
  s.restart = 0;
  s.full = (p.solver == GPO_SOLVER_FULL && g->dev.C > 0) ? 1 : 0;
  g->pcg_full = s.full;
  s.sigma = 1.0;
  s.inv_n = 1.0;
  s.inv_n_f = 1.0f;
  s.beta_f = 0.0f;
  s.active = 1;
  s.pcg_done = 1;   // until the camera blocks start a PCG solve
}

gpo_status gpo_host::upload_scalars(gpo_graph* g, const Scalars& s) {
  if (gpo_status st = ensure_runtime(g); st != GPO_OK) return st;
  *g->h_sc = s;
  GPO_CUDA(g, cudaMemcpyAsync(g->dev.sc, g->h_sc, sizeof(Scalars), cudaMemcpyHostToDevice, g->stream));
  // the pinned staging buffer is reused: make sure the copy has been consumed
  GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  return GPO_OK;
}

constexpr int kPcgGroup = 8;

// Captures kPcgGroup PCG iterations of `ls` as a CUDA graph on g's stream (the
// kernels read every per-iteration value from device memory, so one graph serves
// every group).  On any capture error the graph path is switched off for g.
static void capture_pcg_group(gpo_graph* g, const gpo::LaunchSet& ls) {
  gpo_host::drop_pcg_graph(g);
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    g->pcg_graph_off = true;
    return;
  }
  int c[3] = {0, 0, 0};
  for (int i = 0; i < kPcgGroup; ++i) {
    if (g->pcg_full) {   // full system: product, camera half, update over cameras and points
      c[0] += g->ks->full_spmv(ls, g->prec, g->stream);
      c[2] += g->ks->cam_apply(ls, g->prec, g->stream);
      c[2] += g->ks->full_update(ls, g->prec, g->stream);
      continue;
    }
    c[0] += g->ks->pcg_spmv(ls, g->prec, g->stream);
    const int fused = g->ks->pcg_camera(ls, g->prec, g->stream);
    c[1] += fused;
    if (!fused) {
      c[2] += g->ks->cam_apply(ls, g->prec, g->stream);
      c[2] += g->ks->pcg_update(ls, g->prec, g->stream);
    }
  }
  const cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
  if (e != cudaSuccess || !graph || cudaGraphInstantiate(&g->pcg_exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    g->pcg_exec = nullptr;
    g->pcg_graph_off = true;
  } else {
    g->pcg_ls = ls;
    g->pcg_exec_full = g->pcg_full;
    for (int k = 0; k < 3; ++k) g->pcg_counts[k] = c[k];
  }
  if (graph) cudaGraphDestroy(graph);
}

// PCG iterations with early exit: iterations are launched in groups; after each
// group the done flag is copied back, and the flag of the previous group decides
// whether to launch more (one group of look-ahead keeps the GPU busy).  Full groups
// replay a captured CUDA graph unless profiling is on (which times every launch).
static gpo_status pcg_solve(gpo_graph* g, const gpo::LaunchSet& ls, int max_it) {
  if (gpo_status s = gpo_host::ensure_runtime(g); s != GPO_OK) return s;
  const int kGroup = kPcgGroup;
  int launched = 0, slot = 0, pending = -1;
  // restart iterations (at most one per four PCG iterations) are launched on top of
  // max_it; the device stops at max_it counted PCG iterations
  const int max_launch = max_it + max_it / 4 + 1;
  while (launched < max_launch) {
    const int n = std::min(kGroup, max_launch - launched);
    const bool graph_ok = !g->prof.on && !g->pcg_graph_off && n == kGroup;
    auto same = [&] {   // the captured group is of this launch set and solver
      return g->pcg_exec && g->pcg_exec_full == g->pcg_full && std::memcmp(&g->pcg_ls, &ls, sizeof(ls)) == 0;
    };
    if (graph_ok && !same() && launched > 0)
      capture_pcg_group(g, ls);   // after one direct group, so kernel attributes are set
    if (graph_ok && same()) {
      GPO_CUDA(g, cudaGraphLaunch(g->pcg_exec, g->stream));
      g->prof.launches[KK_SPMV] += g->pcg_counts[0];
      g->prof.launches[KK_PCG_CAMERA] += g->pcg_counts[1];
      g->prof.launches[KK_CAM_APPLY] += g->pcg_counts[2] / 2;
      g->prof.launches[KK_PCG_UPDATE] += g->pcg_counts[2] / 2;
    } else {
      for (int i = 0; i < n; ++i) {
        g->cur_pcg_k = launched + i + 1;
        if (g->pcg_full) {
          run(g, KK_SPMV, [&] { return g->ks->full_spmv(ls, g->prec, g->stream); });
          run(g, KK_CAM_APPLY, [&] { return g->ks->cam_apply(ls, g->prec, g->stream); });
          run(g, KK_PCG_UPDATE, [&] { return g->ks->full_update(ls, g->prec, g->stream); });
          continue;
        }
        run(g, KK_SPMV, [&] { return g->ks->pcg_spmv(ls, g->prec, g->stream); });
        if (g->prof.on) {   // timed separately: the camera half and the update
          run(g, KK_CAM_APPLY, [&] { return g->ks->cam_apply(ls, g->prec, g->stream); });
          run(g, KK_PCG_UPDATE, [&] { return g->ks->pcg_update(ls, g->prec, g->stream); });
        } else if (!g->ks->pcg_camera(ls, g->prec, g->stream)) {
          run(g, KK_CAM_APPLY, [&] { return g->ks->cam_apply(ls, g->prec, g->stream); });
          run(g, KK_PCG_UPDATE, [&] { return g->ks->pcg_update(ls, g->prec, g->stream); });
        } else {
          g->prof.launches[KK_PCG_CAMERA] += 1;
        }
      }
    }
    launched += n;
    GPO_CUDA(g, cudaMemcpyAsync(&g->h_flag[2 * slot], ls.running, 2 * sizeof(int),
                                cudaMemcpyDeviceToHost, g->stream));
    GPO_CUDA(g, cudaEventRecord(g->ev[slot], g->stream));
    if (pending >= 0) {
      GPO_CUDA(g, cudaEventSynchronize(g->ev[pending]));
      if (g->h_flag[2 * pending + 1])
        return fail(g, GPO_ERR_TIMEOUT, "a bounded device wait in the Schur product gave up");
      if (g->h_flag[2 * pending] == 0) break;   // no problem is still iterating
    }
    pending = slot;
    slot ^= 1;
  }
  if (pending >= 0) {
    GPO_CUDA(g, cudaEventSynchronize(g->ev[pending]));
    if (g->h_flag[2 * pending + 1])
      return fail(g, GPO_ERR_TIMEOUT, "a bounded device wait in the Schur product gave up");
  }
  GPO_CUDA(g, cudaGetLastError());
  return GPO_OK;
}

// The point rows of the full-system PCG: seven [P][3] vectors of the accumulation type
// and the point blocks' partial sums, allocated on the first full-system solve (with
// the graph's allocator) and published in the graph's device descriptor.
static gpo_status ensure_full(gpo_graph* g) {
  if (g->full_buf) return GPO_OK;
  const size_t P = (size_t)g->dev.P, sA = at_size(g->prec);
  const size_t vec = (3 * std::max<size_t>(P, 1) * sA + 255) & ~(size_t)255;
  const size_t npb = std::max<size_t>((P + 255) / 256, 1);
  const size_t bytes = 7 * vec + 2 * npb * sizeof(double);
  if (g->desc.memory_budget && g->arena_bytes + bytes > g->desc.memory_budget)
    return fail(g, GPO_ERR_OOM, "the full-system solver needs %zu bytes more, beyond the budget of %zu", bytes,
                (size_t)g->desc.memory_budget);
  void* b = nullptr;
  if (g->desc.alloc && g->desc.free) {
    b = g->desc.alloc(bytes, g->desc.alloc_ctx);
    if (!b) return fail(g, GPO_ERR_OOM, "allocator hook returned NULL for %zu bytes", bytes);
  } else if (cudaMalloc(&b, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(g, GPO_ERR_OOM, "cudaMalloc(%zu) failed for the full-system solver", bytes);
  }
  g->full_buf = b;
  g->full_bytes = bytes;
  char* c = static_cast<char*>(b);
  void** v[7] = {&g->dev.xq, &g->dev.rq, &g->dev.zq, &g->dev.pq, &g->dev.pq2, &g->dev.yq, &g->dev.xqbest};
  for (int i = 0; i < 7; ++i) *v[i] = c + i * vec;
  g->dev.pt_part = reinterpret_cast<double*>(c + 7 * vec);
  GPO_CUDA(g, cudaMemsetAsync(b, 0, bytes, g->stream));
  GPO_CUDA(g, cudaMemcpyAsync(g->dev_desc, &g->dev, sizeof(DevBA), cudaMemcpyHostToDevice, g->stream));
  GPO_CUDA(g, cudaStreamSynchronize(g->stream));   // the host copy of the descriptor stays valid
  return GPO_OK;
}

gpo_status gpo_host::solve_system(gpo_graph* g, const gpo::LaunchSet& ls, int max_it, bool force_lin) {
  if (g->pcg_full) {
    if (gpo_status s = ensure_full(g); s != GPO_OK) return s;
  }
  run(g, KK_LINEARIZE, [&] { return g->ks->linearize(ls, g->prec, force_lin, g->stream); });
  run(g, KK_SCHUR, [&] { return g->ks->schur_prepare(ls, g->prec, g->stream); });
  GPO_CUDA(g, cudaMemsetAsync(ls.running, 0, 6 * sizeof(int), g->stream));   // flags and work counters
  if (g->pcg_full) run(g, KK_FULL_INIT, [&] { return g->ks->full_init(ls, g->prec, g->stream); });
  run(g, KK_CAM_FINALIZE, [&] { return g->ks->cam_finalize(ls, g->prec, g->stream); });
  GPO_CUDA(g, cudaGetLastError());
  gpo_status s = pcg_solve(g, ls, max_it);
  if (s != GPO_OK) return s;
  g->cur_pcg_k = 0;
  run(g, KK_BACKSUB, [&] { return g->ks->backsub(ls, g->prec, g->stream); });
  GPO_CUDA(g, cudaGetLastError());
  return GPO_OK;
}

gpo_status gpo_host::finish_iteration(gpo_graph* g, const gpo::LaunchSet& ls) {
  run(g, KK_RETRACT, [&] { return g->ks->retract(ls, g->prec, g->stream); });
  run(g, KK_COST, [&] { return g->ks->cost(ls, true, g->stream); });
  run(g, KK_DECIDE, [&] { return g->ks->decide(ls, g->prec, g->stream); });
  run(g, KK_COMMIT, [&] { return g->ks->commit(ls, g->stream); });
  GPO_CUDA(g, cudaGetLastError());
  return GPO_OK;
}

gpo_status gpo_host::launch_initial_cost(gpo_graph* g, const gpo::LaunchSet& ls) {
  run(g, KK_CAM_PREPARE, [&] { return g->ks->cam_prepare(ls, false, g->stream); });
  run(g, KK_COST, [&] { return g->ks->cost(ls, false, g->stream); });
  run(g, KK_COST_REDUCE, [&] { return g->ks->cost_init(ls, g->stream); });
  GPO_CUDA(g, cudaGetLastError());
  return GPO_OK;
}

static gpo_status compute_cost(gpo_graph* g, double* out) {
  gpo_status s = gpo_host::launch_initial_cost(g, g->ls);
  if (s != GPO_OK) return s;
  GPO_CUDA(g, cudaMemcpyAsync(g->h_sc, g->dev.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, g->stream));
  GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  *out = g->h_sc->cost;
  return GPO_OK;
}

gpo_lm_params gpo_host::params_or_default(const gpo_lm_params* p) {
  gpo_lm_params d;
  gpo_lm_params_default(&d);
  return p ? *p : d;
}

gpo_status gpo_host::download_begin(gpo_graph* g, std::vector<double>& pts) {
  if (!g->finalized) return GPO_OK;
  const DevBA& d = g->dev;
  pts.resize(3 * (size_t)d.P);
  if (d.C) GPO_CUDA(g, cudaMemcpyAsync(g->cam_state.data(), d.cam, (size_t)cam_ss(g) * d.C * sizeof(double),
                                      cudaMemcpyDeviceToHost, g->stream));
  if (d.P) GPO_CUDA(g, cudaMemcpyAsync(pts.data(), d.pt, 3 * (size_t)d.P * sizeof(double),
                                      cudaMemcpyDeviceToHost, g->stream));
  return GPO_OK;
}

void gpo_host::download_end(gpo_graph* g, const std::vector<double>& pts) {
  if (!g->finalized) return;
  for (int p = 0; p < g->dev.P; ++p)
    for (int k = 0; k < 3; ++k) g->pt_state[3 * (size_t)p + k] = pts[3 * (size_t)g->pt_old2new[p] + k];
}

gpo_status gpo_host::download_state(gpo_graph* g) {
  std::vector<double> pts;
  gpo_status s = download_begin(g, pts);
  if (s != GPO_OK) return s;
  if (g->finalized) GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  download_end(g, pts);
  return GPO_OK;
}

gpo_status gpo_host::ensure_stream(gpo_graph* g) {
  if (g->stream) return GPO_OK;
  GPO_CUDA(g, cudaSetDevice(g->desc.device));
  GPO_CUDA(g, cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
  g->own_stream = true;
  return GPO_OK;
}

gpo_status gpo_host::ensure_runtime(gpo_graph* g) {
  if (g->h_sc) return GPO_OK;
  if (gpo_status s = ensure_stream(g); s != GPO_OK) return s;
  GPO_CUDA(g, cudaMallocHost(&g->h_flag, 4 * sizeof(int)));
  GPO_CUDA(g, cudaMallocHost(&g->h_changed, sizeof(int)));
  GPO_CUDA(g, cudaMalloc(&g->d_changed, sizeof(int)));
  GPO_CUDA(g, cudaEventCreateWithFlags(&g->ev[0], cudaEventDisableTiming));
  GPO_CUDA(g, cudaEventCreateWithFlags(&g->ev[1], cudaEventDisableTiming));
  GPO_CUDA(g, cudaMallocHost(&g->h_sc, sizeof(Scalars)));   // last: marks the runtime as ready
  return GPO_OK;
}

using namespace gpo_host;

// ============================================================== C ABI

extern "C" {

gpo_status gpo_graph_desc_default(gpo_graph_desc* out) {
  if (!out) return GPO_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->precision = GPO_FP64;
  return GPO_OK;
}

gpo_status gpo_lm_params_default(gpo_lm_params* out) {
  if (!out) return GPO_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->initial_damping = 1e-4;
  out->lambda_min = 1e-16;
  out->lambda_max = 1e32;
  out->diag_min = 1e-6;
  out->diag_max = 1e32;
  out->damping_mode = 0;
  out->pcg_max_iters = 100;
  out->pcg_tol = 1e-6;
  out->pcg_tol_relative = 1;
  out->pcg_rejection_ratio = 10.0;
  out->pcg_normalize = -1;
  out->pcg_restart_every = -1;
  out->solver = GPO_SOLVER_SCHUR;
  return GPO_OK;
}

const char* gpo_version(void) { return "gpo 0.1 sm_103a"; }

const char* gpo_last_error(const gpo_graph* g) { return g ? g->err.c_str() : g_create_err.c_str(); }

gpo_status gpo_graph_create(const gpo_graph_desc* desc, gpo_graph** out) {
  if (!desc || !out) return fail(nullptr, GPO_ERR_ARG, "null argument");
  if (desc->precision < GPO_FP64 || desc->precision > GPO_FP32_BF16)
    return fail(nullptr, GPO_ERR_ARG, "unknown precision %d", desc->precision);
  if ((desc->alloc == nullptr) != (desc->free == nullptr))
    return fail(nullptr, GPO_ERR_ARG, "alloc and free hooks must be given together");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || desc->device < 0 || desc->device >= ndev)
    return fail(nullptr, GPO_ERR_CUDA, "no CUDA device %d (%s)", desc->device,
                e != cudaSuccess ? cudaGetErrorString(e) : "out of range");
  gpo_graph* g = new (std::nothrow) gpo_graph();
  if (!g) return fail(nullptr, GPO_ERR_OOM, "host allocation failed");
  g->desc = *desc;
  g->prec = static_cast<Prec>(desc->precision);
  // dynamic Jacobians store no rows: BF16 and FP32 storage are then one mode, FP32 rows
  // evaluated where they are used
  if (desc->spmv_variant == 4 && g->prec == Prec::BF16) g->prec = Prec::F32;
  // the stream, pinned staging and events are created at the first finalize (a graph
  // handed to a server runs on the server's stream and never needs its own)
  if (desc->cuda_stream) g->stream = static_cast<cudaStream_t>(desc->cuda_stream);
  if (desc->reserve_vertices > 0) {
    g->v_kind.reserve(desc->reserve_vertices);
    g->v_local.reserve(desc->reserve_vertices);
  }
  if (desc->reserve_edges > 0) {
    g->e_cam.reserve(desc->reserve_edges);
    g->e_pt.reserve(desc->reserve_edges);
    g->e_obs.reserve(2 * desc->reserve_edges);
  }
  *out = g;
  return GPO_OK;
}

gpo_status gpo_graph_destroy(gpo_graph* g) {
  if (!g) return GPO_OK;
  if (g->stream) cudaStreamSynchronize(g->stream);
  release_device(g);
  if (g->h_sc) cudaFreeHost(g->h_sc);
  if (g->h_flag) cudaFreeHost(g->h_flag);
  if (g->h_changed) cudaFreeHost(g->h_changed);
  if (g->d_changed) cudaFree(g->d_changed);
  for (auto& ev : g->prof.pool)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : g->ev)
    if (ev) cudaEventDestroy(ev);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
  return GPO_OK;
}

gpo_status gpo_add_vertices(gpo_graph* g, int32_t kind, int32_t block_size, int64_t n, int64_t* first_id) {
  if (!g) return GPO_ERR_ARG;
  if (g->finalized) return fail(g, GPO_ERR_STATE, "topology is frozen after the first optimize");
  if (kind != GPO_V_BA_CAMERA9 && kind != GPO_V_POINT3 && kind != GPO_V_NAV15)
    return fail(g, GPO_ERR_ARG, "unknown vertex kind %d", kind);
  if (block_size != tangent_dim(kind))
    return fail(g, GPO_ERR_ARG, "block size %d does not match kind %d (%d)", block_size, kind, tangent_dim(kind));
  if (n < 0) return fail(g, GPO_ERR_ARG, "negative count");
  if (is_camera(kind) && g->cam_kind >= 0 && g->cam_kind != kind)
    return fail(g, GPO_ERR_ARG, "a graph holds one camera kind (it already has kind %d)", g->cam_kind);
  const int64_t id0 = (int64_t)g->v_kind.size();
  const int64_t loc0 = is_camera(kind) ? (int64_t)g->cam_fixed.size() : (int64_t)g->pt_fixed.size();
  if (loc0 + n > INT32_MAX / 16) return fail(g, GPO_ERR_UNSUPPORTED, "too many vertices of kind %d", kind);
  g->v_kind.insert(g->v_kind.end(), n, (int8_t)kind);
  for (int64_t i = 0; i < n; ++i) g->v_local.push_back(loc0 + i);
  if (is_camera(kind)) {
    if (n > 0) g->cam_kind = kind;
    g->cam_fixed.insert(g->cam_fixed.end(), n, 0);
    const int w = state_dim(kind);
    const size_t at = g->cam_state.size();
    g->cam_state.insert(g->cam_state.end(), (size_t)w * n, 0.0);
    if (kind == GPO_V_NAV15)
      for (int64_t i = 0; i < n; ++i) g->cam_state[at + (size_t)w * i + 3] = 1.0;   // qw
  } else {
    g->pt_fixed.insert(g->pt_fixed.end(), n, 0);
    g->pt_state.insert(g->pt_state.end(), 3 * n, 0.0);
  }
  g->prep.reset();
  g->state_same = false;
  if (first_id) *first_id = id0;
  return GPO_OK;
}

gpo_status gpo_set_fisheye(gpo_graph* g, const double* k) {
  if (!g) return GPO_ERR_ARG;
  if (!k) return fail(g, GPO_ERR_ARG, "null coefficients");
  if (g->finalized) return fail(g, GPO_ERR_STATE, "the rig is frozen after the first optimize");
  if (!g->camk_set) return fail(g, GPO_ERR_STATE, "set the stereo rig first");
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(k[i])) return fail(g, GPO_ERR_ARG, "coefficient %d is not finite", i);
  g->camk[17] = 1.0;
  for (int i = 0; i < 4; ++i) g->camk[18 + i] = k[i];
  g->prep.reset();
  g->state_same = false;
  return GPO_OK;
}

gpo_status gpo_set_stereo_camera(gpo_graph* g, const double* rig) {
  if (!g) return GPO_ERR_ARG;
  if (!rig) return fail(g, GPO_ERR_ARG, "null rig");
  if (g->finalized) return fail(g, GPO_ERR_STATE, "the rig is frozen after the first optimize");
  for (int k = 0; k < 17; ++k)
    if (!std::isfinite(rig[k])) return fail(g, GPO_ERR_ARG, "rig value %d is not finite", k);
  std::memset(g->camk, 0, sizeof(g->camk));
  std::memcpy(g->camk, rig, 17 * sizeof(double));
  g->camk_set = true;
  g->prep.reset();
  g->state_same = false;
  return GPO_OK;
}

// Observation edges (camera, point) of the graph's camera kind.  A monocular edge is
// stored as a stereo edge whose third residual row is whitened to zero: observation
// (u, v, 0) and the square root of its 2 x 2 information embedded with a zero third
// row, so the stereo kernels evaluate it unchanged.
static gpo_status add_obs_edges(gpo_graph* g, int32_t kind, int64_t n, const int64_t* ids, const double* meas,
                                const double* info, int32_t loss_kind, double loss_delta) {
  const bool mono = kind == GPO_E_MONO;
  const int ck = kind == GPO_E_BA_REPROJ ? GPO_V_BA_CAMERA9 : GPO_V_NAV15;
  const int m = kind == GPO_E_BA_REPROJ ? 2 : 3, nq = tri(m);
  const int mu = mono ? 2 : m;   // the caller's residual size
  if (g->cam_kind >= 0 && g->cam_kind != ck)
    return fail(g, GPO_ERR_ARG, "edge kind %d does not fit the graph's camera kind %d", kind, g->cam_kind);
  if (n > 0 && !meas) return fail(g, GPO_ERR_ARG, "null measurements");
  const int64_t V = (int64_t)g->v_kind.size();
  // validate everything first: a failed call leaves the graph unchanged
  for (int64_t i = 0; i < n; ++i) {
    const int64_t c = ids[2 * i], p = ids[2 * i + 1];
    if (c < 0 || c >= V || p < 0 || p >= V || g->v_kind[c] != ck || g->v_kind[p] != GPO_V_POINT3)
      return fail(g, GPO_ERR_ARG, "edge %lld: ids must be (%s, point)", (long long)i,
                  ck == GPO_V_NAV15 ? "navigation state" : "camera");
  }
  std::vector<double> packed;   // packed upper square roots of the information, if given
  bool non_identity = false;
  if (info || mono) {
    packed.resize((size_t)nq * n);
    for (int64_t i = 0; i < n; ++i) {
      double Uu[9], U[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      for (int k = 0; k < mu * mu; ++k) Uu[k] = (k % (mu + 1)) == 0 ? 1.0 : 0.0;   // identity, mu x mu
      if (info && !sqrt_info(info + (size_t)mu * mu * i, mu, Uu))
        return fail(g, GPO_ERR_ARG, "edge %lld: information matrix is not symmetric positive definite", (long long)i);
      for (int a = 0; a < mu; ++a)
        for (int b = 0; b < mu; ++b) U[a * m + b] = Uu[a * mu + b];   // mono: third row stays zero
      int t = 0;
      for (int a = 0; a < m; ++a)
        for (int b = a; b < m; ++b, ++t) {
          packed[(size_t)nq * i + t] = U[a * m + b];
          if (U[a * m + b] != (a == b ? 1.0 : 0.0)) non_identity = true;
        }
    }
  }
  const size_t base = g->e_cam.size();
  const int64_t eid0 = (int64_t)g->ed_kind.size();
  g->e_cam.resize(base + n);
  g->e_pt.resize(base + n);
  g->e_eid.resize(base + n);
  g->e_delta.resize(base + n, loss_kind == GPO_LOSS_HUBER ? loss_delta : 0.0);
  g->e_active.resize(base + n, 1);
  if (mono) {
    for (int64_t i = 0; i < n; ++i) {
      g->e_obs.push_back(meas[2 * i]);
      g->e_obs.push_back(meas[2 * i + 1]);
      g->e_obs.push_back(0.0);
    }
  } else {
    g->e_obs.insert(g->e_obs.end(), meas, meas + (size_t)m * n);
  }
  for (int64_t i = 0; i < n; ++i) {
    g->e_cam[base + i] = (int32_t)g->v_local[ids[2 * i]];
    g->e_pt[base + i] = (int32_t)g->v_local[ids[2 * i + 1]];
    g->e_eid[base + i] = eid0 + i;
  }
  // square roots of the information are stored once some edge has a non-identity one
  if (non_identity && !g->any_info) {
    g->any_info = true;
    g->e_sqinfo.assign((size_t)nq * base, 0.0);
    for (size_t e = 0; e < base; ++e)
      for (int a = 0, t = 0; a < m; ++a)
        for (int b = a; b < m; ++b, ++t) g->e_sqinfo[(size_t)nq * e + t] = a == b ? 1.0 : 0.0;
  }
  if (g->any_info) {
    if (info || mono) {
      g->e_sqinfo.insert(g->e_sqinfo.end(), packed.begin(), packed.end());
    } else {
      for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < m; ++a)
          for (int b = a; b < m; ++b) g->e_sqinfo.push_back(a == b ? 1.0 : 0.0);
    }
  }
  g->ed_kind.resize(eid0 + n, (int8_t)kind);
  g->ed_local.resize(eid0 + n);
  for (int64_t i = 0; i < n; ++i) g->ed_local[eid0 + i] = (int64_t)base + i;
  if (n > 0) g->cam_kind = ck;
  g->prep.reset();
  g->state_same = false;
  return GPO_OK;
}

// Camera-side edges between navigation states.
static gpo_status add_nav_edges(gpo_graph* g, int32_t kind, int64_t n, const int64_t* ids, const double* meas,
                                const double* info, int32_t loss_kind, double loss_delta) {
  if (loss_kind != GPO_LOSS_NONE && kind != GPO_E_IMU)
    return fail(g, GPO_ERR_UNSUPPORTED, "edge kind %d takes no robust loss", kind);
  if (g->cam_kind >= 0 && g->cam_kind != GPO_V_NAV15)
    return fail(g, GPO_ERR_ARG, "edge kind %d needs navigation states", kind);
  const int arity = kind == GPO_E_BIAS_PRIOR ? 1 : 2;
  const int m = kind == GPO_E_IMU ? 9 : 6;
  const int mlen = kind == GPO_E_IMU ? gpo::kImuMeas : (kind == GPO_E_BIAS_PRIOR ? 6 : 0);
  if (n > 0 && mlen > 0 && !meas) return fail(g, GPO_ERR_ARG, "null measurements");
  const int64_t V = (int64_t)g->v_kind.size();
  const size_t base = g->x_kind.size();
  auto undo = [&] {
    g->x_i.resize(base); g->x_j.resize(base); g->x_kind.resize(base); g->x_eid.resize(base);
    g->x_rec.resize(base * gpo::kXRec); g->x_active.resize(base);
  };
  for (int64_t i = 0; i < n; ++i) {
    const int64_t a = ids[arity * i], b = arity == 2 ? ids[arity * i + 1] : -1;
    const bool ok = a >= 0 && a < V && g->v_kind[a] == GPO_V_NAV15 &&
                    (arity == 1 || (b >= 0 && b < V && b != a && g->v_kind[b] == GPO_V_NAV15));
    if (!ok) {
      undo();
      return fail(g, GPO_ERR_ARG, "edge %lld: ids must be %s navigation state%s", (long long)i,
                  arity == 2 ? "two distinct" : "one", arity == 2 ? "s" : "");
    }
    double U[81];
    for (int k = 0; k < m * m; ++k) U[k] = (k % (m + 1)) == 0 ? 1.0 : 0.0;
    if (info && !sqrt_info(info + (size_t)m * m * i, m, U)) {
      undo();
      return fail(g, GPO_ERR_ARG, "edge %lld: information matrix is not symmetric positive definite", (long long)i);
    }
    if (kind == GPO_E_IMU && !(meas[(size_t)mlen * i + 60] > 0.0)) {
      undo();
      return fail(g, GPO_ERR_ARG, "edge %lld: preintegration time must be positive", (long long)i);
    }
    const size_t r0 = g->x_rec.size();
    g->x_rec.resize(r0 + gpo::kXRec, 0.0);
    for (int k = 0; k < mlen; ++k) g->x_rec[r0 + k] = meas[(size_t)mlen * i + k];
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < m; ++q) g->x_rec[r0 + gpo::kXU + p * gpo::kXRows + q] = U[p * m + q];
    g->x_rec[r0 + gpo::kXDelta] = loss_kind == GPO_LOSS_HUBER ? loss_delta : 0.0;
    g->x_i.push_back((int32_t)g->v_local[a]);
    g->x_j.push_back(b >= 0 ? (int32_t)g->v_local[b] : -1);
    g->x_kind.push_back((int8_t)(kind == GPO_E_IMU ? gpo::XK_IMU : (kind == GPO_E_BIAS_RW ? gpo::XK_BIAS_RW
                                                                                           : gpo::XK_BIAS_PRIOR)));
    g->x_eid.push_back((int64_t)g->ed_kind.size() + i);
    g->x_active.push_back(1);
  }
  for (int64_t i = 0; i < n; ++i) {
    g->ed_kind.push_back((int8_t)kind);
    g->ed_local.push_back((int64_t)base + i);
  }
  g->prep.reset();
  g->state_same = false;
  return GPO_OK;
}

gpo_status gpo_add_edges(gpo_graph* g, int32_t kind, int64_t n, const int64_t* vertex_ids, const double* meas,
                         const double* info, int32_t loss_kind, double loss_delta, int64_t* first_id) {
  if (!g) return GPO_ERR_ARG;
  if (g->finalized) return fail(g, GPO_ERR_STATE, "topology is frozen after the first optimize");
  if (kind < GPO_E_BA_REPROJ || kind > GPO_E_MONO) return fail(g, GPO_ERR_ARG, "unknown edge kind %d", kind);
  if (n < 0 || (n > 0 && !vertex_ids)) return fail(g, GPO_ERR_ARG, "null ids or negative count");
  if (loss_kind != GPO_LOSS_NONE && loss_kind != GPO_LOSS_HUBER) return fail(g, GPO_ERR_ARG, "unknown loss %d", loss_kind);
  if (loss_kind == GPO_LOSS_HUBER && !(loss_delta > 0.0 && std::isfinite(loss_delta)))
    return fail(g, GPO_ERR_ARG, "Huber threshold must be positive and finite");
  const int64_t first = (int64_t)g->ed_kind.size();
  const gpo_status s = (kind == GPO_E_BA_REPROJ || kind == GPO_E_STEREO || kind == GPO_E_MONO)
                           ? add_obs_edges(g, kind, n, vertex_ids, meas, info, loss_kind, loss_delta)
                           : add_nav_edges(g, kind, n, vertex_ids, meas, info, loss_kind, loss_delta);
  if (s == GPO_OK && first_id) *first_id = first;
  return s;
}

gpo_status gpo_set_fixed(gpo_graph* g, int64_t vid, int32_t fixed) {
  if (!g) return GPO_ERR_ARG;
  if (g->finalized) return fail(g, GPO_ERR_STATE, "fixed flags are frozen after the first optimize");
  if (vid < 0 || vid >= (int64_t)g->v_kind.size()) return fail(g, GPO_ERR_ARG, "no vertex %lld", (long long)vid);
  if (is_camera(g->v_kind[vid])) g->cam_fixed[g->v_local[vid]] = fixed ? 1 : 0;
  else g->pt_fixed[g->v_local[vid]] = fixed ? 1 : 0;
  g->prep.reset();
  g->state_same = false;
  return GPO_OK;
}

gpo_status gpo_set_edge_active(gpo_graph* g, int64_t eid, int32_t active) {
  if (!g) return GPO_ERR_ARG;
  if (g->finalized) return fail(g, GPO_ERR_STATE, "edge activity is frozen after the first optimize");
  if (eid < 0 || eid >= (int64_t)g->ed_kind.size()) return fail(g, GPO_ERR_ARG, "no edge %lld", (long long)eid);
  const int k = g->ed_kind[eid];
  if (k == GPO_E_BA_REPROJ || k == GPO_E_STEREO || k == GPO_E_MONO) g->e_active[g->ed_local[eid]] = active ? 1 : 0;
  else g->x_active[g->ed_local[eid]] = active ? 1 : 0;
  g->prep.reset();
  g->state_same = false;
  return GPO_OK;
}

static gpo_status check_range(gpo_graph* g, int64_t first, int64_t n, int* kind_out) {
  if (n < 0 || first < 0 || first + n > (int64_t)g->v_kind.size())
    return fail(g, GPO_ERR_ARG, "vertex range [%lld, %lld) out of bounds", (long long)first, (long long)(first + n));
  if (n == 0) { *kind_out = -1; return GPO_OK; }
  const int k = g->v_kind[first];
  for (int64_t i = 1; i < n; ++i)
    if (g->v_kind[first + i] != k) return fail(g, GPO_ERR_ARG, "vertex range mixes kinds");
  // the range must also be contiguous in the kind's local numbering
  if (g->v_local[first + n - 1] - g->v_local[first] != n - 1)
    return fail(g, GPO_ERR_ARG, "vertex range is not contiguous within its kind");
  *kind_out = k;
  return GPO_OK;
}

// The device address of page-locked host memory mapped into the device's address space
// (e.g. from cudaHostAlloc), or null for pageable memory.
static const double* mapped_host(const double* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? static_cast<const double*>(at.devicePointer) : nullptr;
}

gpo_status gpo_set_initial(gpo_graph* g, int64_t first, int64_t n, const double* state, int32_t on_device) {
  if (!g) return GPO_ERR_ARG;
  int kind;
  gpo_status s = check_range(g, first, n, &kind);
  if (s != GPO_OK || n == 0) return s;
  if (!state) return fail(g, GPO_ERR_ARG, "null state");
  const int w = state_dim(kind);
  const int64_t loc = g->v_local[first];
  if (!g->finalized) {
    g->cost_valid = false;
    g->prep.reset();
    g->state_same = false;
    std::vector<double>& dst = is_camera(kind) ? g->cam_state : g->pt_state;
    if (on_device) {
      GPO_CUDA(g, cudaMemcpy(dst.data() + loc * w, state, n * w * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(dst.data() + loc * w, state, n * w * sizeof(double));
    }
    return GPO_OK;
  }
  if ((s = ensure_runtime(g)) != GPO_OK) return s;
  cudaStream_t st = g->stream;
  // the rows are written through a kernel that reads device or mapped pinned host
  // memory directly (pageable memory through a device copy) and flags any value whose
  // bits change; points live on the device in sorted order (the id -> row map is
  // resident)
  GPO_CUDA(g, cudaMemsetAsync(g->d_changed, 0, sizeof(int), st));
  const double* src = on_device ? state : mapped_host(state);
  double* tmp = nullptr;
  if (!src) {
    GPO_CUDA(g, cudaMallocAsync(&tmp, n * w * sizeof(double), st));
    GPO_CUDA(g, cudaMemcpyAsync(tmp, state, n * w * sizeof(double), cudaMemcpyHostToDevice, st));
    src = tmp;
  }
  double* dst = is_camera(kind) ? g->dev.cam + loc * w : g->dev.pt;
  const int32_t* idx = is_camera(kind) ? nullptr : g->pt_old2new_d + loc;
  k_assign_rows<<<(int)((n * w + 255) / 256), 256, 0, st>>>(dst, src, idx, (int)n, w, g->d_changed);
  GPO_CUDA(g, cudaGetLastError());
  if (tmp) GPO_CUDA(g, cudaFreeAsync(tmp, st));
  GPO_CUDA(g, cudaMemcpyAsync(g->h_changed, g->d_changed, sizeof(int), cudaMemcpyDeviceToHost, st));
  GPO_CUDA(g, cudaStreamSynchronize(st));
  if (*g->h_changed) {
    g->cost_valid = false;
    g->state_same = false;
  }
  return GPO_OK;
}

gpo_status gpo_get_state(gpo_graph* g, int64_t first, int64_t n, double* out, int32_t on_device) {
  if (!g) return GPO_ERR_ARG;
  int kind;
  gpo_status s = check_range(g, first, n, &kind);
  if (s != GPO_OK || n == 0) return s;
  if (!out) return fail(g, GPO_ERR_ARG, "null output");
  const int w = state_dim(kind);
  const int64_t loc = g->v_local[first];
  if (!g->finalized) {
    const std::vector<double>& src = is_camera(kind) ? g->cam_state : g->pt_state;
    if (on_device) GPO_CUDA(g, cudaMemcpy(out, src.data() + loc * w, n * w * sizeof(double), cudaMemcpyHostToDevice));
    else std::memcpy(out, src.data() + loc * w, n * w * sizeof(double));
    return GPO_OK;
  }
  cudaStream_t st = g->stream;
  if (is_camera(kind)) {
    GPO_CUDA(g, cudaMemcpyAsync(out, g->dev.cam + loc * w, n * w * sizeof(double),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  } else {
    // the gather writes device or mapped pinned host memory directly, pageable memory
    // through a device copy
    double* dst = on_device ? out : const_cast<double*>(mapped_host(out));
    double* tmp = nullptr;
    if (!dst) GPO_CUDA(g, cudaMallocAsync(&tmp, n * 3 * sizeof(double), st));
    k_gather_rows<<<(int)((n * 3 + 255) / 256), 256, 0, st>>>(dst ? dst : tmp, g->dev.pt, g->pt_old2new_d + loc, (int)n, 3);
    if (tmp) {
      GPO_CUDA(g, cudaMemcpyAsync(out, tmp, n * 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
      GPO_CUDA(g, cudaFreeAsync(tmp, st));
    }
  }
  GPO_CUDA(g, cudaStreamSynchronize(st));
  return GPO_OK;
}

gpo_status gpo_optimize(gpo_graph* g, int32_t max_iters, const gpo_lm_params* params, gpo_report* out) {
  if (!g) return GPO_ERR_ARG;
  if (max_iters < 0) return fail(g, GPO_ERR_ARG, "negative iteration count");
  GPO_CUDA(g, cudaSetDevice(g->desc.device));
  gpo_status s = finalize(g);
  if (s != GPO_OK) return s;
  const gpo_lm_params prm = params_or_default(params);
  if (!(prm.initial_damping > 0.0)) return fail(g, GPO_ERR_ARG, "initial damping must be positive");
  if (prm.solver == GPO_SOLVER_FULL && !g->dev.J && g->dev.E > 0)
    return fail(g, GPO_ERR_UNSUPPORTED, "the full-system solver reads stored rows; dynamic Jacobians keep none");
  // a run that continues from the state the last run left (unchanged since) takes its
  // cost, and its linearisation if its last step was rejected: the same values a fresh
  // evaluation gives, without the kernels
  const bool cont = g->state_same && g->cost_valid && g->last_solver == prm.solver;
  Scalars sc;
  fill_scalars(g, prm, prm.initial_damping, sc);
  if (cont) {
    sc.need_lin = g->last_need_lin;
    sc.cost = g->last_cost;
  }
  if ((s = upload_scalars(g, sc)) != GPO_OK) return s;
  double F0;
  if (cont) F0 = g->last_cost;
  else if ((s = compute_cost(g, &F0)) != GPO_OK) return s;
  if (!std::isfinite(F0)) return fail(g, GPO_ERR_NUMERIC, "initial cost is not finite (%g)", F0);
  for (int it = 0; it < max_iters; ++it) {
    g->cur_lm_iter = it;
    if ((s = solve_system(g, g->ls, sc.max_it, false)) != GPO_OK) return s;
    if ((s = finish_iteration(g, g->ls)) != GPO_OK) return s;
  }
  g->cur_lm_iter = -1;
  GPO_CUDA(g, cudaMemcpyAsync(g->h_sc, g->dev.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, g->stream));
  const int nh = std::min(max_iters, gpo::kMaxHistory);
  g->hist.resize(nh);
  if (nh)
    GPO_CUDA(g, cudaMemcpyAsync(g->hist.data(), g->dev.hist, nh * sizeof(gpo::IterRecord),
                                cudaMemcpyDeviceToHost, g->stream));
  GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  if (g->prof.on) prof_resolve(g);
  g->last_cost = g->h_sc->cost;
  g->cost_valid = true;
  g->last_need_lin = g->h_sc->need_lin;
  g->last_solver = prm.solver;
  g->state_same = true;
  if (out) {
    out->initial_cost = F0;
    out->final_cost = g->h_sc->cost;
    out->final_lambda = g->h_sc->lambda;
    out->iterations = g->h_sc->iter;
    out->accepted = g->h_sc->n_accepted;
    out->pcg_iters_total = g->h_sc->pcg_total;
    out->reserved0 = 0;
    out->final_nu = g->h_sc->nu;
  }
  return GPO_OK;
}

gpo_status gpo_get_cost(gpo_graph* g, double* cost) {
  if (!g || !cost) return GPO_ERR_ARG;
  GPO_CUDA(g, cudaSetDevice(g->desc.device));
  gpo_status s = finalize(g);
  if (s != GPO_OK) return s;
  if (g->cost_valid) {
    *cost = g->last_cost;
    return GPO_OK;
  }
  Scalars sc;
  gpo_lm_params prm;
  gpo_lm_params_default(&prm);
  fill_scalars(g, prm, prm.initial_damping, sc);
  if ((s = upload_scalars(g, sc)) != GPO_OK) return s;
  if ((s = compute_cost(g, cost)) != GPO_OK) return s;
  g->last_cost = *cost;
  g->cost_valid = true;
  return GPO_OK;
}

gpo_status gpo_get_history(gpo_graph* g, gpo_iter_record* out, int32_t cap, int32_t* n_out) {
  if (!g || (!out && cap > 0)) return GPO_ERR_ARG;
  const int n = std::min<int>(cap, (int)g->hist.size());
  for (int i = 0; i < n; ++i) {
    const gpo::IterRecord& h = g->hist[i];
    out[i].cost = h.cost;
    out[i].cand_cost = h.cand_cost;
    out[i].model_decrease = h.model_decrease;
    out[i].rho = h.rho;
    out[i].lambda = h.lambda;
    out[i].pcg_residual = h.pcg_residual;
    out[i].accepted = h.accepted;
    out[i].pcg_iters = h.pcg_iters;
    out[i].pcg_products = h.pcg_products;
    out[i].pcg_failed = h.pcg_failed;
  }
  if (n_out) *n_out = n;
  return GPO_OK;
}

gpo_status gpo_set_profiling(gpo_graph* g, int32_t enable) {
  if (!g) return GPO_ERR_ARG;
  if (g->stream) GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  Profiler& p = g->prof;
  p.marks.clear();
  p.pool_used = 0;
  for (int k = 0; k < KK_COUNT; ++k) {
    p.launches[k] = p.timed[k] = p.active[k] = 0;
    p.ms[k] = p.active_ms[k] = 0.0;
  }
  p.on = enable != 0;
  return GPO_OK;
}

gpo_status gpo_get_profile(gpo_graph* g, gpo_kernel_profile* out, int32_t cap, int32_t* n_out) {
  if (!g || (!out && cap > 0)) return GPO_ERR_ARG;
  if (g->stream) GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  if (!g->prof.marks.empty()) prof_resolve(g);
  const int n = std::min<int>(cap, KK_COUNT);
  for (int k = 0; k < n; ++k) {
    std::memset(&out[k], 0, sizeof(out[k]));
    std::snprintf(out[k].name, sizeof(out[k].name), "%s", kKernelNames[k]);
    out[k].launches = g->prof.launches[k];
    out[k].timed_launches = g->prof.timed[k];
    out[k].active_launches = g->prof.active[k];
    out[k].total_ms = g->prof.ms[k];
    out[k].active_ms = g->prof.active_ms[k];
  }
  if (n_out) *n_out = n;
  return GPO_OK;
}

gpo_status gpo_graph_info(gpo_graph* g, gpo_graph_info_t* out) {
  if (!g || !out) return GPO_ERR_ARG;
  if (!g->finalized) return fail(g, GPO_ERR_STATE, "the graph is not on the device");
  const DevBA& d = g->dev;
  out->cameras = d.C;
  out->points = d.P;
  out->edges = d.E;
  out->extra_edges = d.NX;
  out->chunks = d.NCH;
  out->slots = d.NS;
  out->chunk_edges = g->ch_max;
  out->spmv_variant = g->desc.spmv_variant;
  out->spmv_kernel = d.E > 0 ? g->ks->spmv_kind(g->ls, g->prec) : 0;
  out->j_bytes = d.J ? (int64_t)(g->j_elems * jt_size(g->prec)) : 0;
  return GPO_OK;
}

gpo_status gpo_graph_plan(gpo_graph* g, size_t* bytes) {
  if (!g || !bytes) return GPO_ERR_ARG;
  return finalize(g, bytes);
}

gpo_status gpo_memory_footprint(gpo_graph* g, size_t* bytes) {
  if (!g || !bytes) return GPO_ERR_ARG;
  *bytes = g->arena_bytes + g->full_bytes;
  return GPO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- diagnostics

static double read_j(const std::vector<char>& raw, size_t i, Prec pr) {
  if (pr == Prec::F64) return reinterpret_cast<const double*>(raw.data())[i];
  if (pr == Prec::F32) return reinterpret_cast<const float*>(raw.data())[i];
  const __nv_bfloat16 b = reinterpret_cast<const __nv_bfloat16*>(raw.data())[i];
  uint16_t bits;
  std::memcpy(&bits, &b, 2);
  uint32_t f = (uint32_t)bits << 16;
  float out;
  std::memcpy(&out, &f, 4);
  return out;
}

static double read_a(const std::vector<char>& raw, size_t i, Prec pr) {
  return pr == Prec::F64 ? reinterpret_cast<const double*>(raw.data())[i]
                         : (double)reinterpret_cast<const float*>(raw.data())[i];
}

template <class T>
static gpo_status fetch(gpo_graph* g, std::vector<char>& dst, const T* src, size_t bytes) {
  dst.resize(bytes);
  if (bytes)
    GPO_CUDA(g, cudaMemcpyAsync(dst.data(), src, bytes, cudaMemcpyDeviceToHost, g->stream));
  return GPO_OK;
}

extern "C" {

// Linearises every edge and writes the rows of the edges `sel[0..n_sel)` (all edges in
// id order when sel is null) to r_out / J_out, one output row per selected edge.
static gpo_status debug_linearize_rows(gpo_graph* g, const int64_t* sel, int64_t n_sel, double* r_out,
                                       double* J_out) {
  if (!g) return GPO_ERR_ARG;
  GPO_CUDA(g, cudaSetDevice(g->desc.device));
  gpo_status s = finalize(g);
  if (s != GPO_OK) return s;
  if (!g->dev.J)
    return fail(g, GPO_ERR_UNSUPPORTED, "dynamic Jacobians keep no rows to return (gpo_debug_autodiff_edges evaluates them)");
  const gpo::KernelSet& ks = *g->ks;
  const int M = ks.M, DC = ks.DC, DB = ks.DB, NJ = ks.NJ;
  const bool nav = ks.model == gpo::ModelKind::STEREO;
  const int R = nav ? gpo::kXRows : 2, K = nav ? gpo::kXCols : 12;
  const DevBA& d = g->dev;
  double* dbg = nullptr;
  GPO_CUDA(g, cudaMallocAsync(&dbg, std::max<size_t>(1, (size_t)M * d.E) * sizeof(double), g->stream));
  DevBA dd = d;
  dd.dbg_r = dbg;
  Scalars sc;
  gpo_lm_params prm;
  gpo_lm_params_default(&prm);
  fill_scalars(g, prm, prm.initial_damping, sc);
  if ((s = upload_scalars(g, sc)) != GPO_OK) return s;
  GPO_CUDA(g, cudaMemcpyAsync(g->dev_desc, &dd, sizeof(DevBA), cudaMemcpyHostToDevice, g->stream));
  ks.cam_prepare(g->ls, false, g->stream);
  ks.linearize(g->ls, g->prec, true, g->stream);
  GPO_CUDA(g, cudaMemcpyAsync(g->dev_desc, &g->dev, sizeof(DevBA), cudaMemcpyHostToDevice, g->stream));
  GPO_CUDA(g, cudaGetLastError());
  std::vector<char> rraw, jraw, xjraw, xrraw;
  if ((s = fetch(g, rraw, dbg, (size_t)M * d.E * sizeof(double))) != GPO_OK) return s;
  if ((s = fetch(g, jraw, static_cast<const char*>(d.J), g->j_elems * jt_size(g->prec))) != GPO_OK) return s;
  if ((s = fetch(g, xjraw, d.xe_J, (size_t)d.NX * gpo::kXJ * sizeof(double))) != GPO_OK) return s;
  if ((s = fetch(g, xrraw, d.xe_r, (size_t)d.NX * gpo::kXRows * sizeof(double))) != GPO_OK) return s;
  GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  GPO_CUDA(g, cudaFreeAsync(dbg, g->stream));
  const size_t n_ids = g->ed_kind.size();
  // output row of each edge id (-1: not selected)
  std::vector<int64_t> row_of;
  size_t n_out = n_ids;
  if (sel) {
    row_of.assign(n_ids, -1);
    for (int64_t k = 0; k < n_sel; ++k) {
      if (sel[k] < 0 || sel[k] >= (int64_t)n_ids) return fail(g, GPO_ERR_ARG, "no edge %lld", (long long)sel[k]);
      row_of[sel[k]] = k;
    }
    n_out = (size_t)n_sel;
  }
  if (r_out) std::fill(r_out, r_out + (size_t)R * n_out, 0.0);
  if (J_out) std::fill(J_out, J_out + (size_t)R * K * n_out, 0.0);
  const double* rv = reinterpret_cast<const double*>(rraw.data());
  for (int k = 0; k < d.NCH; ++k) {
    const int e0 = g->h_ch_e0[k], n = g->h_ch_e0[k + 1] - e0;
    for (int i = 0; i < n; ++i) {
      int64_t id = g->e_eid[g->sorted_edge[e0 + i]];
      if (sel && (id = row_of[id]) < 0) continue;
      if (r_out)
        for (int a = 0; a < M; ++a) r_out[(size_t)R * id + a] = rv[(size_t)M * (e0 + i) + a];
      if (J_out) {
        // element k of row e in the tiled layout (see kJTile)
        const size_t e = (size_t)(e0 + i), sj = jt_size(g->prec), Q = (size_t)NJ * sj / 16;
        auto at = [&](size_t k) {
          const size_t unit = ((e / gpo::kJTile) * Q + k * sj / 16) * gpo::kJTile + e % gpo::kJTile;
          return (unit * 16 + (k * sj) % 16) / sj;
        };
        for (int a = 0; a < M; ++a) {
          double* row = J_out + ((size_t)R * id + a) * K;
          for (int j = 0; j < DC; ++j) row[j] = read_j(jraw, at((size_t)DC * a + j), g->prec);
          for (int j = 0; j < 3; ++j) row[DB + j] = read_j(jraw, at((size_t)M * DC + 3 * a + j), g->prec);
        }
      }
    }
  }
  const double* xj = reinterpret_cast<const double*>(xjraw.data());
  const double* xr = reinterpret_cast<const double*>(xrraw.data());
  for (int t = 0; t < d.NX; ++t) {
    int64_t id = g->x_eid[g->x_sorted[t]];
    if (sel && (id = row_of[id]) < 0) continue;
    if (r_out)
      for (int a = 0; a < gpo::kXRows; ++a) r_out[(size_t)R * id + a] = xr[(size_t)gpo::kXRows * t + a];
    if (J_out)
      for (int k = 0; k < gpo::kXJ; ++k) J_out[(size_t)R * K * id + k] = xj[(size_t)gpo::kXJ * t + k];
  }
  return GPO_OK;
}

gpo_status gpo_debug_linearize(gpo_graph* g, double* r_out, double* J_out) {
  if (g) g->state_same = false;   // the call overwrites the run's device buffers
  return debug_linearize_rows(g, nullptr, 0, r_out, J_out);
}

gpo_status gpo_debug_linearize_edges(gpo_graph* g, const int64_t* edge_ids, int64_t n, double* r_out,
                                     double* J_out) {
  if (g) g->state_same = false;   // the call overwrites the run's device buffers
  if (!g || n < 0 || (n > 0 && !edge_ids)) return GPO_ERR_ARG;
  return debug_linearize_rows(g, edge_ids, n, r_out, J_out);
}

gpo_status gpo_debug_autodiff_edges(gpo_graph* g, const int64_t* edge_ids, int64_t n, double* r_out,
                                    double* J_out) {
  if (g) g->state_same = false;   // the call overwrites the run's device buffers
  if (!g || n < 0 || (n > 0 && !edge_ids)) return GPO_ERR_ARG;
  GPO_CUDA(g, cudaSetDevice(g->desc.device));
  gpo_status s = finalize(g);
  if (s != GPO_OK) return s;
  const gpo::KernelSet& ks = *g->ks;
  const int M = ks.M, DC = ks.DC, DB = ks.DB, N = DC + 3;
  const bool nav = ks.model == gpo::ModelKind::STEREO;
  const int R = nav ? gpo::kXRows : 2, K = nav ? gpo::kXCols : 12;
  const DevBA& d = g->dev;
  Scalars sc;
  gpo_lm_params prm;
  gpo_lm_params_default(&prm);
  fill_scalars(g, prm, prm.initial_damping, sc);
  if ((s = upload_scalars(g, sc)) != GPO_OK) return s;
  double *rb = nullptr, *jb = nullptr;
  GPO_CUDA(g, cudaMallocAsync(&rb, std::max<size_t>(1, (size_t)M * d.E) * sizeof(double), g->stream));
  GPO_CUDA(g, cudaMallocAsync(&jb, std::max<size_t>(1, (size_t)M * N * d.E) * sizeof(double), g->stream));
  ks.cam_prepare(g->ls, false, g->stream);
  run(g, KK_AUTODIFF, [&] { return ks.autodiff(g->ls, d.E, rb, jb, g->stream); });
  GPO_CUDA(g, cudaGetLastError());
  std::vector<char> rraw, jraw;
  if ((s = fetch(g, rraw, rb, (size_t)M * d.E * sizeof(double))) != GPO_OK) return s;
  if ((s = fetch(g, jraw, jb, (size_t)M * N * d.E * sizeof(double))) != GPO_OK) return s;
  GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  GPO_CUDA(g, cudaFreeAsync(rb, g->stream));
  GPO_CUDA(g, cudaFreeAsync(jb, g->stream));
  if (g->prof.on) prof_resolve(g);
  const size_t n_ids = g->ed_kind.size();
  std::vector<int64_t> row_of;
  size_t n_out = n_ids;
  if (edge_ids) {
    row_of.assign(n_ids, -1);
    for (int64_t k = 0; k < n; ++k) {
      if (edge_ids[k] < 0 || edge_ids[k] >= (int64_t)n_ids)
        return fail(g, GPO_ERR_ARG, "no edge %lld", (long long)edge_ids[k]);
      row_of[edge_ids[k]] = k;
    }
    n_out = (size_t)n;
  }
  if (r_out) std::fill(r_out, r_out + (size_t)R * n_out, 0.0);
  if (J_out) std::fill(J_out, J_out + (size_t)R * K * n_out, 0.0);
  const double* rv = reinterpret_cast<const double*>(rraw.data());
  const double* jv = reinterpret_cast<const double*>(jraw.data());
  for (int e = 0; e < d.E; ++e) {   // sorted position
    int64_t id = g->e_eid[g->sorted_edge[e]];
    if (edge_ids && (id = row_of[id]) < 0) continue;
    for (int a = 0; a < M; ++a) {
      if (r_out) r_out[(size_t)R * id + a] = rv[(size_t)M * e + a];
      if (J_out) {
        double* row = J_out + ((size_t)R * id + a) * K;
        const double* src = jv + ((size_t)M * e + a) * N;
        for (int j = 0; j < DC; ++j) row[j] = src[j];
        for (int j = 0; j < 3; ++j) row[DB + j] = src[DC + j];
      }
    }
  }
  return GPO_OK;
}

gpo_status gpo_debug_step(gpo_graph* g, double lambda, const gpo_lm_params* params, double* dx_out, int32_t* pcg_iters) {
  if (g) g->state_same = false;   // the call overwrites the run's device buffers
  if (!g || !dx_out) return GPO_ERR_ARG;
  GPO_CUDA(g, cudaSetDevice(g->desc.device));
  gpo_status s = finalize(g);
  if (s != GPO_OK) return s;
  const gpo_lm_params prm = params_or_default(params);
  Scalars sc;
  fill_scalars(g, prm, lambda, sc);
  if ((s = upload_scalars(g, sc)) != GPO_OK) return s;
  g->ks->cam_prepare(g->ls, false, g->stream);
  if ((s = solve_system(g, g->ls, sc.max_it, true)) != GPO_OK) return s;
  const DevBA& d = g->dev;
  const int DB = g->ks->DB;
  const size_t sA = at_size(g->prec);
  std::vector<char> sraw, xraw, xbraw, praw;
  if ((s = fetch(g, sraw, reinterpret_cast<const char*>(d.sc), sizeof(Scalars))) != GPO_OK) return s;
  if ((s = fetch(g, xraw, static_cast<const char*>(d.x), (size_t)DB * d.C * sA)) != GPO_OK) return s;
  if ((s = fetch(g, xbraw, static_cast<const char*>(d.xbest), (size_t)DB * d.C * sA)) != GPO_OK) return s;
  if ((s = fetch(g, praw, static_cast<const char*>(d.dp), 3 * (size_t)d.P * sA)) != GPO_OK) return s;
  GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  const Scalars* hs = reinterpret_cast<const Scalars*>(sraw.data());
  const std::vector<char>& xs = hs->use_best ? xbraw : xraw;
  if (pcg_iters) *pcg_iters = hs->pcg_it;
  size_t off = 0;
  for (size_t v = 0; v < g->v_kind.size(); ++v) {
    const int64_t loc = g->v_local[v];
    if (is_camera(g->v_kind[v])) {
      for (int k = 0; k < DB; ++k)
        dx_out[off + k] = g->cam_fixed[loc] ? 0.0 : read_a(xs, (size_t)DB * loc + k, g->prec);
      off += DB;
    } else {
      const int np = g->pt_old2new[loc];
      for (int k = 0; k < 3; ++k) dx_out[off + k] = g->pt_fixed[loc] ? 0.0 : read_a(praw, 3 * (size_t)np + k, g->prec);
      off += 3;
    }
  }
  return GPO_OK;
}

gpo_status gpo_debug_wait_timeout(gpo_graph* g) {
  if (g) g->state_same = false;   // the call overwrites the run's device buffers
  if (!g) return GPO_ERR_ARG;
  GPO_CUDA(g, cudaSetDevice(g->desc.device));
  gpo_status s = finalize(g);
  if (s != GPO_OK) return s;
  gpo_lm_params prm;
  gpo_lm_params_default(&prm);
  Scalars sc;
  fill_scalars(g, prm, prm.initial_damping, sc);
  if ((s = upload_scalars(g, sc)) != GPO_OK) return s;
  g->ks->cam_prepare(g->ls, false, g->stream);
  g->ks->linearize(g->ls, g->prec, true, g->stream);
  g->ks->schur_prepare(g->ls, g->prec, g->stream);
  GPO_CUDA(g, cudaMemsetAsync(g->ls.running, 0, 6 * sizeof(int), g->stream));
  g->ks->cam_finalize(g->ls, g->prec, g->stream);
  gpo::LaunchSet ls = g->ls;
  ls.debug_wait = 1;   // one CTA more than the grid: nothing completes the barrier
  const int fused = g->ks->pcg_camera(ls, g->prec, g->stream);
  GPO_CUDA(g, cudaGetLastError());
  int flags[2] = {0, 0};
  GPO_CUDA(g, cudaMemcpyAsync(flags, ls.running, sizeof(flags), cudaMemcpyDeviceToHost, g->stream));
  GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  GPO_CUDA(g, cudaMemsetAsync(g->ls.running, 0, 6 * sizeof(int), g->stream));   // leave clean counters
  GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  if (!fused) return fail(g, GPO_ERR_UNSUPPORTED, "the camera blocks do not fit one resident wave");
  if (flags[1]) return fail(g, GPO_ERR_TIMEOUT, "the camera kernel's grid barrier gave up");
  return fail(g, GPO_ERR_STATE, "the grid barrier did not give up");
}

gpo_status gpo_debug_schur(gpo_graph* g, double lambda, const gpo_lm_params* params, double* S_out, double* g_out) {
  if (g) g->state_same = false;   // the call overwrites the run's device buffers
  if (!g) return GPO_ERR_ARG;
  GPO_CUDA(g, cudaSetDevice(g->desc.device));
  gpo_status s = finalize(g);
  if (s != GPO_OK) return s;
  const gpo_lm_params prm = params_or_default(params);
  Scalars sc;
  fill_scalars(g, prm, lambda, sc);
  if ((s = upload_scalars(g, sc)) != GPO_OK) return s;
  const gpo::KernelSet& ks = *g->ks;
  ks.cam_prepare(g->ls, false, g->stream);
  ks.linearize(g->ls, g->prec, true, g->stream);
  ks.schur_prepare(g->ls, g->prec, g->stream);
  GPO_CUDA(g, cudaMemsetAsync(g->ls.running, 0, sizeof(int), g->stream));
  ks.cam_finalize(g->ls, g->prec, g->stream);
  GPO_CUDA(g, cudaGetLastError());
  const DevBA& d = g->dev;
  const int DB = ks.DB, TB = tri(DB);
  const size_t sA = at_size(g->prec);
  std::vector<char> Sraw, graw;
  if ((s = fetch(g, Sraw, static_cast<const char*>(d.S), (size_t)TB * d.C * sA)) != GPO_OK) return s;
  if ((s = fetch(g, graw, static_cast<const char*>(d.g), (size_t)DB * d.C * sA)) != GPO_OK) return s;
  GPO_CUDA(g, cudaStreamSynchronize(g->stream));
  for (int c = 0; c < d.C; ++c) {
    if (S_out)
      for (int i = 0; i < DB; ++i)
        for (int j = 0; j < DB; ++j) {
          const int a = std::min(i, j), b = std::max(i, j);
          const int t = a * DB - (a * (a - 1)) / 2 + (b - a);
          S_out[(size_t)DB * DB * c + DB * i + j] = read_a(Sraw, (size_t)TB * c + t, g->prec);
        }
    if (g_out)
      for (int i = 0; i < DB; ++i) g_out[(size_t)DB * c + i] = read_a(graw, (size_t)DB * c + i, g->prec);
  }
  return GPO_OK;
}

}  // extern "C"
