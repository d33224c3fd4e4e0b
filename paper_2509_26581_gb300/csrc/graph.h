// Host-side graph object and LM driver helpers shared by the C-ABI translation
// units (api.cu: single graphs; batch.cu: batched solves and the serving loop).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "gpo.h"
#include "gpo_internal.h"

using gpo::DevBA;
using gpo::Prec;
using gpo::Scalars;

// Per-kernel launch counts (always) and CUDA-event timings (when enabled) of the
// kernels the library launches on the graph's stream.
enum KernelKind {
  KK_CAM_PREPARE, KK_COST, KK_COST_REDUCE, KK_LINEARIZE, KK_SCHUR, KK_CAM_FINALIZE, KK_SPMV,
  KK_CAM_APPLY, KK_PCG_UPDATE, KK_BACKSUB, KK_RETRACT, KK_DECIDE, KK_COMMIT, KK_PCG_CAMERA,
  KK_FULL_INIT, KK_AUTODIFF, KK_COUNT
};
inline const char* const kKernelNames[KK_COUNT] = {
    "cam_prepare", "cost", "cost_reduce", "linearize", "schur_prepare", "cam_finalize", "spmv",
    "cam_apply", "pcg_update", "backsub", "retract", "decide", "commit", "pcg_camera", "full_init", "autodiff"};

struct Profiler {
  bool on = false;
  int64_t launches[KK_COUNT] = {};
  int64_t timed[KK_COUNT] = {};
  int64_t active[KK_COUNT] = {};
  double ms[KK_COUNT] = {};
  double active_ms[KK_COUNT] = {};
  struct Mark { int kind, lm_iter, pcg_k; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
};

struct Prepared;                       // host-side plan of a graph's device image (api.cu)
struct PrepDeleter {
  void operator()(Prepared* p) const;
};

struct gpo_graph {
  gpo_graph_desc desc{};
  Prec prec = Prec::F64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;

  // vertices: global id -> (kind, index within kind).  A graph holds one camera kind
  // (BA cameras or navigation states) besides points.
  int cam_kind = -1;
  std::vector<int8_t> v_kind;
  std::vector<int64_t> v_local;
  std::vector<double> cam_state;   // [C][SS] (host copy until finalize)
  std::vector<double> pt_state;    // [P][3]
  std::vector<uint8_t> cam_fixed, pt_fixed;

  // edges: global id -> (kind, index within the kind's table)
  std::vector<int8_t> ed_kind;
  std::vector<int64_t> ed_local;
  // observation edges (BA reprojection or stereo reprojection), M rows each
  std::vector<int32_t> e_cam, e_pt;
  std::vector<int64_t> e_eid;      // edge id
  std::vector<double> e_obs;       // [E][M]
  std::vector<double> e_sqinfo;    // [E][tri(M)] packed upper Cholesky factor (identity if no info)
  std::vector<double> e_delta;     // [E]
  std::vector<uint8_t> e_active;
  bool any_info = false;
  // camera-side edges (inertial, bias random walk, bias prior)
  std::vector<int32_t> x_i, x_j;
  std::vector<int8_t> x_kind;
  std::vector<int64_t> x_eid;
  std::vector<double> x_rec;       // [NX][kXRec]
  std::vector<uint8_t> x_active;
  double camk[24] = {};            // stereo rig (and fisheye coefficients)
  bool camk_set = false;

  // finalized topology
  std::unique_ptr<Prepared, PrepDeleter> prep;   // planned, not yet uploaded
  bool finalized = false;
  const gpo::KernelSet* ks = nullptr;
  int ch_max = 0;
  std::vector<int64_t> sorted_edge;   // sorted position -> observation edge index
  std::vector<int32_t> x_sorted;      // sorted position -> camera-side edge index
  std::vector<int32_t> pt_new2old, pt_old2new;
  const int32_t* pt_old2new_d = nullptr;   // device copy of pt_old2new (in the arena)
  std::vector<int32_t> h_ch_e0;
  size_t j_elems = 0;

  // device
  void* arena = nullptr;
  size_t arena_bytes = 0;
  void* full_buf = nullptr;        // point rows of the full-system PCG (allocated on first use)
  size_t full_bytes = 0;
  DevBA dev{};
  gpo::LaunchSet ls{};             // one-problem launch set over `dev`
  DevBA* dev_desc = nullptr;       // device copy of `dev` (ls.probs)
  Scalars* h_sc = nullptr;         // pinned
  int* h_flag = nullptr;           // pinned [2]
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<gpo::IterRecord> hist;
  double last_cost = NAN;
  bool cost_valid = false;
  // The device state is the one the last gpo_optimize left and no call has changed it
  // since (gpo_set_initial with the same values keeps it): the next gpo_optimize takes
  // that run's cost and, if its last step was rejected, its linearisation.
  bool state_same = false;
  int last_need_lin = 1;           // the run's need_lin at its end (0: rows at the state)
  int32_t last_solver = -1;
  int* d_changed = nullptr;        // device flag: gpo_set_initial changed a value
  int* h_changed = nullptr;        // pinned
  Profiler prof;
  int cur_lm_iter = -1;
  int cur_pcg_k = 0;
  // a group of PCG iterations captured as a CUDA graph, for the launch set it was
  // captured with (replayed by the PCG loop while profiling is off)
  cudaGraphExec_t pcg_exec = nullptr;
  gpo::LaunchSet pcg_ls{};
  int pcg_counts[3] = {0, 0, 0};   // kernels per group: Schur product, fused camera kernel, separate camera kernels
  bool pcg_graph_off = false;      // capture failed once: launch directly
  int pcg_full = 0;                // solver of the last scalars filled (1: full system)
  int pcg_exec_full = -1;          // solver the captured group was recorded for
};


namespace gpo_host {

// Camera state and tangent sizes of the graph's camera kind.
inline int cam_ss(const gpo_graph* g) { return g->cam_kind == GPO_V_NAV15 ? 16 : 9; }
inline int cam_db(const gpo_graph* g) { return g->cam_kind == GPO_V_NAV15 ? 15 : 9; }
inline const gpo::KernelSet& kernels_of(const gpo_graph* g) {
  return gpo::kernels_for(g->cam_kind == GPO_V_NAV15 ? gpo::ModelKind::STEREO : gpo::ModelKind::BA);
}

gpo_status fail(gpo_graph* g, gpo_status st, const char* fmt, ...);
gpo_status finalize(gpo_graph* g, size_t* plan_bytes = nullptr);
void release_device(gpo_graph* g);
void fill_scalars(gpo_graph* g, const gpo_lm_params& p, double lambda, Scalars& s);
gpo_status upload_scalars(gpo_graph* g, const Scalars& s);
gpo_lm_params params_or_default(const gpo_lm_params* p);
// One LM iteration's solve (linearise, Schur, PCG, back-substitution) over `ls`
// on g's stream, counting launches in g's profiler.
gpo_status solve_system(gpo_graph* g, const gpo::LaunchSet& ls, int max_it, bool force_lin);
// Retraction, candidate cost, decision and commit over `ls`.
gpo_status finish_iteration(gpo_graph* g, const gpo::LaunchSet& ls);
// Camera render blocks, F(x) and its per-problem reduction over `ls` (no sync).
gpo_status launch_initial_cost(gpo_graph* g, const gpo::LaunchSet& ls);
void prof_resolve(gpo_graph* g);
// Drops the captured PCG group (its launch set is gone).
void drop_pcg_graph(gpo_graph* g);
// Copies the final device state back into the graph's host arrays (user order).
gpo_status download_state(gpo_graph* g);
// The same in two halves: enqueue the copies (points into `pts`), then, after the
// caller has synchronised the graph's stream, scatter the points to user order.
gpo_status download_begin(gpo_graph* g, std::vector<double>& pts);
void download_end(gpo_graph* g, const std::vector<double>& pts);
// Creates the graph's stream unless one was given or adopted (done by the first full
// finalize), and its pinned staging and events (done by the calls that need them).
gpo_status ensure_stream(gpo_graph* g);
gpo_status ensure_runtime(gpo_graph* g);

}  // namespace gpo_host

#define GPO_CUDA(g, call)                                                                    \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return gpo_host::fail((g), GPO_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
