// Internal declarations shared by the CUDA translation units of libgpo.
//
// Device data layout (one problem, or many concatenated problems in a batch):
//  * edges are sorted point-major (all edges of a point are contiguous) and
//    partitioned into chunks of whole points with at most `ch_max` edges; every
//    per-edge kernel runs one CTA per chunk, so per-point reductions stay inside a
//    CTA and need no atomics;
//  * inside a chunk, the distinct cameras form "slots"; a CTA reduces its edges'
//    camera contributions per slot in a fixed order (edges pre-sorted by slot) and
//    writes one partial per slot; a camera sums its slots' partials in chunk order.
//    Every reduction therefore has a fixed order: runs are bit-reproducible;
//  * Jacobians are stored edge-major, one row per edge in point-major edge order
//    (BA: 24 values, 48 / 96 / 192 bytes in BF16 / FP32 / FP64; stereo: 27 values
//    padded to 32): 16-byte vector accesses;
//  * the edge model (BAL reprojection on 9-dim cameras, or stereo reprojection on
//    15-dim navigation states plus inertial / bias edges between them) is a
//    compile-time parameter of the kernels; a graph picks its kernel set at finalize.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gpo {

constexpr int kThreads = 256;       // CTA size of the chunk kernels
constexpr int kPtDim = 3;
constexpr int kCamPerBlock = 8;     // cameras (warps) per CTA in camera kernels
constexpr int kMaxDevices = 64;     // per-device launch caches
constexpr int kGroupEdges = 64;     // edges of a warp group (two per lane) of a chunk
constexpr int kMaxGroups = 16;      // warp groups per chunk
constexpr int kMaxHistory = 4096;

// Edge models (the kernel set a graph runs).
enum class ModelKind { BA = 0, STEREO = 1 };

// Camera-side ("extra") edges of the navigation model: inertial (9 rows), bias random
// walk (6 rows) between keyframes i and j, bias prior (6 rows) on keyframe i.
enum XKind { XK_IMU = 0, XK_BIAS_RW = 1, XK_BIAS_PRIOR = 2 };
constexpr int kXRows = 9;           // largest residual of an extra edge
constexpr int kXCols = 30;          // two 15-dim navigation blocks
constexpr int kXJ = kXRows * kXCols;
// Record of an extra edge (doubles): the measurement, then the upper-triangular
// square root U of the information matrix (Omega = U^T U), row-major kXRows x kXRows.
//  IMU:   dR (9, row-major), dv (3), dp (3), JRg, Jvg, Jva, Jpg, Jpa (9 each), T, bg0 (3), ba0 (3)
//  prior: bg_prior (3), ba_prior (3)
constexpr int kImuMeas = 67;
constexpr int kXU = 72;             // offset of U in the record
constexpr int kXDelta = kXU - 1;    // Huber threshold of the whitened residual (0: no loss)
constexpr int kXRec = kXU + kXRows * kXRows;   // 153

__host__ __device__ inline int pad8(int n) { return (n + 7) & ~7; }

// Per-problem scalars of the LM / PCG state machine (device resident).
struct Scalars {
  // LM
  double lambda, nu, cost, cand_cost, model_dec, rho;
  double lambda_min, lambda_max, diag_min, diag_max;
  int damping_mode, need_lin, accepted, n_accepted, iter, pcg_total;
  // PCG
  double gnorm;          // |g|
  double rz;             // r^T z of the (scaled) current residual
  double pAp, alpha, beta, inv_n;
  double sigma;          // true residual = sigma * stored residual
  double rnorm;          // true |r|
  double rmin;           // min_j |r_j| (rejection-ratio guard)
  double tol_abs;        // stop when |r| <= tol_abs
  double ratio;          // rejection ratio (<= 0: off)
  double pcg_tol;        // PCG tolerance (relative to |g| if pcg_rel)
  int pcg_rel;
  int pcg_it, pcg_done, use_best, save_best, normalize, max_it;
  int pidx;              // which direction buffer holds p_{k-1} (0: p, 1: p2)
  unsigned int ticket;   // last-CTA counter of the reductions
  int active;            // the problem takes part in the current launches
  int lm_max;            // LM iterations to run (the problem deactivates after them)
  int restart_every;     // true-residual restart period in PCG iterations (0: off)
  int restart;           // the current PCG iteration is a restart: the product is S x,
                         // the update sets r = g - S x and restarts the direction
  int pcg_products;      // Schur products of the current solve (iterations + restarts)
  int full;              // PCG on the full damped system (cameras and points) instead of
                         // the camera Schur complement
  int pcg_fail;          // the solve broke down before its first step (r^T M r or p^T S p
                         // not positive, or not finite): no step; a failed linear solve,
                         // the LM step is rejected
  int pcg_breakdown;     // the solve broke down after a step (the damped system is at the
                         // edge of positive definiteness in the working precision): the
                         // iterate is a descent step, but the damping is not lowered
  int have_best;         // the rejection-ratio guard has saved an iterate
  float beta_f, inv_n_f; // beta and inv_n rounded to FP32 once, where they are set (the
                         // FP32 kernels read these: a conversion from FP64 per thread
                         // would occupy the part's small FP64 pipe)
};

struct IterRecord {       // mirrors gpo_iter_record
  double cost, cand_cost, model_decrease, rho, lambda, pcg_residual;
  int accepted, pcg_iters, pcg_products, pcg_failed;
};

// Raw device pointers of one problem.  Arrays marked AT are of the accumulation type
// (double in FP64 mode, float otherwise); J is of the storage type (double, float or
// __nv_bfloat16).  Sizes by model: SS = camera state (9 BA, 16 navigation), DB =
// camera tangent block (9 / 15), DC = camera columns of an observation's Jacobian
// (9 / 6), M = observation rows (2 / 3), NJ = Jacobian row (24 / 32), NPA = slot
// partial row (54 / 27), TB = packed camera block (45 / 120).
struct DevBA {
  int C, P, E, NCH, NS;
  int NX;                    // extra (camera-side) edges
  int model;                 // ModelKind
  double camk[24];           // stereo rig: fx fy cx cy baseline, R_cb (9, row-major), t_cb (3),
                             // [17] projection (0 pinhole, 1 Kannala-Brandt fisheye), [18..21] k1..k4
  // topology (point-major edge order)
  const int* e_cam;          // [E]
  const int* e_pt;           // [E]
  const double* obs;         // [E][M]
  const double* e_delta;     // [E] Huber threshold, <= 0: plain squares
  const double* e_sqinfo;    // [E][tri(M)] packed upper Cholesky factor of Omega, or null
  const int* pt_off;         // [P+1]
  const int* ch_e0;          // [NCH+1]
  const int* ch_p0;          // [NCH+1]
  const int* ch_s0;          // [NCH+1]
  const uint16_t* e_pos;     // [E] position of the edge in its chunk's slot-sorted order
  const uint16_t* e_slot;    // [E] slot of the edge inside its chunk
  const uint16_t* ch_sorted; // [E] per chunk: local edge ids sorted by (slot, id)
  const uint32_t* e_meta;    // [E + 4] packed pos | slot << 10 | local point << 20 (chunks <= 1024)
  const uint16_t* ch_grp;    // [NCH][kMaxGroups] local edge offset where warp group g of the
                             // chunk ends (groups of whole points, <= kGroupEdges edges
                             // unless one point has more)
  const int4* slot_rec;      // [NS] local edge range [x, y) in slot order, camera z, partial row w
  const int* slot_e0;        // [NS+1] range of a slot in ch_sorted (global positions)
  const int* slot_cam;       // [NS]
  const int* slot_pos;       // [NS] row of the slot's partial in camera-major order
  const int* cam_s_off;      // [C+1]
  const int* cam_s_list;     // [NS] slots of each camera, chunk order
  const uint8_t* cam_fixed;  // [C]
  const uint8_t* pt_fixed;   // [P]
  // extra edges, sorted by (first vertex, id)
  const int* xe_i;           // [NX] first camera
  const int* xe_j;           // [NX] second camera, -1 for a unary edge
  const int* xe_kind;        // [NX] XKind
  const double* xe_rec;      // [NX][kXRec]
  const int* xo_off;         // [C+1] extra edges whose first camera is c
  const int* xk_off;         // [C+1] extra edges touching camera c ...
  const int* xk_list;        // [2 NX] ... as 2 x + side (side 1: c is the second camera)
  double* xe_J;              // [NX][kXRows][kXCols] whitened Jacobian (FP64)
  double* xe_r;              // [NX][kXRows] whitened residual
  double* xe_cost;           // [NX] 1/2 |r|^2 at the last evaluated state
  double* xe_md;             // [NX] -1/2 |J dx|^2
  void* xe_H;                // AT [NX][15][15] J_i^T J_j of two-keyframe edges (row-major)
  // FP64 state
  double* cam;               // [C][SS]
  double* cam_cand;          // [C][SS]
  double* camrb;             // [C][16] render block (BA: R t f k1 k2 pad; nav: R p pad)
  double* camrb_cand;        // [C][16]
  float* camrbf;             // [C][16] the render block rounded to FP32 (mixed-precision rows)
  float* camrbf_cand;        // [C][16]
  double* pt;                // [P][3]
  double* pt_cand;           // [P][3]
  // linear system
  void* J;                   // JT [E][NJ] edge-major rows
  void* Hpp;                 // AT [P][6] undamped point blocks
  void* bp;                  // AT [P][3]
  void* Hinv;                // AT [P][6] damped inverses
  void* pt_rec;              // [P] records of 32 (FP32) / 64 (FP64) bytes: H_pp^-1 (6 AT), local edge range (2 int)
  void* dp;                  // AT [P][3] point step
  void* partA;               // AT [NS][NPA]
  void* partB;               // AT [NS][NPA]
  void* partV;               // AT [NS][DC]
  void* Hcl;                 // AT [C][TB] H_cc + lambda D_c
  void* bc;                  // AT [C][DB]
  void* S;                   // AT [C][TB] Schur diagonal blocks
  void* Minv;                // AT [C][TB] block-Jacobi preconditioner S_cc^-1
  void* g;                   // AT [C][DB] reduced right-hand side
  void* x; void* r; void* z; void* p; void* p2; void* y; void* xbest;   // AT [C][DB]
  // full-system PCG, point part (allocated on first use): AT [P][3] each
  void* xq; void* rq; void* zq; void* pq; void* pq2; void* yq; void* xqbest;
  double* pt_part;           // [npb][2] per-point-block partial sums (full-system PCG)
  double* cost_part;         // [NCH]
  double* md_part;           // [NCH]
  double* cblk_part;         // [ncblk][2]
  Scalars* sc;               // [1]
  IterRecord* hist;          // [kMaxHistory]
  double* dbg_r;             // optional [E][M] weighted residual output
  int ch_max;                // max edges per chunk
  int ns_max, np_max;        // max slots / points of a chunk
  int ncblk;                 // CTAs of the camera kernels
};

enum class Prec { F64 = 0, F32 = 1, BF16 = 2 };

// A launch over several independent problems (one problem for a plain graph).
// Every CTA finds its problem through a schedule table and binds that problem's
// DevBA (device copy) in shared memory:
//  * chunk CTAs (per-edge kernels): ch_prob[b], local chunk b - ch_base[problem];
//  * camera CTAs (8 cameras, one warp each): cb_prob[b], local block b - cb_base[..];
//  * point CTAs (256 points): pb_prob[b], local block b - pb_base[..];
//  * problem CTAs (decisions, reductions): CTA b is problem b.
struct LaunchSet {
  const DevBA* probs;
  const int* ch_prob; const int* ch_base;
  const int* cb_prob; const int* cb_base;
  const int* pb_prob; const int* pb_base;
  int* running;          // [2]: problems whose PCG is still iterating; [1] error flag (a
                         // bounded device wait gave up)
  int* err;              // = running + 1
  int* work;             // = running + 2: [0] next chunk handed out by the pipelined Schur
                         // product, [1] its CTAs that have finished (both back to 0 at
                         // the end of every launch); [2] arrivals at the camera kernel's
                         // grid barrier (back to 0 at every barrier), [3] its generation
  int spmv_variant;      // Schur-product kernel: 0 auto, 1 staged (bulk copies), 2 classic,
                         // 3 pipelined, 4 dynamic Jacobians
  int debug_wait;        // test hook, 0 in production: the camera kernel's grid barrier
                         // waits for this many CTAs more than the grid, so that its
                         // bounded wait gives up
  int nprob, n_ch, n_cb, n_pb;
  int ch_max;            // largest chunk over the problems (shared-memory sizing)
  int ns_max, np_max;    // most slots / points in one chunk over the problems
};

// Kernel set of one edge model.  Every launcher is asynchronous on `st` and returns
// the number of kernels it launched.
struct KernelSet {
  ModelKind model;
  int SS, DB, DC, M, NJ, NPA;     // sizes (see DevBA)
  int (*cam_prepare)(const LaunchSet& ls, bool candidate, cudaStream_t st);
  int (*cost)(const LaunchSet& ls, bool candidate, cudaStream_t st);
  int (*cost_init)(const LaunchSet& ls, cudaStream_t st);
  int (*linearize)(const LaunchSet& ls, Prec pr, bool force, cudaStream_t st);
  int (*schur_prepare)(const LaunchSet& ls, Prec pr, cudaStream_t st);
  int (*cam_finalize)(const LaunchSet& ls, Prec pr, cudaStream_t st);
  int (*pcg_spmv)(const LaunchSet& ls, Prec pr, cudaStream_t st);     // the Schur product (hot loop)
  int (*cam_apply)(const LaunchSet& ls, Prec pr, cudaStream_t st);    // y = S p camera side, alpha
  int (*pcg_update)(const LaunchSet& ls, Prec pr, cudaStream_t st);   // x, r, z; stopping rules, beta
  int (*pcg_camera)(const LaunchSet& ls, Prec pr, cudaStream_t st);   // cam_apply + pcg_update in one launch
  // full-system PCG (cameras and points; the paper's form): point-side start, the
  // product with the whole damped H, the update over camera and point blocks
  int (*full_init)(const LaunchSet& ls, Prec pr, cudaStream_t st);
  int (*full_spmv)(const LaunchSet& ls, Prec pr, cudaStream_t st);
  int (*full_update)(const LaunchSet& ls, Prec pr, cudaStream_t st);
  // forward-mode automatic differentiation of the observation edges (checker)
  int (*autodiff)(const LaunchSet& ls, int n_edges, double* r, double* J, cudaStream_t st);
  int (*backsub)(const LaunchSet& ls, Prec pr, cudaStream_t st);
  int (*retract)(const LaunchSet& ls, Prec pr, cudaStream_t st);
  int (*decide)(const LaunchSet& ls, Prec pr, cudaStream_t st);
  int (*commit)(const LaunchSet& ls, cudaStream_t st);
  int (*max_supported_ch)(Prec pr);
  int (*spmv_kind)(const LaunchSet& ls, Prec pr);   // the Schur-product kernel pcg_spmv runs
};
const KernelSet& kernels_ba();       // ba_kernels.cu
const KernelSet& kernels_stereo();   // vi_kernels.cu
inline const KernelSet& kernels_for(ModelKind m) { return m == ModelKind::STEREO ? kernels_stereo() : kernels_ba(); }
inline int default_ch_max(Prec) { return 512; }

// Jacobian rows are stored in tiles of kJTile consecutive edges, each row cut into
// 16-byte pieces and piece q of a tile's rows stored contiguously: piece q of row e is
// 16-byte unit ((e / kJTile) * Q + q) * kJTile + e % kJTile, Q = row bytes / 16.
constexpr int kJTile = 32;

}  // namespace gpo
