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
//  * Jacobians are stored edge-major, one 24-value row per edge in point-major edge
//    order (48 / 96 / 192 bytes in BF16 / FP32 / FP64: 16-byte vector accesses).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gpo {

constexpr int kThreads = 256;       // CTA size of the chunk kernels
constexpr int kCamDim = 9;          // BA camera tangent size
constexpr int kPtDim = 3;
constexpr int kJComp = 24;          // 2 x (9 + 3) Jacobian values per edge
constexpr int kCamTri = 45;         // packed upper triangle of a 9x9 block
constexpr int kPartA = 54;          // H_cc (45) + b_c (9)
constexpr int kCamPerBlock = 8;     // cameras (warps) per CTA in camera kernels
constexpr int kMaxHistory = 4096;

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
  int pad_;
};

struct IterRecord {       // mirrors gpo_iter_record
  double cost, cand_cost, model_decrease, rho, lambda, pcg_residual;
  int accepted, pcg_iters;
};

// Raw device pointers of one (possibly batched) BA problem set.  Arrays marked AT
// are of the accumulation type (double in FP64 mode, float otherwise); J is of the
// storage type (double, float or __nv_bfloat16).
struct DevBA {
  int C, P, E, NCH, NS;
  // topology (point-major edge order)
  const int* e_cam;          // [E]
  const int* e_pt;           // [E]
  const double* obs;         // [E][2]
  const double* e_delta;     // [E] Huber threshold, <= 0: plain squares
  const double* e_sqinfo;    // [E][3] upper Cholesky factor of Omega (u00 u01 u11) or null
  const int* pt_off;         // [P+1]
  const int* ch_e0;          // [NCH+1]
  const int* ch_p0;          // [NCH+1]
  const int* ch_s0;          // [NCH+1]
  const uint16_t* e_pos;     // [E] position of the edge in its chunk's slot-sorted order
  const uint16_t* e_slot;    // [E] slot of the edge inside its chunk
  const uint16_t* ch_sorted; // [E] per chunk: local edge ids sorted by (slot, id)
  const int* slot_e0;        // [NS+1] range of a slot in ch_sorted (global positions)
  const int* slot_cam;       // [NS]
  const int* slot_pos;       // [NS] row of the slot's partial in camera-major order
  const int* cam_s_off;      // [C+1]
  const int* cam_s_list;     // [NS] slots of each camera, chunk order
  const uint8_t* cam_fixed;  // [C]
  const uint8_t* pt_fixed;   // [P]
  // FP64 state
  double* cam;               // [C][9]
  double* cam_cand;          // [C][9]
  double* camrb;             // [C][16] R (9) t (3) f k1 k2 pad
  double* camrb_cand;        // [C][16]
  double* pt;                // [P][3]
  double* pt_cand;           // [P][3]
  // linear system
  void* J;                   // JT [E][24] edge-major rows
  void* Hpp;                 // AT [P][6] undamped point blocks
  void* bp;                  // AT [P][3]
  void* Hinv;                // AT [P][6] damped inverses
  void* dp;                  // AT [P][3] point step
  void* partA;               // AT [NS][54]
  void* partB;               // AT [NS][54]
  void* partV;               // AT [NS][9]
  void* Hcl;                 // AT [C][45] H_cc + lambda D_c
  void* bc;                  // AT [C][9]
  void* S;                   // AT [C][45] Schur diagonal blocks
  void* Minv;                // AT [C][45] block-Jacobi preconditioner S_cc^-1
  void* g;                   // AT [C][9] reduced right-hand side
  void* x; void* r; void* z; void* p; void* p2; void* y; void* xbest;   // AT [C][9]
  double* cost_part;         // [NCH]
  double* md_part;           // [NCH]
  double* cblk_part;         // [ncblk][2]
  Scalars* sc;               // [1]
  IterRecord* hist;          // [kMaxHistory]
  double* dbg_r;             // optional [E][2] weighted residual output
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
  int* running;          // problems whose PCG is still iterating
  int nprob, n_ch, n_cb, n_pb;
  int ch_max;            // largest chunk over the problems (shared-memory sizing)
  int ns_max, np_max;    // most slots / points in one chunk over the problems
};

// Kernel launchers (ba_kernels.cu).  All are asynchronous on `st`.
int launch_cam_prepare(const LaunchSet& ls, bool candidate, cudaStream_t st);
int launch_cost(const LaunchSet& ls, bool candidate, cudaStream_t st);
int launch_cost_init(const LaunchSet& ls, cudaStream_t st);
int launch_linearize(const LaunchSet& ls, Prec pr, bool force, cudaStream_t st);
int launch_schur_prepare(const LaunchSet& ls, Prec pr, cudaStream_t st);
int launch_cam_finalize(const LaunchSet& ls, Prec pr, cudaStream_t st);
int launch_pcg_spmv(const LaunchSet& ls, Prec pr, cudaStream_t st);      // the Schur product (hot loop)
int launch_cam_apply(const LaunchSet& ls, Prec pr, cudaStream_t st);     // y = S p camera side, alpha
int launch_pcg_update(const LaunchSet& ls, Prec pr, cudaStream_t st);    // x, r, z; stopping rules, beta
int launch_backsub(const LaunchSet& ls, Prec pr, cudaStream_t st);
int launch_retract(const LaunchSet& ls, Prec pr, cudaStream_t st);
int launch_decide(const LaunchSet& ls, Prec pr, cudaStream_t st);
int launch_commit(const LaunchSet& ls, cudaStream_t st);
size_t smem_bytes_linearize(Prec pr, int ch_max);
int default_ch_max(Prec pr);
int max_supported_ch(Prec pr);

}  // namespace gpo
