/*
 * gpo.h -- C ABI of the GB300-native Levenberg-Marquardt graph optimiser.
 *
 * The library solves weighted nonlinear least squares over a hypergraph of
 * vertices (parameter blocks) and edges (constraints):
 *     argmin_x 1/2 sum_e rho(r_e(x)^T Omega_e r_e(x))            (Eq. 1, Eq. 7)
 * with Levenberg-Marquardt (Eq. 3-6).  Each iteration linearises every edge,
 * eliminates the 3-D points with a Schur complement, solves the reduced camera
 * system by block-Jacobi preconditioned conjugate gradients without storing it
 * (Sec. IV-E) and back-substitutes the points.  Vertices live in FP64; the
 * linear system is FP64, FP32 or BF16 storage with FP32 accumulation (Sec. IV-E,
 * Listing 3's Graph<FP, SP>).
 *
 * Conventions for every call:
 *  - Return value: GPO_OK (0) or a negative gpo_status.  No C++ exception
 *    crosses the ABI.  On error, gpo_last_error(g) gives a message; the graph
 *    stays usable unless the status is GPO_ERR_CUDA.
 *  - Host pointers are owned by the caller and only read or written during the
 *    call.  Device pointers (on_device = 1) must be CUDA device memory of the
 *    graph's device; copies run on the graph's stream and the call waits for them.
 *  - All device memory of a graph is owned by the library (allocated through the
 *    optional allocator hook of gpo_graph_desc) and released by gpo_graph_destroy.
 *  - A graph is not thread-safe: one host thread at a time per graph.
 *  - Vertex and edge ids are int64, assigned consecutively from 0 in the order
 *    of the add calls (vertices and edges have separate counters).
 */
#ifndef GPO_H
#define GPO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpo_graph gpo_graph;

typedef enum {
  GPO_OK = 0,
  GPO_ERR_ARG = -1,          /* invalid argument (null pointer, bad id, bad size, bad kind) */
  GPO_ERR_OOM = -2,          /* device memory or the memory budget exhausted */
  GPO_ERR_STATE = -3,        /* call not allowed in the graph's state (e.g. add after optimize) */
  GPO_ERR_NUMERIC = -4,      /* non-finite cost at the initial state */
  GPO_ERR_CUDA = -5,         /* a CUDA call failed; the message names it */
  GPO_ERR_TIMEOUT = -6,      /* a bounded device wait gave up */
  GPO_ERR_UNSUPPORTED = -7   /* valid request that this build does not support */
} gpo_status;

/* Precision of the linear system (Listing 3: Graph<FP, SP>).  Vertex states, the
 * retraction, the total cost and the gain ratio are always FP64. */
typedef enum {
  GPO_FP64 = 0,       /* Jacobians, Hessian blocks and PCG in FP64 */
  GPO_FP32 = 1,       /* Jacobians, Hessian blocks and PCG in FP32 */
  GPO_FP32_BF16 = 2   /* Jacobians stored in BF16, accumulation and PCG in FP32;
                         gradient from the unrounded FP32 Jacobian; preconditioner
                         and point-block inverses kept in FP32 (Sec. IV-E) */
} gpo_precision;

/* Vertex kinds (Listing 1's dimension = tangent block size; state size in brackets).
 *  GPO_V_BA_CAMERA9: BAL camera [wx wy wz tx ty tz f k1 k2], tangent 9;
 *                    rotation updated as w <- Log(Exp(dw) Exp(w)), rest additive.
 *  GPO_V_POINT3:     3-D point [X Y Z], tangent 3, additive; eliminated by Schur.
 *  GPO_V_NAV15:      keyframe navigation state [qx qy qz qw px py pz vx vy vz
 *                    bgx bgy bgz bax bay baz] (16 doubles; q a unit quaternion of the
 *                    body-to-world rotation R, p and v in the world frame, gyroscope and
 *                    accelerometer biases), tangent 15 [dtheta dp dv dbg dba]:
 *                    R <- R Exp(dtheta), p <- p + R dp, the rest additive (Sec. V-C's
 *                    IMU-camera pose, velocity and bias vertices as one block).
 * A graph holds points and ONE camera kind (GPO_V_BA_CAMERA9 or GPO_V_NAV15). */
enum { GPO_V_BA_CAMERA9 = 0, GPO_V_POINT3 = 1, GPO_V_NAV15 = 2 };

/* Edge kinds (vertex ids per edge in brackets; meas length; residual size m).
 *  GPO_E_BA_REPROJ  {camera9, point}; meas 2 [u v] pixels; m = 2 (Eq. 7, Sec. V BAL).
 *    r = f (1 + k1 |p|^2 + k2 |p|^4) p - meas with P = R(w) X + t, p = -P_xy / P_z.
 *  GPO_E_STEREO     {nav15, point}; meas 3 [u_l v_l u_r] pixels; m = 3 (Sec. V-C).
 *    X_b = R^T (X - p), X_c = R_cb X_b + t_cb (rig of gpo_set_stereo_camera),
 *    r = [fx X_c/Z_c + cx, fy Y_c/Z_c + cy, fx (X_c - b)/Z_c + cx] - meas.
 *  GPO_E_IMU        {nav15 i, nav15 j}; meas = a preintegrated IMU record of
 *    GPO_IMU_MEAS_LEN doubles (gpo_imu_preintegrate); m = 9 (Eq. 8 r_I):
 *      r_R = Log((dR Exp(JRg dbg))^T R_i^T R_j),
 *      r_v = R_i^T (v_j - v_i - g T) - (dv + Jvg dbg + Jva dba),
 *      r_p = R_i^T (p_j - p_i - v_i T - g T^2 / 2) - (dp + Jpg dbg + Jpa dba),
 *    dbg = bg_i - bg0, dba = ba_i - ba0, g = (0, 0, -9.81).
 *  GPO_E_BIAS_RW    {nav15 i, nav15 j}; meas unused (may be NULL); m = 6 (Eq. 8 r_b):
 *    r = [bg_j - bg_i, ba_j - ba_i].
 *  GPO_E_BIAS_PRIOR {nav15}; meas 6 [bg ba] prior; m = 6: r = [bg, ba] - meas.
 *  GPO_E_MONO       {nav15, point3}; meas 2 pixels [u v] in the left camera of the
 *    stereo rig; m = 2: the first two rows of GPO_E_STEREO's residual.  Info is 2 x 2.
 *    Stored as a stereo edge whose third row is whitened to zero (edges of both kinds
 *    share the graph and its kernels).
 * GPO_E_IMU may take the Huber loss on its whitened 9-dim residual (the robust inertial
 * edge of the paper's VI descriptors); GPO_E_BIAS_RW and GPO_E_BIAS_PRIOR take no
 * robust loss (GPO_ERR_UNSUPPORTED). */
enum { GPO_E_BA_REPROJ = 0, GPO_E_STEREO = 1, GPO_E_IMU = 2, GPO_E_BIAS_RW = 3,
       GPO_E_BIAS_PRIOR = 4, GPO_E_MONO = 5 };

/* Preintegrated IMU record (doubles, matrices row-major):
 *   [0..9)  dR   [9..12) dv   [12..15) dp   [15..24) JRg  [24..33) Jvg  [33..42) Jva
 *   [42..51) Jpg [51..60) Jpa [60] T        [61..64) bg0  [64..67) ba0 */
enum { GPO_IMU_MEAS_LEN = 67 };

enum { GPO_LOSS_NONE = 0, GPO_LOSS_HUBER = 1 };

typedef struct {
  int32_t precision;          /* gpo_precision */
  int32_t device;             /* CUDA device ordinal */
  int64_t reserve_vertices;   /* capacity hints (Listing 3/4: reserve); 0 = none */
  int64_t reserve_edges;
  void* cuda_stream;          /* cudaStream_t to run on; NULL = the library creates one */
  /* Optional allocator hook for all device memory (e.g. a framework's caching
   * allocator).  alloc returns device memory of at least `bytes` bytes aligned to
   * 256 bytes, or NULL; free releases it.  NULL alloc = cudaMalloc / cudaFree. */
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* alloc_ctx;
  size_t memory_budget;       /* bytes; 0 = unlimited.  Exceeding it gives GPO_ERR_OOM. */
  int32_t chunk_edges;        /* edges per CTA chunk of the per-edge kernels (32..2048;
                                 0 = default: 512); raised to the longest track.  A
                                 tuning knob: the chunking groups the per-camera partial
                                 sums, so results agree up to rounding. */
  int32_t spmv_variant;       /* Schur-product kernel: 0 = automatic (pipelined for BF16
                                 and FP32 storage, classic for FP64), 1 = staged
                                 (persistent CTAs streaming chunks into shared memory
                                 with bulk copies), 2 = classic (one CTA per chunk),
                                 3 = pipelined (persistent CTAs prefetching the next
                                 chunk's indices while the current one runs),
                                 4 = dynamic Jacobians (no rows are stored: every kernel
                                 that needs an edge's rows evaluates them from the
                                 state in the accumulation type, FP32 with FP32 or BF16
                                 storage, which are then one mode; Sec. IV-D, Table II.
                                 Needs points of at most 512 observations, else
                                 GPO_ERR_UNSUPPORTED at the first optimize; not with
                                 the full-system solver, batches or servers, and
                                 gpo_debug_linearize has no rows to return),
                                 5 = warp groups (each warp owns runs of whole points:
                                 rows read once into registers, point sums by a
                                 segmented warp scan, one barrier per chunk; BF16 and
                                 FP32 storage).  1, 3 and 5 need chunks of at most 1024
                                 edges, 4 of at most 512, else classic runs (5 with
                                 FP64 storage too).  0..3 give bit-identical results;
                                 5 sums each point's terms in another order and 4 uses
                                 unrounded rows, so their products agree with the
                                 others up to rounding. */
} gpo_graph_desc;

/* Linear solver of the LM step (gpo_lm_params.solver). */
enum {
  GPO_SOLVER_SCHUR = 0,   /* PCG on the camera Schur complement, points by back-substitution */
  GPO_SOLVER_FULL = 1     /* PCG on the full damped system of cameras and points (Sec. IV-E) */
};

/* Levenberg-Marquardt and PCG options (Listing 5: LevenbergMarquardtOptions and
 * PCGSolver(max_it, tol, rejection_ratio)). */
typedef struct {
  double initial_damping;     /* lambda_0 (Listing 5 initial_damping); default 1e-4 */
  double lambda_min;          /* damping clamp; default 1e-16 */
  double lambda_max;          /* default 1e32 */
  double diag_min;            /* D^T D = clamp(diag(H), diag_min, diag_max) (Sec. IV-E) */
  double diag_max;            /* defaults 1e-6, 1e32 */
  int32_t damping_mode;       /* 0 = clamped diag(H) (Marquardt), 1 = identity (Eq. 4) */
  int32_t pcg_max_iters;      /* default 100 */
  double pcg_tol;             /* default 1e-6 */
  int32_t pcg_tol_relative;   /* 1: stop at |r| <= tol |g|; 0: stop at |r| <= tol */
  double pcg_rejection_ratio; /* stop when |r_k| > ratio * min_j |r_j| and return the
                                 best iterate; <= 0 or inf disables; default 10 */
  int32_t pcg_normalize;      /* keep the PCG residual at unit norm each iteration
                                 (Sec. IV-E); -1 = on for FP32/BF16, off for FP64 */
  int32_t pcg_restart_every;  /* residual restarts: after every this many PCG
                                 iterations one extra Schur product recomputes the
                                 true residual r = g - S x from the current solution
                                 and the direction restarts from z = M r; the
                                 recursively updated residual of FP32/BF16 arithmetic
                                 drifts from the true one.  -1 (default) or 0 = off
                                 (a restart discards the Krylov directions, which slows
                                 convergence); otherwise >= 4 (smaller values are
                                 raised to 4). */
  int32_t solver;             /* GPO_SOLVER_SCHUR (default) or GPO_SOLVER_FULL: the paper's
                                 block-Jacobi PCG on all vertices at once (camera blocks
                                 (H_cc + lambda D_c)^-1 and point blocks (H_pp +
                                 lambda D_p)^-1 as preconditioner, products from the
                                 stored Jacobians, one pass over them per iteration).
                                 An exact solve of either gives the same step; the
                                 tolerance and iteration cap apply to the solved system's
                                 residual.  The full form allocates seven [P][3] vectors
                                 on its first use (counted by gpo_memory_footprint and
                                 held to the graph's memory budget: GPO_ERR_OOM).
                                 Graphs without cameras, and graphs solved together
                                 (gpo_optimize_batch, a server), use the Schur form. */
  double initial_nu;          /* Nielsen's multiplier nu at the start (after a rejected
                                 step lambda *= nu, nu *= 2; after an accepted one nu = 2).
                                 Values below 2 (the default 0) start from 2.  With
                                 initial_damping = the previous report's final_lambda
                                 and initial_nu = its final_nu, a sequence of calls
                                 continues one LM run exactly. */
} gpo_lm_params;

typedef struct {
  double initial_cost;        /* F(x_0) = 1/2 sum rho, FP64 */
  double final_cost;          /* F at the returned state */
  double final_lambda;
  int32_t iterations;         /* LM iterations run (= max_iters) */
  int32_t accepted;           /* accepted steps */
  int32_t pcg_iters_total;
  int32_t reserved0;
  double final_nu;            /* Nielsen's nu after the last iteration (see initial_nu) */
} gpo_report;

/* One LM iteration's record (gpo_get_history). */
typedef struct {
  double cost;                /* F(x) before the step */
  double cand_cost;           /* F(x [+] dx) */
  double model_decrease;      /* L(0) - L(dx) = -b^T dx - 1/2 |J dx|^2 */
  double rho;                 /* gain ratio */
  double lambda;              /* damping used for this step */
  double pcg_residual;        /* final |r| / |g| of the PCG solve */
  int32_t accepted;
  int32_t pcg_iters;
  int32_t pcg_products;       /* Schur products run: PCG iterations plus residual restarts */
  int32_t pcg_failed;         /* 1: the PCG broke down before its first step (r^T M r or
                                 p^T S p not positive or not finite: the damped system
                                 is not positive definite in the working precision), or
                                 the best iterate kept by the rejection-ratio guard is
                                 the zero start; the linear solve failed, so the step
                                 was rejected (lambda grows).  2: it broke down after a
                                 step; the iterate was judged as any step, but lambda
                                 was not lowered.  0: neither */
} gpo_iter_record;

/* Defaults for the two option structs.  Never fail for non-null pointers. */
gpo_status gpo_graph_desc_default(gpo_graph_desc* out);
gpo_status gpo_lm_params_default(gpo_lm_params* out);

/* Creates an empty graph (Listing 3: Graph<FP, SP> graph).  *out receives the handle.
 * Errors: GPO_ERR_ARG (null, bad precision or device), GPO_ERR_CUDA. */
gpo_status gpo_graph_create(const gpo_graph_desc* desc, gpo_graph** out);

/* Releases the graph and all its device memory.  NULL is a no-op. */
gpo_status gpo_graph_destroy(gpo_graph* g);

/* Adds n vertices of `kind` (Listing 4: add_vertex).  block_size must equal the
 * kind's tangent dimension (9 camera, 3 point, 15 navigation).  *first_id (optional)
 * receives the id of the first new vertex; the others follow consecutively.  Initial
 * state is zero (navigation states: identity rotation) until gpo_set_initial.
 * Errors: GPO_ERR_ARG (also for a second camera kind), GPO_ERR_STATE (after optimize). */
gpo_status gpo_add_vertices(gpo_graph* g, int32_t kind, int32_t block_size, int64_t n,
                            int64_t* first_id);

/* Adds n edges of `kind` (Listing 4: add_factor(ids, obs, precision, data, loss)).
 *  vertex_ids: n * arity int64 ids, row-major, in the kind's slot order.
 *  meas:       n * meas_len doubles (see the edge kinds).
 *  info:       n * m * m doubles, row-major symmetric positive definite information
 *              matrices Omega (m = residual size), or NULL for identity (Sec. IV-A:
 *              a null precision matrix means identity).
 *  loss_kind:  GPO_LOSS_NONE or GPO_LOSS_HUBER with threshold loss_delta > 0 in
 *              whitened units (rho(s) = s for s <= delta^2, 2 delta sqrt(s) - delta^2
 *              otherwise, Eq. 7).
 * Errors: GPO_ERR_ARG (unknown ids, wrong vertex kinds, non-SPD info, delta <= 0),
 *         GPO_ERR_STATE (after optimize). */
gpo_status gpo_add_edges(gpo_graph* g, int32_t kind, int64_t n, const int64_t* vertex_ids,
                         const double* meas, const double* info, int32_t loss_kind,
                         double loss_delta, int64_t* first_id);

/* Intrinsics and extrinsics of the stereo rig shared by the graph's GPO_E_STEREO
 * edges: rig[17] = [fx fy cx cy baseline, R_cb (9, row-major, body-to-camera
 * rotation), t_cb (3)].  Required before the first optimize of a graph with stereo
 * edges.  Errors: GPO_ERR_ARG (null), GPO_ERR_STATE (after the first optimize). */
gpo_status gpo_set_stereo_camera(gpo_graph* g, const double* rig);

/* Makes both cameras of the stereo rig Kannala-Brandt (equidistant) fisheye cameras
 * with coefficients k[4] = [k1 k2 k3 k4] (the fisheye descriptor of the paper's VI
 * system): for X_c = (x, y, z), theta = atan2(|(x, y)|, z),
 * theta_d = theta (1 + k1 theta^2 + k2 theta^4 + k3 theta^6 + k4 theta^8), and the
 * projection (fx theta_d x / r + cx, fy theta_d y / r + cy) replaces (fx x / z + cx,
 * fy y / z + cy) in the stereo and monocular residuals (the right camera's point is
 * (x - baseline, y, z)).  Call after gpo_set_stereo_camera (which resets to pinhole).
 * Errors: GPO_ERR_ARG (null, not finite), GPO_ERR_STATE (no rig yet, or after the first
 * optimize). */
gpo_status gpo_set_fisheye(gpo_graph* g, const double* k);

/* On-manifold IMU preintegration (Forster et al., T-RO 2017) of n gyroscope and
 * accelerometer samples gyro[n][3] (rad/s), acc[n][3] (m/s^2) taken every dt seconds,
 * at bias estimates bg0[3], ba0[3], with white-noise densities sigma_g, sigma_a:
 *   dR_{k+1} = dR_k Exp((w_k - bg0) dt), dv_{k+1} = dv_k + dR_k (a_k - ba0) dt,
 *   dp_{k+1} = dp_k + dv_k dt + dR_k (a_k - ba0) dt^2 / 2,
 * with first-order bias Jacobians and the covariance of (dphi, dv, dp) propagated from
 * the discrete noise sigma / sqrt(dt).  meas_out receives the GPO_IMU_MEAS_LEN record
 * for GPO_E_IMU; cov_out (9x9, optional) the covariance; info_out (9x9, optional) its
 * inverse, the information matrix to pass to gpo_add_edges.  Host only: needs no GPU.
 * Errors: GPO_ERR_ARG (null input, n < 1, dt <= 0, sigma <= 0),
 *         GPO_ERR_NUMERIC (covariance not positive definite). */
gpo_status gpo_imu_preintegrate(const double* gyro, const double* acc, int64_t n, double dt,
                                const double* bg0, const double* ba0, double sigma_g,
                                double sigma_a, double* meas_out, double* cov_out,
                                double* info_out);

/* Fixes or frees a vertex (Listing 5: set_fixed).  A fixed vertex keeps its state
 * bit for bit; its edges still constrain the other vertices.
 * Errors: GPO_ERR_ARG, GPO_ERR_STATE (after the first optimize). */
gpo_status gpo_set_fixed(gpo_graph* g, int64_t vertex_id, int32_t fixed);

/* Enables or disables an edge (Listing 5: set_active).  A disabled edge contributes
 * neither cost nor rows.  Errors: GPO_ERR_ARG, GPO_ERR_STATE (after the first optimize). */
gpo_status gpo_set_edge_active(gpo_graph* g, int64_t edge_id, int32_t active);

/* Sets the states of vertices first_id .. first_id + n - 1, which must all be of
 * one kind, from `state` (n rows of the kind's state size, FP64).  on_device = 1:
 * `state` is a device pointer; a pinned host pointer is read in place by the device.
 * Allowed before and between optimize calls.  After the first optimize, rows whose
 * values are bit for bit the ones the graph holds leave it as it was (see
 * gpo_optimize).  Errors: GPO_ERR_ARG, GPO_ERR_CUDA. */
gpo_status gpo_set_initial(gpo_graph* g, int64_t first_id, int64_t n, const double* state,
                           int32_t on_device);

/* Runs max_iters Levenberg-Marquardt iterations (Listing 5: levenberg_marquardt).
 * The first call freezes the topology (sorts edges point-major, plans and
 * allocates device memory).  params NULL = defaults; out (optional) receives the
 * report.  Every call starts from params->initial_damping and params->initial_nu and
 * evaluates F at the current state; passing the previous report's final_lambda and
 * final_nu continues the previous call's LM run step for step.  When no call has
 * changed the graph or its state since the previous gpo_optimize (with the same
 * solver), that run's cost is taken as F, and if its last step was rejected its
 * linearisation is kept: the values a fresh evaluation gives, without the kernels.
 * Errors: GPO_ERR_ARG, GPO_ERR_OOM, GPO_ERR_NUMERIC (non-finite initial cost),
 *         GPO_ERR_UNSUPPORTED (a point seen more than the supported maximum of
 *         times), GPO_ERR_CUDA. */
gpo_status gpo_optimize(gpo_graph* g, int32_t max_iters, const gpo_lm_params* params,
                        gpo_report* out);

/* F(x) = 1/2 sum_e rho(s_e) at the current state, FP64 (Eq. 1, Eq. 7). */
gpo_status gpo_get_cost(gpo_graph* g, double* cost);

/* Copies the states of vertices first_id .. first_id + n - 1 (one kind) to `out`. */
gpo_status gpo_get_state(gpo_graph* g, int64_t first_id, int64_t n, double* out,
                         int32_t on_device);

/* Copies up to `cap` per-iteration records of the last optimize; *n_out receives
 * the number written. */
gpo_status gpo_get_history(gpo_graph* g, gpo_iter_record* out, int32_t cap, int32_t* n_out);

/* Device bytes held by the graph (planned arena plus state buffers). */
gpo_status gpo_memory_footprint(gpo_graph* g, size_t* bytes);

/* Sizes of a finalized graph (gpo_graph_info). */
typedef struct {
  int64_t cameras;            /* camera or navigation-state vertices */
  int64_t points;
  int64_t edges;              /* active observation edges */
  int64_t extra_edges;        /* active inertial / bias edges */
  int64_t chunks;             /* CTA chunks of the per-edge kernels */
  int64_t slots;              /* (chunk, camera) pairs: rows of the camera-side partials */
  int32_t chunk_edges;        /* edges per chunk in effect */
  int32_t spmv_variant;       /* as requested in gpo_graph_desc */
  int32_t spmv_kernel;        /* the Schur-product kernel the PCG runs, in spmv_variant's
                                 numbering (1 staged, 2 classic, 3 pipelined, 4 dynamic,
                                 5 warp groups; 0: no observation edges) */
  int32_t reserved0;
  int64_t j_bytes;            /* device bytes of the stored Jacobian rows (0 with dynamic
                                 Jacobians, which store none) */
} gpo_graph_info_t;

/* Fills *out for a graph that has been optimized (or otherwise finalized).
 * Errors: GPO_ERR_ARG, GPO_ERR_STATE (not finalized). */
gpo_status gpo_graph_info(gpo_graph* g, gpo_graph_info_t* out);

/* Plans the graph on the host -- sorted topology, chunks, slots and the device memory
 * plan -- without touching the device, and returns the bytes its device image will
 * take.  Optional: gpo_optimize and gpo_server_submit plan when needed and reuse a plan
 * made here (until the next add / set call on the graph).  Needs no GPU and may run
 * concurrently for different graphs (e.g. on worker threads that build requests for a
 * server).  Errors: GPO_ERR_ARG, GPO_ERR_STATE (missing stereo rig),
 * GPO_ERR_UNSUPPORTED, GPO_ERR_OOM (host). */
gpo_status gpo_graph_plan(gpo_graph* g, size_t* bytes);

/* Per-kernel statistics of the kernels the library launches (gpo_get_profile). */
typedef struct {
  char name[32];              /* kernel class, e.g. "spmv" (the PCG Schur product) */
  int64_t launches;           /* kernels launched since gpo_set_profiling (always counted) */
  int64_t timed_launches;     /* launches bracketed by CUDA events (profiling on) */
  int64_t active_launches;    /* timed launches that did work: a Schur-product launch after
                                 its PCG solve stopped returns at once, and so does the
                                 linearisation after a rejected LM step; neither is active */
  double total_ms;            /* summed event time of the timed launches */
  double active_ms;           /* summed event time of the active launches */
} gpo_kernel_profile;

/* Resets the counters; enable = 1 also records a pair of CUDA events around every
 * kernel launch on the graph's stream (timings for gpo_get_profile).  Waits for the
 * stream.  Errors: GPO_ERR_ARG, GPO_ERR_CUDA. */
gpo_status gpo_set_profiling(gpo_graph* g, int32_t enable);

/* Writes up to `cap` per-kernel-class records (waits for the stream first);
 * *n_out receives the number written. */
gpo_status gpo_get_profile(gpo_graph* g, gpo_kernel_profile* out, int32_t cap, int32_t* n_out);

/* Message of the last failed call on g (g may be NULL for creation errors).
 * The pointer stays valid until the next call on g. */
const char* gpo_last_error(const gpo_graph* g);

/* Library version string, e.g. "gpo 0.1 sm_103a". */
const char* gpo_version(void);

/* ---------------------------------------------------------------------------
 * Batched solves and serving.  Many small independent problems (e.g. the local
 * bundle-adjustment windows of a SLAM back end) share every kernel launch: each
 * launch covers the chunks and camera blocks of all graphs in the set, and each graph
 * keeps its own LM and PCG state, so its result is the same as when it is solved
 * alone with gpo_optimize (bit for bit: the reductions of a graph never mix with
 * another graph's).  The paper has no batched mode; this is the library's extension.
 * ------------------------------------------------------------------------ */

/* Solves n graphs together for max_iters LM iterations.  The graphs must share
 * precision and device and be distinct; they are finalized if needed and keep their
 * device state (as after gpo_optimize).  Work runs on graphs[0]'s stream; reports
 * (optional) receives n reports in graph order.  Errors as gpo_optimize; on error
 * the message is on graphs[0]. */
gpo_status gpo_optimize_batch(gpo_graph* const* graphs, int32_t n, int32_t max_iters,
                              const gpo_lm_params* params, gpo_report* reports);

typedef struct gpo_server gpo_server;

typedef struct {
  int32_t precision;          /* of every graph it serves */
  int32_t device;
  void* cuda_stream;          /* NULL = the server creates one */
  size_t memory_budget;       /* device bytes of resident graphs; 0 = unlimited */
  int32_t max_resident;       /* slots: graphs solved concurrently (default 1024) */
  int32_t reserved0;
} gpo_server_desc;

/* Serving loop (continuous batching).  Requests are queued by gpo_server_submit;
 * each gpo_server_step admits queued graphs in arrival order while a slot is free
 * and their planned device memory fits the budget, runs ONE LM iteration for every
 * resident graph in shared launches, and retires graphs that have run their
 * iterations: their final state is copied back into the graph (host side; read it
 * with gpo_get_state) and their device memory is released.  A graph is owned by the
 * server from submit until its ticket is reported done; the caller destroys it. */
gpo_status gpo_server_desc_default(gpo_server_desc* out);
gpo_status gpo_server_create(const gpo_server_desc* desc, gpo_server** out);
gpo_status gpo_server_destroy(gpo_server* sv);
/* Queues g (not yet optimized) for max_iters iterations; *ticket identifies it.
 * Errors: GPO_ERR_ARG (precision or device mismatch), GPO_ERR_STATE (g already on the
 * device), GPO_ERR_OOM (g alone exceeds the budget), GPO_ERR_UNSUPPORTED. */
gpo_status gpo_server_submit(gpo_server* sv, gpo_graph* g, int32_t max_iters,
                             const gpo_lm_params* params, int64_t* ticket);
/* Admission, one LM iteration of the resident graphs, retirement.  Outputs (optional):
 * graphs resident after the step, still queued, and retired by this step. */
gpo_status gpo_server_step(gpo_server* sv, int32_t* n_resident, int32_t* n_queued,
                           int32_t* n_finished);
/* *done = 1 and the report once the ticket's graph has been retired (each ticket is
 * reported once). */
gpo_status gpo_server_poll(gpo_server* sv, int64_t ticket, int32_t* done, gpo_report* report);
/* Device bytes held by resident graphs. */
gpo_status gpo_server_memory(gpo_server* sv, size_t* used_bytes);
const char* gpo_server_last_error(const gpo_server* sv);

/* ---------------------------------------------------------------------------
 * Cost evaluation without device allocation.  The paper has no counterpart; this is
 * for callers that cannot allocate device memory where they need a cost (a fully
 * handed-out memory pool, a real-time or callback thread that must not enter the
 * CUDA allocator, device memory owned by another framework).
 *
 * F = 1/2 sum_e rho(|r_e|^2) of a BA problem with identity information, every buffer
 * caller-owned device memory of `device`: cams [C][9] and points [P][3] (FP64 states in
 * the layouts of GPO_V_BA_CAMERA9 / GPO_V_POINT3), cam_idx / pt_idx [n_edges] int32,
 * obs [n_edges][2] pixels; huber_delta > 0 selects the Huber loss, <= 0 plain squares.
 * *cost_out (a device double) receives F when the work queued on cuda_stream (NULL =
 * the legacy default stream) completes; the call does not wait for it.
 * No device memory is allocated: the reduction's scratch is a static device array of
 * 64 KB held by every GPU that loads the library until the process exits, which
 * bounds n_edges to 2,097,152 (larger gives GPO_ERR_ARG).  The first call on a device
 * looks up that array's address (make it before any stream capture).  All calls on a
 * device share the array and its last contents; the call clears the part that must
 * start at zero, but calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller.
 * Errors: GPO_ERR_ARG (null buffer, bad device, n_edges out of range), GPO_ERR_CUDA. */
gpo_status gpo_ba_cost_noalloc(int32_t device, void* cuda_stream, const double* cams,
                               const double* points, const int32_t* cam_idx,
                               const int32_t* pt_idx, const double* obs, int64_t n_edges,
                               double huber_delta, double* cost_out);

/* ---------------------------------------------------------------------------
 * Generic edge kinds (Sec. III: a constraint is declared by its residual over its
 * vertices; the library differentiates it in forward mode).  Kinds are compiled into
 * the library; a generic graph has n vertices of one dimension (2 for the kinds below)
 * and is solved by LM with block-Jacobi PCG on the full damped system, in FP64 (the
 * damping, PCG and Huber options of gpo_lm_params apply).  The circle kind is the
 * paper's running example: points pulled onto a circle.
 * ------------------------------------------------------------------------ */
enum {
  GPO_GE_CIRCLE = 0,    /* arity 1, meas [R]: r = x^2 + y^2 - R^2 */
  GPO_GE_DISTANCE = 1   /* arity 2, meas [d]: r = |x_i - x_j|^2 - d^2 */
};
typedef struct gpo_generic gpo_generic;
/* x0: n_vertices * vertex_dim doubles (copied).  cuda_stream NULL: an own stream.
 * Errors: GPO_ERR_ARG (vertex_dim != 2, n_vertices out of range, bad device),
 * GPO_ERR_OOM, GPO_ERR_CUDA. */
gpo_status gpo_generic_create(int32_t vertex_dim, int64_t n_vertices, const double* x0, int32_t device,
                              void* cuda_stream, gpo_generic** out);
gpo_status gpo_generic_destroy(gpo_generic* g);
/* n edges of a registered kind: vertex_ids n * arity, meas n * (kind's length);
 * loss as in gpo_add_edges.  Edge ids continue across calls. */
gpo_status gpo_generic_add_edges(gpo_generic* g, int32_t kind, int64_t n, const int64_t* vertex_ids,
                                 const double* meas, int32_t loss_kind, double loss_delta, int64_t* first_id);
gpo_status gpo_generic_set_fixed(gpo_generic* g, int64_t vertex_id, int32_t fixed);
gpo_status gpo_generic_set_edge_active(gpo_generic* g, int64_t edge_id, int32_t active);
/* max_iters LM iterations (Nielsen damping, gain ratio in FP64); the states are kept
 * between calls.  Errors: GPO_ERR_ARG, GPO_ERR_OOM, GPO_ERR_CUDA. */
gpo_status gpo_generic_optimize(gpo_generic* g, int32_t max_iters, const gpo_lm_params* params, gpo_report* out);
/* out: n_vertices * vertex_dim doubles. */
gpo_status gpo_generic_get_state(gpo_generic* g, double* out);

/* ---------------------------------------------------------------------------
 * FP64 throughput probe (measurement).  The linearisation and cost kernels evaluate
 * the geometry, residuals and cost in FP64 (the state, retraction and cost are FP64 in
 * every precision mode), so their roofline is the FP64 pipe, whose rate this measures.
 *
 * Launches n_ctas CTAs of 256 threads on cuda_stream (NULL = the legacy default
 * stream); every thread runs iters x 32 FP64 fused multiply-adds in eight independent
 * chains and writes one double to out[thread] (out: caller-owned device memory of
 * n_ctas * 256 doubles).  One launch performs n_ctas * 256 * iters * 32 FMAs, i.e.
 * twice that many FP64 flops; the caller times it on the stream.  The call does not
 * wait.  Errors: GPO_ERR_ARG (n_ctas or iters <= 0, out NULL), GPO_ERR_CUDA. */
gpo_status gpo_fp64_fma_probe(void* cuda_stream, int32_t n_ctas, int32_t iters, double* out);

/* ---------------------------------------------------------------------------
 * Diagnostic entry points (used by the parity tests; same kernels as optimize).
 * ------------------------------------------------------------------------ */

/* Linearises every edge at the current state in the graph's precision.
 * Layout per edge id, (R, K) = (2, 12) for graphs of BA cameras, (9, 30) for graphs of
 * navigation states:
 * r_out: n_edges * R doubles: the whitened residual (observation edges:
 *        Huber-weighted, sqrt(rho') U r), rows beyond the edge's m are zero;
 * J_out: n_edges * R * K doubles, row-major per residual row, with the same
 *        weighting: observation edges have the camera block in columns [0, DB)
 *        (DB = 9 or 15; a stereo edge fills the first 6, the pose) and the point in
 *        [DB, DB + 3); camera-side edges have keyframe i in [0, 15) and j in [15, 30).
 *        Observation-edge values are as stored (rounded to the storage precision);
 *        camera-side edges are FP64.  Disabled edges are written as zeros.
 * Either pointer may be NULL. */
gpo_status gpo_debug_linearize(gpo_graph* g, double* r_out, double* J_out);

/* The same for the n edges edge_ids[0..n) only: row k of r_out / J_out belongs to
 * edge_ids[k] (for sampled checks of large graphs).  Errors: GPO_ERR_ARG (unknown id). */
gpo_status gpo_debug_linearize_edges(gpo_graph* g, const int64_t* edge_ids, int64_t n, double* r_out,
                                     double* J_out);

/* Forward-mode automatic differentiation of the observation edges (Sec. IV-D: the
 * paper's edges are differentiated by a forward-mode generator, with analytic
 * Jacobians beside it): every edge's residual is evaluated on dual numbers at the
 * current state in FP64, with the whitening, Huber IRLS weight and fixed-vertex zero
 * columns of the analytic path, and returned in gpo_debug_linearize_edges' layout
 * (edge_ids[k] -> row k; camera-side edges give zero rows).  Unlike
 * gpo_debug_linearize_edges the rows are FP64 in every precision.  A checker of the
 * analytic Jacobians and the prototyping path for new edge kinds; with profiling on its
 * kernel is timed as "autodiff".  Errors: GPO_ERR_ARG (unknown id), GPO_ERR_CUDA. */
gpo_status gpo_debug_autodiff_edges(gpo_graph* g, const int64_t* edge_ids, int64_t n, double* r_out,
                                    double* J_out);

/* Solves one damped system (H + lambda D^T D) dx = -b at the current state with
 * the full path (Schur, PCG, back-substitution) and given PCG options, without
 * changing the state.  dx_out: one row per vertex in id order, each of the
 * vertex's tangent size (fixed vertices give zeros).  pcg_iters (optional). */
gpo_status gpo_debug_step(gpo_graph* g, double lambda, const gpo_lm_params* params,
                          double* dx_out, int32_t* pcg_iters);

/* Camera Schur blocks at damping lambda: S_out[C][DB][DB] the diagonal blocks
 * S_cc = H_cc + lambda D_c - sum_p W H_pp^-1 W^T, g_out[C][DB] the reduced right-hand
 * side -b_c + sum_p W H_pp^-1 b_p, cameras in id order (DB = 9 for BA cameras, 15 for
 * navigation states; H_cc includes the camera-side edges).  Either may be NULL. */
gpo_status gpo_debug_schur(gpo_graph* g, double lambda, const gpo_lm_params* params,
                           double* S_out, double* g_out);

/* Failure-detection test of the bounded device waits: prepares one PCG solve and
 * launches the fused camera kernel (camera half of the Schur product and PCG update)
 * with its grid barrier waiting for one CTA more than the grid, so that nothing can
 * complete it.  The barrier's bounded wait (1 s) gives up, the kernel raises the
 * error flag and returns.  Returns GPO_ERR_TIMEOUT when that happened (the expected
 * result), GPO_ERR_UNSUPPORTED when the graph's camera blocks do not fit one resident
 * wave (the fused kernel is then not used), GPO_ERR_STATE otherwise.  The graph's
 * device counters are left clean and the context usable: a later gpo_optimize runs
 * as if this call had not been made. */
gpo_status gpo_debug_wait_timeout(gpo_graph* g);

#ifdef __cplusplus
}
#endif
#endif /* GPO_H */
