/*
 * dba.h -- C ABI of a GB300 (sm_103a) implementation of distributed bundle
 * adjustment by consensus ADMM (Ramamurthy, Lin, Aravkin, Pankanti, Viguier,
 * "Distributed Bundle Adjustment", arXiv 1708.07954).
 *
 * Problem (Sec. 2.1-2.2 of the paper): m cameras y_j = (alpha, beta, gamma,
 * tx, ty, tz) with R = Rz(gamma) Ry(beta) Rx(alpha), n points x_i in R^3,
 * observations z_ij (pixels) for the pairs (i, j) listed by the caller.  The
 * pixel model is z = f (R x + t)_{1,2} / (R x + t)_3 + (cx, cy) (Eq. 1 with the
 * focal matrix K applied and a known principal point).
 *
 * Method (Sec. 3.1): every observation o = (i, j) owns a private copy of its
 * point and camera (9 unknowns) and the duals r_o (3), s_o (6).  One ADMM
 * iteration is
 *   (9)       local solve of every observation's robust subproblem,
 *   (10),(11) consensus means of the copies plus scaled duals per point/camera,
 *   (12),(13) dual ascent with the new consensus.
 * Equation numbers follow the order of the paper's LaTeX source.
 *
 * Conventions for every entry point:
 *   - host pointers are caller-owned and only read (inputs) or written
 *     (outputs) during the call; the library owns all device memory;
 *   - observations are accepted and returned in caller order;
 *   - arrays are row-major, float64, C-contiguous: cams [m][6], pts [n][3],
 *     z [l][2], copies/duals [l][9] = (point part 3, camera part 6);
 *   - every call returns a dba_status and never aborts; dba_last_error() gives
 *     the message of the last failure on that context;
 *   - a context is not thread-safe; separate contexts are independent.
 */
#ifndef DBA_H
#define DBA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dba_ctx dba_ctx;

typedef enum {
  DBA_OK = 0,
  DBA_EINVAL = -1,   /* bad argument: index out of range, n <= 0, non-finite input, bad config */
  DBA_ENOMEM = -2,   /* device or host allocation failed */
  DBA_ECUDA = -3,    /* a CUDA call failed (message in dba_last_error) */
  DBA_ESTATE = -4,   /* call out of order, e.g. dba_iterate before dba_set_observations */
  DBA_ENUMERIC = -5, /* a local solve produced a non-finite value */
  DBA_ETIMEOUT = -6  /* a bounded device-side wait gave up */
} dba_status;

typedef enum {
  DBA_LOSS_L2 = 0,        /* phi_m(e) = |e|^2, Eq. (2) */
  DBA_LOSS_HUBER = 1,     /* |e|^2 if |e| <= delta else 2 delta |e| - delta^2 (Sec. 3.1) */
  DBA_LOSS_STUDENT_T = 2  /* nu log(1 + |e|^2 / nu) (robust loss cited in Sec. 1) */
} dba_loss;

typedef enum {
  DBA_PREC_F64 = 0,       /* local solves, consensus and duals in FP64 */
  DBA_PREC_F32_LOCAL = 1  /* local solves in FP32; consensus, duals, objective in FP64 */
} dba_precision;

typedef struct {
  double focal, cx, cy;   /* pinhole intrinsics (pixels), shared by all cameras */
  int loss;               /* dba_loss */
  double loss_param;      /* Huber delta (pixels) or Student's t nu */
  double rho_x, rho_y;    /* consensus penalties of Eq. (8), > 0: points; camera translations */
  double rho_angle;       /* penalty of the camera Euler angles; <= 0: rho_y (the paper's single
                             camera penalty).  Angles are radians and translations lengths, so
                             their data curvatures differ by ~depth^2 */
  int inner_steps;        /* damped Gauss-Newton steps per local solve, >= 0 */
  double lm_lambda0;      /* first damping = lm_lambda0 * mean(diag H) */
  double lm_lambda_min;   /* lower clamp of the damping after an accepted step */
  double eps_depth;       /* a copy with depth (R x + t)_3 <= eps_depth is rejected */
  double lm_model_tol;    /* kappa >= 0: a local step whose predicted decrease is below
                             kappa u (|L| + 2 w |e| (|z_1| + |z_2|)), the rounding noise of the
                             local objective L in the working precision (u = 2^-24 or 2^-53),
                             is accepted without comparing objective values; 0 = always
                             compare */
  int precision;          /* dba_precision */
  int tile_obs;           /* observations per tile and thread block: 64, 128 or 256; 0 = by
                             precision (256 FP32-local, 128 FP64); -1 = autotune: time each
                             size on the problem at dba_set_observations and keep the fastest
                             (cached per process by precision, size and mean track length) */
  int use_graph;          /* 1: replay each iteration as a CUDA graph; 0: plain launches */
  void* cuda_stream;      /* cudaStream_t to launch on; NULL = a stream owned by the context */
  int local_solver;       /* dba_local_solver: how each local subproblem (Eq. 9) is solved */
  int finalize_threads;   /* threads per block of the segmented reduction that completes
                             Eqs. (10)-(11) over the per-tile partial sums (one block per
                             camera and per track spanning several tiles): 32, 64, 128 or
                             256; 0 = 128, or with tile_obs = -1 timed together with the
                             tile size and the fastest pair kept */
} dba_config;

typedef enum {
  DBA_SOLVER_GN = 0,      /* inner_steps damped Gauss-Newton steps (the paper's choice for l2) */
  DBA_SOLVER_LBFGS = 1    /* inner_steps L-BFGS iterations (the paper's choice for Huber, Sec. 3.1):
                             coordinates scaled by sqrt(rho), memory 4, two-loop recursion with
                             H0 = (s.y / y.y) I, backtracking Armijo line search (c1 = 1e-4, at
                             most 10 halvings) from step 1, the same rounding-noise acceptance */
} dba_local_solver;

typedef struct {
  long long iters_done;   /* ADMM iterations run on this context since the state was set */
  double rmse_obs;        /* sqrt(mean |z - f(x_i, y_j)|^2) at consensus, valid observations */
  double rmse_gt;         /* sqrt(mean over inliers |f(x_i, y_j) - f(x*_i, y*_j)|^2); 0 without ground truth */
  double objective;       /* sum of phi_m(z - f(x_i, y_j)) at consensus: Eq. (2) with phi_m */
  double primal_res;      /* sqrt(sum over copies |copy - consensus|^2) */
  double dual_res;        /* sqrt(sum over copies rho^2 |consensus - previous consensus|^2) */
  long long n_invalid;    /* observations with consensus depth <= eps_depth (excluded above) */
  double seconds;         /* device time of the dba_iterate call (CUDA events) */
} dba_stats;

/* Fills *cfg with defaults: focal 500, principal point (320, 240), Huber 2 px,
 * rho 1 (angles: rho_y), 5 inner steps, lambda0 1e-3, lambda_min 1e-12, eps_depth 1e-6,
 * lm_model_tol 16,
 * FP32 local solves, automatic tile size, graphs on, own stream, Gauss-Newton local solver,
 * finalize_threads 0. */
void dba_config_default(dba_config* cfg);

/* Creates a context on the current CUDA device for one problem of Sec. 2.2 solved by
 * the consensus ADMM of Sec. 3.1: *cfg carries the known intrinsics of Eq. (1), the
 * misfit phi_m of Eq. (2), the penalties rho of the augmented Lagrangian, Eq. (8), and
 * how each local subproblem, Eq. (9), is solved.  *cfg is copied; *out receives the
 * context (owned by the caller, freed by dba_destroy).  EINVAL for a null argument or an
 * invalid configuration, ECUDA when no CUDA device is usable, ENOMEM when host memory
 * runs out; the message is in dba_last_error(NULL).  No device memory is allocated
 * until dba_set_observations. */
dba_status dba_create(const dba_config* cfg, dba_ctx** out);

/* Loads one problem (Sec. 2.2: unknowns 6m + 3n, one observation per listed
 * pair).  pt_idx/cam_idx [n_obs] index pts0/cams0; z [n_obs][2] pixels;
 * cams0 [n_cams][6], pts0 [n_pts][3] the initial estimate.  Copies start at
 * the initial estimate and duals at zero (the paper does not state an
 * initialisation).  A camera or point with no observation keeps its value.
 * EINVAL on an index out of range, n_obs <= 0, n_cams/n_pts <= 0 or a
 * non-finite value.  Replaces any previous problem of this context. */
dba_status dba_set_observations(dba_ctx* ctx, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                                const int32_t* pt_idx, const int32_t* cam_idx, const double* z,
                                const double* cams0, const double* pts0);

/* Optional: ground-truth cameras [n_cams][6] and points [n_pts][3]; enables
 * dba_stats.rmse_gt, the RMS distance between the consensus projections and
 * the noise-free projections of the ground truth.  inlier [n_obs] (caller
 * order, nullable = all) selects the observations it averages over: pass 0 for
 * observations whose pixel is an outlier rather than a noisy measurement. */
dba_status dba_set_ground_truth(dba_ctx* ctx, const double* cams_gt, const double* pts_gt,
                                const uint8_t* inlier);

/* Declares that the loaded problem is a batch of n_scenes independent scenes:
 * observations [obs_off[s], obs_off[s+1]) (caller order) use only cameras
 * [cam_off[s], cam_off[s+1]) and points [pt_off[s], pt_off[s+1]).  The offsets
 * are nondecreasing, start at 0 and end at n_obs, n_cams, n_pts.  The scenes are
 * solved together, one tile kernel launch per iteration, with no coupling
 * (each consensus segment lies inside one scene); this call only enables
 * dba_scene_stats.  EINVAL if an observation leaves its scene. */
dba_status dba_set_scenes(dba_ctx* ctx, int32_t n_scenes, const int64_t* obs_off, const int32_t* cam_off,
                          const int32_t* pt_off);

/* Per-scene metrics at the current consensus after dba_set_scenes: rmse_obs,
 * rmse_gt (0 without ground truth) and the objective, each [n_scenes]; any
 * pointer may be NULL. */
dba_status dba_scene_stats(dba_ctx* ctx, double* rmse_obs, double* rmse_gt, double* objective);

/* Runs n_iters >= 0 ADMM iterations, Eqs. (9)-(13), on the context's stream
 * and waits for them.  stats (nullable) receives the metrics at the final
 * consensus.  ESTATE before dba_set_observations, ENUMERIC if a local solve
 * produced a non-finite value (the state is then unspecified). */
dba_status dba_iterate(dba_ctx* ctx, int n_iters, dba_stats* stats);

/* Runs up to max_iters iterations and stops after the first iteration whose
 * consensus has rmse_gt <= target_rmse_gt (needs ground truth; ESTATE
 * otherwise).  Metrics are evaluated after every iteration; stats receives
 * those of the last one. */
dba_status dba_iterate_until(dba_ctx* ctx, int max_iters, double target_rmse_gt, dba_stats* stats);

/* Metrics of the current state without iterating. */
dba_status dba_evaluate(dba_ctx* ctx, dba_stats* stats);

/* Copies the consensus estimate, the point and camera means of Eqs. (10)-(11) after
 * the last iteration (Sec. 3.1), to cams [n_cams][6] and pts [n_pts][3] (caller-owned
 * host arrays; a camera or point without observations keeps its input value).
 * EINVAL for a null pointer, ESTATE before dba_set_observations. */
dba_status dba_get_params(dba_ctx* ctx, double* cams, double* pts);

/* Copies the ADMM state of Sec. 3.1 after the last iteration: every observation's
 * private copy (x_o, y_o) of Eq. (9) to copies [n_obs][9] and its duals (r_o, s_o)
 * after Eqs. (12)-(13) to duals [n_obs][9], caller order, caller-owned host arrays.
 * Either pointer may be NULL.  ESTATE before dba_set_observations. */
dba_status dba_get_state(dba_ctx* ctx, double* copies, double* duals);

/* Replaces the whole ADMM state of Sec. 3.1 (checkpoint resume): the copies of
 * Eq. (9) and duals of Eqs. (12)-(13) [n_obs][9] in caller order, the consensus of
 * Eqs. (10)-(11) cams [n_cams][6] and pts [n_pts][3] (host arrays, only read), and the
 * iteration counter k >= 0 that dba_stats.iters_done continues from.  The next
 * iteration forms the consensus sums in full, so any duals are accepted (after an
 * iteration of the method they sum to zero per point and camera).  EINVAL for a null
 * array, a non-finite value or k < 0; ESTATE before dba_set_observations.  Clears the
 * device error flags. */
dba_status dba_set_state(dba_ctx* ctx, const double* copies, const double* duals,
                         const double* cams, const double* pts, int64_t k);

/* Device time per kernel, averaged over the launches of the last dba_profile
 * call: names[i] (static strings) and ms[i] for i < *count (in: capacity). */
dba_status dba_profile(dba_ctx* ctx, int n_iters, const char** names, double* ms, int* count);

/* The internal observation order and tile table that dba_set_observations builds
 * for these indices and tile size (64, 128 or 256), computed on the host only (no
 * device), for inspection and tests.  Outputs, caller-allocated, any may be NULL:
 *   perm[n_obs]        caller index of the observation at each internal position;
 *   point[n_obs]       internal point id at each position (points ordered by their
 *                      smallest observing camera, then caller index; each point's
 *                      observations contiguous and ordered by camera, then caller index);
 *   point_perm[n_pts]  caller id of each internal point (unobserved points last);
 *   cam_rank[n_obs]    the position's rank in its tile's camera order;
 *   tile_start[n_obs + 1]  first position of each tile, then n_obs after the last;
 *   *n_tiles           number of tiles (a track longer than tile_obs is cut into
 *                      tiles of its own; other tiles hold whole tracks).
 * EINVAL as dba_set_observations or for another tile size; message in
 * dba_last_error(NULL). */
dba_status dba_build_layout(int32_t n_cams, int32_t n_pts, int64_t n_obs, const int32_t* pt_idx,
                            const int32_t* cam_idx, int tile_obs, int64_t* perm, int32_t* point,
                            int32_t* point_perm, int32_t* cam_rank, int64_t* tile_start, int64_t* n_tiles);

/* Fault injection for tests of failure detection.  While `on` is nonzero, the
 * tile kernel announces each tile's tensor copies on its mbarrier without
 * issuing them, so the bounded wait for them (about two seconds) runs out:
 * the kernel sets an error bit and returns, and dba_iterate reports
 * DBA_ETIMEOUT.  The CUDA context stays usable; the iteration's state is not,
 * so restore one with dba_set_state (which also clears the error bit) before
 * iterating again.  EINVAL on a null context, ESTATE before
 * dba_set_observations. */
dba_status dba_inject_copy_stall(dba_ctx* ctx, int on);

/* Fault injection for tests of the ABI's exception guard (no counterpart in the paper).
 * The next n entry points called on this host thread fail as if their first host
 * allocation had thrown: each returns DBA_ENOMEM with "out of host memory" as its
 * message, touching none of its arguments.  n = 0 cancels; EINVAL for n < 0.  Every
 * entry point that returns a dba_status runs its whole body under the guard, so no C++
 * exception crosses this ABI. */
dba_status dba_inject_host_alloc_failure(int n);

/* Sizes of the internal observation layout after dba_set_observations, for
 * traffic models: out[0] tiles, out[1] observations per tile (block size),
 * out[2] point runs, out[3] camera runs (= camera partial slots), out[4]
 * points whose track spans several tiles, out[5] their partial slots, out[6]
 * threads per block of the partial-sum reduction (finalize_threads in use).
 * *count: in capacity, out entries written. */
dba_status dba_layout(dba_ctx* ctx, int64_t* out, int* count);

/* Allocation-free evaluation.  For callers that cannot let the library call cudaMalloc:
 * processes whose device memory belongs to another allocator (a framework's caching
 * allocator, a fixed pool reserved up front), loops replayed as CUDA graphs or with
 * real-time budgets where an allocation would stall or fail, and embedders that do not let
 * a library own device memory.  The paper has no counterpart; this is an interface of this
 * library only, and it uses no context.
 *
 * At the caller's cameras and points it computes, over all observations, out[0] = sum of
 * |z - f(x_i, y_j)|^2, out[1] = sum of phi_m (Eq. 2 with the configured misfit), out[2] = the
 * number of observations evaluated, out[3] = the number not evaluated (depth <= eps_depth, or
 * an index outside [0, n_pts) / [0, n_cams)).  FP64 throughout.
 * All arrays are DEVICE pointers the caller owns, laid out as elsewhere in this header:
 * pt_idx, cam_idx int32 [n_obs]; z float64 [n_obs][2]; cams [n_cams][6]; pts [n_pts][3];
 * out float64 [4], written only.  Uses cfg->focal, cx, cy, loss, loss_param, eps_depth.
 * Launches on `stream` (a cudaStream_t; NULL = the default stream) and returns without
 * waiting: out is complete when the stream reaches that point.
 * Limit: 0 <= n_obs <= DBA_NOALLOC_MAX_OBS; larger sizes return DBA_EINVAL.
 * Scratch: one file-scope device array of 4096 x 4 doubles (128 KiB), which every GPU that
 * loads this library holds until the process exits.  All calls share it and each call
 * overwrites what it reads, so nothing needs clearing, but calls whose kernels may overlap
 * on the GPU (other streams, other host threads on the same device) race: serialise them.
 * The first call on each device looks up the array's device address with that device
 * current; make that first call before capturing a stream into a graph.
 * Errors: DBA_EINVAL for null pointers, bad sizes or configuration, DBA_ECUDA for a launch
 * failure; the message is in dba_last_error(NULL). */
#define DBA_NOALLOC_MAX_OBS 16777216
dba_status dba_evaluate_noalloc(const dba_config* cfg, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                                const int32_t* pt_idx, const int32_t* cam_idx, const double* z,
                                const double* cams, const double* pts, double* out, void* stream);

/* ---- Learned warm start (no counterpart in the paper) ------------------------------------
 * A small network (32-64-64-64-16, GELU) predicts, for every observation, a start for its
 * local solve (Eq. 9) from the residual, Jacobian, offset and dual at the plain start, all in
 * coordinates scaled by sqrt(rho).  Inference runs on BF16 tensor cores (tcgen05, FP32
 * accumulation) before each iteration's local solves; each local solve starts from the
 * learned candidate only if that lowers Eq. (9), and the Levenberg-Marquardt solve
 * refines whichever start it keeps.  The network is trained on the GPU by this library's own FP32
 * forward/backward/Adam kernels on targets harvested from long local solves.  The dba_mlp_*
 * calls run on a stream of the network that is ordered after work queued on the legacy
 * default stream and return when done; buffers filled on other streams must be complete. */
typedef struct dba_mlp dba_mlp;
#define DBA_MLP_N_PARAMS 11552  /* W1 64x32, b1, W2 64x64, b2, W3 64x64, b3, W4 16x64, b4, input
                                   mean[32], input std[32], target scale[16] (FP32, row-major) */
#define DBA_MLP_N_FEATURES 32
#define DBA_MLP_N_TARGETS 16

/* New network with He-normal weights from `seed`; identity normaliser. */
dba_status dba_mlp_create(uint64_t seed, dba_mlp** out);
void dba_mlp_destroy(dba_mlp* mlp);
const char* dba_mlp_last_error(const dba_mlp* mlp);
/* Host copies of the parameters [DBA_MLP_N_PARAMS]. */
dba_status dba_mlp_get_params(const dba_mlp* mlp, float* params);
dba_status dba_mlp_set_params(dba_mlp* mlp, const float* params);
/* Features [cap][32] and targets [cap][16] (DEVICE buffers owned by the caller) of the local
 * problems of observations 0, stride, 2 stride, ... of ctx's current state (internal order),
 * the targets from target_steps damped Gauss-Newton steps.  The state is only read. */
dba_status dba_mlp_harvest(dba_ctx* ctx, int64_t stride, int target_steps, float* feats, float* targets,
                           int64_t cap, int64_t* n_out);
/* Input mean/std and target scale from n harvested rows (device buffers). */
dba_status dba_mlp_fit_normalizer(dba_mlp* mlp, const float* feats, const float* targets, int64_t n);
/* Mean squared error over the 9 used outputs of n rows and its gradient (host
 * [DBA_MLP_N_PARAMS], normaliser entries 0). */
dba_status dba_mlp_loss_grad(dba_mlp* mlp, const float* feats, const float* targets, int64_t n, double* loss,
                             float* grad);
/* Adam (beta 0.9/0.999) over `epochs` shuffled passes of minibatches; last epoch's mean loss. */
dba_status dba_mlp_train(dba_mlp* mlp, const float* feats, const float* targets, int64_t n, int epochs,
                         int batch, float lr, uint64_t seed, double* last_loss);
/* Tensor-core inference on n feature rows (device) -> out [n][16] (device), in target-scale units. */
dba_status dba_mlp_predict(dba_mlp* mlp, const float* feats, int64_t n, float* out);
/* Uses (a copy of) the network to warm-start ctx's local solves; NULL disables. */
dba_status dba_set_warm_start(dba_ctx* ctx, const dba_mlp* mlp);

/* Message of the last failed call on ctx (or of the last failed dba_create
 * when ctx is NULL).  Never NULL. */
const char* dba_last_error(const dba_ctx* ctx);

/* Frees the context and its device memory.  NULL is ignored. */
void dba_destroy(dba_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Block subproblems: the generalized update step (Sec. 3.1.4, Eq. 14).
 *
 * Instead of one observation, each update solves a block of up to
 * block_points points and block_cams cameras together with all observations
 * between them, over one copy of each of its points and cameras; consensus
 * (Eqs. 10-11) averages copy + dual / rho over a point's (camera's) copies and
 * the dual ascent (Eqs. 12-13) runs per copy.  Blocks: points ranked by
 * (smallest observing camera index, point index) and cut into groups of
 * block_points consecutive ranks; cameras cut into groups of block_cams
 * consecutive indices; one block per (point group, camera group) pair that
 * holds observations.  block_points = block_cams = 1 is the per-observation
 * method of dba_iterate.  Each block's subproblem takes inner_steps damped
 * Gauss-Newton steps with the damping, acceptance and noise rules of the
 * per-observation solve (points eliminated, the reduced camera system
 * factorised).  The context owns its device memory; inputs are host arrays in
 * caller order, copied in.  Not thread-safe per context.
 * ------------------------------------------------------------------------- */
typedef struct dba_block_ctx dba_block_ctx;
#define DBA_BLOCK_MAX_POINTS 64
#define DBA_BLOCK_MAX_CAMERAS 4

/* Validates cfg as dba_create does (tile_obs, use_graph are ignored; local_solver
 * must be DBA_SOLVER_GN) and 1 <= block_points <= 64, 1 <= block_cams <= 4 (EINVAL). */
dba_status dba_block_create(const dba_config* cfg, int block_points, int block_cams, dba_block_ctx** out);
/* Same arrays and checks as dba_set_observations, and a (point, camera) pair
 * may appear once (EINVAL); builds the blocks and starts with copies at the
 * initial estimate and zero duals. */
dba_status dba_block_set_observations(dba_block_ctx* ctx, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                                      const int32_t* pt_idx, const int32_t* cam_idx, const double* z,
                                      const double* cams0, const double* pts0);
/* Reference pixels z_ref [n_obs][2] (e.g. noise-free projections) for rmse_gt,
 * over observations with inlier[o] != 0 (inlier NULL: all). */
dba_status dba_block_set_reference_pixels(dba_block_ctx* ctx, const double* z_ref, const uint8_t* inlier);
/* n_iters iterations; stats (nullable) as dba_iterate, residuals over copies. */
dba_status dba_block_iterate(dba_block_ctx* ctx, int n_iters, dba_stats* stats);
/* Iterates until rmse_gt <= target (metrics after every iteration, included in
 * stats->seconds) or max_iters; needs reference pixels (ESTATE). */
dba_status dba_block_iterate_until(dba_block_ctx* ctx, int max_iters, double target_rmse_gt, dba_stats* stats);
/* Runs n_iters iterations (no metrics) with CUDA events around each launch and
 * writes the mean device milliseconds into ms_out[3]: the block solves (Eq. 14, with
 * the previous iteration's dual ascent, Eqs. 12-13, applied as they start), the point
 * consensus (Eq. 10) and the camera consensus (Eq. 11). */
dba_status dba_block_profile(dba_block_ctx* ctx, int n_iters, double* ms_out);
/* Consensus cameras [m][6] and points [n][3]. */
dba_status dba_block_get_params(dba_block_ctx* ctx, double* cams_out, double* pts_out);
/* Number of blocks, point copies and camera copies (any pointer may be NULL). */
dba_status dba_block_layout(const dba_block_ctx* ctx, int64_t* n_blocks, int64_t* n_point_copies,
                            int64_t* n_camera_copies);
/* The block layout dba_block_set_observations builds, computed on the host only (no
 * device), for inspection and tests.  Same index checks as dba_block_set_observations
 * and 1 <= block_points <= DBA_BLOCK_MAX_POINTS, 1 <= block_cams <= DBA_BLOCK_MAX_CAMERAS
 * (EINVAL, message in dba_block_last_error(NULL)).  Outputs, caller-allocated, any may
 * be NULL:
 *   obs_order[n_obs]   caller index of each observation in block order (blocks by
 *                      (point group, camera group); inside a block by point rank, then
 *                      camera);
 *   blocks[6 n_obs]    per block in launch (size-class) order: first observation, count;
 *                      first point copy, count; first camera copy, count;
 *   pc_point[n_obs]    point of each point copy (copies in block order);
 *   cc_camera[n_obs]   camera of each camera copy;
 *   counts[3]          blocks, point copies, camera copies;
 *   size_classes[DBA_BLOCK_SIZE_CLASSES]  blocks per size class. */
dba_status dba_block_build_layout(int32_t n_cams, int32_t n_pts, int64_t n_obs, const int32_t* pt_idx,
                                  const int32_t* cam_idx, int block_points, int block_cams, int64_t* obs_order,
                                  int32_t* blocks, int32_t* pc_point, int32_t* cc_camera, int64_t* counts,
                                  int64_t* size_classes);
/* Blocks in each size class of the solve kernel, in launch order: one camera and at
 * most 8 points (lane groups of 1, 2, 4 or 8 by the block's points), at most 2
 * cameras and 16 points (16 lanes; two-camera blocks of at most 4 or 8 points in 4 or
 * 8), at most 32 points (32 lanes), the rest (32 lanes, two point copies each).
 * counts: DBA_BLOCK_SIZE_CLASSES entries, caller-owned. */
#define DBA_BLOCK_SIZE_CLASSES 4
dba_status dba_block_size_classes(const dba_block_ctx* ctx, int64_t* counts);
/* Kernel launches one iteration of dba_block_iterate makes with the loaded layout: one
 * block-solve launch per nonempty range of blocks that share a kernel and lane-group
 * width, then the point and the camera consensus.  Launch bookkeeping of this library;
 * the paper has no counterpart.  launches: caller-owned. */
dba_status dba_block_launches_per_iteration(const dba_block_ctx* ctx, int32_t* launches);
/* Algorithmic floating-point operations of one iteration's block solves (every
 * Gauss-Newton step counted in full with its trial objective; add/mul 1, fma 2,
 * reciprocal/square root/sine/cosine 1), counted from the loaded layout. */
dba_status dba_block_algorithmic_flops(const dba_block_ctx* ctx, double* per_iteration);
/* Message of the last failed call on ctx (ctx NULL: of the last failed create). */
const char* dba_block_last_error(const dba_block_ctx* ctx);
void dba_block_destroy(dba_block_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DBA_H */
