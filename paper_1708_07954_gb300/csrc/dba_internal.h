// Internal interface between the host C ABI (dba_api.cu) and the kernels
// (dba_kernels.cu).  Not installed; not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dba {

// Device control word read by every kernel of an iteration, so that one
// captured CUDA graph serves every iteration: which consensus buffer is
// current, whether the previous iteration's dual ascent (Eqs. 12-13) is still
// to be applied, and a sticky error flag.
struct alignas(16) DevCtl {
  int cur;          // index (0/1) of the current consensus buffer
  int pending;      // 1: copies are offsets from the previous consensus, duals lag by one step
  int err;          // bit 0: non-finite local solve; bit 1: warm-start network wait timed out;
                    // bit 2: tile kernel tensor-copy wait timed out
  int exact;        // 1: duals may not sum to zero per point/camera (first iteration after set_state)
  unsigned long long k;   // iterations run
  unsigned int done;      // finalize-kernel block counter
  unsigned int inject;    // fault injection for tests: bit 0 = the tile kernel announces its
                          // tensor copies but does not issue them (its bounded wait runs out)
  unsigned int metric_done;  // metrics-kernel block counter (the last block reduces)
};

// One tile of the observation layout: observations [o0, o0 + n), point runs
// [r0, r0 + nr) covering internal points [pt_lo, pt_lo + nr), camera runs [c0, c0 + nc).
struct alignas(16) TileInfo {
  int o0, n, r0, nr, c0, nc, pt_lo, pad;
};

struct Params {
  double focal, cx, cy;
  int loss;
  double loss_param;
  double rho_x, rho_y, rho_a;  // points, camera translations, camera angles
  int inner_steps;
  double lambda0, lambda_min, eps_depth, model_tol;
  int solver;  // dba_local_solver
};

// All device pointers of one problem.  Observation arrays are in internal
// (tile) order; per-observation vectors are structure-of-arrays with row stride
// `pitch` (n_obs rounded up to kObsPitchAlign, so every row starts on a 128-byte
// boundary as the tile kernel's tensor copies require).
struct DevProblem {
  int n_cams, n_pts;
  long long n_obs;
  long long pitch;              // row stride of delta, adual and mlp_start
  int n_tiles;
  int tile_obs;                 // block size of the tile kernel
  int fin_threads;              // block size of finalize: 32, 64, 128 or 256
  int n_cam_slots, n_pt_slots, n_split_pts;
  // static structure
  const int* obs_pt;            // [l] internal point id
  const int* obs_cam_rank;      // [l] camera | (position in the tile's camera order) << 24
  const void* z;                // [l] float2 (FP32 path) or double2 (FP64 path)
  const void* zt;               // [l] same type: ground-truth projections, or nullptr
  const unsigned char* inlier;  // [l] 1: counted in rmse_gt (nullptr: all)
  const TileInfo* tiles;        // [n_tiles]
  const int2* pseg;             // (start, length) of each point run inside its tile
  const int* pseg_slot;         // -1: the whole track is in this tile; else partial slot
  const int2* cseg;             // (start, length) of each camera run in the tile's camera order
  const int* cseg_slot;         // partial slot of each camera run
  const int* cam_slot_off;      // [m+1] camera -> its partial slots
  const int* cam_count;         // [m] observations per camera
  const int* split_pt;          // [n_split_pts] points whose track spans several tiles
  const int* split_slot_off;    // [n_split_pts+1]
  const int* pt_count;          // [n] observations per point
  // state
  void* delta;                  // [9][pitch] T: copy minus the consensus it was solved against
  double* adual;                // [9][pitch] scaled duals (r/rho_x, s/rho_y)
  double* X[2];                 // [n][3] point consensus, ping-pong
  double* Y[2];                 // [m][6] camera consensus, ping-pong
  void* Xm;                     // [n][3] T copy of the current point consensus
  void* DX;                     // [n][3] T: previous minus current point consensus
  void* Ym;                     // [m][6]
  void* DY;                     // [m][6]
  double* pt_part;              // [n_pt_slots][3]
  double* cam_part;             // [n_cam_slots][6]
  const void* mlp_start;        // [9][pitch] T: learned candidate start (nullptr: none)
  double* metric_part;          // [metric blocks][8]
  double* metric_out;           // [8]
  void* cam_pose;               // [n_cams][12] T: R (row-major) and t of each consensus camera
  DevCtl* ctl;
};

// Tensor maps of the observation arrays the tile kernel stages with TMA (built on the
// host per problem; passed to the kernel as a grid constant).
struct TileMaps {
  CUtensorMap delta;  // [9][n_obs] T, row stride pitch
  CUtensorMap adual;  // [9][n_obs] double
  CUtensorMap z;      // [n_obs] float2 as 64-bit words, or [n_obs][2] double
  CUtensorMap pt;     // [n_obs] int32
  CUtensorMap cam;    // [n_obs] int32 (obs_cam_rank)
};

constexpr int kCamMask = 0xffffff;  // camera index bits of obs_cam_rank
constexpr long long kObsPitchAlign = 32;  // elements: 128 bytes of float, 256 of double
inline long long obs_pitch(long long n_obs) { return (n_obs + kObsPitchAlign - 1) / kObsPitchAlign * kObsPitchAlign; }
constexpr int kMetricBlocks = 1024;
constexpr int kMetricThreads = 256;

// One-time kernel set-up on the current device (shared-memory opt-in, occupancy); call
// before any stream capture.
cudaError_t prepare_tile_kernels();

// Kernel launchers (return the launch error).  fp32 selects the FP32 local-solve path.
// Encodes the tile kernel's tensor maps for P (its pointers, n_obs, pitch, tile_obs).
cudaError_t encode_tile_maps(const DevProblem& P, bool fp32, TileMaps* M);
cudaError_t launch_tile_iterate(const DevProblem& P, const TileMaps& M, const Params& prm, bool fp32,
                                cudaStream_t s);
cudaError_t launch_finalize(const DevProblem& P, bool fp32, cudaStream_t s);
// gt_only: only the reference-pixel sums (rmse_gt and its count) and the valid counts.
cudaError_t launch_metrics(const DevProblem& P, const Params& prm, bool fp32, int cur, int pending,
                           cudaStream_t s, bool gt_only = false);
cudaError_t launch_settle(const DevProblem& P, bool fp32, int cur, cudaStream_t s);
cudaError_t launch_project_truth(const DevProblem& P, const Params& prm, bool fp32,
                                 const double* cams_gt, const double* pts_gt, void* zt_out,
                                 cudaStream_t s);

// Per-scene metrics: out[5 * scene + k] += (sum e^2, objective, sum gt^2, valid count,
// gt count) over observations whose internal scene id is `scene` (out zeroed by the caller).
cudaError_t launch_scene_metrics(const DevProblem& P, const Params& prm, bool fp32, const int* scene_of_obs,
                                 double* out, cudaStream_t s);

// Learned warm start (dba_mlp.cu): tensor-core inference writing P.mlp_start from the
// state, feature/target harvest, and the BF16 operand blob built from FP32 parameters.
cudaError_t launch_mlp_warmstart(const DevProblem& P, const Params& prm, bool fp32, const unsigned char* blob,
                                 const float* params, cudaStream_t s);
cudaError_t launch_mlp_harvest(const DevProblem& P, const Params& prm, bool fp32, int pending, long long stride,
                               long long cap, int target_steps, float* feats, float* targs, cudaStream_t s);

// Allocation-free reprojection statistics (file-scope device scratch; see dba_evaluate_noalloc).
cudaError_t launch_eval_noalloc(const Params& prm, long long n_obs, int n_cams, int n_pts, const int* pt_idx,
                                const int* cam_idx, const double* z, const double* cams, const double* pts,
                                double* out, cudaStream_t s);

}  // namespace dba

#include <vector>
namespace dba {
void mlp_make_blob(const float* params, std::vector<unsigned char>& blob);
}  // namespace dba
