// Block subproblems: the generalized update step of Sec. 3.1.4, Eq. (14).
//
// Each update solves, instead of one observation, a block of up to pi points and
// kappa cameras with all observations between them, over one copy of each of its
// points and cameras.  Blocks are formed by this reading of the paper: points
// ranked by (smallest observing camera index, point index) and cut into groups of
// pi consecutive ranks, cameras cut into groups of kappa consecutive indices, one
// block per (point group, camera group) pair holding observations.
//
// GPU mapping: one group of G lanes per block (G = 8, 16 or 32 by the block's size,
// several blocks per warp), one lane per point copy (two per lane above 32 points;
// pi <= 64), camera copies (kappa <= 4) shared by the group in shared memory.  Each damped
// Gauss-Newton step eliminates the points (3x3 per lane) and solves the reduced camera
// system (at most 24 x 24).  Three solve kernels:
//   one camera (6 x 6): terms summed by a reduce-scatter over the group (butterflies in
//     groups of one or two lanes), factored in every lane's registers;
//   two or four camera slots, at most 32 points (12 x 12 or 24 x 24): terms formed in
//     registers, summed by the reduce-scatter, factored in registers a row per lane;
//   above 32 points (two copies a lane): terms staged in shared memory, summed
//     entry-parallel, factored lane-per-row in shared memory.
// Consensus (Eqs. 10-11 over copies) and dual ascent (Eqs. 12-13) run in FP64 over copy
// lists.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "../../include/dba.h"
#include "dba_device.cuh"
#include "dba_internal.h"
#include "dba_guard.h"

namespace dba {
namespace {

constexpr int kBlkWarps = 4;  // most warps per CTA (fewer where shared memory would not hold them)
constexpr int kBlkClasses = 4;
constexpr int kLin = 21;      // per observation: A = dz/dx (2x3), B = dz/dy (2x6), 2w, e (2)

struct BlockInfo {
  int o0, no;  // observations (block order)
  int p0, np;  // point copies
  int c0, nc;  // camera copies
};

struct BlockProblem {
  int n_cams, n_pts, n_blocks;
  long long n_obs, n_pc, n_cc;
  const BlockInfo* blocks;
  const int* pc_obs;             // [n_pc + 1] first observation of each point copy
  const int* pc_pt;              // [n_pc]
  const int* cc_cam;             // [n_cc]
  const unsigned char* obs_lc;   // [n_obs] local camera of each observation
  const int* obs_pt;             // [n_obs] point id
  const int* obs_cam;            // [n_obs] camera id
  const void* z;                 // [n_obs] pixel pairs in T
  const double* zt;              // [2 n_obs] reference pixels or null
  const unsigned char* inlier;   // [n_obs] or null
  void* pc_delta;                // [3][n_pc] T: copy minus the consensus it was solved against
  double* pc_a;                  // [3][n_pc] scaled duals r / rho
  void* cc_delta;                // [6][n_cc]
  double* cc_a;                  // [6][n_cc]
  double* X[2];                  // [3 n_pts] consensus, ping-pong
  double* Y[2];                  // [6 n_cams]
  const int* pt_cp_off;          // [n_pts + 1] CSR point -> its copies
  const int* pt_cp;
  const int* cam_cp_off;         // [n_cams + 1]
  const int* cam_cp;
  double* sums;                  // [8] metric accumulators
  void* cam_pose;                // [n_cams][12] T: R (row-major) and t of each consensus camera
  // T mirrors of the current consensus and of its last change (previous minus current),
  // written by the consensus kernels; they let the next block solves re-base the copies
  // and apply the deferred dual ascent without FP64 gathers
  void* Xm;                      // [3 n_pts]
  void* DX;                      // [3 n_pts]
  void* Ym;                      // [6 n_cams]
  void* DY;                      // [6 n_cams]
  int pending;                   // 1: the last iteration's dual ascent (Eqs. 12-13) is still to apply
  int* err;                      // bit 0: non-finite copy
};

// A block's lane group: G consecutive lanes of a warp (G = 8, 16 or 32).  Every vote,
// shuffle and barrier names the group's lanes only, so groups of one warp may diverge.
template <int G>
struct Grp {
  int lane;       // lane in the warp: column of the per-lane shared arrays
  int gl;         // lane in the group
  int base;       // first warp lane of the group
  unsigned mask;  // the group's lanes
  __device__ explicit Grp(int warp_lane)
      : lane(warp_lane), gl(warp_lane & (G - 1)), base(warp_lane & ~(G - 1)),
        mask(G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (warp_lane & ~(G - 1)))) {}
  __device__ void sync() const { __syncwarp(mask); }
  template <typename T>
  __device__ T sum(T v) const {
#pragma unroll
    for (int m = G / 2; m > 0; m >>= 1) v += __shfl_xor_sync(mask, v, m, G);
    return v;
  }
  __device__ bool all(bool p) const { return __all_sync(mask, p); }
  template <typename T>
  __device__ T bcast(T v, int src) const { return __shfl_sync(mask, v, src, G); }
};

// Lane gl of a group of G receives the sum over the group of v[gl] (v is overwritten).
// Stage h: the lane keeps the half of its values whose index has bit h equal to its own lane
// bit h, adds the partner's partial sums of that half and hands over the other half.
template <typename T, int G>
__device__ __forceinline__ T reduce_scatter(T (&v)[G], const Grp<G>& grp) {
#pragma unroll
  for (int h = G / 2; h >= 1; h >>= 1) {
    const bool up = (grp.gl & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? v[i] : v[i + h];
      const T keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(grp.mask, send, h, G);
    }
  }
  return v[0];
}

// State of one block solve shared by its lane group; KC = the most cameras a block holds.
template <typename T, int KC>
struct BlkShared {
  static constexpr int kU = 6 * KC;
  T S[kU][kU + 1];            // reduced camera system, then its Cholesky factor
  T rhs[kU];
  T g[kU];                    // camera part of the block gradient
  T dy[kU];                   // camera step
  T vbar[KC][6];              // camera consensus
  T d[KC][6];                 // camera copy offsets
  T dt[KC][6];                // trial offsets
  T a[KC][6];                 // camera scaled duals
};

// Per-warp shared memory: per-copy arrays (one column per point copy held by the warp:
// 32 x PPL, padded) and the shared state of the warp's 32 / G blocks.
template <typename T, int KC, int G, int PPL>
struct BlkSmem {
  static constexpr int kPairs = KC * (KC + 1) / 2;
  // rows padded by one word: the reduction reads one copy's column across rows, which an
  // unpadded row of 32 words would put in a single bank
  static constexpr int kCols = 32 * PPL + 1;
  T lin[KC][kLin][kCols];     // each copy's observation slots: A = dz/dx (2x3), B = dz/dy (2x6), 2w, e
  T U[KC][2][kCols];          // 2w A W_p g_p per slot
  T Q[kPairs][4][kCols];      // per camera pair c1 <= c2: 2x2 weight of the point's Schur term
  signed char slot[KC][32 * PPL];  // slot of each copy's observation on camera c (-1: none)
  BlkShared<T, KC> grp[32 / G];
};

template <int KC>
__device__ __forceinline__ int pair_index(int c1, int c2) {  // c1 <= c2
  return c1 * KC - c1 * (c1 - 1) / 2 + (c2 - c1);
}

// One point copy held by a lane: its consensus, offset and scaled dual, and its
// observations in the block (at most one per camera).
template <typename T, int KC>
struct BlkPt {
  bool act;          // the lane holds this copy
  int nob;           // its observations
  int oc[KC];        // local camera of observation k
  int slot[KC];      // observation on local camera c (-1: none)
  T oz0[KC], oz1[KC];
  T xbar[3], ax[3];
};

// Eq. (14) at (point offsets dp of this lane's copies, camera offsets dc): misfits of
// the lane's observations + its points' dual and penalty terms, summed over the group,
// plus the cameras' terms.  +inf when an observation is behind its camera.
template <typename T, int KC, int G, int PPL>
__device__ __forceinline__ T block_objective(const Prm<T>& q, const Grp<G>& grp, const BlkPt<T, KC> (&pt)[PPL],
                                             const T (&dp)[PPL][3], const BlkShared<T, KC>& Z, const T (*dc)[6],
                                             int nc) {
  T s = 0;
  bool ok = true;
#pragma unroll
  for (int j = 0; j < PPL; ++j) {
    if (!pt[j].act) continue;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      if (k < pt[j].nob) {
        const int c = pt[j].oc[k];
        T v[9];
#pragma unroll
        for (int u = 0; u < 3; ++u) v[u] = pt[j].xbar[u] + dp[j][u];
#pragma unroll
        for (int u = 0; u < 6; ++u) v[3 + u] = Z.vbar[c][u] + dc[c][u];
        Pose<T> P;
        pose_at(v, q.eps, P);
        if (!P.valid) {
          ok = false;
        } else {
          const T iz = Num<T>::rcp(P.p[2]);
          const T e0 = pt[j].oz0[k] - (q.focal * P.p[0] * iz + q.cx);
          const T e1 = pt[j].oz1[k] - (q.focal * P.p[1] * iz + q.cy);
          s += misfit<T>(q.loss, q.lp, e0 * e0 + e1 * e1);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) s += q.rho_x * dp[j][u] * (pt[j].ax[u] + T(0.5) * dp[j][u]);
  }
  s = grp.sum(s);
  ok = grp.all(ok);
  T sc = 0;
  for (int c = 0; c < nc; ++c)
#pragma unroll
    for (int u = 0; u < 6; ++u) sc += q.rho(3 + u) * dc[c][u] * (Z.a[c][u] + T(0.5) * dc[c][u]);
  return ok ? s + sc : Num<T>::inf();
}

// One coordinate of a copy at the start of a block solve: its consensus (the T mirror), its
// offset re-based on that consensus and its scaled dual.  With a pending dual ascent (every
// iteration but the first) the previous iteration's Eqs. (12)-(13) are applied here, now
// that the new consensus exists: the offset becomes d0 = offset + (previous - current
// consensus) and the dual a + d0, in FP64, written back.
template <typename T>
__device__ __forceinline__ void deferred_ascent(const BlockProblem& B, T cons, T change, T offset, double* a,
                                                T& vbar, T& d0, T& aT) {
  vbar = cons;
  if (B.pending) {
    d0 = offset + change;
    const double an = *a + to_f64<T>(d0);
    *a = an;
    aT = from_f64<T>(an);
  } else {
    d0 = offset;
    aT = from_f64<T>(*a);
  }
}

// Point copy p of a block sits on group lane p % G, register slot p / G, shared-memory
// column base + p (PPL = 2 only with G = 32, so a warp's columns never overlap).
template <typename T, int KC, int G, int PPL>
__device__ void solve_block(const BlockProblem& B, const Prm<T>& q, const BlockInfo& bi,
                            BlkSmem<T, KC, G, PPL>& W, const Grp<G>& grp, int cur) {
  static_assert(PPL == 1 || G == 32, "two point copies per lane need whole-warp groups");
  static_assert(6 * KC <= G, "one lane per row of the reduced camera system");
  const int gl = grp.gl;  // lane in the group: first point copy, row of the camera system
  BlkShared<T, KC>& Z = W.grp[grp.base / G];
  using V2 = typename Num<T>::V2;
  const int np = bi.np, nc = bi.nc, n_u = 6 * nc;
  T* pdel = static_cast<T*>(B.pc_delta);
  T* cdel = static_cast<T*>(B.cc_delta);
  BlkPt<T, KC> pt[PPL];
  T dp[PPL][3];
#pragma unroll
  for (int j = 0; j < PPL; ++j) {
    const int p = gl + G * j;
    const int col = grp.base + p;
    BlkPt<T, KC>& P = pt[j];
    P.act = p < np;
    P.nob = 0;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      P.oc[k] = 0;
      P.oz0[k] = P.oz1[k] = 0;
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) P.xbar[u] = dp[j][u] = P.ax[u] = 0;
    if (P.act) {
      const long long pc = (long long)bi.p0 + p;
      const int i = B.pc_pt[pc];
#pragma unroll
      for (int u = 0; u < 3; ++u)
        deferred_ascent<T>(B, static_cast<const T*>(B.Xm)[3 * (long long)i + u],
                           static_cast<const T*>(B.DX)[3 * (long long)i + u], pdel[u * B.n_pc + pc],
                           B.pc_a + u * B.n_pc + pc, P.xbar[u], dp[j][u], P.ax[u]);
      const int ob0 = B.pc_obs[pc];
      P.nob = B.pc_obs[pc + 1] - ob0;
      const V2* zz = static_cast<const V2*>(B.z);
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k < P.nob) {
          P.oc[k] = B.obs_lc[ob0 + k];
          const V2 z = zz[ob0 + k];
          P.oz0[k] = z.x;
          P.oz1[k] = z.y;
        }
    }
    // slot of this copy's observation on each camera of the block (-1: none)
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      P.slot[c] = -1;
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k < P.nob && P.oc[k] == c) P.slot[c] = k;
      W.slot[c][col] = (signed char)P.slot[c];
    }
  }
  if (gl < n_u) {
    const int c = gl / 6, u = gl % 6;
    const long long cc = (long long)bi.c0 + c;
    const int j = B.cc_cam[cc];
    deferred_ascent<T>(B, static_cast<const T*>(B.Ym)[6 * (long long)j + u],
                       static_cast<const T*>(B.DY)[6 * (long long)j + u], cdel[u * B.n_cc + cc],
                       B.cc_a + u * B.n_cc + cc, Z.vbar[c][u], Z.d[c][u], Z.a[c][u]);
  }
  grp.sync();

  T L = block_objective<T, KC, G, PPL>(q, grp, pt, dp, Z, Z.d, nc);
  T lambda = T(-1);
  for (int step = 0; step < q.steps; ++step) {
    // linearise this lane's observations at the current copies
    T Hpp[PPL][6], gp[PPL][3];
    T noise = 0, trc = 0;
#pragma unroll
    for (int j = 0; j < PPL; ++j) {
      const int col = grp.lane + 32 * j;
#pragma unroll
      for (int u = 0; u < 6; ++u) Hpp[j][u] = 0;
#pragma unroll
      for (int u = 0; u < 3; ++u) gp[j][u] = 0;
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        if (k < pt[j].nob) {
          const int c = pt[j].oc[k];
          T v[9];
#pragma unroll
          for (int u = 0; u < 3; ++u) v[u] = pt[j].xbar[u] + dp[j][u];
#pragma unroll
          for (int u = 0; u < 6; ++u) v[3 + u] = Z.vbar[c][u] + Z.d[c][u];
          Pose<T> P;
          pose_at(v, q.eps, P);
          T J0[9], J1[9], e0 = 0, e1 = 0, w = 0;
          if (P.valid) {
            linearize(P, pt[j].oz0[k], pt[j].oz1[k], q, J0, J1, e0, e1, w);
          } else {
#pragma unroll
            for (int u = 0; u < 9; ++u) J0[u] = J1[u] = 0;
          }
          const T tw = T(2) * w;
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            W.lin[k][u][col] = J0[u];
            W.lin[k][3 + u][col] = J1[u];
          }
#pragma unroll
          for (int u = 0; u < 6; ++u) {
            W.lin[k][6 + u][col] = J0[3 + u];
            W.lin[k][12 + u][col] = J1[3 + u];
          }
          W.lin[k][18][col] = tw;
          W.lin[k][19][col] = e0;
          W.lin[k][20][col] = e1;
          Hpp[j][0] += tw * (J0[0] * J0[0] + J1[0] * J1[0]);
          Hpp[j][1] += tw * (J0[0] * J0[1] + J1[0] * J1[1]);
          Hpp[j][2] += tw * (J0[0] * J0[2] + J1[0] * J1[2]);
          Hpp[j][3] += tw * (J0[1] * J0[1] + J1[1] * J1[1]);
          Hpp[j][4] += tw * (J0[1] * J0[2] + J1[1] * J1[2]);
          Hpp[j][5] += tw * (J0[2] * J0[2] + J1[2] * J1[2]);
#pragma unroll
          for (int u = 0; u < 3; ++u) gp[j][u] -= tw * (J0[u] * e0 + J1[u] * e1);
#pragma unroll
          for (int u = 3; u < 9; ++u) trc += tw * (J0[u] * J0[u] + J1[u] * J1[u]);
          noise += tw * Num<T>::sqrt_(e0 * e0 + e1 * e1) * (fabs(pt[j].oz0[k]) + fabs(pt[j].oz1[k]));
        }
      }
      if (pt[j].act)
#pragma unroll
        for (int u = 0; u < 3; ++u) gp[j][u] += q.rho_x * (pt[j].ax[u] + dp[j][u]);
    }
    if (lambda < T(0)) {
      T tr = trc;
#pragma unroll
      for (int j = 0; j < PPL; ++j)
        if (pt[j].act) tr += Hpp[j][0] + Hpp[j][3] + Hpp[j][5] + T(3) * q.rho_x;
      tr = grp.sum(tr);
      for (int c = 0; c < nc; ++c)
#pragma unroll
        for (int u = 0; u < 6; ++u) tr += q.rho(3 + u);
      lambda = q.lambda0 * tr / T(3 * np + n_u);
    }
    // W_p = (H_pp + (rho_x + lambda) I)^-1 by cofactors (symmetric positive definite)
    T Wp[PPL][6];
#pragma unroll
    for (int j = 0; j < PPL; ++j) {
      const int col = grp.lane + 32 * j;
      Wp[j][0] = 1, Wp[j][1] = 0, Wp[j][2] = 0, Wp[j][3] = 1, Wp[j][4] = 0, Wp[j][5] = 1;
      if (pt[j].act) {
        const T dg = q.rho_x + lambda;
        const T h00 = Hpp[j][0] + dg, h01 = Hpp[j][1], h02 = Hpp[j][2], h11 = Hpp[j][3] + dg, h12 = Hpp[j][4],
                h22 = Hpp[j][5] + dg;
        const T c00 = h11 * h22 - h12 * h12, c01 = h02 * h12 - h01 * h22, c02 = h01 * h12 - h02 * h11;
        const T c11 = h00 * h22 - h02 * h02, c12 = h01 * h02 - h00 * h12, c22 = h00 * h11 - h01 * h01;
        const T idet = Num<T>::rcp(h00 * c00 + h01 * c01 + h02 * c02);
        Wp[j][0] = c00 * idet;
        Wp[j][1] = c01 * idet;
        Wp[j][2] = c02 * idet;
        Wp[j][3] = c11 * idet;
        Wp[j][4] = c12 * idet;
        Wp[j][5] = c22 * idet;
      }
      const T* w6 = Wp[j];
      const T* g3 = gp[j];
      const T Wg0 = w6[0] * g3[0] + w6[1] * g3[1] + w6[2] * g3[2];
      const T Wg1 = w6[1] * g3[0] + w6[3] * g3[1] + w6[4] * g3[2];
      const T Wg2 = w6[2] * g3[0] + w6[4] * g3[1] + w6[5] * g3[2];
      // this point's terms of the reduced system: U_k = 2w_k A_k W_p g_p and, per camera
      // pair, Q = [c1 = c2] 2w_1 I - (2w_1 A_1) W_p (2w_2 A_2)^T
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k < pt[j].nob) {
          const T tw = W.lin[k][18][col];
          W.U[k][0][col] = tw * (W.lin[k][0][col] * Wg0 + W.lin[k][1][col] * Wg1 + W.lin[k][2][col] * Wg2);
          W.U[k][1][col] = tw * (W.lin[k][3][col] * Wg0 + W.lin[k][4][col] * Wg1 + W.lin[k][5][col] * Wg2);
        }
#pragma unroll
      for (int c1 = 0; c1 < KC; ++c1)
#pragma unroll
        for (int c2 = c1; c2 < KC; ++c2) {
          const int k1 = pt[j].slot[c1], k2 = pt[j].slot[c2];
          if (pt[j].act && k1 >= 0 && k2 >= 0) {
            const T tw1 = W.lin[k1][18][col], tw2 = W.lin[k2][18][col];
            const T a20 = W.lin[k2][0][col], a21 = W.lin[k2][1][col], a22 = W.lin[k2][2][col];
            const T a23 = W.lin[k2][3][col], a24 = W.lin[k2][4][col], a25 = W.lin[k2][5][col];
            // columns of W_p A_2^T
            const T w0 = w6[0] * a20 + w6[1] * a21 + w6[2] * a22, w1 = w6[1] * a20 + w6[3] * a21 + w6[4] * a22,
                    w2 = w6[2] * a20 + w6[4] * a21 + w6[5] * a22;
            const T x0 = w6[0] * a23 + w6[1] * a24 + w6[2] * a25, x1 = w6[1] * a23 + w6[3] * a24 + w6[4] * a25,
                    x2 = w6[2] * a23 + w6[4] * a24 + w6[5] * a25;
            const T a10 = W.lin[k1][0][col], a11 = W.lin[k1][1][col], a12 = W.lin[k1][2][col];
            const T a13 = W.lin[k1][3][col], a14 = W.lin[k1][4][col], a15 = W.lin[k1][5][col];
            const T sw = tw1 * tw2, dgw = c1 == c2 ? tw1 : T(0);
            const int pr = pair_index<KC>(c1, c2);
            W.Q[pr][0][col] = dgw - sw * (a10 * w0 + a11 * w1 + a12 * w2);
            W.Q[pr][1][col] = -sw * (a10 * x0 + a11 * x1 + a12 * x2);
            W.Q[pr][2][col] = -sw * (a13 * w0 + a14 * w1 + a15 * w2);
            W.Q[pr][3][col] = dgw - sw * (a13 * x0 + a14 * x1 + a15 * x2);
          }
        }
    }
    grp.sync();
    // reduced camera system, one entry per lane at a time, summed over the block's points:
    //   S(c1 r, c2 s) = sum_p B_1[:, r]^T Q B_2[:, s],  g_c = -sum 2w B^T e + rho (a + d),
    //   rhs_c = sum_p B^T U - g_c
    const int nS = 21 * nc + 18 * nc * (nc - 1);
    const int nV = nS + 12 * nc;
    for (int v = gl; v < nV; v += G) {
      T acc = 0;
      if (v < nS) {
        int c1 = 0, c2 = 0, e = v;
        bool found = false;
        for (c1 = 0; c1 < nc && !found; ++c1)
          for (c2 = c1; c2 < nc; ++c2) {
            const int size = c1 == c2 ? 21 : 36;
            if (e < size) {
              found = true;
              break;
            }
            e -= size;
          }
        --c1;  // the outer loop stepped past the pair it found
        int r, s;
        if (c1 == c2) {
          r = 0;
          while (e >= 6 - r) {
            e -= 6 - r;
            ++r;
          }
          s = r + e;
        } else {
          r = e / 6;
          s = e % 6;
        }
        const int pr = pair_index<KC>(c1, c2);
        for (int l = 0; l < np; ++l) {
          const int lb = grp.base + l;
          const int k1 = W.slot[c1][lb], k2 = W.slot[c2][lb];
          if (k1 >= 0 && k2 >= 0) {
            const T b10 = W.lin[k1][6 + r][lb], b11 = W.lin[k1][12 + r][lb];
            const T b20 = W.lin[k2][6 + s][lb], b21 = W.lin[k2][12 + s][lb];
            acc += b10 * (W.Q[pr][0][lb] * b20 + W.Q[pr][1][lb] * b21) +
                   b11 * (W.Q[pr][2][lb] * b20 + W.Q[pr][3][lb] * b21);
          }
        }
        Z.S[6 * c1 + r][6 * c2 + s] = acc;
        Z.S[6 * c2 + s][6 * c1 + r] = acc;
      } else {
        const int w = v - nS, c = w / 12, u = w % 6;
        const bool isg = (w % 12) < 6;
        for (int l = 0; l < np; ++l) {
          const int lb = grp.base + l;
          const int k = W.slot[c][lb];
          if (k >= 0) {
            const T b0 = W.lin[k][6 + u][lb], b1 = W.lin[k][12 + u][lb];
            if (isg)
              acc -= W.lin[k][18][lb] * (b0 * W.lin[k][19][lb] + b1 * W.lin[k][20][lb]);
            else
              acc += b0 * W.U[k][0][lb] + b1 * W.U[k][1][lb];
          }
        }
        if (isg)
          Z.g[6 * c + u] = acc + q.rho(3 + u) * (Z.a[c][u] + Z.d[c][u]);
        else
          Z.rhs[6 * c + u] = acc;
      }
    }
    grp.sync();
    if (gl < n_u) {
      Z.rhs[gl] -= Z.g[gl];
      Z.S[gl][gl] += q.rho(3 + gl % 6) + lambda;
    }
    grp.sync();
    // Cholesky S = L L^T, lane i owning row i
    bool spd = true;
    for (int k = 0; k < n_u; ++k) {
      const T piv = Z.S[k][k];
      if (!(piv > T(0))) {
        spd = false;
        break;
      }
      const T lkk = Num<T>::sqrt_(piv);
      if (gl > k && gl < n_u) Z.S[gl][k] = Num<T>::div(Z.S[gl][k], lkk);
      grp.sync();
      if (gl == k) Z.S[k][k] = lkk;
      if (gl > k && gl < n_u) {
        const T lik = Z.S[gl][k];
        for (int jj = k + 1; jj <= gl; ++jj) Z.S[gl][jj] -= lik * Z.S[jj][k];
      }
      grp.sync();
    }
    if (!spd) {
      lambda *= T(10);
      continue;
    }
    // L y = rhs, then L^T dy = y; lane i holds entry i
    T y = gl < n_u ? Z.rhs[gl] : T(0);
    for (int k = 0; k < n_u; ++k) {
      const T yk = Num<T>::div(grp.bcast(y, k), Z.S[k][k]);
      if (gl == k) y = yk;
      else if (gl > k && gl < n_u) y -= Z.S[gl][k] * yk;
    }
    for (int k = n_u - 1; k >= 0; --k) {
      const T xk = Num<T>::div(grp.bcast(y, k), Z.S[k][k]);
      if (gl == k) y = xk;
      else if (gl < k) y -= Z.S[k][gl] * xk;
    }
    if (gl < n_u) Z.dy[gl] = y;
    grp.sync();
    // point steps dx = -W_p (g_p + H_pc dy); predicted decrease (lambda |d|^2 - g.d) / 2
    T xt[PPL][3];
    T gd = 0, dd = 0;
#pragma unroll
    for (int j = 0; j < PPL; ++j) {
      const int col = grp.lane + 32 * j;
      T dx[3] = {0, 0, 0};
      if (pt[j].act) {
        T t0 = gp[j][0], t1 = gp[j][1], t2 = gp[j][2];
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          if (k < pt[j].nob) {
            const int c = pt[j].oc[k];
            T r0 = 0, r1 = 0;
#pragma unroll
            for (int u = 0; u < 6; ++u) {
              r0 += W.lin[k][6 + u][col] * Z.dy[6 * c + u];
              r1 += W.lin[k][12 + u][col] * Z.dy[6 * c + u];
            }
            const T tw = W.lin[k][18][col];
            r0 *= tw;
            r1 *= tw;
            t0 += W.lin[k][0][col] * r0 + W.lin[k][3][col] * r1;
            t1 += W.lin[k][1][col] * r0 + W.lin[k][4][col] * r1;
            t2 += W.lin[k][2][col] * r0 + W.lin[k][5][col] * r1;
          }
        }
        dx[0] = -(Wp[j][0] * t0 + Wp[j][1] * t1 + Wp[j][2] * t2);
        dx[1] = -(Wp[j][1] * t0 + Wp[j][3] * t1 + Wp[j][4] * t2);
        dx[2] = -(Wp[j][2] * t0 + Wp[j][4] * t1 + Wp[j][5] * t2);
      }
      gd += gp[j][0] * dx[0] + gp[j][1] * dx[1] + gp[j][2] * dx[2];
      dd += dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
#pragma unroll
      for (int u = 0; u < 3; ++u) xt[j][u] = dp[j][u] + dx[u];
    }
    gd = grp.sum(gd);
    dd = grp.sum(dd);
    for (int u = 0; u < n_u; ++u) {
      gd += Z.g[u] * Z.dy[u];
      dd += Z.dy[u] * Z.dy[u];
    }
    const T pred = T(0.5) * (lambda * dd - gd);
    const T noise_sum = grp.sum(noise);
    const bool trust = isfinite(L) && q.model_tol > T(0) &&
                       pred <= q.model_tol * Num<T>::unit_roundoff * (fabs(L) + noise_sum);
    if (gl < n_u) Z.dt[gl / 6][gl % 6] = Z.d[gl / 6][gl % 6] + Z.dy[gl];
    grp.sync();
    const T Lt = block_objective<T, KC, G, PPL>(q, grp, pt, xt, Z, Z.dt, nc);
    const bool valid = Lt < Num<T>::inf();
    if (valid && (trust || Lt < L)) {
#pragma unroll
      for (int j = 0; j < PPL; ++j)
#pragma unroll
        for (int u = 0; u < 3; ++u) dp[j][u] = xt[j][u];
      if (gl < n_u) Z.d[gl / 6][gl % 6] = Z.dt[gl / 6][gl % 6];
      L = Lt;  // Eq. (14) at the accepted point, trusted step or not
      const T lr = Num<T>::tenth(lambda);
      lambda = lr > q.lambda_min ? lr : q.lambda_min;
    } else {
      lambda *= T(10);
    }
    grp.sync();
  }
  bool finite = true;
#pragma unroll
  for (int j = 0; j < PPL; ++j)
    if (pt[j].act) {
      const long long pc = (long long)bi.p0 + gl + G * j;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        pdel[u * B.n_pc + pc] = dp[j][u];
        finite = finite && isfinite(dp[j][u]);
      }
    }
  if (gl < n_u) {
    const T v = Z.d[gl / 6][gl % 6];
    cdel[(gl % 6) * B.n_cc + bi.c0 + gl / 6] = v;
    finite = finite && isfinite(v);
  }
  if (!finite) atomicOr(B.err, 1);
  grp.sync();
}

// ------------------------------------------------------------ one-camera blocks
// A block with a single camera (every block when block_cams = 1; the 8-lane class always)
// has a 6 x 6 reduced camera system.  Each lane forms the terms of its point copies (each
// holds the block's one observation of its point); a reduce-scatter over the group sums
// them into a small per-group buffer that every lane reads back (butterflies in groups of
// one or two lanes, where a butterfly stage adds the same two partial sums on both lanes
// of a pair), so all lanes hold the same bits, factor the system in registers and take the
// same step, acceptance and damping.  Same arithmetic as solve_block: points eliminated by their 3x3 inverses,
// Schur weights Q = 2w I - (2w)^2 A W_p A^T, right-hand side sum B^T U - g_c.
template <typename T, int G, int PPL>
struct OneCam {
  const Grp<G>& grp;
  const Prm<T>& q;
  T cb[6], ca[6];                    // camera consensus and scaled dual
  bool act[PPL];
  T xb[PPL][3], ax[PPL][3], z0[PPL], z1[PPL];
  __device__ OneCam(const Grp<G>& g, const Prm<T>& qq) : grp(g), q(qq) {}

  // Eq. (14) at point offsets dp and camera offset dc, summed over the group; +inf when an
  // observation is behind the camera
  __device__ T objective(const T (&dp)[PPL][3], const T (&dc)[6]) const {
    T s = 0;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < PPL; ++j) {
      if (!act[j]) continue;
      T v[9];
#pragma unroll
      for (int u = 0; u < 3; ++u) v[u] = xb[j][u] + dp[j][u];
#pragma unroll
      for (int u = 0; u < 6; ++u) v[3 + u] = cb[u] + dc[u];
      Pose<T> P;
      pose_at(v, q.eps, P);
      if (!P.valid) {
        ok = false;
      } else {
        const T iz = Num<T>::rcp(P.p[2]);
        const T e0 = z0[j] - (q.focal * P.p[0] * iz + q.cx);
        const T e1 = z1[j] - (q.focal * P.p[1] * iz + q.cy);
        s += misfit<T>(q.loss, q.lp, e0 * e0 + e1 * e1);
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) s += q.rho_x * dp[j][u] * (ax[j][u] + T(0.5) * dp[j][u]);
    }
    s = grp.sum(s);
    ok = grp.all(ok);
    T sc = 0;
#pragma unroll
    for (int u = 0; u < 6; ++u) sc += q.rho(3 + u) * dc[u] * (ca[u] + T(0.5) * dc[u]);
    return ok ? s + sc : Num<T>::inf();
  }
};

// L1 prefetch of the copy rows of block nb (the group's next block), so that its start
// does not wait on them: offsets and duals of its point copies (one per lane), their point
// and observation indices, and its camera copy's rows.
template <typename T, int G>
__device__ __forceinline__ void prefetch_block(const BlockProblem& B, const BlockInfo& nb, int gl) {
  const T* pdel = static_cast<const T*>(B.pc_delta);
  const T* cdel = static_cast<const T*>(B.cc_delta);
  if (gl < nb.np) {
    const long long pc = (long long)nb.p0 + gl;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      asm volatile("prefetch.global.L1 [%0];" ::"l"(pdel + u * B.n_pc + pc));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(B.pc_a + u * B.n_pc + pc));
    }
    asm volatile("prefetch.global.L1 [%0];" ::"l"(B.pc_pt + pc));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(B.pc_obs + pc));
  }
  for (int u = gl; u < 6; u += G) {
    const long long cc = nb.c0;
    asm volatile("prefetch.global.L1 [%0];" ::"l"(cdel + u * B.n_cc + cc));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(B.cc_a + u * B.n_cc + cc));
    if (u == 0) asm volatile("prefetch.global.L1 [%0];" ::"l"(B.cc_cam + cc));
  }
}

template <typename T, int G>
__device__ void solve_block_1cam(const BlockProblem& B, const Prm<T>& q, const BlockInfo& bi, const Grp<G>& grp,
                                 int cur, const BlockInfo* next, T* red) {
  constexpr int PPL = 1;  // one point copy per lane (blocks of at most 32 points)
  using V2 = typename Num<T>::V2;
  const int gl = grp.gl, np = bi.np;
  T* pdel = static_cast<T*>(B.pc_delta);
  T* cdel = static_cast<T*>(B.cc_delta);
  OneCam<T, G, PPL> K(grp, q);
  T cd[6], dp[PPL][3];
  const long long cc = bi.c0;
  {
    // every lane forms the camera's six coordinates (the same bits); lane u mod G writes back
    // the deferred dual ascent of coordinate u
    const int jc = B.cc_cam[cc];
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const T off = cdel[u * B.n_cc + cc];
      const T ch = static_cast<const T*>(B.DY)[6 * (long long)jc + u];
      K.cb[u] = static_cast<const T*>(B.Ym)[6 * (long long)jc + u];
      const double a = B.cc_a[u * B.n_cc + cc];
      if (B.pending) {
        cd[u] = off + ch;
        const double an = a + to_f64<T>(cd[u]);
        if (gl == u % G) B.cc_a[u * B.n_cc + cc] = an;
        K.ca[u] = from_f64<T>(an);
      } else {
        cd[u] = off;
        K.ca[u] = from_f64<T>(a);
      }
    }
  }
  const long long pc = (long long)bi.p0 + gl;
  K.act[0] = gl < np;
  K.z0[0] = K.z1[0] = 0;
#pragma unroll
  for (int u = 0; u < 3; ++u) K.xb[0][u] = K.ax[0][u] = dp[0][u] = 0;
  if (K.act[0]) {
    const int i = B.pc_pt[pc];
#pragma unroll
    for (int u = 0; u < 3; ++u)
      deferred_ascent<T>(B, static_cast<const T*>(B.Xm)[3 * (long long)i + u],
                         static_cast<const T*>(B.DX)[3 * (long long)i + u], pdel[u * B.n_pc + pc],
                         B.pc_a + u * B.n_pc + pc, K.xb[0][u], dp[0][u], K.ax[0][u]);
    const V2 z = static_cast<const V2*>(B.z)[B.pc_obs[pc]];  // the copy's one observation
    K.z0[0] = z.x;
    K.z1[0] = z.y;
  }
  if (next) prefetch_block<T, G>(B, *next, gl);
  T L = K.objective(dp, cd);
  T lambda = T(-1);
  for (int step = 0; step < q.steps; ++step) {
    // linearisation of this lane's observation at the current copies
    T J0[9], J1[9], tw = 0, e0 = 0, e1 = 0;
    {
      T v[9], w = 0;
#pragma unroll
      for (int u = 0; u < 3; ++u) v[u] = K.xb[0][u] + dp[0][u];
#pragma unroll
      for (int u = 0; u < 6; ++u) v[3 + u] = K.cb[u] + cd[u];
      Pose<T> P;
      pose_at(v, q.eps, P);
      if (K.act[0] && P.valid) {
        linearize(P, K.z0[0], K.z1[0], q, J0, J1, e0, e1, w);
      } else {
#pragma unroll
        for (int u = 0; u < 9; ++u) J0[u] = J1[u] = 0;
      }
      tw = T(2) * w;
    }
    // point block of H, point gradient, camera misfit gradient, noise scale
    const T h00 = tw * (J0[0] * J0[0] + J1[0] * J1[0]), h01 = tw * (J0[0] * J0[1] + J1[0] * J1[1]),
            h02 = tw * (J0[0] * J0[2] + J1[0] * J1[2]), h11 = tw * (J0[1] * J0[1] + J1[1] * J1[1]),
            h12 = tw * (J0[1] * J0[2] + J1[1] * J1[2]), h22 = tw * (J0[2] * J0[2] + J1[2] * J1[2]);
    T gp[3], gc[6];
#pragma unroll
    for (int u = 0; u < 3; ++u)
      gp[u] = K.act[0] ? -tw * (J0[u] * e0 + J1[u] * e1) + q.rho_x * (K.ax[0][u] + dp[0][u]) : T(0);
#pragma unroll
    for (int u = 0; u < 6; ++u) gc[u] = -tw * (J0[3 + u] * e0 + J1[3 + u] * e1);
    T noise = tw * Num<T>::sqrt_(e0 * e0 + e1 * e1) * (fabs(K.z0[0]) + fabs(K.z1[0]));
    if (lambda < T(0)) {
      T trc = K.act[0] ? h00 + h11 + h22 + T(3) * q.rho_x : T(0);
#pragma unroll
      for (int u = 3; u < 9; ++u) trc += tw * (J0[u] * J0[u] + J1[u] * J1[u]);
      T tr = grp.sum(trc);
#pragma unroll
      for (int u = 0; u < 6; ++u) tr += q.rho(3 + u);
      lambda = q.lambda0 * tr / T(3 * np + 6);
    }
    // W_p = (H_pp + (rho_x + lambda) I)^-1 by cofactors
    T w6[6];
    {
      const T dg = q.rho_x + lambda;
      const T a00 = h00 + dg, a11 = h11 + dg, a22 = h22 + dg;
      const T c00 = a11 * a22 - h12 * h12, c01 = h02 * h12 - h01 * a22, c02 = h01 * h12 - h02 * a11;
      const T c11 = a00 * a22 - h02 * h02, c12 = h01 * h02 - a00 * h12, c22 = a00 * a11 - h01 * h01;
      const T idet = Num<T>::rcp(a00 * c00 + h01 * c01 + h02 * c02);
      w6[0] = c00 * idet, w6[1] = c01 * idet, w6[2] = c02 * idet;
      w6[3] = c11 * idet, w6[4] = c12 * idet, w6[5] = c22 * idet;
    }
    // this point's terms of the reduced camera system: S += B^T Q B, rhs += B^T U
    T S[21], rhs[6];
    {
      const T Wg0 = w6[0] * gp[0] + w6[1] * gp[1] + w6[2] * gp[2];
      const T Wg1 = w6[1] * gp[0] + w6[3] * gp[1] + w6[4] * gp[2];
      const T Wg2 = w6[2] * gp[0] + w6[4] * gp[1] + w6[5] * gp[2];
      const T w0 = w6[0] * J0[0] + w6[1] * J0[1] + w6[2] * J0[2], w1 = w6[1] * J0[0] + w6[3] * J0[1] + w6[4] * J0[2],
              w2 = w6[2] * J0[0] + w6[4] * J0[1] + w6[5] * J0[2];
      const T x0 = w6[0] * J1[0] + w6[1] * J1[1] + w6[2] * J1[2], x1 = w6[1] * J1[0] + w6[3] * J1[1] + w6[4] * J1[2],
              x2 = w6[2] * J1[0] + w6[4] * J1[1] + w6[5] * J1[2];
      const T sw = tw * tw;
      const T q00 = tw - sw * (J0[0] * w0 + J0[1] * w1 + J0[2] * w2);
      const T q01 = -sw * (J0[0] * x0 + J0[1] * x1 + J0[2] * x2);
      const T q10 = -sw * (J1[0] * w0 + J1[1] * w1 + J1[2] * w2);
      const T q11 = tw - sw * (J1[0] * x0 + J1[1] * x1 + J1[2] * x2);
      const T U0 = tw * (J0[0] * Wg0 + J0[1] * Wg1 + J0[2] * Wg2);
      const T U1 = tw * (J1[0] * Wg0 + J1[1] * Wg1 + J1[2] * Wg2);
      int e = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        const T b0r = J0[3 + r], b1r = J1[3 + r];
#pragma unroll
        for (int c = r; c < 6; ++c, ++e) S[e] = b0r * (q00 * J0[3 + c] + q01 * J1[3 + c]) +
                                                b1r * (q10 * J0[3 + c] + q11 * J1[3 + c]);
        rhs[r] = b0r * U0 + b1r * U1;
      }
    }
    // sums over the block's points (every lane receives the same bits): in groups of 4 or
    // more lanes a reduce-scatter of the 34 values, G at a time, into the group's buffer,
    // read back by every lane; below that butterflies
    if constexpr (G >= 4) {
      constexpr int kV = 34, kC = (kV + G - 1) / G;
      T vals[kC * G];
#pragma unroll
      for (int e = 0; e < 21; ++e) vals[e] = S[e];
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        vals[21 + u] = rhs[u];
        vals[27 + u] = gc[u];
      }
      vals[33] = noise;
#pragma unroll
      for (int e = kV; e < kC * G; ++e) vals[e] = 0;
#pragma unroll
      for (int k = 0; k < kC; ++k) {
        T v[G];
#pragma unroll
        for (int i = 0; i < G; ++i) v[i] = vals[k * G + i];
        const T sum = reduce_scatter<T, G>(v, grp);
        if (k * G + grp.gl < kV) red[k * G + grp.gl] = sum;
      }
      grp.sync();
#pragma unroll
      for (int e = 0; e < 21; ++e) S[e] = red[e];
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        rhs[u] = red[21 + u];
        gc[u] = red[27 + u] + q.rho(3 + u) * (K.ca[u] + cd[u]);  // camera gradient with its penalty
      }
      noise = red[33];
      grp.sync();  // the buffer is free for the next step
    } else {
#pragma unroll
      for (int e = 0; e < 21; ++e) S[e] = grp.sum(S[e]);
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        rhs[u] = grp.sum(rhs[u]);
        gc[u] = grp.sum(gc[u]) + q.rho(3 + u) * (K.ca[u] + cd[u]);  // camera gradient with its penalty
      }
      noise = grp.sum(noise);
    }
    // (S + diag(rho_c) + lambda I) dy = rhs - g_c by a Cholesky factorisation in registers
    T A[6][6];
    {
      int e = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c, ++e) A[r][c] = A[c][r] = S[e];
    }
#pragma unroll
    for (int u = 0; u < 6; ++u) A[u][u] += q.rho(3 + u) + lambda;
    bool spd = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
      for (int m = 0; m < k; ++m) A[k][k] -= A[k][m] * A[k][m];
      spd = spd && A[k][k] > T(0);
      const T lkk = Num<T>::sqrt_(A[k][k]);
      A[k][k] = lkk;
      const T ilkk = Num<T>::rcp(lkk);
#pragma unroll
      for (int i2 = k + 1; i2 < 6; ++i2) {
#pragma unroll
        for (int m = 0; m < k; ++m) A[i2][k] -= A[i2][m] * A[k][m];
        A[i2][k] *= ilkk;
      }
    }
    if (!spd) {
      lambda *= T(10);
      continue;
    }
    T dy[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      T y = rhs[k] - gc[k];
#pragma unroll
      for (int m = 0; m < k; ++m) y -= A[k][m] * dy[m];
      dy[k] = Num<T>::div(y, A[k][k]);
    }
#pragma unroll
    for (int k = 5; k >= 0; --k) {
      T y = dy[k];
#pragma unroll
      for (int m = k + 1; m < 6; ++m) y -= A[m][k] * dy[m];
      dy[k] = Num<T>::div(y, A[k][k]);
    }
    // point step dx = -W_p (g_p + 2w A^T B dy); predicted decrease (lambda |d|^2 - g.d) / 2
    T xt[PPL][3], gd = 0, dd = 0;
    {
      T bd0 = 0, bd1 = 0;
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        bd0 += J0[3 + u] * dy[u];
        bd1 += J1[3 + u] * dy[u];
      }
      T t3[3], dx[3] = {0, 0, 0};
#pragma unroll
      for (int u = 0; u < 3; ++u) t3[u] = gp[u] + tw * (J0[u] * bd0 + J1[u] * bd1);
      if (K.act[0]) {
        dx[0] = -(w6[0] * t3[0] + w6[1] * t3[1] + w6[2] * t3[2]);
        dx[1] = -(w6[1] * t3[0] + w6[3] * t3[1] + w6[4] * t3[2]);
        dx[2] = -(w6[2] * t3[0] + w6[4] * t3[1] + w6[5] * t3[2]);
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        gd += gp[u] * dx[u];
        dd += dx[u] * dx[u];
        xt[0][u] = dp[0][u] + dx[u];
      }
    }
    gd = grp.sum(gd);
    dd = grp.sum(dd);
    T ct[6];
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      gd += gc[u] * dy[u];
      dd += dy[u] * dy[u];
      ct[u] = cd[u] + dy[u];
    }
    const T pred = T(0.5) * (lambda * dd - gd);
    const bool trust = isfinite(L) && q.model_tol > T(0) &&
                       pred <= q.model_tol * Num<T>::unit_roundoff * (fabs(L) + noise);
    const T Lt = K.objective(xt, ct);
    if (Lt < Num<T>::inf() && (trust || Lt < L)) {
#pragma unroll
      for (int u = 0; u < 3; ++u) dp[0][u] = xt[0][u];
#pragma unroll
      for (int u = 0; u < 6; ++u) cd[u] = ct[u];
      L = Lt;  // Eq. (14) at the accepted point, trusted step or not
      const T lr = Num<T>::tenth(lambda);
      lambda = lr > q.lambda_min ? lr : q.lambda_min;
    } else {
      lambda *= T(10);
    }
  }
  bool finite = true;
  if (K.act[0]) {
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      pdel[u * B.n_pc + pc] = dp[0][u];
      finite = finite && isfinite(dp[0][u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 6; ++u)
    if (gl == u % G) {
      cdel[u * B.n_cc + cc] = cd[u];
      finite = finite && isfinite(cd[u]);
    }
  if (!finite) atomicOr(B.err, 1);
}

// One-camera blocks [lo, hi) of one size class, one group of G lanes per block.
template <typename T, int G>
__global__ void __launch_bounds__(kBlkWarps * 32)
    block_solve_1cam_kernel(BlockProblem B, Prm<T> q, int cur, int lo, int hi) {
  constexpr int kPer = 32 / G;
  __shared__ T red[kBlkWarps * kPer][G >= 4 ? 36 : 1];  // each group's sums (groups of >= 4 lanes)
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const Grp<G> grp(threadIdx.x & 31);
  const int stride = gridDim.x * warps * kPer;
  int b = lo + (blockIdx.x * warps + warp) * kPer + grp.base / G;
  BlockInfo bi{};
  if (b < hi) bi = B.blocks[b];
  for (; b < hi; b += stride) {
    // the next block's record is loaded now and its rows prefetched once this block's own
    // loads are in, so that both arrive while this block is solved
    const bool more = b + stride < hi;
    BlockInfo nb{};
    if (more) nb = B.blocks[b + stride];
    solve_block_1cam<T, G>(B, q, bi, grp, cur, more ? &nb : nullptr, red[warp * kPer + grp.base / G]);
    bi = nb;
  }
}

// ------------------------------------------------------------ one-point blocks
// A block of one point and nc <= 4 cameras (one observation per camera) has 3 + 6 nc unknowns.
// One thread solves it by eliminating the cameras instead of the point: each camera's block
// of the damped normal matrix is diagonal plus rank 2 (its one observation), so it is
// inverted through its 2 x 2 capacitance matrix (Sherman-Morrison-Woodbury, as the
// per-observation solve does), which leaves a 3 x 3 system for the point.  Same damped
// normal equations, damping start, acceptance and noise rules as the other block solves.
template <typename T>
struct PointCam {
  T vbar[6], a[6], z0, z1;
};

// y = (D + tw B^T B)^-1 v with D = diag(iD)^-1 (iD: the inverse diagonal) and B the 2 x 6
// camera rows: D^-1 v - tw D^-1 B^T S^-1 B D^-1 v, S = I + tw B D^-1 B^T (det >= 1)
template <typename T>
__device__ __forceinline__ void cam_block_solve(const T (&iD)[6], const T (&Bc)[2][6], T tw, const T (&v)[6],
                                                T (&y)[6]) {
  T s00 = 0, s01 = 0, s11 = 0, t0 = 0, t1 = 0;
#pragma unroll
  for (int u = 0; u < 6; ++u) {
    const T q = iD[u] * v[u];
    y[u] = q;
    s00 += Bc[0][u] * iD[u] * Bc[0][u];
    s01 += Bc[0][u] * iD[u] * Bc[1][u];
    s11 += Bc[1][u] * iD[u] * Bc[1][u];
    t0 += Bc[0][u] * q;
    t1 += Bc[1][u] * q;
  }
  const T S00 = T(1) + tw * s00, S01 = tw * s01, S11 = T(1) + tw * s11;
  const T idet = Num<T>::rcp(S00 * S11 - S01 * S01);
  const T w0 = (S11 * t0 - S01 * t1) * idet, w1 = (S00 * t1 - S01 * t0) * idet;
#pragma unroll
  for (int u = 0; u < 6; ++u) y[u] -= tw * iD[u] * (Bc[0][u] * w0 + Bc[1][u] * w1);
}

template <typename T>
__device__ void solve_block_point(const BlockProblem& B, const Prm<T>& q, const BlockInfo& bi) {
  constexpr int KC = 4;  // most cameras of a block
  using V2 = typename Num<T>::V2;
  const int nc = bi.nc, n_u = 6 * nc;
  T* pdel = static_cast<T*>(B.pc_delta);
  T* cdel = static_cast<T*>(B.cc_delta);
  PointCam<T> C[KC];
  T cd[KC][6];  // camera offsets
  bool has[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    has[c] = c < nc;
#pragma unroll
    for (int u = 0; u < 6; ++u) C[c].vbar[u] = cd[c][u] = C[c].a[u] = 0;
    C[c].z0 = C[c].z1 = 0;
    if (has[c]) {
      const long long cc = (long long)bi.c0 + c;
      const int j = B.cc_cam[cc];
#pragma unroll
      for (int u = 0; u < 6; ++u)
        deferred_ascent<T>(B, static_cast<const T*>(B.Ym)[6 * (long long)j + u],
                           static_cast<const T*>(B.DY)[6 * (long long)j + u], cdel[u * B.n_cc + cc],
                           B.cc_a + u * B.n_cc + cc, C[c].vbar[u], cd[c][u], C[c].a[u]);
    }
  }
  const long long pc = bi.p0;
  T xb[3], ax[3], dp[3];
  {
    const int i = B.pc_pt[pc];
#pragma unroll
    for (int u = 0; u < 3; ++u)
      deferred_ascent<T>(B, static_cast<const T*>(B.Xm)[3 * (long long)i + u],
                         static_cast<const T*>(B.DX)[3 * (long long)i + u], pdel[u * B.n_pc + pc],
                         B.pc_a + u * B.n_pc + pc, xb[u], dp[u], ax[u]);
    // one observation per camera of the block
    const int ob0 = B.pc_obs[pc], nob = B.pc_obs[pc + 1] - ob0;
    const V2* zz = static_cast<const V2*>(B.z);
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k < nob) {
        const int c = B.obs_lc[ob0 + k];
        const V2 z = zz[ob0 + k];
#pragma unroll
        for (int s = 0; s < KC; ++s)
          if (c == s) {
            C[s].z0 = z.x;
            C[s].z1 = z.y;
          }
      }
  }
  // Eq. (14) at point offset p and camera offsets dc; +inf when an observation is behind its camera
  auto objective = [&](const T (&p)[3], const T (&dc)[KC][6]) -> T {
    T s = 0;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      if (!has[c]) continue;
      T v[9];
#pragma unroll
      for (int u = 0; u < 3; ++u) v[u] = xb[u] + p[u];
#pragma unroll
      for (int u = 0; u < 6; ++u) v[3 + u] = C[c].vbar[u] + dc[c][u];
      Pose<T> P;
      pose_at(v, q.eps, P);
      if (!P.valid) {
        ok = false;
      } else {
        const T iz = Num<T>::rcp(P.p[2]);
        const T e0 = C[c].z0 - (q.focal * P.p[0] * iz + q.cx);
        const T e1 = C[c].z1 - (q.focal * P.p[1] * iz + q.cy);
        s += misfit<T>(q.loss, q.lp, e0 * e0 + e1 * e1);
      }
#pragma unroll
      for (int u = 0; u < 6; ++u) s += q.rho(3 + u) * dc[c][u] * (C[c].a[u] + T(0.5) * dc[c][u]);
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) s += q.rho_x * p[u] * (ax[u] + T(0.5) * p[u]);
    return ok ? s : Num<T>::inf();
  };
  T L = objective(dp, cd);
  T lambda = T(-1);
  for (int step = 0; step < q.steps; ++step) {
    // linearisation of each observation (camera slots without one, or behind the camera: zero)
    T Ap[KC][2][3], Bc[KC][2][6], tw[KC], gc[KC][6];
    T h[6] = {0, 0, 0, 0, 0, 0}, gx[3] = {0, 0, 0}, trc = 0, noise = 0;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      T J0[9], J1[9], e0 = 0, e1 = 0, w = 0;
      bool lin = false;
      if (has[c]) {
        T v[9];
#pragma unroll
        for (int u = 0; u < 3; ++u) v[u] = xb[u] + dp[u];
#pragma unroll
        for (int u = 0; u < 6; ++u) v[3 + u] = C[c].vbar[u] + cd[c][u];
        Pose<T> P;
        pose_at(v, q.eps, P);
        if (P.valid) {
          linearize(P, C[c].z0, C[c].z1, q, J0, J1, e0, e1, w);
          lin = true;
        }
      }
      if (!lin) {
#pragma unroll
        for (int u = 0; u < 9; ++u) J0[u] = J1[u] = 0;
        e0 = e1 = w = 0;
      }
      const T t = T(2) * w;
      tw[c] = t;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        Ap[c][0][u] = J0[u];
        Ap[c][1][u] = J1[u];
      }
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        Bc[c][0][u] = J0[3 + u];
        Bc[c][1][u] = J1[3 + u];
        gc[c][u] = -t * (J0[3 + u] * e0 + J1[3 + u] * e1) + (has[c] ? q.rho(3 + u) * (C[c].a[u] + cd[c][u]) : T(0));
      }
      h[0] += t * (J0[0] * J0[0] + J1[0] * J1[0]);
      h[1] += t * (J0[0] * J0[1] + J1[0] * J1[1]);
      h[2] += t * (J0[0] * J0[2] + J1[0] * J1[2]);
      h[3] += t * (J0[1] * J0[1] + J1[1] * J1[1]);
      h[4] += t * (J0[1] * J0[2] + J1[1] * J1[2]);
      h[5] += t * (J0[2] * J0[2] + J1[2] * J1[2]);
#pragma unroll
      for (int u = 0; u < 3; ++u) gx[u] -= t * (J0[u] * e0 + J1[u] * e1);
#pragma unroll
      for (int u = 3; u < 9; ++u) trc += t * (J0[u] * J0[u] + J1[u] * J1[u]);
      noise += t * Num<T>::sqrt_(e0 * e0 + e1 * e1) * (fabs(C[c].z0) + fabs(C[c].z1));
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) gx[u] += q.rho_x * (ax[u] + dp[u]);
    if (lambda < T(0)) {
      T tr = trc + h[0] + h[3] + h[5] + T(3) * q.rho_x;
      for (int c = 0; c < nc; ++c)
#pragma unroll
        for (int u = 0; u < 6; ++u) tr += q.rho(3 + u);
      lambda = q.lambda0 * tr / T(3 + n_u);
    }
    // cameras eliminated: S = H_xx - sum_c H_xc H_cc^-1 H_cx, r = -g_x + sum_c H_xc H_cc^-1 g_c,
    // with H_cx = 2w B^T A (6 x 3) and H_cc = diag(rho_c) + lambda I + 2w B^T B
    T iD[6];
#pragma unroll
    for (int u = 0; u < 6; ++u) iD[u] = Num<T>::rcp(q.rho(3 + u) + lambda);
    T S[6], r[3];
    {
      const T dg = q.rho_x + lambda;
      S[0] = h[0] + dg, S[1] = h[1], S[2] = h[2], S[3] = h[3] + dg, S[4] = h[4], S[5] = h[5] + dg;
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) r[u] = -gx[u];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      if (!has[c]) continue;
      // H_xc = 2w A^T B (its rows hx[k] = columns of H_cx); M_k = H_cc^-1 H_cx[:, k],
      // m = H_cc^-1 g_c; S -= H_xc M, r += H_xc m
      T hx[3][6], Mk[3][6], m[6];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int u = 0; u < 6; ++u) hx[k][u] = tw[c] * (Ap[c][0][k] * Bc[c][0][u] + Ap[c][1][k] * Bc[c][1][u]);
        cam_block_solve<T>(iD, Bc[c], tw[c], hx[k], Mk[k]);
      }
      cam_block_solve<T>(iD, Bc[c], tw[c], gc[c], m);
      T p00 = 0, p01 = 0, p02 = 0, p11 = 0, p12 = 0, p22 = 0, q0 = 0, q1 = 0, q2 = 0;
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        p00 += hx[0][u] * Mk[0][u];
        p01 += hx[0][u] * Mk[1][u];
        p02 += hx[0][u] * Mk[2][u];
        p11 += hx[1][u] * Mk[1][u];
        p12 += hx[1][u] * Mk[2][u];
        p22 += hx[2][u] * Mk[2][u];
        q0 += hx[0][u] * m[u];
        q1 += hx[1][u] * m[u];
        q2 += hx[2][u] * m[u];
      }
      S[0] -= p00, S[1] -= p01, S[2] -= p02, S[3] -= p11, S[4] -= p12, S[5] -= p22;
      r[0] += q0, r[1] += q1, r[2] += q2;
    }
    // the point step by cofactors (S symmetric positive definite when H is)
    const T c00 = S[3] * S[5] - S[4] * S[4], c01 = S[2] * S[4] - S[1] * S[5], c02 = S[1] * S[4] - S[2] * S[3];
    const T c11 = S[0] * S[5] - S[2] * S[2], c12 = S[1] * S[2] - S[0] * S[4], c22 = S[0] * S[3] - S[1] * S[1];
    const T det = S[0] * c00 + S[1] * c01 + S[2] * c02;
    if (!(det > T(0)) || !(S[0] > T(0)) || !(c22 > T(0))) {
      lambda *= T(10);
      continue;
    }
    const T idet = Num<T>::rcp(det);
    T dx[3];
    dx[0] = (c00 * r[0] + c01 * r[1] + c02 * r[2]) * idet;
    dx[1] = (c01 * r[0] + c11 * r[1] + c12 * r[2]) * idet;
    dx[2] = (c02 * r[0] + c12 * r[1] + c22 * r[2]) * idet;
    // camera steps dy_c = -H_cc^-1 (g_c + H_cx dx); predicted decrease (lambda |d|^2 - g.d) / 2
    T gd = gx[0] * dx[0] + gx[1] * dx[1] + gx[2] * dx[2], dd = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    T xt[3], ct[KC][6];
#pragma unroll
    for (int u = 0; u < 3; ++u) xt[u] = dp[u] + dx[u];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      T v[6], y[6];
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        const T a0 = Ap[c][0][0] * dx[0] + Ap[c][0][1] * dx[1] + Ap[c][0][2] * dx[2];
        const T a1 = Ap[c][1][0] * dx[0] + Ap[c][1][1] * dx[1] + Ap[c][1][2] * dx[2];
        v[u] = gc[c][u] + tw[c] * (Bc[c][0][u] * a0 + Bc[c][1][u] * a1);
      }
      cam_block_solve<T>(iD, Bc[c], tw[c], v, y);
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        const T dy = has[c] ? -y[u] : T(0);
        gd += gc[c][u] * dy;
        dd += dy * dy;
        ct[c][u] = cd[c][u] + dy;
      }
    }
    const T pred = T(0.5) * (lambda * dd - gd);
    const bool trust = isfinite(L) && q.model_tol > T(0) &&
                       pred <= q.model_tol * Num<T>::unit_roundoff * (fabs(L) + noise);
    const T Lt = objective(xt, ct);
    if (Lt < Num<T>::inf() && (trust || Lt < L)) {
#pragma unroll
      for (int u = 0; u < 3; ++u) dp[u] = xt[u];
#pragma unroll
      for (int c = 0; c < KC; ++c)
#pragma unroll
        for (int u = 0; u < 6; ++u) cd[c][u] = ct[c][u];
      L = Lt;  // Eq. (14) at the accepted point, trusted step or not
      const T lr = Num<T>::tenth(lambda);
      lambda = lr > q.lambda_min ? lr : q.lambda_min;
    } else {
      lambda *= T(10);
    }
  }
  bool finite = true;
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    pdel[u * B.n_pc + pc] = dp[u];
    finite = finite && isfinite(dp[u]);
  }
#pragma unroll
  for (int c = 0; c < KC; ++c)
    if (has[c])
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        cdel[u * B.n_cc + bi.c0 + c] = cd[c][u];
        finite = finite && isfinite(cd[c][u]);
      }
  if (!finite) atomicOr(B.err, 1);
}

// One-point blocks [lo, hi), one thread per block.
template <typename T>
__global__ void __launch_bounds__(kBlkWarps * 32, (sizeof(T) == 4 ? 2 : 1))
    block_solve_point_kernel(BlockProblem B, Prm<T> q, int cur, int lo, int hi) {
  for (long long b = lo + blockIdx.x * (long long)blockDim.x + threadIdx.x; b < hi;
       b += (long long)gridDim.x * blockDim.x)
    solve_block_point<T>(B, q, B.blocks[b]);
}

// ------------------------------------------------------------ blocks of two or four cameras
// A block with at most KC cameras (KC = 2 or 4) and at most G <= 32 points has a reduced camera
// system of at most 6 KC x 6 KC.  Each lane keeps its point copy's linearisation in registers
// (at most one observation per camera) and forms its terms of the whole system: the 6 x 6
// blocks of B^T Q B, the right-hand side B^T U and the camera misfit gradient.  A
// reduce-scatter over the group (recursive halving) sums them, G values at a time, so that each
// value passes through one shuffle instead of log2(G); lane i receives the sum of value i and
// writes it into the group's system in shared memory.  The system is then factored in
// registers, a row per lane (6 KC / G rows a lane below 6 KC lanes), pivots and columns by
// shuffles.  Same arithmetic as solve_block; the sums run in another order.
template <typename T, int KC>
struct CamShared {
  // the reduced camera system's upper triangle S(row <= col) at kLd row + col, then the
  // right-hand side sums B^T U, the camera misfit gradients and the rounding-noise scale
  static constexpr int kN = 6 * KC, kLd = kN + 1;
  static constexpr int kRhs = kN * kLd, kG = kRhs + kN, kNoise = kG + kN, kSys = kNoise + 1;
  T sys[kSys];
  T vbar[KC][6];
  T d[KC][6];
  T dt[KC][6];
  T a[KC][6];
};

// The values one lane contributes to the reduced system, in this order: the upper triangles
// of the KC diagonal 6 x 6 blocks (21 each), the off-diagonal blocks of the camera pairs
// c1 < c2 (36 each, row-major), the right-hand sides B^T U (6 per camera), the camera misfit
// gradients (6 per camera) and the rounding-noise scale; the rest of the last group of G is zero.
template <int KC>
__host__ __device__ constexpr int sys_values() {
  return 21 * KC + 36 * (KC * (KC - 1) / 2) + 12 * KC + 1;
}

struct SysEntry {
  int kind;  // 0: S(row, col), 1: rhs(row), 2: g(row), 3: noise, 4: none
  int row, col;
};

template <int KC>
__host__ __device__ constexpr SysEntry sys_entry(int e) {
  if (e < 21 * KC) {
    const int c = e / 21;
    int t = e - 21 * c, r = 0;
    while (t >= 6 - r) {
      t -= 6 - r;
      ++r;
    }
    return SysEntry{0, 6 * c + r, 6 * c + r + t};
  }
  e -= 21 * KC;
  for (int c1 = 0; c1 < KC; ++c1)
    for (int c2 = c1 + 1; c2 < KC; ++c2) {
      if (e < 36) return SysEntry{0, 6 * c1 + e / 6, 6 * c2 + e % 6};
      e -= 36;
    }
  if (e < 6 * KC) return SysEntry{1, e, 0};
  e -= 6 * KC;
  if (e < 6 * KC) return SysEntry{2, e, 0};
  e -= 6 * KC;
  return e == 0 ? SysEntry{3, 0, 0} : SysEntry{4, 0, 0};
}

// where value e lands in CamShared::sys, or -1
template <int KC>
__host__ __device__ constexpr int sys_dst(int e) {
  using Sh = CamShared<float, KC>;
  const SysEntry se = sys_entry<KC>(e);
  return se.kind == 0   ? Sh::kLd * se.row + se.col
         : se.kind == 1 ? Sh::kRhs + se.row
         : se.kind == 2 ? Sh::kG + se.row
         : se.kind == 3 ? Sh::kNoise
                        : -1;
}

// index of the camera pair c1 <= c2 among the KC (KC + 1) / 2 pairs
__host__ __device__ constexpr int cam_pair(int KC, int c1, int c2) {
  return c1 * KC - c1 * (c1 - 1) / 2 + (c2 - c1);
}


// One lane's terms of the reduced system: the camera rows B_c of its observations' Jacobians,
// U_c, the Schur weights Q of the camera pairs, the IRLS weights 2w_c, the residuals and the
// rounding-noise scale (camera slots without an observation: zero).
template <typename T, int KC>
struct SysTerms {
  T Bc[KC][2][6], U[KC][2], Q[KC * (KC + 1) / 2][4], tw[KC], ez[KC][2], noise;
};

// value E of the list above, E a compile-time index
template <int E, typename T, int KC>
__device__ __forceinline__ T sys_value(const SysTerms<T, KC>& m) {
  constexpr SysEntry se = sys_entry<KC>(E);
  if constexpr (se.kind == 0) {
    constexpr int c1 = se.row / 6, r = se.row % 6, c2 = se.col / 6, s = se.col % 6, pr = cam_pair(KC, c1, c2);
    const T b10 = m.Bc[c1][0][r], b11 = m.Bc[c1][1][r], b20 = m.Bc[c2][0][s], b21 = m.Bc[c2][1][s];
    return b10 * (m.Q[pr][0] * b20 + m.Q[pr][1] * b21) + b11 * (m.Q[pr][2] * b20 + m.Q[pr][3] * b21);
  } else if constexpr (se.kind == 1) {
    constexpr int c = se.row / 6, r = se.row % 6;
    return m.Bc[c][0][r] * m.U[c][0] + m.Bc[c][1][r] * m.U[c][1];
  } else if constexpr (se.kind == 2) {
    constexpr int c = se.row / 6, r = se.row % 6;
    return -m.tw[c] * (m.Bc[c][0][r] * m.ez[c][0] + m.Bc[c][1][r] * m.ez[c][1]);
  } else if constexpr (se.kind == 3) {
    return m.noise;
  } else {
    return T(0);
  }
}

// values K G ... K G + G - 1: summed over the group, value K G + gl landing on lane gl, which
// writes it to its place in the system (dst: sys_dst of every value, a per-CTA table)
template <typename T, int G, int KC, int K, int... I>
__device__ __forceinline__ void sys_chunk(const SysTerms<T, KC>& m, const Grp<G>& grp, CamShared<T, KC>& Z,
                                          const short* dst, std::integer_sequence<int, I...>) {
  T v[G] = {sys_value<K * G + I, T, KC>(m)...};
  const T sum = reduce_scatter<T, G>(v, grp);
  const int o = dst[K * G + grp.gl];
  if (o >= 0) Z.sys[o] = sum;
}

template <typename T, int G, int KC, int... K>
__device__ __forceinline__ void sys_reduce(const SysTerms<T, KC>& m, const Grp<G>& grp, CamShared<T, KC>& Z,
                                           const short* dst, std::integer_sequence<int, K...>) {
  (sys_chunk<T, G, KC, K>(m, grp, Z, dst, std::make_integer_sequence<int, G>{}), ...);
}

// values padded to whole groups of G lanes (the size of the per-CTA destination table)
template <int KC, int G>
__host__ __device__ constexpr int sys_slots() {
  return (sys_values<KC>() + G - 1) / G * G;
}

// One lane's point copy in a block of at most KC cameras: consensus, scaled dual, its
// observation on each camera slot (has[c]) and the pixels.
template <typename T, int KC>
struct CamPt {
  bool act, has[KC];
  T xb[3], ax[3], z0[KC], z1[KC];

  // Eq. (14) at point offsets dp and camera offsets dc (nc cameras), summed over the group;
  // +inf when an observation is behind its camera
  template <int G>
  __device__ T objective(const Prm<T>& q, const Grp<G>& grp, const T (&dp)[3], const CamShared<T, KC>& Z,
                         const T (*dc)[6], int nc) const {
    T s = 0;
    bool ok = true;
    if (act) {
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        if (!has[c]) continue;
        T v[9];
#pragma unroll
        for (int u = 0; u < 3; ++u) v[u] = xb[u] + dp[u];
#pragma unroll
        for (int u = 0; u < 6; ++u) v[3 + u] = Z.vbar[c][u] + dc[c][u];
        Pose<T> P;
        pose_at(v, q.eps, P);
        if (!P.valid) {
          ok = false;
        } else {
          const T iz = Num<T>::rcp(P.p[2]);
          const T e0 = z0[c] - (q.focal * P.p[0] * iz + q.cx);
          const T e1 = z1[c] - (q.focal * P.p[1] * iz + q.cy);
          s += misfit<T>(q.loss, q.lp, e0 * e0 + e1 * e1);
        }
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) s += q.rho_x * dp[u] * (ax[u] + T(0.5) * dp[u]);
    }
    s = grp.sum(s);
    ok = grp.all(ok);
    T sc = 0;
    for (int c = 0; c < nc; ++c)
#pragma unroll
      for (int u = 0; u < 6; ++u) sc += q.rho(3 + u) * dc[c][u] * (Z.a[c][u] + T(0.5) * dc[c][u]);
    return ok ? s + sc : Num<T>::inf();
  }
};

// L1 prefetch of the copy rows of block nb (the group's next block): its point copies' offsets,
// duals and indices (one per lane) and its camera copies' rows (one coordinate per lane).
template <typename T, int G>
__device__ __forceinline__ void prefetch_block_cams(const BlockProblem& B, const BlockInfo& nb, int gl) {
  const T* pdel = static_cast<const T*>(B.pc_delta);
  const T* cdel = static_cast<const T*>(B.cc_delta);
  if (gl < nb.np) {
    const long long pc = (long long)nb.p0 + gl;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      asm volatile("prefetch.global.L1 [%0];" ::"l"(pdel + u * B.n_pc + pc));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(B.pc_a + u * B.n_pc + pc));
    }
    asm volatile("prefetch.global.L1 [%0];" ::"l"(B.pc_pt + pc));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(B.pc_obs + pc));
  }
  for (int r = gl; r < 6 * nb.nc; r += G) {
    const long long cc = (long long)nb.c0 + r / 6;
    const int u = r % 6;
    asm volatile("prefetch.global.L1 [%0];" ::"l"(cdel + u * B.n_cc + cc));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(B.cc_a + u * B.n_cc + cc));
    if (u == 0) asm volatile("prefetch.global.L1 [%0];" ::"l"(B.cc_cam + cc));
  }
}

template <typename T, int G, int KC>
__device__ void solve_block_cams(const BlockProblem& B, const Prm<T>& q, const BlockInfo& bi, const Grp<G>& grp,
                                 CamShared<T, KC>& Z, const short* dst, const BlockInfo* next) {
  // rows of the camera system held by a lane: gl + G t, t < R
  constexpr int N = 6 * KC, R = (N + G - 1) / G;
  using Sh = CamShared<T, KC>;
  using V2 = typename Num<T>::V2;
  const int gl = grp.gl, np = bi.np, nc = bi.nc, n_u = 6 * nc;
  T* pdel = static_cast<T*>(B.pc_delta);
  T* cdel = static_cast<T*>(B.cc_delta);
  // camera copies: row r = 6 c + u is coordinate u of camera c; absent camera slots are
  // zero, so that the sums over all KC slots below need no test
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int r = gl + G * t;
    if (r < n_u) {
      const int c = r / 6, u = r % 6;
      const long long cc = (long long)bi.c0 + c;
      const int j = B.cc_cam[cc];
      deferred_ascent<T>(B, static_cast<const T*>(B.Ym)[6 * (long long)j + u],
                         static_cast<const T*>(B.DY)[6 * (long long)j + u], cdel[u * B.n_cc + cc],
                         B.cc_a + u * B.n_cc + cc, Z.vbar[c][u], Z.d[c][u], Z.a[c][u]);
    } else if (r < N) {
      Z.vbar[r / 6][r % 6] = Z.d[r / 6][r % 6] = Z.a[r / 6][r % 6] = 0;
    }
  }
  const long long pc = (long long)bi.p0 + gl;
  CamPt<T, KC> K;
  T dp[3];
  K.act = gl < np;
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    K.has[c] = false;
    K.z0[c] = K.z1[c] = 0;
  }
#pragma unroll
  for (int u = 0; u < 3; ++u) K.xb[u] = K.ax[u] = dp[u] = 0;
  if (K.act) {
    const int i = B.pc_pt[pc];
#pragma unroll
    for (int u = 0; u < 3; ++u)
      deferred_ascent<T>(B, static_cast<const T*>(B.Xm)[3 * (long long)i + u],
                         static_cast<const T*>(B.DX)[3 * (long long)i + u], pdel[u * B.n_pc + pc],
                         B.pc_a + u * B.n_pc + pc, K.xb[u], dp[u], K.ax[u]);
    // at most one observation per camera of the block
    const int ob0 = B.pc_obs[pc], nob = B.pc_obs[pc + 1] - ob0;
    const V2* zz = static_cast<const V2*>(B.z);
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k < nob) {
        const int c = B.obs_lc[ob0 + k];
        const V2 z = zz[ob0 + k];
#pragma unroll
        for (int s = 0; s < KC; ++s)
          if (c == s) {
            K.has[s] = true;
            K.z0[s] = z.x;
            K.z1[s] = z.y;
          }
      }
  }
  if (next) prefetch_block_cams<T, G>(B, *next, gl);
  grp.sync();

  T L = K.objective(q, grp, dp, Z, Z.d, nc);
  T lambda = T(-1);
  for (int step = 0; step < q.steps; ++step) {
    // linearisation of this lane's observations (camera slots without one: zero)
    SysTerms<T, KC> m;
    T Ap[KC][2][3];
    T h[6] = {0, 0, 0, 0, 0, 0}, gp[3] = {0, 0, 0}, trc = 0;
    m.noise = 0;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      T J0[9], J1[9], e0 = 0, e1 = 0, w = 0;
      bool lin = false;
      if (K.act && K.has[c]) {
        T v[9];
#pragma unroll
        for (int u = 0; u < 3; ++u) v[u] = K.xb[u] + dp[u];
#pragma unroll
        for (int u = 0; u < 6; ++u) v[3 + u] = Z.vbar[c][u] + Z.d[c][u];
        Pose<T> P;
        pose_at(v, q.eps, P);
        if (P.valid) {
          linearize(P, K.z0[c], K.z1[c], q, J0, J1, e0, e1, w);
          lin = true;
        }
      }
      if (!lin) {
#pragma unroll
        for (int u = 0; u < 9; ++u) J0[u] = J1[u] = 0;
        e0 = e1 = w = 0;
      }
      const T t = T(2) * w;
      m.tw[c] = t;
      m.ez[c][0] = e0;
      m.ez[c][1] = e1;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        Ap[c][0][u] = J0[u];
        Ap[c][1][u] = J1[u];
      }
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        m.Bc[c][0][u] = J0[3 + u];
        m.Bc[c][1][u] = J1[3 + u];
      }
      h[0] += t * (J0[0] * J0[0] + J1[0] * J1[0]);
      h[1] += t * (J0[0] * J0[1] + J1[0] * J1[1]);
      h[2] += t * (J0[0] * J0[2] + J1[0] * J1[2]);
      h[3] += t * (J0[1] * J0[1] + J1[1] * J1[1]);
      h[4] += t * (J0[1] * J0[2] + J1[1] * J1[2]);
      h[5] += t * (J0[2] * J0[2] + J1[2] * J1[2]);
#pragma unroll
      for (int u = 0; u < 3; ++u) gp[u] -= t * (J0[u] * e0 + J1[u] * e1);
#pragma unroll
      for (int u = 3; u < 9; ++u) trc += t * (J0[u] * J0[u] + J1[u] * J1[u]);
      m.noise += t * Num<T>::sqrt_(e0 * e0 + e1 * e1) * (fabs(K.z0[c]) + fabs(K.z1[c]));
    }
    if (K.act)
#pragma unroll
      for (int u = 0; u < 3; ++u) gp[u] += q.rho_x * (K.ax[u] + dp[u]);
    if (lambda < T(0)) {
      T tr = trc;
      if (K.act) tr += h[0] + h[3] + h[5] + T(3) * q.rho_x;
      tr = grp.sum(tr);
      for (int c = 0; c < nc; ++c)
#pragma unroll
        for (int u = 0; u < 6; ++u) tr += q.rho(3 + u);
      lambda = q.lambda0 * tr / T(3 * np + n_u);
    }
    // W_p = (H_pp + (rho_x + lambda) I)^-1 by cofactors (identity on lanes without a copy)
    T w6[6] = {1, 0, 0, 1, 0, 1};
    if (K.act) {
      const T dg = q.rho_x + lambda;
      const T a00 = h[0] + dg, a01 = h[1], a02 = h[2], a11 = h[3] + dg, a12 = h[4], a22 = h[5] + dg;
      const T c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
      const T c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
      const T idet = Num<T>::rcp(a00 * c00 + a01 * c01 + a02 * c02);
      w6[0] = c00 * idet, w6[1] = c01 * idet, w6[2] = c02 * idet;
      w6[3] = c11 * idet, w6[4] = c12 * idet, w6[5] = c22 * idet;
    }
    // U_c = 2w_c A_c W_p g_p and, per camera pair c1 <= c2, the Schur weight
    // Q = [c1 = c2] 2w_1 I - (2w_1 A_1) W_p (2w_2 A_2)^T
    {
      const T Wg0 = w6[0] * gp[0] + w6[1] * gp[1] + w6[2] * gp[2];
      const T Wg1 = w6[1] * gp[0] + w6[3] * gp[1] + w6[4] * gp[2];
      const T Wg2 = w6[2] * gp[0] + w6[4] * gp[1] + w6[5] * gp[2];
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        m.U[c][0] = m.tw[c] * (Ap[c][0][0] * Wg0 + Ap[c][0][1] * Wg1 + Ap[c][0][2] * Wg2);
        m.U[c][1] = m.tw[c] * (Ap[c][1][0] * Wg0 + Ap[c][1][1] * Wg1 + Ap[c][1][2] * Wg2);
      }
#pragma unroll
      for (int c2 = 0; c2 < KC; ++c2) {
        const T* a2r0 = Ap[c2][0];
        const T* a2r1 = Ap[c2][1];
        const T w0 = w6[0] * a2r0[0] + w6[1] * a2r0[1] + w6[2] * a2r0[2];
        const T w1 = w6[1] * a2r0[0] + w6[3] * a2r0[1] + w6[4] * a2r0[2];
        const T w2 = w6[2] * a2r0[0] + w6[4] * a2r0[1] + w6[5] * a2r0[2];
        const T x0 = w6[0] * a2r1[0] + w6[1] * a2r1[1] + w6[2] * a2r1[2];
        const T x1 = w6[1] * a2r1[0] + w6[3] * a2r1[1] + w6[4] * a2r1[2];
        const T x2 = w6[2] * a2r1[0] + w6[4] * a2r1[1] + w6[5] * a2r1[2];
#pragma unroll
        for (int c1 = 0; c1 <= c2; ++c1) {
          const int pr = cam_pair(KC, c1, c2);
          const T* a1r0 = Ap[c1][0];
          const T* a1r1 = Ap[c1][1];
          const T sw = m.tw[c1] * m.tw[c2], dgw = c1 == c2 ? m.tw[c1] : T(0);
          m.Q[pr][0] = dgw - sw * (a1r0[0] * w0 + a1r0[1] * w1 + a1r0[2] * w2);
          m.Q[pr][1] = -sw * (a1r0[0] * x0 + a1r0[1] * x1 + a1r0[2] * x2);
          m.Q[pr][2] = -sw * (a1r1[0] * w0 + a1r1[1] * w1 + a1r1[2] * w2);
          m.Q[pr][3] = dgw - sw * (a1r1[0] * x0 + a1r1[1] * x1 + a1r1[2] * x2);
        }
      }
    }
    // sums over the block's points, G values at a time
    sys_reduce<T, G, KC>(m, grp, Z, dst, std::make_integer_sequence<int, sys_slots<KC, G>() / G>{});
    grp.sync();
    // row r < n_u of S + diag(rho_c) + lambda I (entries j <= r), g_r (the camera gradient
    // with its penalty) and the right-hand side rhs_r - g_r, on lane r mod G; a block with
    // fewer than KC cameras is padded to N x N by identity rows with a zero right-hand side,
    // which leave its factor and solution as they are
    T a[R][N], lc[R][N], y[R], gi[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int r = gl + G * t;
      const bool row = r < n_u;
      const int c = row ? r / 6 : 0, u = row ? r % 6 : 0;
      const T shift = q.rho(3 + u) + lambda;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        a[t][j] = row && j <= r ? Z.sys[Sh::kLd * j + r] + (j == r ? shift : T(0)) : T(j == r ? 1 : 0);
        lc[t][j] = 0;
      }
      gi[t] = y[t] = 0;
      if (row) {
        gi[t] = Z.sys[Sh::kG + r] + q.rho(3 + u) * (Z.a[c][u] + Z.d[c][u]);
        y[t] = Z.sys[Sh::kRhs + r] - gi[t];
      }
    }
    // Cholesky factor in registers: each held row r of L (a) and, below the diagonal,
    // column r (lc[j] = L_jr); pivots and columns pass by shuffles.  Row k sits on lane
    // k mod G in slot k / G; the tests on G t skip rows a slot cannot hold.
    bool spd = true;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const T piv = grp.bcast(a[k / G][k], k % G);
      spd = spd && piv > T(0);
      const T lkk = Num<T>::sqrt_(piv);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        if (G * t + G - 1 < k) continue;
        const int r = gl + G * t;
        if (r == k) a[t][k] = lkk;
        else if (r > k) a[t][k] = Num<T>::div(a[t][k], lkk);
      }
#pragma unroll N
      for (int j = k + 1; j < N; ++j) {
        const T ljk = grp.bcast(a[j / G][k], j % G);
        if (gl == k % G) lc[k / G][j] = ljk;
#pragma unroll
        for (int t = 0; t < R; ++t) {
          if (G * t + G - 1 < j) continue;
          if (gl + G * t >= j) a[t][j] -= a[t][k] * ljk;
        }
      }
    }
    if (!spd) {
      lambda *= T(10);
      continue;
    }
    // L y = rhs - g, then L^T dy = y; row r's entry on lane r mod G (zero beyond n_u)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (gl == k % G) y[k / G] = Num<T>::div(y[k / G], a[k / G][k]);
      const T yk = grp.bcast(y[k / G], k % G);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        if (G * t + G - 1 <= k) continue;
        if (gl + G * t > k) y[t] -= a[t][k] * yk;
      }
    }
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
      if (gl == k % G) y[k / G] = Num<T>::div(y[k / G], a[k / G][k]);
      const T xk = grp.bcast(y[k / G], k % G);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        if (G * t >= k) continue;
        if (gl + G * t < k) y[t] -= lc[t][k] * xk;
      }
    }
    // point step dx = -W_p (g_p + sum_c 2w_c A_c^T B_c dy_c); predicted decrease
    // (lambda |d|^2 - g.d) / 2
    T xt[3], gd = 0, dd = 0;
    {
      T t3[3] = {gp[0], gp[1], gp[2]};
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        T r0 = 0, r1 = 0;
#pragma unroll
        for (int u = 0; u < 6; ++u) {
          const T dyu = grp.bcast(y[(6 * c + u) / G], (6 * c + u) % G);
          r0 += m.Bc[c][0][u] * dyu;
          r1 += m.Bc[c][1][u] * dyu;
        }
        r0 *= m.tw[c];
        r1 *= m.tw[c];
#pragma unroll
        for (int u = 0; u < 3; ++u) t3[u] += Ap[c][0][u] * r0 + Ap[c][1][u] * r1;
      }
      T dx[3] = {0, 0, 0};
      if (K.act) {
        dx[0] = -(w6[0] * t3[0] + w6[1] * t3[1] + w6[2] * t3[2]);
        dx[1] = -(w6[1] * t3[0] + w6[3] * t3[1] + w6[4] * t3[2]);
        dx[2] = -(w6[2] * t3[0] + w6[4] * t3[1] + w6[5] * t3[2]);
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        gd += gp[u] * dx[u];
        dd += dx[u] * dx[u];
        xt[u] = dp[u] + dx[u];
      }
    }
#pragma unroll
    for (int t = 0; t < R; ++t)
      if (gl + G * t < n_u) {  // the camera terms of the rows this lane holds
        gd += gi[t] * y[t];
        dd += y[t] * y[t];
      }
    gd = grp.sum(gd);
    dd = grp.sum(dd);
    const T pred = T(0.5) * (lambda * dd - gd);
    const bool trust = isfinite(L) && q.model_tol > T(0) &&
                       pred <= q.model_tol * Num<T>::unit_roundoff * (fabs(L) + Z.sys[Sh::kNoise]);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int r = gl + G * t;
      if (r < n_u) Z.dt[r / 6][r % 6] = Z.d[r / 6][r % 6] + y[t];
    }
    grp.sync();
    const T Lt = K.objective(q, grp, xt, Z, Z.dt, nc);
    if (Lt < Num<T>::inf() && (trust || Lt < L)) {
#pragma unroll
      for (int u = 0; u < 3; ++u) dp[u] = xt[u];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const int r = gl + G * t;
        if (r < n_u) Z.d[r / 6][r % 6] = Z.dt[r / 6][r % 6];
      }
      L = Lt;  // Eq. (14) at the accepted point, trusted step or not
      const T lr = Num<T>::tenth(lambda);
      lambda = lr > q.lambda_min ? lr : q.lambda_min;
    } else {
      lambda *= T(10);
    }
    grp.sync();
  }
  bool finite = true;
  if (K.act) {
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      pdel[u * B.n_pc + pc] = dp[u];
      finite = finite && isfinite(dp[u]);
    }
  }
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int r = gl + G * t;
    if (r < n_u) {
      const T v = Z.d[r / 6][r % 6];
      cdel[(r % 6) * B.n_cc + bi.c0 + r / 6] = v;
      finite = finite && isfinite(v);
    }
  }
  if (!finite) atomicOr(B.err, 1);
  grp.sync();
}

// Blocks [lo, hi) of one size class with at most KC cameras and G points, one group of G
// lanes per block, the groups' systems in static shared memory.
template <typename T, int G, int KC>
__device__ __forceinline__ void block_solve_cams(const BlockProblem& B, const Prm<T>& q, int lo, int hi) {
  constexpr int kPer = 32 / G, kSlots = sys_slots<KC, G>();
  __shared__ CamShared<T, KC> sh[kBlkWarps * kPer];
  __shared__ short dst[kSlots];
  for (int e = threadIdx.x; e < kSlots; e += blockDim.x) dst[e] = (short)sys_dst<KC>(e);
  __syncthreads();
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const Grp<G> grp(threadIdx.x & 31);
  CamShared<T, KC>& Z = sh[warp * kPer + grp.base / G];
  const int stride = gridDim.x * warps * kPer;
  int b = lo + (blockIdx.x * warps + warp) * kPer + grp.base / G;
  BlockInfo bi{};
  if (b < hi) bi = B.blocks[b];
  for (; b < hi; b += stride) {
    const bool more = b + stride < hi;
    BlockInfo nb{};
    if (more) nb = B.blocks[b + stride];
    solve_block_cams<T, G, KC>(B, q, bi, grp, Z, dst, more ? &nb : nullptr);
    bi = nb;
  }
}

// at most two cameras: 4 CTAs of 4 warps per SM in FP32 (128 registers)
template <typename T, int G>
__global__ void __launch_bounds__(kBlkWarps * 32, (sizeof(T) == 4 ? 4 : 1))
    block_solve_2cam_kernel(BlockProblem B, Prm<T> q, int cur, int lo, int hi) {
  block_solve_cams<T, G, 2>(B, q, lo, hi);
}

// at most four cameras (a 24 x 24 system, a row per lane): 2 CTAs of 4 warps per SM
template <typename T, int G>
__global__ void __launch_bounds__(kBlkWarps * 32, (sizeof(T) == 4 ? 2 : 1))
    block_solve_4cam_kernel(BlockProblem B, Prm<T> q, int cur, int lo, int hi) {
  block_solve_cams<T, G, 4>(B, q, lo, hi);
}

// Blocks [lo, hi) of one size class, each solved by a group of G lanes holding PPL
// point copies each (32 / G groups per warp, blockDim.x / 32 warps per CTA); groups
// stride through the range independently.
// Resident CTAs per SM the register allocation is held to (4 warps each): the FP32
// one-camera variants fit in 72 registers a thread, the two-camera ones in 96.
template <typename T, int KC, int PPL>
constexpr int blk_min_ctas() {
  return sizeof(T) > 4 || PPL > 1 ? 1 : KC == 1 ? 7 : KC == 2 ? 5 : 1;
}

template <typename T, int KC, int G, int PPL>
__global__ void __launch_bounds__(kBlkWarps * 32, (blk_min_ctas<T, KC, PPL>()))
    block_solve_kernel(BlockProblem B, Prm<T> q, int cur, int lo, int hi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kPer = 32 / G;
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const Grp<G> grp(threadIdx.x & 31);
  BlkSmem<T, KC, G, PPL>& W = reinterpret_cast<BlkSmem<T, KC, G, PPL>*>(smem_raw)[warp];
  const int stride = gridDim.x * warps * kPer;
  for (int b = lo + (blockIdx.x * warps + warp) * kPer + grp.base / G; b < hi; b += stride) {
    const BlockInfo bi = B.blocks[b];
    solve_block<T, KC, G, PPL>(B, q, bi, W, grp, cur);
  }
}

// Eqs. (10)-(11) over copies.  After any full iteration the scaled duals of a point's (a
// camera's) copies sum to zero (Eqs. 10 and 12 summed over the copies; the oracle's tests
// pin it), and the duals are zero before the first, so the mean of copy + dual / rho is
// the consensus the copies were solved against plus the mean of their offsets.  Offsets
// are summed in T (points) or FP64 (cameras), the mean added to the FP64 consensus; the T
// mirror and the change are written for the next block solves.  A point or camera without
// copies keeps its value.
// Points (a few copies each): one thread per point.
template <typename T>
__global__ void __launch_bounds__(256) block_point_consensus_kernel(BlockProblem B, int cur) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= B.n_pts) return;
  const int nxt = cur ^ 1;
  const int i = (int)t, k0 = B.pt_cp_off[i], k1 = B.pt_cp_off[i + 1];
  const T* del = static_cast<const T*>(B.pc_delta);
  T acc[3] = {0, 0, 0};
  for (int k = k0; k < k1; ++k) {
    const int cp = B.pt_cp[k];
#pragma unroll
    for (int u = 0; u < 3; ++u) acc[u] += del[u * B.n_pc + cp];
  }
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const long long e = 3 * (long long)i + u;
    const T inc = k1 > k0 ? acc[u] / (T)(k1 - k0) : T(0);
    const double x = B.X[cur][e] + to_f64<T>(inc);
    B.X[nxt][e] = x;
    static_cast<T*>(B.Xm)[e] = from_f64<T>(x);
    static_cast<T*>(B.DX)[e] = -inc;
  }
}

// Cameras (thousands of copies each): one CTA of 256 threads per camera, strided partial
// sums of the offsets in FP64 and a fixed reduction tree.
template <typename T>
__global__ void __launch_bounds__(256) block_camera_consensus_kernel(BlockProblem B, int cur) {
  __shared__ double red[6][256];
  const int j = blockIdx.x, nxt = cur ^ 1;
  const int k0 = B.cam_cp_off[j], k1 = B.cam_cp_off[j + 1];
  const T* del = static_cast<const T*>(B.cc_delta);
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const int cp = B.cam_cp[k];
#pragma unroll
    for (int u = 0; u < 6; ++u) s[u] += to_f64<T>(del[u * B.n_cc + cp]);
  }
#pragma unroll
  for (int u = 0; u < 6; ++u) red[u][threadIdx.x] = s[u];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int u = 0; u < 6; ++u) red[u][threadIdx.x] += red[u][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 6) {
    const int u = threadIdx.x;
    const long long e = 6 * (long long)j + u;
    const double yo = B.Y[cur][e];
    const double yn = k1 > k0 ? yo + red[u][0] / (double)(k1 - k0) : yo;
    B.Y[nxt][e] = yn;
    static_cast<T*>(B.Ym)[e] = from_f64<T>(yn);
    static_cast<T*>(B.DY)[e] = from_f64<T>(yo - yn);
  }
}

// Primal (|copy - consensus|^2) and dual (rho^2 |change of consensus|^2) residual terms of
// the last iteration, one thread per point or camera copy in storage order: right after an
// iteration the offsets are still relative to the previous consensus Y[cur ^ 1] (the dual
// ascent is deferred), so copy - new consensus = offset - (new - previous consensus).
template <typename T>
__global__ void __launch_bounds__(256) block_residual_kernel(BlockProblem B, Prm<double> q, int cur) {
  __shared__ double red[2][256];
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int prv = cur ^ 1;
  double pr = 0.0, dr = 0.0;
  if (t < B.n_pc) {
    const T* del = static_cast<const T*>(B.pc_delta);
    const long long i = B.pc_pt[t];
    for (int u = 0; u < 3; ++u) {
      const double inc = B.X[cur][3 * i + u] - B.X[prv][3 * i + u];
      const double d = to_f64<T>(del[u * B.n_pc + t]) - inc;
      pr += d * d;
      const double r = q.rho_x * inc;
      dr += r * r;
    }
  } else if (t < B.n_pc + B.n_cc) {
    const long long k = t - B.n_pc;
    const T* del = static_cast<const T*>(B.cc_delta);
    const long long j = B.cc_cam[k];
    for (int u = 0; u < 6; ++u) {
      const double inc = B.Y[cur][6 * j + u] - B.Y[prv][6 * j + u];
      const double d = to_f64<T>(del[u * B.n_cc + k]) - inc;
      pr += d * d;
      const double r = q.rho(3 + u) * inc;
      dr += r * r;
    }
  }
  red[0][threadIdx.x] = pr;
  red[1][threadIdx.x] = dr;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&B.sums[6], red[0][0]);
    atomicAdd(&B.sums[7], red[1][0]);
  }
}

// Rotation and translation of every consensus camera Y[c] (R = Rz Ry Rx, Sec. 2.1), so that
// the metrics project each observation without evaluating its camera's angles again.
template <typename T>
__global__ void block_camera_pose_kernel(BlockProblem B, int c) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= B.n_cams) return;
  T v[9] = {0, 0, 0};
#pragma unroll
  for (int u = 0; u < 6; ++u) v[3 + u] = from_f64<T>(B.Y[c][6 * (long long)j + u]);
  Pose<T> P;
  pose_at(v, T(0), P);  // x = 0: p = t
  T* out = static_cast<T*>(B.cam_pose) + 12 * (long long)j;
#pragma unroll
  for (int u = 0; u < 9; ++u) out[u] = P.R[u];
#pragma unroll
  for (int u = 0; u < 3; ++u) out[9 + u] = v[6 + u];
}

// Reprojection terms of Eq. (2) at consensus X[c], Y[c]: sums of |e|^2, phi_m, |f - z_ref|^2
// (reference pixels, inliers), valid, invalid and reference counts.  A thread's own
// observations (a few) are summed in T, the block and grid reductions in FP64.
template <typename T>
__global__ void block_metrics_kernel(BlockProblem B, Prm<T> q, int c) {
  __shared__ double red[6][256];
  using V2 = typename Num<T>::V2;
  const T* pose = static_cast<const T*>(B.cam_pose);
  T acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < B.n_obs;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = B.obs_pt[o], j = B.obs_cam[o];
    const T x0 = from_f64<T>(B.X[c][3 * (long long)i]), x1 = from_f64<T>(B.X[c][3 * (long long)i + 1]),
            x2 = from_f64<T>(B.X[c][3 * (long long)i + 2]);
    const T* Rt = pose + 12 * (long long)j;
    const T p0 = Rt[0] * x0 + Rt[1] * x1 + Rt[2] * x2 + Rt[9];
    const T p1 = Rt[3] * x0 + Rt[4] * x1 + Rt[5] * x2 + Rt[10];
    const T p2 = Rt[6] * x0 + Rt[7] * x1 + Rt[8] * x2 + Rt[11];
    if (!(p2 > q.eps)) {
      acc[4] += T(1);
      continue;
    }
    const V2 zz = static_cast<const V2*>(B.z)[o];
    const T iz = T(1) / p2;
    const T zp0 = q.focal * p0 * iz + q.cx, zp1 = q.focal * p1 * iz + q.cy;
    const T e0 = zz.x - zp0, e1 = zz.y - zp1;
    const T s = e0 * e0 + e1 * e1;
    acc[0] += s;
    acc[1] += misfit<T>(q.loss, q.lp, s);
    acc[3] += T(1);
    if (B.zt && (!B.inlier || B.inlier[o])) {
      const double g0 = to_f64<T>(zp0) - B.zt[2 * o], g1 = to_f64<T>(zp1) - B.zt[2 * o + 1];
      acc[2] += from_f64<T>(g0 * g0 + g1 * g1);
      acc[5] += T(1);
    }
  }
  for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = to_f64<T>(acc[k]);
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) atomicAdd(&B.sums[k], red[k][0]);
}

int blocks_of(long long n, int per) { return (int)((n + per - 1) / per); }

}  // namespace
}  // namespace dba

// ------------------------------------------------------------ host side
struct dba_block_ctx {
  dba_config cfg{};
  dba::Params prm{};
  bool fp32 = true;
  int pi = 1, kappa = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool has_problem = false;
  int cur = 0;
  long long iters = 0;
  int cls[dba::kBlkClasses + 1] = {};  // block list cut into size classes: [cls[k], cls[k + 1])
  int small[dba::kBlkClasses][4] = {};  // in class k: first block of more than 1, 2, 4, 8 points
  std::string err = "no error";
  // host copy of the layout (caller order <-> block order)
  std::vector<long long> blk_obs;  // block order -> caller observation
  std::vector<dba::BlockInfo> h_blocks;
  dba::BlockProblem B{};
  std::vector<void*> allocs;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double flops_start = 0.0, flops_step = 0.0;  // algorithmic FP work of the block solves

  dba_status fail(dba_status s, const std::string& msg) {
    err = msg;
    return s;
  }
  dba_status cuda_fail(cudaError_t e, const char* where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return DBA_ECUDA;
  }
  template <typename P>
  cudaError_t alloc(P** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess) allocs.push_back(q);
    *p = static_cast<P*>(q);
    return e;
  }
  void free_all() {
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    B = dba::BlockProblem{};
    has_problem = false;
  }
};

namespace {
thread_local std::string g_block_error = "no error";

#define BLK_CUDA(call, where)                           \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, where); \
  } while (0)

template <typename T>
cudaError_t upload(dba_block_ctx* ctx, T** dst, const std::vector<T>& src) {
  cudaError_t e = ctx->alloc(dst, sizeof(T) * src.size());
  if (e != cudaSuccess || src.empty()) return e;
  return cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, ctx->stream);
}

// Blocks [lo, hi) of one size class: lane groups of G with PPL point copies per lane,
// at most KC cameras per block.
template <typename T, int KC, int G, int PPL>
cudaError_t launch_block_class(dba_block_ctx* ctx, int lo, int hi) {
  if (hi <= lo) return cudaSuccess;
  using Smem = dba::BlkSmem<T, KC, G, PPL>;
  constexpr int kWarps = sizeof(Smem) * dba::kBlkWarps <= 200 * 1024 ? dba::kBlkWarps : 2;
  static_assert(sizeof(Smem) * kWarps <= 220 * 1024, "block solve shared memory");
  const size_t smem = sizeof(Smem) * kWarps;
  static std::atomic<int> cached{0};  // CTAs of a full wave
  int grid = cached.load();
  if (!grid) {
    // resident CTAs per SM from the resources one CTA takes (registers, shared memory)
    cudaError_t e = cudaFuncSetAttribute(dba::block_solve_kernel<T, KC, G, PPL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncAttributes fa;
    int dev = 0, sms = 0, smem_sm = 0, smem_rsv = 0, regs_sm = 0;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, dba::block_solve_kernel<T, KC, G, PPL>);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    const int threads = kWarps * 32;
    int per_sm = 2048 / threads;
    per_sm = std::min(per_sm, regs_sm / std::max(1, (fa.numRegs + 7) / 8 * 8 * threads));
    per_sm = std::min(per_sm, smem_sm / ((int)smem + smem_rsv + (int)fa.sharedSizeBytes));
    grid = std::max(per_sm, 1) * sms;
    cached.store(grid);
  }
  const int need = dba::blocks_of(hi - lo, kWarps * (32 / G));
  const int g = std::max(1, std::min(need, grid));
  dba::block_solve_kernel<T, KC, G, PPL><<<g, kWarps * 32, smem, ctx->stream>>>(
      ctx->B, dba::make_prm<T>(ctx->prm), ctx->cur, lo, hi);
  return cudaGetLastError();
}

// One-camera blocks [lo, hi): the register-resident solve, groups of G lanes.
template <typename T, int G>
cudaError_t launch_block_class_1cam(dba_block_ctx* ctx, int lo, int hi) {
  if (hi <= lo) return cudaSuccess;
  constexpr int kThreads = dba::kBlkWarps * 32;
  static std::atomic<int> cached{0};  // CTAs of a full wave
  int grid = cached.load();
  if (!grid) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dba::block_solve_1cam_kernel<T, G>,
                                                                  kThreads, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    grid = std::max(per_sm, 1) * sms;
    cached.store(grid);
  }
  const int need = dba::blocks_of(hi - lo, dba::kBlkWarps * (32 / G));
  const int g = std::max(1, std::min(need, grid));
  dba::block_solve_1cam_kernel<T, G><<<g, kThreads, 0, ctx->stream>>>(ctx->B, dba::make_prm<T>(ctx->prm), ctx->cur,
                                                                       lo, hi);
  return cudaGetLastError();
}

// Blocks [lo, hi) with at most KC = 2 or 4 cameras and G points: the register solve, groups of
// G lanes.
template <typename T, int G, int KC = 2>
cudaError_t launch_block_class_2cam(dba_block_ctx* ctx, int lo, int hi) {
  if (hi <= lo) return cudaSuccess;
  constexpr int kThreads = dba::kBlkWarps * 32;
  auto kernel = [] {
    if constexpr (KC == 2) return dba::block_solve_2cam_kernel<T, G>;
    else return dba::block_solve_4cam_kernel<T, G>;
  }();
  static std::atomic<int> cached{0};  // CTAs of a full wave
  int grid = cached.load();
  if (!grid) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    grid = std::max(per_sm, 1) * sms;
    cached.store(grid);
  }
  const int need = dba::blocks_of(hi - lo, dba::kBlkWarps * (32 / G));
  const int g = std::max(1, std::min(need, grid));
  kernel<<<g, kThreads, 0, ctx->stream>>>(ctx->B, dba::make_prm<T>(ctx->prm), ctx->cur, lo, hi);
  return cudaGetLastError();
}

// One-point blocks [lo, hi): one thread per block, cameras eliminated.
template <typename T>
cudaError_t launch_block_class_point(dba_block_ctx* ctx, int lo, int hi) {
  if (hi <= lo) return cudaSuccess;
  constexpr int kThreads = dba::kBlkWarps * 32;
  static std::atomic<int> cached{0};  // CTAs of a full wave
  int grid = cached.load();
  if (!grid) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dba::block_solve_point_kernel<T>,
                                                                  kThreads, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    grid = std::max(per_sm, 1) * sms;
    cached.store(grid);
  }
  const int need = dba::blocks_of(hi - lo, kThreads);
  const int g = std::max(1, std::min(need, grid));
  dba::block_solve_point_kernel<T><<<g, kThreads, 0, ctx->stream>>>(ctx->B, dba::make_prm<T>(ctx->prm), ctx->cur,
                                                                     lo, hi);
  return cudaGetLastError();
}

template <typename T, int G, int PPL>
cudaError_t launch_block_class_kc(dba_block_ctx* ctx, int k) {
  const int lo = ctx->cls[k], hi = ctx->cls[k + 1];
  if (ctx->kappa == 1) {
    if constexpr (PPL == 1) return launch_block_class_1cam<T, G>(ctx, lo, hi);
    return launch_block_class<T, 1, G, PPL>(ctx, lo, hi);
  }
  if constexpr (PPL == 1) {
    // the 16-lane class holds at most 2 cameras (its blocks of at most 8 points in groups of
    // 8 lanes), the 32-lane one at most block_cams
    // blocks of one point (the first of each class) eliminate their cameras instead
    const int m1 = ctx->small[k][0];
    cudaError_t e = launch_block_class_point<T>(ctx, lo, m1);
    if (e != cudaSuccess) return e;
    if constexpr (G == 16) {
      const int m4 = ctx->small[k][2], m8 = ctx->small[k][3];
      e = launch_block_class_2cam<T, 4>(ctx, m1, m4);
      if (e == cudaSuccess) e = launch_block_class_2cam<T, 8>(ctx, m4, m8);
      return e == cudaSuccess ? launch_block_class_2cam<T, 16>(ctx, m8, hi) : e;
    } else {
      if (ctx->kappa == 2) return launch_block_class_2cam<T, G>(ctx, m1, hi);
      return launch_block_class_2cam<T, G, 4>(ctx, m1, hi);
    }
  } else {
    if (ctx->kappa == 2) return launch_block_class<T, 2, G, PPL>(ctx, lo, hi);
    return launch_block_class<T, 4, G, PPL>(ctx, lo, hi);
  }
}

// The size classes of the block list, in its order: one camera and at most 8 points
// (groups of 1, 2, 4 or 8 lanes by the block's points), at most 2 cameras and 16 points
// (16 lanes; 8 for two cameras and at most 8 points), at most 32 points (32 lanes), the rest
// (32 lanes holding two point copies each).  Blocks with one camera (the first class; the
// next two when block_cams = 1) take the one-camera solve, blocks of the next two classes
// the two-camera solve (the 32-lane class: the four-slot solve when block_cams >= 3), the
// rest the shared-memory solve.
template <typename T>
cudaError_t launch_block_solve(dba_block_ctx* ctx) {
  // block_solve_launches counts the nonempty ranges launched here; keep the two in step
  const int* c0 = ctx->small[0];
  cudaError_t e = launch_block_class_1cam<T, 1>(ctx, ctx->cls[0], c0[0]);
  if (e == cudaSuccess) e = launch_block_class_1cam<T, 2>(ctx, c0[0], c0[1]);
  if (e == cudaSuccess) e = launch_block_class_1cam<T, 4>(ctx, c0[1], c0[2]);
  if (e == cudaSuccess) e = launch_block_class_1cam<T, 8>(ctx, c0[2], ctx->cls[1]);
  if (e == cudaSuccess) e = launch_block_class_kc<T, 16, 1>(ctx, 1);
  if (e == cudaSuccess) e = launch_block_class_kc<T, 32, 1>(ctx, 2);
  if (e == cudaSuccess) e = launch_block_class_kc<T, 32, 2>(ctx, 3);
  return e;
}

// Block-solve launches of one iteration: the nonempty ranges launch_block_solve launches.
int block_solve_launches(const dba_block_ctx* ctx) {
  std::vector<std::pair<int, int>> r;
  const int* c0 = ctx->small[0];
  r.push_back({ctx->cls[0], c0[0]});
  r.push_back({c0[0], c0[1]});
  r.push_back({c0[1], c0[2]});
  r.push_back({c0[2], ctx->cls[1]});
  if (ctx->kappa == 1) {
    r.push_back({ctx->cls[1], ctx->cls[2]});
    r.push_back({ctx->cls[2], ctx->cls[3]});
  } else {
    r.push_back({ctx->cls[1], ctx->small[1][0]});  // one point
    r.push_back({ctx->small[1][0], ctx->small[1][2]});
    r.push_back({ctx->small[1][2], ctx->small[1][3]});
    r.push_back({ctx->small[1][3], ctx->cls[2]});
    r.push_back({ctx->cls[2], ctx->small[2][0]});  // one point
    r.push_back({ctx->small[2][0], ctx->cls[3]});
  }
  r.push_back({ctx->cls[3], ctx->cls[4]});
  int n = 0;
  for (const auto& x : r) n += x.second > x.first;
  return n;
}

// One iteration: block solves, consensus, dual ascent.  ev (nullable) receives an event
// before each of the three launches and one after the last.
cudaError_t launch_iteration(dba_block_ctx* ctx, cudaEvent_t* ev = nullptr) {
  cudaError_t e;
  if (ev && (e = cudaEventRecord(ev[0], ctx->stream)) != cudaSuccess) return e;
  e = ctx->fp32 ? launch_block_solve<float>(ctx) : launch_block_solve<double>(ctx);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], ctx->stream)) != cudaSuccess) return e;
  const int gp = dba::blocks_of(ctx->B.n_pts, 256);
  if (ctx->fp32)
    dba::block_point_consensus_kernel<float><<<gp, 256, 0, ctx->stream>>>(ctx->B, ctx->cur);
  else
    dba::block_point_consensus_kernel<double><<<gp, 256, 0, ctx->stream>>>(ctx->B, ctx->cur);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[2], ctx->stream)) != cudaSuccess) return e;
  if (ctx->fp32)
    dba::block_camera_consensus_kernel<float><<<ctx->B.n_cams, 256, 0, ctx->stream>>>(ctx->B, ctx->cur);
  else
    dba::block_camera_consensus_kernel<double><<<ctx->B.n_cams, 256, 0, ctx->stream>>>(ctx->B, ctx->cur);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[3], ctx->stream)) != cudaSuccess) return e;
  ctx->cur ^= 1;
  ctx->B.pending = 1;  // the next block solves apply this iteration's dual ascent
  return cudaSuccess;
}

// The metric sums at the current consensus into B.sums[0..5] (cleared first); with
// residuals, the last iteration's primal and dual residual terms into B.sums[6..7].
cudaError_t launch_stats(dba_block_ctx* ctx, bool residuals) {
  cudaError_t e = cudaMemsetAsync(ctx->B.sums, 0, 8 * sizeof(double), ctx->stream);
  if (e != cudaSuccess) return e;
  const int g = std::min(dba::blocks_of(ctx->B.n_obs, 256), 4096), gc = dba::blocks_of(ctx->B.n_cams, 128);
  const dba::Prm<double> q64 = dba::make_prm<double>(ctx->prm);
  const int gr = dba::blocks_of(ctx->B.n_pc + ctx->B.n_cc, 256);
  if (ctx->fp32) {
    if (residuals) dba::block_residual_kernel<float><<<gr, 256, 0, ctx->stream>>>(ctx->B, q64, ctx->cur);
    dba::block_camera_pose_kernel<float><<<gc, 128, 0, ctx->stream>>>(ctx->B, ctx->cur);
    dba::block_metrics_kernel<float><<<g, 256, 0, ctx->stream>>>(ctx->B, dba::make_prm<float>(ctx->prm), ctx->cur);
  } else {
    if (residuals) dba::block_residual_kernel<double><<<gr, 256, 0, ctx->stream>>>(ctx->B, q64, ctx->cur);
    dba::block_camera_pose_kernel<double><<<gc, 128, 0, ctx->stream>>>(ctx->B, ctx->cur);
    dba::block_metrics_kernel<double><<<g, 256, 0, ctx->stream>>>(ctx->B, dba::make_prm<double>(ctx->prm), ctx->cur);
  }
  return cudaGetLastError();
}

// Metrics (and, with residuals, the last iteration's residual terms) at the current state.
dba_status read_stats(dba_block_ctx* ctx, bool residuals, dba_stats* st) {
  BLK_CUDA(launch_stats(ctx, residuals), "metrics");
  double h[8];
  int herr = 0;
  BLK_CUDA(cudaMemcpyAsync(h, ctx->B.sums, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "metrics");
  BLK_CUDA(cudaMemcpyAsync(&herr, ctx->B.err, sizeof herr, cudaMemcpyDeviceToHost, ctx->stream), "metrics");
  BLK_CUDA(cudaStreamSynchronize(ctx->stream), "metrics");
  if (herr & 1) return ctx->fail(DBA_ENUMERIC, "a block solve produced a non-finite value");
  st->iters_done = ctx->iters;
  st->rmse_obs = h[3] > 0 ? std::sqrt(h[0] / h[3]) : 0.0;
  st->objective = h[1];
  st->rmse_gt = h[5] > 0 ? std::sqrt(h[2] / h[5]) : 0.0;
  st->n_invalid = (long long)h[4];
  st->primal_res = residuals ? std::sqrt(h[6]) : 0.0;
  st->dual_res = residuals ? std::sqrt(h[7]) : 0.0;
  return DBA_OK;
}

}  // namespace

// The block layout of Sec. 3.1.4 (Eq. 14) under the reading in the header comment, built
// on the host: observations in block order, blocks (in size-class order), point and
// camera copies, their consensus lists and the algorithmic flop counts.  Returns an empty
// string, or the message for a repeated (point, camera) pair.
struct BlockHostLayout {
  std::vector<long long> blk_obs;  // block order -> caller observation
  std::vector<dba::BlockInfo> blocks;
  int cls[dba::kBlkClasses + 1] = {};
  int small[dba::kBlkClasses][4] = {};
  std::vector<int> pc_obs, pc_pt, cc_cam, obs_pt, obs_cam;
  std::vector<unsigned char> obs_lc;
  std::vector<int> pt_off, cam_off, pt_cp, cam_cp;
  double flops_step = 0.0, flops_start = 0.0;
};

std::string build_block_layout(int n_cams, int n_pts, long long l, const int32_t* pt_idx, const int32_t* cam_idx,
                               int pi, int kappa, BlockHostLayout& H) {
  const int n = n_pts, m = n_cams;
  // point ranks by (smallest observing camera, point index)
  std::vector<int> first(n, INT_MAX);
  for (long long o = 0; o < l; ++o) first[pt_idx[o]] = std::min(first[pt_idx[o]], (int)cam_idx[o]);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return first[a] < first[b]; });
  std::vector<int> rank(n);
  for (int r = 0; r < n; ++r) rank[order[r]] = r;
  const long long n_cg = (m + kappa - 1) / kappa;
  auto key = [&](long long o) { return (long long)(rank[pt_idx[o]] / pi) * n_cg + cam_idx[o] / kappa; };
  std::vector<long long>& idx = H.blk_obs;
  idx.resize(l);
  std::iota(idx.begin(), idx.end(), 0LL);
  std::sort(idx.begin(), idx.end(), [&](long long a, long long b) {
    const long long ka = key(a), kb = key(b);
    if (ka != kb) return ka < kb;
    if (rank[pt_idx[a]] != rank[pt_idx[b]]) return rank[pt_idx[a]] < rank[pt_idx[b]];
    return cam_idx[a] < cam_idx[b];
  });
  for (long long t = 1; t < l; ++t)
    if (pt_idx[idx[t]] == pt_idx[idx[t - 1]] && cam_idx[idx[t]] == cam_idx[idx[t - 1]])
      return "point " + std::to_string(pt_idx[idx[t]]) + " is observed twice by camera " +
             std::to_string(cam_idx[idx[t]]);
  // blocks, point copies (consecutive observations of one point), camera copies
  std::vector<dba::BlockInfo>& blocks = H.blocks;
  blocks.clear();
  std::vector<int>&pc_obs = H.pc_obs, &pc_pt = H.pc_pt, &cc_cam = H.cc_cam, &obs_pt = H.obs_pt, &obs_cam = H.obs_cam;
  obs_pt.assign(l, 0);
  obs_cam.assign(l, 0);
  std::vector<unsigned char>& obs_lc = H.obs_lc;
  obs_lc.assign(l, 0);
  long long o = 0;
  while (o < l) {
    const long long k = key(idx[o]);
    long long e = o;
    while (e < l && key(idx[e]) == k) ++e;
    dba::BlockInfo bi{};
    bi.o0 = (int)o;
    bi.no = (int)(e - o);
    bi.p0 = (int)pc_pt.size();
    bi.c0 = (int)cc_cam.size();
    std::vector<int> cams;
    for (long long t = o; t < e; ++t) cams.push_back(cam_idx[idx[t]]);
    std::sort(cams.begin(), cams.end());
    cams.erase(std::unique(cams.begin(), cams.end()), cams.end());
    for (int c : cams) cc_cam.push_back(c);
    bi.nc = (int)cams.size();
    for (long long t = o; t < e; ++t) {
      const int i = pt_idx[idx[t]];
      if (t == o || pt_idx[idx[t - 1]] != i) {
        pc_pt.push_back(i);
        pc_obs.push_back((int)t);
      }
      obs_pt[t] = i;
      obs_cam[t] = cam_idx[idx[t]];
      obs_lc[t] = (unsigned char)(std::lower_bound(cams.begin(), cams.end(), (int)cam_idx[idx[t]]) - cams.begin());
    }
    bi.np = (int)pc_pt.size() - bi.p0;
    blocks.push_back(bi);
    o = e;
  }
  pc_obs.push_back((int)l);
  const long long n_pc = (long long)pc_pt.size(), n_cc = (long long)cc_cam.size();
  // algorithmic flops of the block solves (add/mul 1, fma 2, rcp/sqrt/sin/cos 1), counted
  // from the kernel's arithmetic, each step a full step with its trial objective:
  //   per observation: pose 44, Jacobian and residual 64, point block and gradient terms 43,
  //     noise bound 7, its 2w A W g term 14, gradient and right-hand side entries 48,
  //     back-substitution 30, trial pose and misfit 64                        -> 314
  //   per point copy: penalty gradient 6, 3x3 inverse 35, W g 15, step 15, model terms 12,
  //     trial penalty 9                                                      -> 92
  //   blocks whose points are eliminated:
  //     per camera pair of a point's observations (Schur weight 60 + 8 per entry of the
  //       reduced system): 228 when both are one observation (21 entries), 348 otherwise;
  //     per block: Cholesky n^3/3 + n^2/2, triangular solves 2 n^2, damping and camera
  //       model/penalty terms 10 n (n = 6 cameras)
  //   blocks of one point and several cameras (cameras eliminated): per camera five
  //     capacitance solves of 140, its H_xc rows 72, the 3 x 3 Schur update 108, the
  //     back-substitution terms 66 -> 946; per block the 3 x 3 solve and damping 60
  //   start of a solve: pose and misfit 64 per observation, penalty 9 per point copy and
  //     per camera copy 24
  {
    double schur = 0.0, per_block = 0.0;
    for (const dba::BlockInfo& bi : blocks) {
      if (bi.np == 1 && bi.nc >= 2) {
        per_block += 946.0 * bi.nc + 60.0;
        continue;
      }
      for (int k = bi.p0; k < bi.p0 + bi.np; ++k) {
        const double c = (double)(pc_obs[k + 1] - pc_obs[k]);
        schur += 228.0 * c + 348.0 * c * (c - 1.0) / 2.0;
      }
      const double nu = 6.0 * bi.nc;
      per_block += nu * nu * nu / 3.0 + nu * nu / 2.0 + 2.0 * nu * nu + 10.0 * nu;
    }
    H.flops_step = 314.0 * (double)l + 92.0 * (double)n_pc + schur + per_block;
    H.flops_start = 64.0 * (double)l + 9.0 * (double)n_pc + 24.0 * (double)n_cc;
  }
  // size classes of the solve kernel (lane groups of 8, 16, 32, 32 with two copies per
  // lane), each contiguous and ordered by points, so that its small blocks can take
  // narrower lane groups
  {
    auto cls_of = [](const dba::BlockInfo& b) {
      return b.nc == 1 && b.np <= 8 ? 0 : b.nc <= 2 && b.np <= 16 ? 1 : b.np <= 32 ? 2 : 3;
    };
    std::stable_sort(blocks.begin(), blocks.end(), [&](const dba::BlockInfo& a, const dba::BlockInfo& b) {
      const int ca = cls_of(a), cb = cls_of(b);
      return ca != cb ? ca < cb : a.np < b.np;
    });
    H.cls[0] = 0;
    for (int k = 0; k < dba::kBlkClasses; ++k) {
      const auto lo = blocks.begin() + H.cls[k];
      const auto hi = std::partition_point(lo, blocks.end(), [&](const dba::BlockInfo& b) { return cls_of(b) <= k; });
      H.cls[k + 1] = (int)(hi - blocks.begin());
      for (int t = 0; t < 4; ++t)
        H.small[k][t] = (int)(std::partition_point(lo, hi, [&](const dba::BlockInfo& b) { return b.np <= (1 << t); }) -
                              blocks.begin());
    }
  }
  // copy lists per point and per camera (consensus)
  std::vector<int>&pt_off = H.pt_off, &cam_off = H.cam_off, &pt_cp = H.pt_cp, &cam_cp = H.cam_cp;
  pt_off.assign(n + 1, 0);
  cam_off.assign(m + 1, 0);
  pt_cp.assign(n_pc, 0);
  cam_cp.assign(n_cc, 0);
  for (long long k = 0; k < n_pc; ++k) ++pt_off[pc_pt[k] + 1];
  for (long long k = 0; k < n_cc; ++k) ++cam_off[cc_cam[k] + 1];
  for (int i = 0; i < n; ++i) pt_off[i + 1] += pt_off[i];
  for (int j = 0; j < m; ++j) cam_off[j + 1] += cam_off[j];
  {
    std::vector<int> fill(pt_off.begin(), pt_off.end() - 1);
    for (long long k = 0; k < n_pc; ++k) pt_cp[fill[pc_pt[k]]++] = (int)k;
    std::vector<int> fc(cam_off.begin(), cam_off.end() - 1);
    for (long long k = 0; k < n_cc; ++k) cam_cp[fc[cc_cam[k]]++] = (int)k;
  }
  return std::string();
}

extern "C" {

dba_status dba_block_create(const dba_config* cfg, int block_points, int block_cams, dba_block_ctx** out) {
  return dba::guarded(&g_block_error, [&]() -> dba_status {
    if (!cfg || !out) {
      g_block_error = "dba_block_create: null argument";
      return DBA_EINVAL;
    }
    *out = nullptr;
    const bool ok = std::isfinite(cfg->focal) && cfg->focal > 0 && std::isfinite(cfg->cx) && std::isfinite(cfg->cy) &&
                    cfg->loss >= 0 && cfg->loss <= 2 &&
                    (cfg->loss == DBA_LOSS_L2 || (std::isfinite(cfg->loss_param) && cfg->loss_param > 0)) &&
                    std::isfinite(cfg->rho_x) && cfg->rho_x > 0 && std::isfinite(cfg->rho_y) && cfg->rho_y > 0 &&
                    std::isfinite(cfg->rho_angle) && cfg->inner_steps >= 0 && cfg->inner_steps <= 1000 &&
                    std::isfinite(cfg->lm_lambda0) && cfg->lm_lambda0 > 0 && std::isfinite(cfg->lm_lambda_min) &&
                    cfg->lm_lambda_min >= 0 && std::isfinite(cfg->eps_depth) && std::isfinite(cfg->lm_model_tol) &&
                    cfg->lm_model_tol >= 0 && (cfg->precision == 0 || cfg->precision == 1) &&
                    cfg->local_solver == DBA_SOLVER_GN;
    if (!ok) {
      g_block_error = "dba_block_create: invalid configuration";
      return DBA_EINVAL;
    }
    if (block_points < 1 || block_points > DBA_BLOCK_MAX_POINTS || block_cams < 1 ||
        block_cams > DBA_BLOCK_MAX_CAMERAS) {
      g_block_error = "dba_block_create: block_points must be in [1, 64] and block_cams in [1, 4]";
      return DBA_EINVAL;
    }
    cudaError_t e = cudaFree(nullptr);
    if (e != cudaSuccess) {
      g_block_error = std::string("dba_block_create: CUDA unavailable: ") + cudaGetErrorString(e);
      return DBA_ECUDA;
    }
    dba_block_ctx* ctx = new (std::nothrow) dba_block_ctx();
    if (!ctx) {
      g_block_error = "dba_block_create: out of host memory";
      return DBA_ENOMEM;
    }
    ctx->cfg = *cfg;
    ctx->fp32 = cfg->precision == DBA_PREC_F32_LOCAL;
    ctx->pi = block_points;
    ctx->kappa = block_cams;
    ctx->prm = dba::Params{cfg->focal, cfg->cx, cfg->cy, cfg->loss, cfg->loss_param, cfg->rho_x, cfg->rho_y,
                           cfg->rho_angle > 0 ? cfg->rho_angle : cfg->rho_y, cfg->inner_steps, cfg->lm_lambda0,
                           cfg->lm_lambda_min, cfg->eps_depth, cfg->lm_model_tol, DBA_SOLVER_GN};
    if (cfg->cuda_stream) {
      ctx->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e != cudaSuccess) {
      g_block_error = std::string("dba_block_create: ") + cudaGetErrorString(e);
      dba_block_destroy(ctx);
      return DBA_ECUDA;
    }
    *out = ctx;
    return DBA_OK;
  });
}

dba_status dba_block_set_observations(dba_block_ctx* ctx, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                                      const int32_t* pt_idx, const int32_t* cam_idx, const double* z,
                                      const double* cams0, const double* pts0) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (n_cams <= 0 || n_pts <= 0 || n_obs <= 0)
      return ctx->fail(DBA_EINVAL, "dba_block_set_observations: n_cams, n_pts and n_obs must be positive");
    if (n_obs > INT_MAX) return ctx->fail(DBA_EINVAL, "dba_block_set_observations: at most 2^31-1 observations");
    if (!pt_idx || !cam_idx || !z || !cams0 || !pts0)
      return ctx->fail(DBA_EINVAL, "dba_block_set_observations: null array");
    for (int64_t o = 0; o < n_obs; ++o) {
      if (pt_idx[o] < 0 || pt_idx[o] >= n_pts || cam_idx[o] < 0 || cam_idx[o] >= n_cams)
        return ctx->fail(DBA_EINVAL, "dba_block_set_observations: observation " + std::to_string(o) +
                                         " indexes outside the cameras or points");
      if (!std::isfinite(z[2 * o]) || !std::isfinite(z[2 * o + 1]))
        return ctx->fail(DBA_EINVAL, "dba_block_set_observations: non-finite pixel");
    }
    for (int64_t k = 0; k < 6LL * n_cams; ++k)
      if (!std::isfinite(cams0[k])) return ctx->fail(DBA_EINVAL, "dba_block_set_observations: non-finite camera");
    for (int64_t k = 0; k < 3LL * n_pts; ++k)
      if (!std::isfinite(pts0[k])) return ctx->fail(DBA_EINVAL, "dba_block_set_observations: non-finite point");
    ctx->free_all();
    const long long l = n_obs;
    const int n = n_pts, m = n_cams;
    BlockHostLayout H;
    {
      const std::string msg = build_block_layout(n_cams, n_pts, l, pt_idx, cam_idx, ctx->pi, ctx->kappa, H);
      if (!msg.empty()) return ctx->fail(DBA_EINVAL, "dba_block_set_observations: " + msg);
    }
    ctx->blk_obs = H.blk_obs;
    ctx->h_blocks = H.blocks;
    for (int k = 0; k <= dba::kBlkClasses; ++k) ctx->cls[k] = H.cls[k];
    for (int k = 0; k < dba::kBlkClasses; ++k)
      for (int t = 0; t < 4; ++t) ctx->small[k][t] = H.small[k][t];
    ctx->flops_step = H.flops_step;
    ctx->flops_start = H.flops_start;
    const std::vector<dba::BlockInfo>& blocks = H.blocks;
    const std::vector<int>&pc_obs = H.pc_obs, &pc_pt = H.pc_pt, &cc_cam = H.cc_cam, &obs_pt = H.obs_pt,
                      &obs_cam = H.obs_cam, &pt_off = H.pt_off, &cam_off = H.cam_off, &pt_cp = H.pt_cp,
                      &cam_cp = H.cam_cp;
    const std::vector<unsigned char>& obs_lc = H.obs_lc;
    const std::vector<long long>& idx = H.blk_obs;
    const long long n_pc = (long long)pc_pt.size(), n_cc = (long long)cc_cam.size();
    // device problem
    dba::BlockProblem& B = ctx->B;
    B.n_cams = m;
    B.n_pts = n;
    B.n_obs = l;
    B.n_blocks = (int)blocks.size();
    B.n_pc = n_pc;
    B.n_cc = n_cc;
    const size_t tsz = ctx->fp32 ? sizeof(float) : sizeof(double);
    std::vector<float> mirror_pts, mirror_cams;  // FP32 mirrors of the initial consensus (uploaded below)
    dba::BlockInfo* d_blocks = nullptr;
    int *d_pc_obs = nullptr, *d_pc_pt = nullptr, *d_cc_cam = nullptr, *d_obs_pt = nullptr, *d_obs_cam = nullptr;
    int *d_pt_off = nullptr, *d_pt_cp = nullptr, *d_cam_off = nullptr, *d_cam_cp = nullptr;
    unsigned char* d_lc = nullptr;
    BLK_CUDA(upload(ctx, &d_blocks, blocks), "upload");
    BLK_CUDA(upload(ctx, &d_pc_obs, pc_obs), "upload");
    BLK_CUDA(upload(ctx, &d_pc_pt, pc_pt), "upload");
    BLK_CUDA(upload(ctx, &d_cc_cam, cc_cam), "upload");
    BLK_CUDA(upload(ctx, &d_obs_pt, obs_pt), "upload");
    BLK_CUDA(upload(ctx, &d_obs_cam, obs_cam), "upload");
    BLK_CUDA(upload(ctx, &d_lc, obs_lc), "upload");
    BLK_CUDA(upload(ctx, &d_pt_off, pt_off), "upload");
    BLK_CUDA(upload(ctx, &d_pt_cp, pt_cp), "upload");
    BLK_CUDA(upload(ctx, &d_cam_off, cam_off), "upload");
    BLK_CUDA(upload(ctx, &d_cam_cp, cam_cp), "upload");
    B.blocks = d_blocks;
    B.pc_obs = d_pc_obs;
    B.pc_pt = d_pc_pt;
    B.cc_cam = d_cc_cam;
    B.obs_pt = d_obs_pt;
    B.obs_cam = d_obs_cam;
    B.obs_lc = d_lc;
    B.pt_cp_off = d_pt_off;
    B.pt_cp = d_pt_cp;
    B.cam_cp_off = d_cam_off;
    B.cam_cp = d_cam_cp;
    // pixels in block order, in the working precision
    {
      std::vector<double> zb(2 * l);
      for (long long t = 0; t < l; ++t) {
        zb[2 * t] = z[2 * idx[t]];
        zb[2 * t + 1] = z[2 * idx[t] + 1];
      }
      void* d_z = nullptr;
      BLK_CUDA(ctx->alloc(&d_z, tsz * 2 * l), "alloc");
      if (ctx->fp32) {
        std::vector<float> zf(zb.begin(), zb.end());
        BLK_CUDA(cudaMemcpyAsync(d_z, zf.data(), sizeof(float) * zf.size(), cudaMemcpyHostToDevice, ctx->stream),
                 "upload");
        BLK_CUDA(cudaStreamSynchronize(ctx->stream), "upload");
      } else {
        BLK_CUDA(cudaMemcpyAsync(d_z, zb.data(), sizeof(double) * zb.size(), cudaMemcpyHostToDevice, ctx->stream),
                 "upload");
        BLK_CUDA(cudaStreamSynchronize(ctx->stream), "upload");
      }
      B.z = d_z;
    }
    // state: copies at the consensus (offsets 0), duals 0
    void *d_pdel = nullptr, *d_cdel = nullptr;
    BLK_CUDA(ctx->alloc(&d_pdel, tsz * 3 * n_pc), "alloc");
    BLK_CUDA(ctx->alloc(&d_cdel, tsz * 6 * n_cc), "alloc");
    BLK_CUDA(ctx->alloc(&B.pc_a, sizeof(double) * 3 * n_pc), "alloc");
    BLK_CUDA(ctx->alloc(&B.cc_a, sizeof(double) * 6 * n_cc), "alloc");
    BLK_CUDA(cudaMemsetAsync(d_pdel, 0, tsz * 3 * n_pc, ctx->stream), "init");
    BLK_CUDA(cudaMemsetAsync(d_cdel, 0, tsz * 6 * n_cc, ctx->stream), "init");
    BLK_CUDA(cudaMemsetAsync(B.pc_a, 0, sizeof(double) * 3 * n_pc, ctx->stream), "init");
    BLK_CUDA(cudaMemsetAsync(B.cc_a, 0, sizeof(double) * 6 * n_cc, ctx->stream), "init");
    B.pc_delta = d_pdel;
    B.cc_delta = d_cdel;
    for (int k = 0; k < 2; ++k) {
      BLK_CUDA(ctx->alloc(&B.X[k], sizeof(double) * 3 * n), "alloc");
      BLK_CUDA(ctx->alloc(&B.Y[k], sizeof(double) * 6 * m), "alloc");
    }
    BLK_CUDA(cudaMemcpyAsync(B.X[0], pts0, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->stream), "upload");
    BLK_CUDA(cudaMemcpyAsync(B.Y[0], cams0, sizeof(double) * 6 * m, cudaMemcpyHostToDevice, ctx->stream), "upload");
    // T mirrors of the consensus and its (zero) last change
    BLK_CUDA(ctx->alloc(&B.Xm, tsz * 3 * (size_t)n), "alloc");
    BLK_CUDA(ctx->alloc(&B.DX, tsz * 3 * (size_t)n), "alloc");
    BLK_CUDA(ctx->alloc(&B.Ym, tsz * 6 * (size_t)m), "alloc");
    BLK_CUDA(ctx->alloc(&B.DY, tsz * 6 * (size_t)m), "alloc");
    BLK_CUDA(cudaMemsetAsync(B.DX, 0, tsz * 3 * (size_t)n, ctx->stream), "init");
    BLK_CUDA(cudaMemsetAsync(B.DY, 0, tsz * 6 * (size_t)m, ctx->stream), "init");
    if (ctx->fp32) {
      mirror_pts.assign(pts0, pts0 + 3 * (size_t)n);
      mirror_cams.assign(cams0, cams0 + 6 * (size_t)m);
      BLK_CUDA(cudaMemcpyAsync(B.Xm, mirror_pts.data(), sizeof(float) * mirror_pts.size(), cudaMemcpyHostToDevice,
                               ctx->stream), "upload");
      BLK_CUDA(cudaMemcpyAsync(B.Ym, mirror_cams.data(), sizeof(float) * mirror_cams.size(), cudaMemcpyHostToDevice,
                               ctx->stream), "upload");
    } else {
      BLK_CUDA(cudaMemcpyAsync(B.Xm, pts0, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->stream), "upload");
      BLK_CUDA(cudaMemcpyAsync(B.Ym, cams0, sizeof(double) * 6 * m, cudaMemcpyHostToDevice, ctx->stream), "upload");
    }
    B.pending = 0;  // duals start at zero: nothing to apply before the first block solves
    BLK_CUDA(ctx->alloc(&B.sums, sizeof(double) * 8), "alloc");
    BLK_CUDA(ctx->alloc(&B.cam_pose, tsz * 12 * (size_t)m), "alloc");
    BLK_CUDA(ctx->alloc(&B.err, sizeof(int)), "alloc");
    BLK_CUDA(cudaMemsetAsync(B.err, 0, sizeof(int), ctx->stream), "init");
    BLK_CUDA(cudaStreamSynchronize(ctx->stream), "upload");
    ctx->cur = 0;
    ctx->iters = 0;
    ctx->has_problem = true;
    return DBA_OK;
  });
}

dba_status dba_block_set_reference_pixels(dba_block_ctx* ctx, const double* z_ref, const uint8_t* inlier) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_block_set_reference_pixels before set_observations");
    if (!z_ref) return ctx->fail(DBA_EINVAL, "dba_block_set_reference_pixels: null array");
    const long long l = ctx->B.n_obs;
    std::vector<double> zb(2 * l);
    std::vector<unsigned char> mb(l, 1);
    for (long long t = 0; t < l; ++t) {
      const long long o = ctx->blk_obs[t];
      zb[2 * t] = z_ref[2 * o];
      zb[2 * t + 1] = z_ref[2 * o + 1];
      if (!std::isfinite(zb[2 * t]) || !std::isfinite(zb[2 * t + 1]))
        return ctx->fail(DBA_EINVAL, "dba_block_set_reference_pixels: non-finite pixel");
      if (inlier) mb[t] = inlier[o] ? 1 : 0;
    }
    double* d_zt = nullptr;
    unsigned char* d_in = nullptr;
    BLK_CUDA(upload(ctx, &d_zt, zb), "upload");
    BLK_CUDA(upload(ctx, &d_in, mb), "upload");
    BLK_CUDA(cudaStreamSynchronize(ctx->stream), "upload");
    ctx->B.zt = d_zt;
    ctx->B.inlier = d_in;
    return DBA_OK;
  });
}

dba_status dba_block_iterate(dba_block_ctx* ctx, int n_iters, dba_stats* stats) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_block_iterate before dba_block_set_observations");
    if (n_iters < 0) return ctx->fail(DBA_EINVAL, "dba_block_iterate: n_iters < 0");
    BLK_CUDA(cudaEventRecord(ctx->ev0, ctx->stream), "iterate");
    for (int it = 0; it < n_iters; ++it) BLK_CUDA(launch_iteration(ctx), "iterate");
    BLK_CUDA(cudaEventRecord(ctx->ev1, ctx->stream), "iterate");
    ctx->iters += n_iters;
    int herr = 0;
    BLK_CUDA(cudaMemcpyAsync(&herr, ctx->B.err, sizeof herr, cudaMemcpyDeviceToHost, ctx->stream), "iterate");
    BLK_CUDA(cudaStreamSynchronize(ctx->stream), "iterate");
    if (herr & 1) return ctx->fail(DBA_ENUMERIC, "a block solve produced a non-finite value");
    if (stats) {
      float ms = 0.f;
      BLK_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1), "iterate");
      const dba_status s = read_stats(ctx, n_iters > 0, stats);
      stats->seconds = 1e-3 * ms;
      return s;
    }
    return DBA_OK;
  });
}

dba_status dba_block_iterate_until(dba_block_ctx* ctx, int max_iters, double target_rmse_gt, dba_stats* stats) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx || !stats) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_block_iterate_until before set_observations");
    if (!ctx->B.zt) return ctx->fail(DBA_ESTATE, "dba_block_iterate_until needs reference pixels");
    if (max_iters < 0 || !(target_rmse_gt > 0)) return ctx->fail(DBA_EINVAL, "dba_block_iterate_until: bad arguments");
    double secs = 0.0;
    bool any = false;
    for (int it = 0; it < max_iters; ++it) {
      // one iteration and the stopping test's metrics, timed on the device
      BLK_CUDA(cudaEventRecord(ctx->ev0, ctx->stream), "iterate_until");
      BLK_CUDA(launch_iteration(ctx), "iterate_until");
      BLK_CUDA(launch_stats(ctx, false), "iterate_until");
      BLK_CUDA(cudaEventRecord(ctx->ev1, ctx->stream), "iterate_until");
      ctx->iters += 1;
      any = true;
      double h[8];
      int herr = 0;
      BLK_CUDA(cudaMemcpyAsync(h, ctx->B.sums, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "iterate_until");
      BLK_CUDA(cudaMemcpyAsync(&herr, ctx->B.err, sizeof herr, cudaMemcpyDeviceToHost, ctx->stream), "iterate_until");
      BLK_CUDA(cudaStreamSynchronize(ctx->stream), "iterate_until");
      if (herr & 1) return ctx->fail(DBA_ENUMERIC, "a block solve produced a non-finite value");
      float ms = 0.f;
      BLK_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1), "iterate_until");
      secs += 1e-3 * ms;
      if (h[5] > 0 && std::sqrt(h[2] / h[5]) <= target_rmse_gt) break;
    }
    // the full statistics of the last iteration, residuals included
    const dba_status s = read_stats(ctx, any, stats);
    if (s != DBA_OK) return s;
    stats->seconds = secs;
    return DBA_OK;
  });
}

dba_status dba_block_profile(dba_block_ctx* ctx, int n_iters, double* ms_out) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx || !ms_out) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_block_profile before set_observations");
    if (n_iters <= 0) return ctx->fail(DBA_EINVAL, "dba_block_profile: n_iters must be positive");
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
    double acc[3] = {0, 0, 0};
    for (int it = 0; it < n_iters && e == cudaSuccess; ++it) {
      e = launch_iteration(ctx, ev);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
        acc[k] += ms;
      }
      ctx->iters += 1;
    }
    for (int k = 0; k < 4; ++k)
      if (ev[k]) cudaEventDestroy(ev[k]);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "dba_block_profile");
    for (int k = 0; k < 3; ++k) ms_out[k] = acc[k] / n_iters;
    return DBA_OK;
  });
}

dba_status dba_block_get_params(dba_block_ctx* ctx, double* cams_out, double* pts_out) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_block_get_params before set_observations");
    if (!cams_out || !pts_out) return ctx->fail(DBA_EINVAL, "dba_block_get_params: null array");
    BLK_CUDA(cudaMemcpyAsync(cams_out, ctx->B.Y[ctx->cur], sizeof(double) * 6 * ctx->B.n_cams, cudaMemcpyDeviceToHost,
                             ctx->stream),
             "get_params");
    BLK_CUDA(cudaMemcpyAsync(pts_out, ctx->B.X[ctx->cur], sizeof(double) * 3 * ctx->B.n_pts, cudaMemcpyDeviceToHost,
                             ctx->stream),
             "get_params");
    BLK_CUDA(cudaStreamSynchronize(ctx->stream), "get_params");
    return DBA_OK;
  });
}

dba_status dba_block_algorithmic_flops(const dba_block_ctx* ctx, double* per_iteration) {
  return dba::guarded(ctx ? &const_cast<dba_block_ctx*>(ctx)->err : nullptr, [&]() -> dba_status {
    if (!ctx || !per_iteration) return DBA_EINVAL;
    if (!ctx->has_problem) return DBA_ESTATE;
    *per_iteration = ctx->flops_start + ctx->cfg.inner_steps * ctx->flops_step;
    return DBA_OK;
  });
}

dba_status dba_block_layout(const dba_block_ctx* ctx, int64_t* n_blocks, int64_t* n_point_copies,
                            int64_t* n_camera_copies) {
  return dba::guarded(ctx ? &const_cast<dba_block_ctx*>(ctx)->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return DBA_ESTATE;
    if (n_blocks) *n_blocks = ctx->B.n_blocks;
    if (n_point_copies) *n_point_copies = ctx->B.n_pc;
    if (n_camera_copies) *n_camera_copies = ctx->B.n_cc;
    return DBA_OK;
  });
}

dba_status dba_block_build_layout(int32_t n_cams, int32_t n_pts, int64_t n_obs, const int32_t* pt_idx,
                                  const int32_t* cam_idx, int block_points, int block_cams, int64_t* obs_order,
                                  int32_t* blocks, int32_t* pc_point, int32_t* cc_camera, int64_t* counts,
                                  int64_t* size_classes) {
  return dba::guarded(&g_block_error, [&]() -> dba_status {
    if (n_cams <= 0 || n_pts <= 0 || n_obs <= 0 || n_obs > INT_MAX || !pt_idx || !cam_idx ||
        block_points < 1 || block_points > DBA_BLOCK_MAX_POINTS || block_cams < 1 ||
        block_cams > DBA_BLOCK_MAX_CAMERAS) {
      g_block_error = "dba_block_build_layout: sizes out of range or null index array";
      return DBA_EINVAL;
    }
    for (int64_t o = 0; o < n_obs; ++o)
      if (pt_idx[o] < 0 || pt_idx[o] >= n_pts || cam_idx[o] < 0 || cam_idx[o] >= n_cams) {
        g_block_error = "dba_block_build_layout: observation " + std::to_string(o) +
                        " indexes outside the cameras or points";
        return DBA_EINVAL;
      }
    try {
      BlockHostLayout H;
      const std::string msg = build_block_layout(n_cams, n_pts, n_obs, pt_idx, cam_idx, block_points, block_cams, H);
      if (!msg.empty()) {
        g_block_error = "dba_block_build_layout: " + msg;
        return DBA_EINVAL;
      }
      if (obs_order)
        for (int64_t o = 0; o < n_obs; ++o) obs_order[o] = H.blk_obs[o];
      if (blocks)
        for (size_t b = 0; b < H.blocks.size(); ++b) {
          const dba::BlockInfo& bi = H.blocks[b];
          const int32_t v[6] = {bi.o0, bi.no, bi.p0, bi.np, bi.c0, bi.nc};
          for (int k = 0; k < 6; ++k) blocks[6 * b + k] = v[k];
        }
      if (pc_point)
        for (size_t k = 0; k < H.pc_pt.size(); ++k) pc_point[k] = H.pc_pt[k];
      if (cc_camera)
        for (size_t k = 0; k < H.cc_cam.size(); ++k) cc_camera[k] = H.cc_cam[k];
      if (counts) {
        counts[0] = (int64_t)H.blocks.size();
        counts[1] = (int64_t)H.pc_pt.size();
        counts[2] = (int64_t)H.cc_cam.size();
      }
      if (size_classes)
        for (int k = 0; k < dba::kBlkClasses; ++k) size_classes[k] = H.cls[k + 1] - H.cls[k];
    } catch (const std::bad_alloc&) {
      g_block_error = "dba_block_build_layout: out of host memory";
      return DBA_ENOMEM;
    }
    return DBA_OK;
  });
}

dba_status dba_block_size_classes(const dba_block_ctx* ctx, int64_t* counts) {
  return dba::guarded(ctx ? &const_cast<dba_block_ctx*>(ctx)->err : nullptr, [&]() -> dba_status {
    if (!ctx || !counts) return DBA_EINVAL;
    if (!ctx->has_problem) return DBA_ESTATE;
    for (int k = 0; k < dba::kBlkClasses; ++k) counts[k] = ctx->cls[k + 1] - ctx->cls[k];
    return DBA_OK;
  });
}

dba_status dba_block_launches_per_iteration(const dba_block_ctx* ctx, int32_t* launches) {
  return dba::guarded(ctx ? &const_cast<dba_block_ctx*>(ctx)->err : nullptr, [&]() -> dba_status {
    if (!ctx || !launches) return DBA_EINVAL;
    if (!ctx->has_problem) return DBA_ESTATE;
    *launches = block_solve_launches(ctx) + 2;  // and the point and camera consensus
    return DBA_OK;
  });
}

const char* dba_block_last_error(const dba_block_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_block_error.c_str();
}

void dba_block_destroy(dba_block_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->free_all();
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

}  // extern "C"
