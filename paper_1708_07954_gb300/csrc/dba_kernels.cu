// CUDA kernels for one consensus-ADMM iteration of distributed bundle
// adjustment (arXiv 1708.07954, Sec. 3.1, Eqs. 9-13), written for sm_103a.
//
// Layout: observations are sorted by point (points ordered by their first
// camera) and cut into tiles of whole point tracks, one tile per thread block,
// one observation per thread.  Per observation the state is
//   delta[9]  (T)      copy minus the consensus it was last solved against,
//   adual[9]  (double) scaled duals a = (r / rho_x, s / rho_y),
// and per point / camera the FP64 consensus (ping-pong buffers) plus a T
// mirror of it and of its last change.  T = float on the reduced-precision
// path, double on the FP64 path; consensus sums and dual ascent are FP64.
//
//  tile_iterate  Eq. (12)-(13) of the previous iteration (dual ascent, deferred
//                until the new consensus exists), Eq. (9) for every
//                observation, Eq. (10) for every point whose whole track is in
//                the tile, and per-tile partial sums for Eq. (11).
//  finalize      Eq. (11) from the partial sums; Eq. (10) for tracks that
//                span several tiles.
//  metrics       reprojection RMSE, objective and residuals at consensus.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include <type_traits>
#include <math_constants.h>

#include <mutex>

#include "../../include/dba.h"
#include "dba_device.cuh"
#include "dba_internal.h"

namespace dba {
namespace {

// ------------------------------------------------------------ tile kernel
// Persistent, software-pipelined: each block walks tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... and while it computes one tile the copies, duals,
// pixels and indices of its next tile stream into shared memory by tensor copies
// (TMA, issued by one thread, completion on an mbarrier) and its run tables by
// cp.async, so no registers hold loads in flight and DRAM latency hides behind
// the local solves.  One thread per observation of a tile.
//
// Steady state: after any full iteration the scaled duals of every point and
// camera sum to zero (sum of Eq. 12 over a track after Eq. 10; the oracle's
// tests pin this), so Eq. (10)/(11) reduce to consensus + mean of the new
// offsets.  Those offsets are summed per run in T inside the tile and in FP64
// across tiles and into the consensus; the dual ascent itself is FP64.  In the
// first iteration after dba_set_state (exact) the duals are arbitrary and the
// summands offset + dual are formed and summed in FP64.

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned int s = static_cast<unsigned int>(__cvta_generic_to_shared(smem));
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int round128(int bytes) { return (bytes + 127) / 128 * 128; }

// The observation rows of a tile reach shared memory by tensor copies (TMA).  A copy's
// innermost coordinate must fall on a 16-byte boundary, so each row is fetched as a
// window starting at the tile's first observation rounded down to 16 bytes, in two
// boxes of kW elements (a box is at most 256 elements wide); box b lands in slab b.
// Element t of the tile is at window position x = t + (o0 mod 16 / size), found by
// win().  Double pixel pairs (16 bytes) are fetched as [n][2] rows, with no offset.
template <int W, int kSlab>
__device__ __forceinline__ int win(int x) {
  return x < W ? x : kSlab + (x - W);
}

template <typename T, int NT>
struct TileStage {
  using V2 = typename Num<T>::V2;
  static constexpr int kWT = NT / 2 + 16 / (int)sizeof(T);  // copies (T)
  static constexpr int kWD = NT / 2 + 2;                     // duals (double)
  static constexpr int kWI = NT / 2 + 4;                     // indices (int32)
  static constexpr int kWZ = sizeof(T) == 4 ? NT / 2 + 2 : NT / 2;  // pixels (float2 / double2)
  static constexpr int kSlabT = round128(9 * kWT * (int)sizeof(T)) / (int)sizeof(T);
  static constexpr int kSlabD = round128(9 * kWD * 8) / 8;
  static constexpr int kSlabI = round128(kWI * 4) / 4;
  static constexpr int kSlabZ = round128(kWZ * (int)sizeof(V2)) / (int)sizeof(V2);
  // bytes the tensor copies of one tile deliver (whole boxes, out-of-range parts filled)
  static constexpr unsigned kTxBytes =
      2u * (9u * kWT * sizeof(T) + 9u * kWD * 8u + kWZ * sizeof(V2) + 2u * kWI * 4u);
  alignas(128) T delta[2 * kSlabT];      // [box][9][kWT]
  alignas(128) double adual[2 * kSlabD]; // [box][9][kWD]
  alignas(128) V2 z[2 * kSlabZ];
  alignas(128) int pt[2 * kSlabI];
  alignas(128) int cam[2 * kSlabI];      // camera | rank << 24
  // run tables and the FP64 consensus of the tile's points (cp.async)
  double X[3 * NT];  // contiguous internal ids
  int2 pseg[NT];
  int pslot[NT];
  int2 cseg[NT];
  int cslot[NT];
};

// dynamic shared memory: 128 bytes of alignment slack, two stages, the run buffer and
// one mbarrier per stage
template <typename T, int NT>
constexpr size_t tile_smem_bytes() {
  return 128 + 2 * sizeof(TileStage<T, NT>) + sizeof(double) * 9 * NT + 2 * sizeof(unsigned long long);
}

__device__ __forceinline__ TileInfo load_tile_info(const TileInfo* tiles, int tile) {
  const int4* p = reinterpret_cast<const int4*>(tiles + tile);
  const int4 a = __ldg(p), b = __ldg(p + 1);
  TileInfo ti;
  ti.o0 = a.x; ti.n = a.y; ti.r0 = a.z; ti.nr = a.w;
  ti.c0 = b.x; ti.nc = b.y; ti.pt_lo = b.z; ti.pad = b.w;
  return ti;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tma_1d(void* dst, const CUtensorMap* map, int x, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done;
}

// The polling loop of mbar_wait, out of line: false once about two seconds (global timer,
// first read after 256 polls) or 2^22 polls have passed without completion.
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity) {
  constexpr unsigned long long kLimitNs = 2000000000ull;
  unsigned long long t0 = 0;
  for (int it = 0; it < (1 << 22); ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255) {
      const unsigned long long now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kLimitNs) return false;
    }
  }
  return false;
}

// Bounded wait for completion `parity` of the mbarrier at bar; false after the limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  return mbar_try(bar, parity) || mbar_wait_slow(bar, parity);
}

// Issues the copies of one tile into stage S: the observation rows by tensor copies from
// thread 0 (completion on bar), the run tables and consensus by cp.async from every
// thread (one commit group).  stall (fault injection): the tensor copies are announced
// on bar but not issued, so the wait for them runs out.
template <typename T, int NT>
__device__ __forceinline__ void stage_tile(const DevProblem& P, const TileMaps& M, TileStage<T, NT>& S,
                                           const TileInfo& ti, int cur, uint32_t bar, bool stall) {
  using St = TileStage<T, NT>;
  const int t = threadIdx.x;
  if (t == 0) {
    // generic-proxy reads of this stage (the tile before last) precede the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(St::kTxBytes) : "memory");
  }
  if (t == 0 && !stall) {
    const int o0 = ti.o0;
    const int xT = o0 & ~(16 / (int)sizeof(T) - 1), xD = o0 & ~1, xI = o0 & ~3;
    tma_2d(S.delta, &M.delta, xT, 0, bar);
    tma_2d(S.delta + St::kSlabT, &M.delta, xT + St::kWT, 0, bar);
    tma_2d(S.adual, &M.adual, xD, 0, bar);
    tma_2d(S.adual + St::kSlabD, &M.adual, xD + St::kWD, 0, bar);
    if constexpr (sizeof(T) == 4) {
      const int xZ = o0 & ~1;
      tma_1d(S.z, &M.z, xZ, bar);
      tma_1d(S.z + St::kSlabZ, &M.z, xZ + St::kWZ, bar);
    } else {
      tma_2d(S.z, &M.z, 0, o0, bar);
      tma_2d(S.z + St::kSlabZ, &M.z, 0, o0 + St::kWZ, bar);
    }
    tma_1d(S.pt, &M.pt, xI, bar);
    tma_1d(S.pt + St::kSlabI, &M.pt, xI + St::kWI, bar);
    tma_1d(S.cam, &M.cam, xI, bar);
    tma_1d(S.cam + St::kSlabI, &M.cam, xI + St::kWI, bar);
  }
  if (t < ti.nr) {
    cp_async<8>(&S.pseg[t], P.pseg + ti.r0 + t);
    cp_async<4>(&S.pslot[t], P.pseg_slot + ti.r0 + t);
  }
  if (t < ti.nc) {
    cp_async<8>(&S.cseg[t], P.cseg + ti.c0 + t);
    cp_async<4>(&S.cslot[t], P.cseg_slot + ti.c0 + t);
  }
  const double* X = P.X[cur] + 3 * (long long)ti.pt_lo;
  for (int e = t; e < 3 * ti.nr; e += NT) cp_async<8>(&S.X[e], X + e);
  cp_async_commit();
  // the T mirror and last change of the tile's point consensus (read by its local solves
  // and dual ascent; written an iteration ago, so mostly out of L2): prefetched into L2,
  // one 128-byte line per thread
  if (t < 64) {
    const T* row = static_cast<const T*>(t < 32 ? P.Xm : P.DX) + 3 * (long long)ti.pt_lo;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(row);
    const uintptr_t a = (lo & ~(uintptr_t)127) + 128 * (uintptr_t)(t & 31);
    if (a < lo + 3 * (uintptr_t)ti.nr * sizeof(T)) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
  }
}

// One tile from its staged inputs: deferred dual ascent, local solves, run sums.  kLoss >= 0
// fixes the misfit at compile time (the loss tests of every local-solve step fold away).
template <typename T, int NT, int kS, int kLoss>
__device__ __forceinline__ void process_tile_body(const DevProblem& P, const Prm<T>& qr, const TileStage<T, NT>& S,
                                                  double (*s_buf)[NT], const TileInfo& ti, int cur, int pending,
                                                  int exact) {
  Prm<T> q = qr;
  if constexpr (kLoss >= 0) q.loss = kLoss;
  const int t = threadIdx.x;
  const long long l = P.pitch;  // row stride of delta, adual, mlp_start
  const long long o = (long long)ti.o0 + t;
  T* __restrict__ delta = static_cast<T*>(P.delta);
  double* __restrict__ adual = P.adual;
  const T* __restrict__ Xm = static_cast<const T*>(P.Xm);
  const T* __restrict__ Ym = static_cast<const T*>(P.Ym);
  const T* __restrict__ DX = static_cast<const T*>(P.DX);
  const T* __restrict__ DY = static_cast<const T*>(P.DY);
  // T view of the run buffer, rows padded by one word so that the run sums, which read
  // the same position of several rows at once, fall in different banks (9 (NT + 1) T
  // words fit in the 9 NT doubles of s_buf for T = float; FP64 uses the unpadded rows)
  constexpr int kRow = sizeof(T) == 4 ? NT + 1 : NT;
  T(*s_t)[kRow] = reinterpret_cast<T(*)[kRow]>(&s_buf[0][0]);

  using St = TileStage<T, NT>;
  if (t < ti.n) {
    // this observation's positions in the staged windows
    const int wT = win<St::kWT, St::kSlabT>(t + (ti.o0 & (16 / (int)sizeof(T) - 1)));
    const int wD = win<St::kWD, St::kSlabD>(t + (ti.o0 & 1));
    const int wI = win<St::kWI, St::kSlabI>(t + (ti.o0 & 3));
    const int wZ = win<St::kWZ, St::kSlabZ>(t + (sizeof(T) == 4 ? (ti.o0 & 1) : 0));
    const int i = S.pt[wI];
    const int cr = S.cam[wI];
    const int j = cr & kCamMask, rk = (int)((unsigned int)cr >> 24);
    T d[9], vbar[9], aT[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) vbar[c] = Xm[3 * i + c];
#pragma unroll
    for (int c = 0; c < 6; ++c) vbar[3 + c] = Ym[6 * j + c];
#pragma unroll
    for (int c = 0; c < 9; ++c) d[c] = S.delta[wT + c * St::kWT];
    if (pending) {
      // Eqs. (12)-(13) of the previous iteration: the copy relative to the new
      // consensus is d0 = delta + (old - new consensus); a += d0 in FP64.
#pragma unroll
      for (int c = 0; c < 3; ++c) d[c] += DX[3 * i + c];
#pragma unroll
      for (int c = 0; c < 6; ++c) d[3 + c] += DY[6 * j + c];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const double a = S.adual[wD + c * St::kWD] + to_f64<T>(d[c]);
        adual[c * l + o] = a;
        aT[c] = from_f64<T>(a);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 9; ++c) aT[c] = from_f64<T>(S.adual[wD + c * St::kWD]);
    }
    const typename Num<T>::V2 zz = S.z[wZ];
    if (P.mlp_start) {
      const T* ms = static_cast<const T*>(P.mlp_start);
      T alt[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) alt[c] = ms[c * l + o];
      if constexpr (kS == DBA_SOLVER_LBFGS)
        local_solve_lbfgs<T, true>(zz.x, zz.y, vbar, aT, d, q, alt);
      else
        local_solve<T, true>(zz.x, zz.y, vbar, aT, d, q, alt);
    } else {
      if constexpr (kS == DBA_SOLVER_LBFGS)
        local_solve_lbfgs<T>(zz.x, zz.y, vbar, aT, d, q);
      else
        local_solve<T>(zz.x, zz.y, vbar, aT, d, q);
    }
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      delta[c * l + o] = d[c];
      finite = finite && isfinite(d[c]);
    }
    if (!finite) atomicOr(&P.ctl->err, 1);
    if (exact) {
      // first iteration after dba_set_state: full summands offset + dual (pending is 0 then)
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const double v = to_f64<T>(d[c]) + S.adual[wD + c * St::kWD];
        if (c < 3) s_buf[c][t] = v; else s_buf[c][rk] = v;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) s_t[c][t] = d[c];
#pragma unroll
      for (int c = 3; c < 9; ++c) s_t[c][rk] = d[c];
    }
  }
  __syncthreads();

  // Eq. (10) per point run and the per-tile partial sums of Eq. (11) per camera run, one
  // thread per (run, coordinate): point tasks first, camera tasks on the threads after
  // them, so a thread takes a second task only when the two lists exceed the block.
  // Point run r is point pt_lo + r.
  const int nxt = cur ^ 1;
  const int n_pt_tasks = 3 * ti.nr, n_tasks = n_pt_tasks + 6 * ti.nc;
  for (int task = t; task < n_tasks; task += NT) {
    if (task < n_pt_tasks) {
      const int r = task / 3, c = task % 3;
      const int2 se = S.pseg[r];
      double sum;
      T acc = 0;
      if (exact) {
        sum = 0.0;
        for (int e = se.x; e < se.x + se.y; ++e) sum += s_buf[c][e];
      } else {
        // one accumulator, so unrolling keeps the summation order
#pragma unroll 4
        for (int e = se.x; e < se.x + se.y; ++e) acc += s_t[c][e];
        sum = to_f64<T>(acc);
      }
      const int slot = S.pslot[r];
      if (slot < 0) {
        const long long k = 3 * ((long long)ti.pt_lo + r) + c;
        const double xo = S.X[task];
        if (std::is_same<T, float>::value && !exact) {
          // FP32 offsets: their mean is formed in FP32 and added to the FP64 consensus, which
          // keeps the divide and the conversions off the FP64 pipe
          const T inc = acc * Num<T>::rcp((T)se.y);
          const double xn = xo + to_f64<T>(inc);
          P.X[nxt][k] = xn;
          static_cast<T*>(P.Xm)[k] = from_f64<T>(xn);
          static_cast<T*>(P.DX)[k] = -inc;
        } else {
          const double xn = xo + sum / (double)se.y;
          P.X[nxt][k] = xn;
          static_cast<T*>(P.Xm)[k] = from_f64<T>(xn);
          static_cast<T*>(P.DX)[k] = from_f64<T>(xo - xn);
        }
      } else {
        P.pt_part[3 * slot + c] = sum;
      }
    } else {
      const int ct = task - n_pt_tasks, r = ct / 6, c = ct % 6;
      const int2 se = S.cseg[r];
      double sum;
      if (exact) {
        sum = 0.0;
        for (int e = se.x; e < se.x + se.y; ++e) sum += s_buf[3 + c][e];
      } else {
        T acc = 0;
#pragma unroll 4
        for (int e = se.x; e < se.x + se.y; ++e) acc += s_t[3 + c][e];
        sum = to_f64<T>(acc);
      }
      P.cam_part[6 * S.cslot[r] + c] = sum;
    }
  }
}

// The FP32 Gauss-Newton kernel (the benchmarked path) has one body per loss; the other
// kernels read the loss at run time.
template <typename T, int NT, int kS>
__device__ __forceinline__ void process_tile(const DevProblem& P, const Prm<T>& q, const TileStage<T, NT>& S,
                                             double (*s_buf)[NT], const TileInfo& ti, int cur, int pending,
                                             int exact) {
  if constexpr (sizeof(T) == 4 && kS == DBA_SOLVER_GN) {
    if (q.loss == DBA_LOSS_HUBER)
      process_tile_body<T, NT, kS, DBA_LOSS_HUBER>(P, q, S, s_buf, ti, cur, pending, exact);
    else if (q.loss == DBA_LOSS_STUDENT_T)
      process_tile_body<T, NT, kS, DBA_LOSS_STUDENT_T>(P, q, S, s_buf, ti, cur, pending, exact);
    else
      process_tile_body<T, NT, kS, DBA_LOSS_L2>(P, q, S, s_buf, ti, cur, pending, exact);
  } else {
    process_tile_body<T, NT, kS, -1>(P, q, S, s_buf, ti, cur, pending, exact);
  }
}

// Resident blocks per SM the register allocation is held to: 16 warps for the FP32 kernels at
// every tile size (4 blocks of 128 threads run four tiles' latency chains side by side where
// 2 blocks at 129 registers fit only 3); the FP64 kernels, bound by the FP64 pipe, keep 2.
template <typename T, int NT>
constexpr int tile_min_blocks() {
  return sizeof(T) == 4 ? 512 / NT : 2;
}

template <typename T, int NT, int kS>
__global__ void __launch_bounds__(NT, (tile_min_blocks<T, NT>()))
    tile_iterate_kernel(DevProblem P, const __grid_constant__ TileMaps M, Prm<T> q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  TileStage<T, NT>* stage = reinterpret_cast<TileStage<T, NT>*>(base);
  double(*s_buf)[NT] = reinterpret_cast<double(*)[NT]>(base + 2 * sizeof(TileStage<T, NT>));
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(base + 2 * sizeof(TileStage<T, NT>) +
                                                                    sizeof(double) * 9 * NT);
  const uint32_t bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);
  // The control word is written by the previous kernel and constant during this one: one
  // read-only-cache load per thread (cached per SM) instead of same-address L2 traffic.
  const int4 ctl = __ldg(reinterpret_cast<const int4*>(P.ctl));
  const int cur = ctl.x, pending = ctl.y, exact = ctl.w;
  const bool stall = (__ldg(&P.ctl->inject) & 1u) != 0;
  int tile = blockIdx.x;
  if (tile >= P.n_tiles) return;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  TileInfo info = load_tile_info(P.tiles, tile);
  stage_tile<T, NT>(P, M, stage[0], info, cur, bar0, stall);
  int next = tile + gridDim.x;
  TileInfo info_next{};
  if (next < P.n_tiles) info_next = load_tile_info(P.tiles, next);
  cp_async_wait<0>();
  bool ok = mbar_wait(bar0, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicOr(&P.ctl->err, 4);
    return;
  }
  for (int k = 0; tile < P.n_tiles; ++k) {
    // the next tile's copies go into the stage the previous tile used (free since the
    // barrier that ended it) and land while this tile is solved; stage s serves tiles
    // k = s, s + 2, ..., and its mbarrier completes once per use (parity (k >> 1) & 1)
    const int sn = (k + 1) & 1;
    if (next < P.n_tiles) stage_tile<T, NT>(P, M, stage[sn], info_next, cur, sn ? bar1 : bar0, stall);
    const int after = next + gridDim.x;
    TileInfo info_after{};
    if (after < P.n_tiles) info_after = load_tile_info(P.tiles, after);  // used two tiles later
    process_tile<T, NT, kS>(P, q, stage[k & 1], s_buf, info, cur, pending, exact);
    cp_async_wait<0>();  // this thread's copies of the next tile have landed
    ok = next >= P.n_tiles || mbar_wait(sn ? bar1 : bar0, ((k + 1) >> 1) & 1);
    // ... and everyone else's, and the tensor copies; this stage and the run buffer are free
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicOr(&P.ctl->err, 4);
      return;
    }
    tile = next;
    next = after;
    info = info_next;
    info_next = info_after;
  }
}

// ------------------------------------------------------------ finalize
// One block of NF threads per segment of partial sums (a camera's, or a point's whose track
// spans several tiles): strided FP64 sums, then a fixed tree over the block.
template <typename T, int NF>
__global__ void __launch_bounds__(NF) finalize_kernel(DevProblem P) {
  __shared__ double red[6][NF];
  const int cur = __ldg(&P.ctl->cur), nxt = cur ^ 1;
  const int b = blockIdx.x, t = threadIdx.x;
  const bool is_cam = b < P.n_cams;
  const int nc = is_cam ? 6 : 3;
  int s0, s1, cnt, id;
  if (is_cam) {
    id = b;
    s0 = P.cam_slot_off[b];
    s1 = P.cam_slot_off[b + 1];
    cnt = P.cam_count[b];
  } else {
    const int sp = b - P.n_cams;
    id = P.split_pt[sp];
    s0 = P.split_slot_off[sp];
    s1 = P.split_slot_off[sp + 1];
    cnt = P.pt_count[id];
  }
  const double* part = is_cam ? P.cam_part : P.pt_part;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int s = s0 + t; s < s1; s += NF)
    for (int c = 0; c < nc; ++c) acc[c] += part[nc * s + c];
  for (int c = 0; c < 6; ++c) red[c][t] = acc[c];
  __syncthreads();
  for (int w = NF / 2; w > 0; w >>= 1) {
    if (t < w)
      for (int c = 0; c < 6; ++c) red[c][t] += red[c][t + w];
    __syncthreads();
  }
  if (t < nc && cnt > 0) {
    double* C = is_cam ? P.Y[cur] : P.X[cur];
    double* Cn = is_cam ? P.Y[nxt] : P.X[nxt];
    T* Cm = static_cast<T*>(is_cam ? P.Ym : P.Xm);
    T* DC = static_cast<T*>(is_cam ? P.DY : P.DX);
    const double co = C[nc * id + t];
    const double cn = co + red[t][0] / (double)cnt;
    Cn[nc * id + t] = cn;
    Cm[nc * id + t] = (T)cn;
    DC[nc * id + t] = (T)(co - cn);
  }
  // The last block to finish advances the control word for the next iteration.
  if (t == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(&P.ctl->done, 1u);
    if (prev == gridDim.x - 1) {
      P.ctl->cur = nxt;
      P.ctl->pending = 1;
      P.ctl->exact = 0;
      P.ctl->k += 1;
      P.ctl->done = 0;
      __threadfence();
    }
  }
}

// ------------------------------------------------------------ metrics
// Rotation and translation of every consensus camera (R = Rz Ry Rx, Sec. 2.1), so that the
// metrics pass projects each observation without re-evaluating its camera's angles.
template <typename T>
__global__ void camera_pose_kernel(DevProblem P) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.n_cams) return;
  const T* Ym = static_cast<const T*>(P.Ym);
  T v[9] = {0, 0, 0};
#pragma unroll
  for (int c = 0; c < 6; ++c) v[3 + c] = Ym[6 * j + c];
  Pose<T> Q;
  pose_at(v, T(0), Q);  // x = 0: u = 0, p = t
  T* out = static_cast<T*>(P.cam_pose) + 12 * (long long)j;
#pragma unroll
  for (int c = 0; c < 9; ++c) out[c] = Q.R[c];
#pragma unroll
  for (int c = 0; c < 3; ++c) out[9 + c] = v[6 + c];
}

// A camera pose row (R row-major, then t; 16-byte aligned) by vector loads.
__device__ __forceinline__ void load_pose(const float* p, float v[12]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 a = q[k];
    v[4 * k] = a.x;
    v[4 * k + 1] = a.y;
    v[4 * k + 2] = a.z;
    v[4 * k + 3] = a.w;
  }
}
__device__ __forceinline__ void load_pose(const double* p, double v[12]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double2 a = q[k];
    v[2 * k] = a.x;
    v[2 * k + 1] = a.y;
  }
}

// Metrics at consensus: sums of |e|^2, phi_m, |f - z_true|^2 (inliers), valid / invalid
// counts, primal and dual residual terms, reference count.  kGtOnly: only the reference
// sums and the counts (the stopping test of dba_iterate_until).
//
// One observation's terms, added to acc (summed in T: a thread's own observations are a few
// dozen; the FP64 pipe sees one conversion and add per sum and thread in the reduction).
template <typename T, bool kGtOnly>
__device__ __forceinline__ void metric_terms(const DevProblem& P, const Prm<T>& q, int i, int j,
                                             typename Num<T>::V2 zz, typename Num<T>::V2 gt, bool counted,
                                             T acc[8]) {
  const T* Xm = static_cast<const T*>(P.Xm);
  const T x0 = Xm[3 * i], x1 = Xm[3 * i + 1], x2 = Xm[3 * i + 2];
  T Rt[12];
  load_pose(static_cast<const T*>(P.cam_pose) + 12 * (long long)j, Rt);
  const T p0 = Rt[0] * x0 + Rt[1] * x1 + Rt[2] * x2 + Rt[9];
  const T p1 = Rt[3] * x0 + Rt[4] * x1 + Rt[5] * x2 + Rt[10];
  const T p2 = Rt[6] * x0 + Rt[7] * x1 + Rt[8] * x2 + Rt[11];
  if (p2 > q.eps) {
    const T iz = T(1) / p2;
    const T zp0 = q.focal * p0 * iz + q.cx, zp1 = q.focal * p1 * iz + q.cy;
    if (!kGtOnly) {
      const T e0 = zz.x - zp0, e1 = zz.y - zp1;
      const T s = e0 * e0 + e1 * e1;
      acc[0] += s;
      acc[1] += misfit<T>(q.loss, q.lp, s);
    }
    if (P.zt && counted) {
      const T g0 = zp0 - gt.x, g1 = zp1 - gt.y;
      acc[2] += g0 * g0 + g1 * g1;
      acc[7] += T(1);
    }
    acc[3] += T(1);
  } else {
    acc[4] += T(1);
  }
}

// Primal and dual residual terms of one copy coordinate c: the copy relative to the current
// consensus (the stored offset plus the pending consensus change) and rho times that change.
template <typename T>
__device__ __forceinline__ void residual_terms(const DevProblem& P, const Prm<T>& q, int pending, int c, int i,
                                               int j, T offset, T acc[8]) {
  const T dc = c < 3 ? static_cast<const T*>(P.DX)[3 * i + c] : static_cast<const T*>(P.DY)[6 * j + c - 3];
  const T cp = offset + (pending ? dc : T(0));
  const T rd = q.rho(c) * dc;
  acc[5] += cp * cp;
  acc[6] += rd * rd;
}

// four consecutive pixel pairs from a 16-byte aligned address
__device__ __forceinline__ void load4(const float2* p, float2 v[4]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  v[0] = make_float2(a.x, a.y);
  v[1] = make_float2(a.z, a.w);
  v[2] = make_float2(b.x, b.y);
  v[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void load4(const double2* p, double2 v[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = p[k];
}
// four consecutive elements of a copy row (16-byte aligned)
__device__ __forceinline__ void load4(const float* p, float v[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void load4(const double* p, double v[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// Each thread takes four consecutive observations per pass with vector loads of their
// indices, pixels, reference pixels, inlier flags and copy rows (every array starts 256-byte
// aligned and the copy rows' pitch is a multiple of 32 elements), so four independent
// gathers of consensus points and camera poses are in flight per thread.
template <typename T, bool kGtOnly>
__global__ void __launch_bounds__(kMetricThreads) metrics_kernel(DevProblem P, Prm<T> q, int pending) {
  using V2 = typename Num<T>::V2;
  __shared__ double red[8][kMetricThreads];
  const long long l = P.n_obs;
  const T* delta = static_cast<const T*>(P.delta);
  const V2* z = static_cast<const V2*>(P.z);
  const V2* zt = static_cast<const V2*>(P.zt);
  T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long n4 = l / 4, stride = (long long)gridDim.x * kMetricThreads;
  for (long long g = blockIdx.x * (long long)kMetricThreads + threadIdx.x; g < n4; g += stride) {
    const long long o = 4 * g;
    const int4 pi = *reinterpret_cast<const int4*>(P.obs_pt + o);
    const int4 ci = *reinterpret_cast<const int4*>(P.obs_cam_rank + o);
    const int ii[4] = {pi.x, pi.y, pi.z, pi.w};
    const int jj[4] = {ci.x & kCamMask, ci.y & kCamMask, ci.z & kCamMask, ci.w & kCamMask};
    V2 zz[4] = {}, gt[4] = {};
    if (!kGtOnly) load4(z + o, zz);
    if (zt) load4(zt + o, gt);
    unsigned int inl = 0x01010101u;
    if (P.inlier) inl = *reinterpret_cast<const unsigned int*>(P.inlier + o);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      metric_terms<T, kGtOnly>(P, q, ii[k], jj[k], zz[k], gt[k], ((inl >> (8 * k)) & 0xffu) != 0, acc);
    if (!kGtOnly) {
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        T v[4];
        load4(delta + c * P.pitch + o, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) residual_terms<T>(P, q, pending, c, ii[k], jj[k], v[k], acc);
      }
    }
  }
  // the last l mod 4 observations
  for (long long o = 4 * n4 + blockIdx.x * (long long)kMetricThreads + threadIdx.x; o < l; o += stride) {
    const int i = P.obs_pt[o], j = P.obs_cam_rank[o] & kCamMask;
    const V2 zz = kGtOnly ? V2{} : z[o];
    const V2 gt = zt ? zt[o] : V2{};
    metric_terms<T, kGtOnly>(P, q, i, j, zz, gt, !P.inlier || P.inlier[o], acc);
    if (!kGtOnly)
#pragma unroll
      for (int c = 0; c < 9; ++c) residual_terms<T>(P, q, pending, c, i, j, delta[c * P.pitch + o], acc);
  }
  for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = to_f64<T>(acc[k]);
  __syncthreads();
  for (int w = kMetricThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 8; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 8) P.metric_part[8 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
  // the last block to finish sums every block's partials (strided, then the same tree) into
  // metric_out and rearms the counter for the next launch
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&P.ctl->metric_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  double tot[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kMetricThreads)
    for (int k = 0; k < 8; ++k) tot[k] += __ldcg(&P.metric_part[8 * b + k]);
  for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = tot[k];
  __syncthreads();
  for (int w = kMetricThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 8; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 8) P.metric_out[threadIdx.x] = red[threadIdx.x][0];
  if (threadIdx.x == 0) P.ctl->metric_done = 0u;
}

// Per-scene metrics of a batch: each block walks a contiguous chunk of
// observations (scene ids are nondecreasing in internal order, so a chunk spans
// few scenes); a thread accumulates while its scene stays the same and flushes
// with FP64 atomics when it changes.
constexpr int kSceneChunk = 4096;

template <typename T>
__global__ void __launch_bounds__(kMetricThreads)
scene_metrics_kernel(DevProblem P, Prm<T> q, const int* scene_of_obs, double* out) {
  using V2 = typename Num<T>::V2;
  const long long l = P.n_obs;
  const T* Xm = static_cast<const T*>(P.Xm);
  const T* Ym = static_cast<const T*>(P.Ym);
  const long long o0 = (long long)blockIdx.x * kSceneChunk;
  const long long o1 = o0 + kSceneChunk < l ? o0 + kSceneChunk : l;
  int scene = -1;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long o = o0 + threadIdx.x; o < o1; o += kMetricThreads) {
    const int sc = scene_of_obs[o];
    if (sc != scene) {
      if (scene >= 0)
        for (int k = 0; k < 5; ++k) atomicAdd(&out[5 * scene + k], acc[k]);
      scene = sc;
      for (int k = 0; k < 5; ++k) acc[k] = 0.0;
    }
    const int i = P.obs_pt[o], j = P.obs_cam_rank[o] & kCamMask;
    T v[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = Xm[3 * i + c];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[3 + c] = Ym[6 * j + c];
    Pose<T> Q;
    pose_at(v, q.eps, Q);
    if (!Q.valid) continue;
    const V2 zz = static_cast<const V2*>(P.z)[o];
    const T iz = T(1) / Q.p[2];
    const T zp0 = q.focal * Q.p[0] * iz + q.cx, zp1 = q.focal * Q.p[1] * iz + q.cy;
    const T e0 = zz.x - zp0, e1 = zz.y - zp1;
    const T sq = e0 * e0 + e1 * e1;
    acc[0] += (double)sq;
    acc[1] += (double)misfit<T>(q.loss, q.lp, sq);
    acc[3] += 1.0;
    if (P.zt && (!P.inlier || P.inlier[o])) {
      const V2 gt = static_cast<const V2*>(P.zt)[o];
      const T g0 = zp0 - gt.x, g1 = zp1 - gt.y;
      acc[2] += (double)(g0 * g0 + g1 * g1);
      acc[4] += 1.0;
    }
  }
  if (scene >= 0)
    for (int k = 0; k < 5; ++k) atomicAdd(&out[5 * scene + k], acc[k]);
}


// ------------------------------------------------------------ settle
// Applies a deferred dual ascent and rebases the copies onto the current
// consensus, so the stored state is the paper's (copy, dual) after Eq. (13).
template <typename T>
__global__ void settle_kernel(DevProblem P) {
  const long long l = P.n_obs;
  T* delta = static_cast<T*>(P.delta);
  const T* DX = static_cast<const T*>(P.DX);
  const T* DY = static_cast<const T*>(P.DY);
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < l;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = P.obs_pt[o], j = P.obs_cam_rank[o] & kCamMask;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const long long k = c * P.pitch + o;
      const T d = delta[k] + (c < 3 ? DX[3 * i + c] : DY[6 * j + c - 3]);
      delta[k] = d;
      P.adual[k] += (double)d;
    }
  }
}

// ------------------------------------------------------------ ground truth
template <typename T>
__global__ void project_truth_kernel(DevProblem P, Prm<double> q, const double* cams,
                                     const double* pts, typename Num<T>::V2* out) {
  const long long l = P.n_obs;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < l;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = P.obs_pt[o], j = P.obs_cam_rank[o] & kCamMask;
    double v[9];
    for (int c = 0; c < 3; ++c) v[c] = pts[3 * i + c];
    for (int c = 0; c < 6; ++c) v[3 + c] = cams[6 * j + c];
    Pose<double> Q;
    pose_at(v, -CUDART_INF, Q);
    const double iz = 1.0 / Q.p[2];
    typename Num<T>::V2 r;
    r.x = (T)(q.focal * Q.p[0] * iz + q.cx);
    r.y = (T)(q.focal * Q.p[1] * iz + q.cy);
    out[o] = r;
  }
}

// ------------------------------------------------------------ allocation-free evaluation
// Reprojection statistics at caller-given parameters for callers that cannot
// allocate device memory.  Per-block partial sums go to a file-scope device
// array instead of an allocated buffer; a second single-block kernel reduces
// them into the caller's output.  Each block handles a fixed chunk of
// observations, so the array bounds the number of observations per call.
constexpr int kNoallocThreads = 256;
constexpr int kNoallocObsPerBlock = 4096;
constexpr int kNoallocMaxBlocks = 4096;  // 4096 x 4 doubles = 128 KiB of scratch
static_assert((long long)kNoallocMaxBlocks * kNoallocObsPerBlock == (long long)DBA_NOALLOC_MAX_OBS,
              "scratch size and the documented observation limit must agree");

__device__ __align__(256) double g_noalloc_partials[kNoallocMaxBlocks * 4];

__global__ void __launch_bounds__(kNoallocThreads)
eval_noalloc_kernel(Prm<double> q, long long l, int n_cams, int n_pts, const int* pt_idx, const int* cam_idx,
                    const double2* z, const double* cams, const double* pts, double* partials) {
  __shared__ double red[4][kNoallocThreads];
  double acc[4] = {0, 0, 0, 0};
  const long long o0 = (long long)blockIdx.x * kNoallocObsPerBlock;
  const long long o1 = o0 + kNoallocObsPerBlock < l ? o0 + kNoallocObsPerBlock : l;
  for (long long o = o0 + threadIdx.x; o < o1; o += kNoallocThreads) {
    const int i = pt_idx[o], j = cam_idx[o];
    if (i < 0 || i >= n_pts || j < 0 || j >= n_cams) {  // not evaluated: index out of range
      acc[3] += 1.0;
      continue;
    }
    double v[9];
    for (int c = 0; c < 3; ++c) v[c] = pts[3 * (long long)i + c];
    for (int c = 0; c < 6; ++c) v[3 + c] = cams[6 * (long long)j + c];
    Pose<double> Q;
    pose_at(v, q.eps, Q);
    if (Q.valid) {
      const double iz = 1.0 / Q.p[2];
      const double2 zz = z[o];
      const double e0 = zz.x - (q.focal * Q.p[0] * iz + q.cx);
      const double e1 = zz.y - (q.focal * Q.p[1] * iz + q.cy);
      const double sq = e0 * e0 + e1 * e1;
      acc[0] += sq;
      acc[1] += misfit<double>(q.loss, q.lp, sq);
      acc[2] += 1.0;
    } else {
      acc[3] += 1.0;
    }
  }
  for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kNoallocThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) partials[4 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(kNoallocThreads)
eval_noalloc_final_kernel(const double* partials, int nblocks, double* out) {
  __shared__ double red[4][kNoallocThreads];
  double acc[4] = {0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += kNoallocThreads)
    for (int k = 0; k < 4; ++k) acc[k] += partials[4 * b + k];
  for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kNoallocThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = red[threadIdx.x][0];
}

int grid_for(long long n, int threads, int cap) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

namespace {
// Persistent grid of the pipelined tile kernel: resident blocks per SM times SMs, set up
// once per instantiation (dynamic shared memory opt-in, occupancy query).
template <typename T, int NT, int kS>
cudaError_t tile_grid(int* grid) {
  // per process and device-independent: first caller computes; racing callers compute the same
  static std::atomic<int> cached{0};
  if (!cached) {
    const int smem = (int)tile_smem_bytes<T, NT>();
    cudaError_t e =
        cudaFuncSetAttribute(tile_iterate_kernel<T, NT, kS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_iterate_kernel<T, NT, kS>, NT, smem);
    if (e != cudaSuccess) return e;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    cached = (per_sm > 0 ? per_sm : 1) * sms;
  }
  *grid = cached;
  return cudaSuccess;
}

template <typename T, int NT, int kS>
cudaError_t launch_tile(const DevProblem& P, const TileMaps& M, const Params& prm, cudaStream_t s) {
  int grid = 0;
  const cudaError_t e = tile_grid<T, NT, kS>(&grid);
  if (e != cudaSuccess) return e;
  if (grid > P.n_tiles) grid = P.n_tiles;
  tile_iterate_kernel<T, NT, kS><<<grid, NT, tile_smem_bytes<T, NT>(), s>>>(P, M, make_prm<T>(prm));
  return cudaGetLastError();
}

template <typename T, int kS>
cudaError_t launch_tile_sized(const DevProblem& P, const TileMaps& M, const Params& prm, cudaStream_t s) {
  switch (P.tile_obs) {
    case 256: return launch_tile<T, 256, kS>(P, M, prm, s);
    case 128: return launch_tile<T, 128, kS>(P, M, prm, s);
    case 64: return launch_tile<T, 64, kS>(P, M, prm, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t prepare_tile_kernels() {
  int g = 0;
  cudaError_t e;
  if ((e = tile_grid<float, 256, DBA_SOLVER_GN>(&g)) != cudaSuccess) return e;
  if ((e = tile_grid<float, 128, DBA_SOLVER_GN>(&g)) != cudaSuccess) return e;
  if ((e = tile_grid<float, 64, DBA_SOLVER_GN>(&g)) != cudaSuccess) return e;
  if ((e = tile_grid<double, 256, DBA_SOLVER_GN>(&g)) != cudaSuccess) return e;
  if ((e = tile_grid<double, 128, DBA_SOLVER_GN>(&g)) != cudaSuccess) return e;
  if ((e = tile_grid<double, 64, DBA_SOLVER_GN>(&g)) != cudaSuccess) return e;
  if ((e = tile_grid<float, 256, DBA_SOLVER_LBFGS>(&g)) != cudaSuccess) return e;
  if ((e = tile_grid<float, 128, DBA_SOLVER_LBFGS>(&g)) != cudaSuccess) return e;
  if ((e = tile_grid<float, 64, DBA_SOLVER_LBFGS>(&g)) != cudaSuccess) return e;
  if ((e = tile_grid<double, 256, DBA_SOLVER_LBFGS>(&g)) != cudaSuccess) return e;
  if ((e = tile_grid<double, 128, DBA_SOLVER_LBFGS>(&g)) != cudaSuccess) return e;
  return tile_grid<double, 64, DBA_SOLVER_LBFGS>(&g);
}

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// rank-1 or rank-2 map of a row-major array: dims[0] innermost (elements), stride1 the
// byte stride of dimension 1, box the copied extent; out-of-range elements read as zero
cudaError_t encode(CUtensorMap* map, CUtensorMapDataType type, int rank, const void* base, cuuint64_t dim0,
                   cuuint64_t dim1, cuuint64_t stride1, cuuint32_t box0, cuuint32_t box1) {
  EncodeTiled fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {dim0, dim1};
  const cuuint64_t strides[1] = {stride1};
  const cuuint32_t box[2] = {box0, box1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, type, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T, int NT>
cudaError_t encode_maps(const DevProblem& P, TileMaps* M) {
  using St = TileStage<T, NT>;
  const cuuint64_t l = (cuuint64_t)P.n_obs, rowT = (cuuint64_t)P.pitch * sizeof(T), rowD = (cuuint64_t)P.pitch * 8;
  const CUtensorMapDataType tT = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  cudaError_t e = encode(&M->delta, tT, 2, P.delta, l, 9, rowT, St::kWT, 9);
  if (e == cudaSuccess) e = encode(&M->adual, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, P.adual, l, 9, rowD, St::kWD, 9);
  if (e == cudaSuccess) {
    if constexpr (sizeof(T) == 4)
      e = encode(&M->z, CU_TENSOR_MAP_DATA_TYPE_INT64, 1, P.z, l, 1, 16, St::kWZ, 1);
    else
      e = encode(&M->z, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, P.z, 2, l, 16, 2, St::kWZ);
  }
  if (e == cudaSuccess) e = encode(&M->pt, CU_TENSOR_MAP_DATA_TYPE_INT32, 1, P.obs_pt, l, 1, 16, St::kWI, 1);
  if (e == cudaSuccess) e = encode(&M->cam, CU_TENSOR_MAP_DATA_TYPE_INT32, 1, P.obs_cam_rank, l, 1, 16, St::kWI, 1);
  return e;
}

template <typename T>
cudaError_t encode_maps_sized(const DevProblem& P, TileMaps* M) {
  switch (P.tile_obs) {
    case 256: return encode_maps<T, 256>(P, M);
    case 128: return encode_maps<T, 128>(P, M);
    case 64: return encode_maps<T, 64>(P, M);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t encode_tile_maps(const DevProblem& P, bool fp32, TileMaps* M) {
  *M = TileMaps{};
  if (P.n_obs <= 0) return cudaSuccess;
  // the kernel's coordinates are 32-bit; the row pitch keeps every row 16-byte aligned
  if (P.n_obs > 0x7fffffffLL || P.pitch % 4 != 0) return cudaErrorInvalidValue;
  return fp32 ? encode_maps_sized<float>(P, M) : encode_maps_sized<double>(P, M);
}

cudaError_t launch_tile_iterate(const DevProblem& P, const TileMaps& M, const Params& prm, bool fp32,
                                cudaStream_t s) {
  if (P.n_tiles == 0) return cudaSuccess;
  if (prm.solver == DBA_SOLVER_LBFGS)
    return fp32 ? launch_tile_sized<float, DBA_SOLVER_LBFGS>(P, M, prm, s)
                : launch_tile_sized<double, DBA_SOLVER_LBFGS>(P, M, prm, s);
  return fp32 ? launch_tile_sized<float, DBA_SOLVER_GN>(P, M, prm, s)
              : launch_tile_sized<double, DBA_SOLVER_GN>(P, M, prm, s);
}

template <typename T>
void launch_finalize_sized(const DevProblem& P, int blocks, cudaStream_t s) {
  switch (P.fin_threads) {
    case 32: finalize_kernel<T, 32><<<blocks, 32, 0, s>>>(P); break;
    case 64: finalize_kernel<T, 64><<<blocks, 64, 0, s>>>(P); break;
    case 256: finalize_kernel<T, 256><<<blocks, 256, 0, s>>>(P); break;
    default: finalize_kernel<T, 128><<<blocks, 128, 0, s>>>(P); break;
  }
}

cudaError_t launch_finalize(const DevProblem& P, bool fp32, cudaStream_t s) {
  const int blocks = P.n_cams + P.n_split_pts;
  if (fp32)
    launch_finalize_sized<float>(P, blocks, s);
  else
    launch_finalize_sized<double>(P, blocks, s);
  return cudaGetLastError();
}

cudaError_t launch_metrics(const DevProblem& P, const Params& prm, bool fp32, int cur, int pending,
                           cudaStream_t s, bool gt_only) {
  (void)cur;
  // one wave of resident blocks (at most kMetricBlocks, the partial-sum slots)
  static std::atomic<int> resident[4] = {};
  const int key = (fp32 ? 0 : 2) + (gt_only ? 1 : 0);
  int cap = resident[key].load();
  if (!cap) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e0 = fp32 ? (gt_only ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, metrics_kernel<float, true>, kMetricThreads, 0)
                                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, metrics_kernel<float, false>, kMetricThreads, 0))
                          : (gt_only ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, metrics_kernel<double, true>, kMetricThreads, 0)
                                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, metrics_kernel<double, false>, kMetricThreads, 0));
    if (e0 == cudaSuccess) e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e0 != cudaSuccess) return e0;
    cap = std::max(1, std::min(kMetricBlocks, per_sm * sms));
    resident[key].store(cap);
  }
  const int g = grid_for(P.n_obs, kMetricThreads, cap);
  const int gc = (P.n_cams + 127) / 128;
  if (fp32) {
    camera_pose_kernel<float><<<gc, 128, 0, s>>>(P);
    if (gt_only)
      metrics_kernel<float, true><<<g, kMetricThreads, 0, s>>>(P, make_prm<float>(prm), pending);
    else
      metrics_kernel<float, false><<<g, kMetricThreads, 0, s>>>(P, make_prm<float>(prm), pending);
  } else {
    camera_pose_kernel<double><<<gc, 128, 0, s>>>(P);
    if (gt_only)
      metrics_kernel<double, true><<<g, kMetricThreads, 0, s>>>(P, make_prm<double>(prm), pending);
    else
      metrics_kernel<double, false><<<g, kMetricThreads, 0, s>>>(P, make_prm<double>(prm), pending);
  }
  return cudaGetLastError();
}

cudaError_t launch_scene_metrics(const DevProblem& P, const Params& prm, bool fp32, const int* scene_of_obs,
                                 double* out, cudaStream_t s) {
  const int g = (int)((P.n_obs + kSceneChunk - 1) / kSceneChunk);
  if (g == 0) return cudaSuccess;
  if (fp32)
    scene_metrics_kernel<float><<<g, kMetricThreads, 0, s>>>(P, make_prm<float>(prm), scene_of_obs, out);
  else
    scene_metrics_kernel<double><<<g, kMetricThreads, 0, s>>>(P, make_prm<double>(prm), scene_of_obs, out);
  return cudaGetLastError();
}

cudaError_t launch_settle(const DevProblem& P, bool fp32, int cur, cudaStream_t s) {
  (void)cur;
  const int g = grid_for(P.n_obs, 256, 152 * 16);
  if (fp32)
    settle_kernel<float><<<g, 256, 0, s>>>(P);
  else
    settle_kernel<double><<<g, 256, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_project_truth(const DevProblem& P, const Params& prm, bool fp32,
                                 const double* cams_gt, const double* pts_gt, void* zt_out,
                                 cudaStream_t s) {
  const int g = grid_for(P.n_obs, 256, 152 * 16);
  const Prm<double> q = make_prm<double>(prm);
  if (fp32)
    project_truth_kernel<float><<<g, 256, 0, s>>>(P, q, cams_gt, pts_gt, static_cast<float2*>(zt_out));
  else
    project_truth_kernel<double><<<g, 256, 0, s>>>(P, q, cams_gt, pts_gt, static_cast<double2*>(zt_out));
  return cudaGetLastError();
}

// Device address of g_noalloc_partials, looked up once per device with that
// device current.  In host code the symbol's name is only a host-side stand-in.
namespace {
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[256] = {nullptr};
}  // namespace

cudaError_t launch_eval_noalloc(const Params& prm, long long n_obs, int n_cams, int n_pts, const int* pt_idx,
                                const int* cam_idx, const double* z, const double* cams, const double* pts,
                                double* out, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
      if (e != cudaSuccess) return e;
      g_noalloc_addr[dev] = static_cast<double*>(ptr);
    }
    scratch = g_noalloc_addr[dev];
  }
  const int blocks = n_obs > 0 ? (int)((n_obs + kNoallocObsPerBlock - 1) / kNoallocObsPerBlock) : 0;
  if (blocks > kNoallocMaxBlocks) return cudaErrorInvalidValue;
  if (blocks > 0) {
    eval_noalloc_kernel<<<blocks, kNoallocThreads, 0, s>>>(make_prm<double>(prm), n_obs, n_cams, n_pts, pt_idx,
                                                           cam_idx, reinterpret_cast<const double2*>(z), cams,
                                                           pts, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  eval_noalloc_final_kernel<<<1, kNoallocThreads, 0, s>>>(scratch, blocks, out);
  return cudaGetLastError();
}

}  // namespace dba

