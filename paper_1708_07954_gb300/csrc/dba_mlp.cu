// Learned warm start for the local solves (no counterpart in the paper).
//
// A 32-64-64-64-16 GELU network maps the features of one local problem
// (warm_features in dba_device.cuh) to the scaled step r (d* - d0) towards the
// solution of a long local solve.  This unit holds
//   - harvest_kernel: features and targets from the current ADMM state;
//   - FP32 training kernels (tiled SGEMM, GELU, loss, Adam);
//   - mlp_infer_kernel: BF16 tensor-core inference with tcgen05.mma (operands
//     in shared memory, FP32 accumulators in tensor memory), either on given
//     features or fused with feature extraction from the ADMM state, writing a
//     candidate start that the local solve keeps only if it lowers Eq. (9).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/dba.h"
#include "dba_device.cuh"
#include "dba_internal.h"
#include "dba_guard.h"

namespace dba {
namespace {

// flat FP32 parameter layout
constexpr int kW1 = 0;                                  // [64][32]
constexpr int kB1 = kW1 + kMlpHidden * kMlpIn;          // [64]
constexpr int kW2 = kB1 + kMlpHidden;                   // [64][64]
constexpr int kB2 = kW2 + kMlpHidden * kMlpHidden;      // [64]
constexpr int kW3 = kB2 + kMlpHidden;                   // [64][64]
constexpr int kB3 = kW3 + kMlpHidden * kMlpHidden;      // [64]
constexpr int kW4 = kB3 + kMlpHidden;                   // [16][64]
constexpr int kB4 = kW4 + kMlpOut * kMlpHidden;         // [16]
constexpr int kTrainable = kB4 + kMlpOut;
constexpr int kInMean = kTrainable;                     // [32]
constexpr int kInStd = kInMean + kMlpIn;                // [32]
constexpr int kOutStd = kInStd + kMlpIn;                // [16]
constexpr int kNParams = kOutStd + kMlpOut;
static_assert(kNParams == DBA_MLP_N_PARAMS, "parameter count must match the header");

// ------------------------------------------------------------ harvest
// Reconstructs each sampled observation's local problem as the next iteration
// would see it (deferred dual ascent applied), computes its features, and runs
// a long local solve from the plain start for the target.  Reads the state only.
template <typename T>
__global__ void harvest_kernel(DevProblem P, Prm<T> q, int pending, long long stride, long long cap, float* feats,
                               float* targs) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= cap) return;
  const long long l = P.pitch, o = k * stride;  // l: row stride of delta and adual
  float* f = feats + k * kMlpIn;
  float* g = targs + k * kMlpOut;
  const int i = P.obs_pt[o], j = P.obs_cam_rank[o] & kCamMask;
  const T* delta = static_cast<const T*>(P.delta);
  const T* Xm = static_cast<const T*>(P.Xm);
  const T* Ym = static_cast<const T*>(P.Ym);
  const T* DX = static_cast<const T*>(P.DX);
  const T* DY = static_cast<const T*>(P.DY);
  T d0[9], vbar[9], aT[9], r[9];
  for (int c = 0; c < 9; ++c) {
    d0[c] = delta[c * l + o] + (pending ? (c < 3 ? DX[3 * i + c] : DY[6 * j + c - 3]) : T(0));
    const double a = P.adual[c * l + o] + (pending ? (double)d0[c] : 0.0);
    aT[c] = (T)a;
    vbar[c] = c < 3 ? Xm[3 * i + c] : Ym[6 * j + c - 3];
  }
  const typename Num<T>::V2 zz = static_cast<const typename Num<T>::V2*>(P.z)[o];
  float feat[kMlpIn];
  const bool ok = warm_features<T>(zz.x, zz.y, vbar, aT, d0, q, feat, r);
  for (int c = 0; c < kMlpIn; ++c) f[c] = feat[c];
  T d[9];
  for (int c = 0; c < 9; ++c) d[c] = d0[c];
  if (ok) local_solve<T>(zz.x, zz.y, vbar, aT, d, q);
  for (int c = 0; c < kMlpOut; ++c) g[c] = (ok && c < 9) ? (float)(r[c] * (d[c] - d0[c])) : 0.f;
}

// ------------------------------------------------------------ activation
// GELU in its tanh form (Hendrycks and Gimpel): x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
constexpr float kGeluC = 0.7978845608028654f;  // sqrt(2/pi)
constexpr float kGeluA = 0.044715f;
// training: CUDA's tanhf
__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.f + tanhf(kGeluC * fmaf(kGeluA * x * x, x, x)));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float t = tanhf(kGeluC * fmaf(kGeluA * x * x, x, x));
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * kGeluC * fmaf(3.f * kGeluA, x * x, 1.f);
}
// inference: the SFU tanh (PTX tanh.approx.f32, relative error about 2^-11, well below the
// BF16 rounding of the activations that follows)
__device__ __forceinline__ float gelu_fast(float x) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(kGeluC * fmaf(kGeluA * x * x, x, x)));
  const float h = 0.5f * x;
  return fmaf(h, t, h);
}

// ------------------------------------------------------------ training (FP32)

// C[M x N] = op(A) op(B) (+ C if accumulate), row-major; op(A) is M x K, op(B) K x N.
constexpr int kGemmTile = 16;
__global__ void sgemm_kernel(int M, int N, int K, const float* A, int lda, int ta, const float* B, int ldb, int tb,
                             float* C, int ldc, int accumulate) {
  __shared__ float sa[kGemmTile][kGemmTile + 1];
  __shared__ float sb[kGemmTile][kGemmTile + 1];
  const int row = blockIdx.y * kGemmTile + threadIdx.y, col = blockIdx.x * kGemmTile + threadIdx.x;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += kGemmTile) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    sa[threadIdx.y][threadIdx.x] =
        (row < M && ka < K) ? (ta ? A[(long long)ka * lda + row] : A[(long long)row * lda + ka]) : 0.f;
    sb[threadIdx.y][threadIdx.x] =
        (kb < K && col < N) ? (tb ? B[(long long)col * ldb + kb] : B[(long long)kb * ldb + col]) : 0.f;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGemmTile; ++k) acc += sa[threadIdx.y][k] * sb[k][threadIdx.x];
    __syncthreads();
  }
  if (row < M && col < N) {
    float* c = C + (long long)row * ldc + col;
    *c = accumulate ? *c + acc : acc;
  }
}

void sgemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, bool ta, const float* B, int ldb, bool tb,
           float* C, int ldc, bool accumulate = false) {
  const dim3 block(kGemmTile, kGemmTile), grid((N + kGemmTile - 1) / kGemmTile, (M + kGemmTile - 1) / kGemmTile);
  sgemm_kernel<<<grid, block, 0, s>>>(M, N, K, A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, C, ldc, accumulate ? 1 : 0);
}

// rows of X gathered by idx (or in order), standardised with the network's input statistics
__global__ void gather_standardize_kernel(const float* X, const int* idx, int n, const float* params, float* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * kMlpIn) return;
  const int r = e / kMlpIn, c = e % kMlpIn;
  const long long src = idx ? idx[r] : r;
  out[e] = (X[src * kMlpIn + c] - params[kInMean + c]) / params[kInStd + c];
}
__global__ void gather_targets_kernel(const float* Y, const int* idx, int n, const float* params, float* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * kMlpOut) return;
  const int r = e / kMlpOut, c = e % kMlpOut;
  const long long src = idx ? idx[r] : r;
  out[e] = Y[src * kMlpOut + c] / params[kOutStd + c];
}
// Z += bias (per column); H = GELU(Z) when H != nullptr
__global__ void bias_act_kernel(float* Z, const float* bias, int n, int width, float* H) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * width) return;
  const float z = Z[e] + bias[e % width];
  Z[e] = z;
  if (H) H[e] = gelu(z);
}
// dY = 2 (Y - T) / (n * 9) on the 9 used outputs; loss partial sums
__global__ void loss_grad_kernel(const float* Y, const float* Tt, int n, float* dY, double* loss) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (e < n * kMlpOut) {
    const int c = e % kMlpOut;
    const float diff = c < kMlpUsedOut ? Y[e] - Tt[e] : 0.f;
    dY[e] = 2.f * diff / (float)(n * kMlpUsedOut);
    l = (double)diff * diff;
  }
  for (int w = 16; w > 0; w >>= 1) l += __shfl_down_sync(0xffffffffu, l, w);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / (double)(n * kMlpUsedOut));
}
// dZ = dH * GELU'(Z)
__global__ void act_back_kernel(const float* dH, const float* Z, int total, float* dZ) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < total) dZ[e] = dH[e] * gelu_grad(Z[e]);
}
// column sums of dZ into grad (bias gradient)
__global__ void colsum_kernel(const float* dZ, int n, int width, float* out) {
  const int c = blockIdx.x;
  float acc = 0.f;
  for (int r = threadIdx.x; r < n; r += blockDim.x) acc += dZ[(long long)r * width + c];
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.f - b1) * gi;
  const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}
// column moments of features and targets for the normaliser
__global__ void moments_kernel(const float* X, const float* Y, long long n, double* acc) {
  const int c = blockIdx.x;  // 0..47
  const bool feat = c < kMlpIn;
  const int width = feat ? kMlpIn : kMlpOut, col = feat ? c : c - kMlpIn;
  const float* A = feat ? X : Y;
  double s = 0.0, s2 = 0.0;
  for (long long r = threadIdx.x; r < n; r += blockDim.x) {
    const double x = A[r * width + col];
    s += x;
    s2 += x * x;
  }
  __shared__ double r1[256], r2[256];
  r1[threadIdx.x] = s;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      r1[threadIdx.x] += r1[threadIdx.x + w];
      r2[threadIdx.x] += r2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    acc[2 * c] = r1[0];
    acc[2 * c + 1] = r2[0];
  }
}

int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace
}  // namespace dba

// ------------------------------------------------------------ network object
struct dba_mlp {
  cudaStream_t stream = nullptr;
  float* params = nullptr;  // [kNParams] FP32 master copy on the device
  float* grad = nullptr;    // [kNParams]
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  long long adam_t = 0;
  // scratch for a batch of up to `cap` rows
  int cap = 0;
  float *x = nullptr, *t = nullptr, *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *z3 = nullptr,
        *h3 = nullptr, *y = nullptr, *dy = nullptr, *d64a = nullptr, *d64b = nullptr;
  int* idx = nullptr;
  double* dloss = nullptr;
  std::string err;
};

namespace dba {
namespace {

cudaError_t mlp_reserve(dba_mlp* m, int rows) {
  if (rows <= m->cap) return cudaSuccess;
  float** bufs64[] = {&m->z1, &m->h1, &m->z2, &m->h2, &m->z3, &m->h3, &m->d64a, &m->d64b};
  for (float** b : bufs64) {
    cudaFree(*b);
    cudaError_t e = cudaMalloc(b, sizeof(float) * (size_t)rows * kMlpHidden);
    if (e != cudaSuccess) return e;
  }
  cudaFree(m->x);
  cudaFree(m->t);
  cudaFree(m->y);
  cudaFree(m->dy);
  cudaFree(m->idx);
  cudaError_t e;
  if ((e = cudaMalloc(&m->x, sizeof(float) * (size_t)rows * kMlpIn)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->t, sizeof(float) * (size_t)rows * kMlpOut)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->y, sizeof(float) * (size_t)rows * kMlpOut)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->dy, sizeof(float) * (size_t)rows * kMlpOut)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->idx, sizeof(int) * (size_t)rows)) != cudaSuccess) return e;
  m->cap = rows;
  return cudaSuccess;
}

// Forward and backward of one batch already staged in m->x (standardised) and m->t;
// leaves the loss in m->dloss and the gradient in m->grad.
cudaError_t mlp_forward_backward(dba_mlp* m, int n) {
  cudaStream_t s = m->stream;
  const float* P = m->params;
  float* G = m->grad;
  const int H = kMlpHidden;
  // forward: Z1 = X W1^T + b1 ...
  sgemm(s, n, H, kMlpIn, m->x, kMlpIn, false, P + kW1, kMlpIn, true, m->z1, H);
  bias_act_kernel<<<blocks_for((long long)n * H, 256), 256, 0, s>>>(m->z1, P + kB1, n, H, m->h1);
  sgemm(s, n, H, H, m->h1, H, false, P + kW2, H, true, m->z2, H);
  bias_act_kernel<<<blocks_for((long long)n * H, 256), 256, 0, s>>>(m->z2, P + kB2, n, H, m->h2);
  sgemm(s, n, H, H, m->h2, H, false, P + kW3, H, true, m->z3, H);
  bias_act_kernel<<<blocks_for((long long)n * H, 256), 256, 0, s>>>(m->z3, P + kB3, n, H, m->h3);
  sgemm(s, n, kMlpOut, H, m->h3, H, false, P + kW4, H, true, m->y, kMlpOut);
  bias_act_kernel<<<blocks_for((long long)n * kMlpOut, 256), 256, 0, s>>>(m->y, P + kB4, n, kMlpOut, nullptr);
  cudaMemsetAsync(m->dloss, 0, sizeof(double), s);
  loss_grad_kernel<<<blocks_for((long long)n * kMlpOut, 256), 256, 0, s>>>(m->y, m->t, n, m->dy, m->dloss);
  // backward
  cudaMemsetAsync(G, 0, sizeof(float) * kNParams, s);
  sgemm(s, kMlpOut, H, n, m->dy, kMlpOut, true, m->h3, H, false, G + kW4, H);    // dW4 = dY^T H3
  colsum_kernel<<<kMlpOut, 256, 0, s>>>(m->dy, n, kMlpOut, G + kB4);
  sgemm(s, n, H, kMlpOut, m->dy, kMlpOut, false, P + kW4, H, false, m->d64a, H);  // dH3 = dY W4
  act_back_kernel<<<blocks_for((long long)n * H, 256), 256, 0, s>>>(m->d64a, m->z3, n * H, m->d64b);
  sgemm(s, H, H, n, m->d64b, H, true, m->h2, H, false, G + kW3, H);              // dW3 = dZ3^T H2
  colsum_kernel<<<H, 256, 0, s>>>(m->d64b, n, H, G + kB3);
  sgemm(s, n, H, H, m->d64b, H, false, P + kW3, H, false, m->d64a, H);           // dH2 = dZ3 W3
  act_back_kernel<<<blocks_for((long long)n * H, 256), 256, 0, s>>>(m->d64a, m->z2, n * H, m->d64b);
  sgemm(s, H, H, n, m->d64b, H, true, m->h1, H, false, G + kW2, H);              // dW2 = dZ2^T H1
  colsum_kernel<<<H, 256, 0, s>>>(m->d64b, n, H, G + kB2);
  sgemm(s, n, H, H, m->d64b, H, false, P + kW2, H, false, m->d64a, H);           // dH1 = dZ2 W2
  act_back_kernel<<<blocks_for((long long)n * H, 256), 256, 0, s>>>(m->d64a, m->z1, n * H, m->d64b);
  sgemm(s, H, kMlpIn, n, m->d64b, H, true, m->x, kMlpIn, false, G + kW1, kMlpIn);  // dW1 = dZ1^T X
  colsum_kernel<<<H, 256, 0, s>>>(m->d64b, n, H, G + kB1);
  return cudaGetLastError();
}

}  // namespace
}  // namespace dba

// ------------------------------------------------------------ tensor-core inference
namespace dba {
namespace {

constexpr int kInferThreads = 128;  // one observation per thread, M = 128 rows per MMA
// BF16 weights in the canonical no-swizzle K-major layout of tcgen05 operands
constexpr int kBlobW1 = 0;
constexpr int kBlobW2 = kBlobW1 + kMlpHidden * kMlpIn * 2;
constexpr int kBlobW3 = kBlobW2 + kMlpHidden * kMlpHidden * 2;
constexpr int kBlobW4 = kBlobW3 + kMlpHidden * kMlpHidden * 2;
constexpr int kBlobBytes = kBlobW4 + kMlpOut * kMlpHidden * 2;

// Byte offset of element (row, k) of a K-major operand with kdim columns: core
// matrices of 8 rows x 16 bytes, adjacent along K at 128 bytes (LBO), 8-row
// groups at kdim/8 * 128 bytes (SBO).
__host__ __device__ constexpr uint32_t kmajor_off(int row, int k, int kdim) {
  return (uint32_t)((row >> 3) * (kdim / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

struct __align__(128) MlpSmem {
  unsigned char w[kBlobBytes];
  // one 128-row activation tile: the layer-1 operand (K = 32 layout) and then, in
  // place, each hidden layer's output (K = 64 layout); a layer's MMA has completed
  // before its epilogue overwrites the tile
  unsigned char act[kInferThreads * kMlpHidden * 2];
  float bias[3 * kMlpHidden + kMlpOut];
  float in_scale[kMlpIn], in_shift[kMlpIn];  // x = f * scale + shift standardises a feature
  float out_scale[kMlpOut];                  // target scale / r: network output -> step in d
  unsigned long long mbar;
  uint32_t tmem;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading (K) and stride (8-row) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N
__device__ __forceinline__ uint32_t umma_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D[128 x n] = A[128 x kdim] B[n x kdim]^T, issued by one thread, completion on mbar
__device__ __forceinline__ void mma_layer(uint32_t tmem, uint32_t a, uint32_t b, int kdim, int n, uint32_t mbar) {
  const uint32_t idesc = umma_idesc(128, n);
  const uint32_t sbo = (uint32_t)(kdim / 8) * 128;
  for (int ks = 0; ks < kdim / 16; ++ks) {
    const uint64_t da = umma_desc(a + ks * 256, 128, sbo);
    const uint64_t db = umma_desc(b + ks * 256, 128, sbo);
    const uint32_t acc = ks > 0 ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// bounded wait for the mbarrier phase; false after the limit
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
  return done != 0;
}

// 16 consecutive accumulator columns of this thread's row
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

// the operand writes of all threads become visible to the tensor cores, and no
// thread runs ahead of the previous tensor-memory reads
__device__ __forceinline__ void operands_ready() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&p);
}

// Hidden layer epilogue: bias + GELU of the accumulator row, BF16 into the
// activation tile; 16 columns at a time, two 16-byte stores per 16 columns (the
// 8 rows of a core matrix fill 128 contiguous bytes: no bank conflicts).
__device__ __forceinline__ void hidden_epilogue(uint32_t trow, const float* bias, unsigned char* act, int row) {
#pragma unroll
  for (int c0 = 0; c0 < kMlpHidden; c0 += 16) {
    float h[16];
    tmem_ld16(trow + c0, h);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int c = c0 + 8 * half;
      uint4 v;
      v.x = pack_bf16x2(gelu_fast(h[8 * half + 0] + bias[c + 0]), gelu_fast(h[8 * half + 1] + bias[c + 1]));
      v.y = pack_bf16x2(gelu_fast(h[8 * half + 2] + bias[c + 2]), gelu_fast(h[8 * half + 3] + bias[c + 3]));
      v.z = pack_bf16x2(gelu_fast(h[8 * half + 4] + bias[c + 4]), gelu_fast(h[8 * half + 5] + bias[c + 5]));
      v.w = pack_bf16x2(gelu_fast(h[8 * half + 6] + bias[c + 6]), gelu_fast(h[8 * half + 7] + bias[c + 7]));
      *reinterpret_cast<uint4*>(act + kmajor_off(row, c, kMlpHidden)) = v;
    }
  }
}

// Prefetches into L2 the state rows of the 128 observations from nb on (offsets and
// duals, nine rows each, pixels, point and camera indices), one 128-byte line per
// thread and pass, clipped to the arrays.
template <typename T>
__device__ __forceinline__ void prefetch_state_l2(const DevProblem& P, long long nb, int t) {
  constexpr int kLT = 128 * (int)sizeof(T) / 128 + 1, kLD = 8 + 1;
  constexpr int kLZ = 128 * 2 * (int)sizeof(T) / 128 + 1, kLI = 4 + 1;
  constexpr int kLines = 9 * kLT + 9 * kLD + kLZ + 2 * kLI;
  const long long n = P.n_obs, l = P.pitch;
  if (nb >= n) return;
  const long long m = (n - nb < 128 ? n - nb : 128);  // observations in the tile
  for (int e = t; e < kLines; e += kInferThreads) {
    const char* base;
    long long bytes;
    int line;
    if (e < 9 * kLT) {
      base = static_cast<const char*>(P.delta) + ((e / kLT) * l + nb) * (long long)sizeof(T);
      bytes = m * (long long)sizeof(T);
      line = e % kLT;
    } else if (e < 9 * kLT + 9 * kLD) {
      const int f = e - 9 * kLT;
      base = reinterpret_cast<const char*>(P.adual + (f / kLD) * l + nb);
      bytes = m * 8;
      line = f % kLD;
    } else if (e < 9 * kLT + 9 * kLD + kLZ) {
      base = static_cast<const char*>(P.z) + nb * 2 * (long long)sizeof(T);
      bytes = m * 2 * (long long)sizeof(T);
      line = e - 9 * kLT - 9 * kLD;
    } else {
      const int f = e - 9 * kLT - 9 * kLD - kLZ;
      base = reinterpret_cast<const char*>((f < kLI ? P.obs_pt : P.obs_cam_rank) + nb);
      bytes = m * 4;
      line = f % kLI;
    }
    // the line holding byte 128 * line of the range, counted from the range's aligned start
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(base) & ~(uintptr_t)127;
    const uintptr_t a = a0 + 128 * (uintptr_t)line;
    if (a < reinterpret_cast<uintptr_t>(base) + (uintptr_t)bytes)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
  }
}

// Persistent inference.  kFromState: features from the ADMM state of every
// observation, output = candidate start d0 + step / r written to P.mlp_start;
// else features from `feats` (n rows), output = the network's 16 standardised
// outputs.  Each CTA holds the weights once and walks tiles of 128 rows, one
// row per thread; the activations of a tile stay in shared memory (BF16
// operands) and tensor memory (FP32 accumulators, 64 columns).
template <typename T, bool kFromState>
__global__ void __launch_bounds__(kInferThreads, 4) mlp_infer_kernel(DevProblem P, Prm<T> q,
                                                                     const unsigned char* blob, const float* params,
                                                                     const float* feats, long long n, float* y_out,
                                                                     int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  const int t = threadIdx.x;
  for (int e = t; e < kBlobBytes / 16; e += kInferThreads)
    reinterpret_cast<int4*>(S.w)[e] = reinterpret_cast<const int4*>(blob)[e];
  for (int e = t; e < kMlpHidden; e += kInferThreads) {
    S.bias[e] = params[kB1 + e];
    S.bias[kMlpHidden + e] = params[kB2 + e];
    S.bias[2 * kMlpHidden + e] = params[kB3 + e];
  }
  if (t < kMlpOut) {
    S.bias[3 * kMlpHidden + t] = params[kB4 + t];
    // the step in d is (output * target scale) / r, r = sqrt(rho) of the component
    S.out_scale[t] = kFromState && t < 9 ? (float)((double)params[kOutStd + t] / sqrt((double)q.rho(t)))
                                         : params[kOutStd + t];
  }
  if (t < kMlpIn) {
    const float sd = params[kInStd + t];
    S.in_scale[t] = 1.f / sd;
    S.in_shift[t] = -params[kInMean + t] / sd;
  }
  const uint32_t mbar = smem_u32(&S.mbar);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (t < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(kMlpHidden));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  operands_ready();
  const uint32_t tmem = S.tmem;
  const uint32_t trow = tmem + ((uint32_t)(32 * (t / 32)) << 16);  // this warp's 32 lanes
  const uint32_t act = smem_u32(S.act), w = smem_u32(S.w);
  const long long l = P.pitch;  // row stride of delta, adual and mlp_start
  const long long rows = kFromState ? P.n_obs : n;
  int pending = 0;
  if (kFromState) pending = __ldg(&P.ctl->pending);
  uint32_t phase = 0;
  bool ok_all = true;
  for (long long base = (long long)blockIdx.x * kInferThreads; base < rows;
       base += (long long)gridDim.x * kInferThreads) {
    const long long o = base + t;
    float f[kMlpIn];
    bool ok = false;
    T d0[9];
    if (kFromState) {
      if (o < rows) {
        const int i = P.obs_pt[o], j = P.obs_cam_rank[o] & kCamMask;
        const T* delta = static_cast<const T*>(P.delta);
        const T* Xm = static_cast<const T*>(P.Xm);
        const T* Ym = static_cast<const T*>(P.Ym);
        const T* DX = static_cast<const T*>(P.DX);
        const T* DY = static_cast<const T*>(P.DY);
        T vbar[9], aT[9], r[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          d0[c] = delta[c * l + o] + (pending ? (c < 3 ? DX[3 * i + c] : DY[6 * j + c - 3]) : T(0));
          aT[c] = from_f64<T>(P.adual[c * l + o] + (pending ? to_f64<T>(d0[c]) : 0.0));
          vbar[c] = c < 3 ? Xm[3 * i + c] : Ym[6 * j + c - 3];
        }
        const typename Num<T>::V2 zz = static_cast<const typename Num<T>::V2*>(P.z)[o];
        ok = warm_features<T>(zz.x, zz.y, vbar, aT, d0, q, f, r);
      }
      // the next tile's state streams into L2 while this tile runs through the network
      prefetch_state_l2<T>(P, base + (long long)gridDim.x * kInferThreads, t);
    } else if (o < rows) {
      const float4* src = reinterpret_cast<const float4*>(feats + o * kMlpIn);
#pragma unroll
      for (int c = 0; c < kMlpIn / 4; ++c) {
        const float4 v = src[c];
        f[4 * c] = v.x;
        f[4 * c + 1] = v.y;
        f[4 * c + 2] = v.z;
        f[4 * c + 3] = v.w;
      }
      ok = true;
    }
#pragma unroll
    for (int c = 0; c < kMlpIn; c += 8) {
      float x[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = ok ? fmaf(f[c + k], S.in_scale[c + k], S.in_shift[c + k]) : 0.f;
      uint4 v;
      v.x = pack_bf16x2(x[0], x[1]);
      v.y = pack_bf16x2(x[2], x[3]);
      v.z = pack_bf16x2(x[4], x[5]);
      v.w = pack_bf16x2(x[6], x[7]);
      *reinterpret_cast<uint4*>(S.act + kmajor_off(t, c, kMlpIn)) = v;
    }
    operands_ready();
    // layer 1: [128 x 32] x [64 x 32]^T
    if (t == 0) mma_layer(tmem, act, w + kBlobW1, kMlpIn, kMlpHidden, mbar);
    ok_all = mbar_wait(mbar, phase) && ok_all;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    hidden_epilogue(trow, S.bias, S.act, t);
    operands_ready();
    // layers 2 and 3: [128 x 64] x [64 x 64]^T
    if (t == 0) mma_layer(tmem, act, w + kBlobW2, kMlpHidden, kMlpHidden, mbar);
    ok_all = mbar_wait(mbar, phase) && ok_all;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    hidden_epilogue(trow, S.bias + kMlpHidden, S.act, t);
    operands_ready();
    if (t == 0) mma_layer(tmem, act, w + kBlobW3, kMlpHidden, kMlpHidden, mbar);
    ok_all = mbar_wait(mbar, phase) && ok_all;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    hidden_epilogue(trow, S.bias + 2 * kMlpHidden, S.act, t);
    operands_ready();
    // layer 4: [128 x 64] x [16 x 64]^T
    if (t == 0) mma_layer(tmem, act, w + kBlobW4, kMlpHidden, kMlpOut, mbar);
    ok_all = mbar_wait(mbar, phase) && ok_all;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float y[16];
    tmem_ld16(trow, y);
    if (kFromState) {
      if (o < rows) {
        T* out = static_cast<T*>(const_cast<void*>(P.mlp_start));
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          const float step = (y[c] + S.bias[3 * kMlpHidden + c]) * S.out_scale[c];
          out[c * l + o] = d0[c] + (ok ? (T)step : T(0));
        }
      }
    } else if (o < rows) {
      float4* dst = reinterpret_cast<float4*>(y_out + o * kMlpOut);
#pragma unroll
      for (int c = 0; c < kMlpOut / 4; ++c)
        dst[c] = make_float4(y[4 * c] + S.bias[3 * kMlpHidden + 4 * c], y[4 * c + 1] + S.bias[3 * kMlpHidden + 4 * c + 1],
                             y[4 * c + 2] + S.bias[3 * kMlpHidden + 4 * c + 2],
                             y[4 * c + 3] + S.bias[3 * kMlpHidden + 4 * c + 3]);
    }
    // the next tile's features overwrite the activation tile: every MMA reading it
    // has completed (waited above), and the tensor-memory reads of this tile are
    // ordered before the next layer-1 MMA by the operands_ready() that precedes it
  }
  if (!ok_all) atomicOr(err, 2);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMlpHidden));
}

// Resident CTAs per SM, from the resources one CTA takes: registers, shared
// memory, and 64 of an SM's 512 tensor-memory columns.
template <typename T, bool kFromState>
cudaError_t infer_grid(int* grid) {
  // per process and device-independent: first caller computes; racing callers compute the same
  static std::atomic<int> cached{0};
  if (cached) {
    *grid = cached;
    return cudaSuccess;
  }
  const int smem = (int)sizeof(MlpSmem);
  cudaError_t e =
      cudaFuncSetAttribute(mlp_infer_kernel<T, kFromState>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, mlp_infer_kernel<T, kFromState>)) != cudaSuccess) return e;
  int dev = 0, sms = 0, smem_sm = 0, smem_rsv = 0, regs_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  if ((e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess) return e;
  const int regs = (fa.numRegs + 7) / 8 * 8;
  int per_sm = 512 / kMlpHidden;
  per_sm = std::min(per_sm, regs_sm / std::max(1, regs * kInferThreads));
  per_sm = std::min(per_sm, smem_sm / (smem + smem_rsv + (int)fa.sharedSizeBytes));
  cached = std::max(per_sm, 1) * sms;
  *grid = cached;
  return cudaSuccess;
}

template <typename T, bool kFromState>
cudaError_t launch_infer(const DevProblem& P, const Params& prm, const unsigned char* blob, const float* params,
                         const float* feats, long long n, float* y_out, int* err, cudaStream_t s) {
  int grid = 0;
  cudaError_t e = infer_grid<T, kFromState>(&grid);
  if (e != cudaSuccess) return e;
  const long long rows = kFromState ? P.n_obs : n;
  long long need = (rows + kInferThreads - 1) / kInferThreads;
  const int g = (int)(need < grid ? (need > 0 ? need : 1) : grid);
  mlp_infer_kernel<T, kFromState><<<g, kInferThreads, sizeof(MlpSmem), s>>>(P, make_prm<T>(prm), blob, params, feats,
                                                                            n, y_out, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mlp_warmstart(const DevProblem& P, const Params& prm, bool fp32, const unsigned char* blob,
                                 const float* params, cudaStream_t s) {
  int* err = &P.ctl->err;
  return fp32 ? launch_infer<float, true>(P, prm, blob, params, nullptr, 0, nullptr, err, s)
              : launch_infer<double, true>(P, prm, blob, params, nullptr, 0, nullptr, err, s);
}

// BF16 weight blob in the operand layout, from FP32 parameters (host).
void mlp_make_blob(const float* params, std::vector<unsigned char>& blob) {
  blob.assign(kBlobBytes, 0);
  auto put = [&](int base, const float* W, int nrow, int kdim) {
    for (int r = 0; r < nrow; ++r)
      for (int k = 0; k < kdim; ++k) {
        const __nv_bfloat16 b = __float2bfloat16(W[r * kdim + k]);
        std::memcpy(&blob[base + kmajor_off(r, k, kdim)], &b, 2);
      }
  };
  put(kBlobW1, params + kW1, kMlpHidden, kMlpIn);
  put(kBlobW2, params + kW2, kMlpHidden, kMlpHidden);
  put(kBlobW3, params + kW3, kMlpHidden, kMlpHidden);
  put(kBlobW4, params + kW4, kMlpOut, kMlpHidden);
}

cudaError_t launch_mlp_harvest(const DevProblem& P, const Params& prm, bool fp32, int pending, long long stride,
                               long long cap, int target_steps, float* feats, float* targs, cudaStream_t s) {
  const int g = (int)((cap + 127) / 128);
  if (g == 0) return cudaSuccess;
  Params p2 = prm;
  p2.inner_steps = target_steps;
  if (fp32)
    harvest_kernel<float><<<g, 128, 0, s>>>(P, make_prm<float>(p2), pending, stride, cap, feats, targs);
  else
    harvest_kernel<double><<<g, 128, 0, s>>>(P, make_prm<double>(p2), pending, stride, cap, feats, targs);
  return cudaGetLastError();
}

}  // namespace dba

// ------------------------------------------------------------ C ABI of the network
namespace {
thread_local std::string g_mlp_error = "no error";
dba_status mlp_fail(dba_mlp* m, cudaError_t e, const char* where) {
  const std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  if (m) m->err = msg;
  g_mlp_error = msg;
  return DBA_ECUDA;
}
#define MLP_CUDA(call, where)                          \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return mlp_fail(m, e_, where); \
  } while (0)
}  // namespace

extern "C" {

dba_status dba_mlp_create(uint64_t seed, dba_mlp** out) {
  return dba::guarded(&g_mlp_error, [&]() -> dba_status {
    if (!out) return DBA_EINVAL;
    *out = nullptr;
    dba_mlp* m = new (std::nothrow) dba_mlp();
    if (!m) return DBA_ENOMEM;
    std::vector<float> h(dba::kNParams, 0.f);
    std::mt19937_64 rng(seed);
    auto init = [&](int base, int nrow, int fan_in, float gain) {
      std::normal_distribution<float> nd(0.f, gain * std::sqrt(2.f / (float)fan_in));
      for (int e = 0; e < nrow * fan_in; ++e) h[base + e] = nd(rng);
    };
    init(dba::kW1, dba::kMlpHidden, dba::kMlpIn, 1.f);
    init(dba::kW2, dba::kMlpHidden, dba::kMlpHidden, 1.f);
    init(dba::kW3, dba::kMlpHidden, dba::kMlpHidden, 1.f);
    init(dba::kW4, dba::kMlpOut, dba::kMlpHidden, 0.1f);
    for (int c = 0; c < dba::kMlpIn; ++c) h[dba::kInStd + c] = 1.f;
    for (int c = 0; c < dba::kMlpOut; ++c) h[dba::kOutStd + c] = 1.f;
    // a blocking stream: orders after work the caller queued on the legacy default stream
    cudaError_t e = cudaStreamCreate(&m->stream);
    if (e == cudaSuccess) e = cudaMalloc(&m->params, sizeof(float) * dba::kNParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, sizeof(float) * dba::kNParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->adam_m, sizeof(float) * dba::kNParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->adam_v, sizeof(float) * dba::kNParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->dloss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(m->params, h.data(), sizeof(float) * dba::kNParams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->adam_m, 0, sizeof(float) * dba::kNParams);
    if (e == cudaSuccess) e = cudaMemset(m->adam_v, 0, sizeof(float) * dba::kNParams);
    if (e != cudaSuccess) {
      g_mlp_error = std::string("dba_mlp_create: ") + cudaGetErrorString(e);
      dba_mlp_destroy(m);
      return DBA_ECUDA;
    }
    *out = m;
    return DBA_OK;
  });
}

void dba_mlp_destroy(dba_mlp* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  float* bufs[] = {m->params, m->grad, m->adam_m, m->adam_v, m->x, m->t, m->z1, m->h1, m->z2, m->h2,
                   m->z3, m->h3, m->y, m->dy, m->d64a, m->d64b};
  for (float* b : bufs) cudaFree(b);
  cudaFree(m->idx);
  cudaFree(m->dloss);
  if (m->stream) cudaStreamDestroy(m->stream);
  delete m;
}

const char* dba_mlp_last_error(const dba_mlp* m) { return m ? m->err.c_str() : g_mlp_error.c_str(); }

dba_status dba_mlp_get_params(const dba_mlp* mc, float* host) {
  return dba::guarded(mc ? &const_cast<dba_mlp*>(mc)->err : nullptr, [&]() -> dba_status {
    dba_mlp* m = const_cast<dba_mlp*>(mc);
    if (!m || !host) return DBA_EINVAL;
    MLP_CUDA(cudaMemcpy(host, m->params, sizeof(float) * dba::kNParams, cudaMemcpyDeviceToHost), "get_params");
    return DBA_OK;
  });
}

dba_status dba_mlp_set_params(dba_mlp* m, const float* host) {
  return dba::guarded(m ? &m->err : nullptr, [&]() -> dba_status {
    if (!m || !host) return DBA_EINVAL;
    for (int k = 0; k < dba::kNParams; ++k)
      if (!std::isfinite(host[k])) {
        m->err = "dba_mlp_set_params: non-finite parameter";
        return DBA_EINVAL;
      }
    MLP_CUDA(cudaMemcpy(m->params, host, sizeof(float) * dba::kNParams, cudaMemcpyHostToDevice), "set_params");
    return DBA_OK;
  });
}

dba_status dba_mlp_fit_normalizer(dba_mlp* m, const float* feats, const float* targets, int64_t n) {
  return dba::guarded(m ? &m->err : nullptr, [&]() -> dba_status {
    if (!m || !feats || !targets || n <= 1) return DBA_EINVAL;
    double* acc = nullptr;
    const int cols = dba::kMlpIn + dba::kMlpOut;
    MLP_CUDA(cudaMalloc(&acc, sizeof(double) * 2 * cols), "normalizer");
    dba::moments_kernel<<<cols, 256, 0, m->stream>>>(feats, targets, n, acc);
    std::vector<double> h(2 * cols);
    cudaError_t e = cudaMemcpyAsync(h.data(), acc, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    cudaFree(acc);
    if (e != cudaSuccess) return mlp_fail(m, e, "normalizer");
    std::vector<float> stats(dba::kNParams - dba::kTrainable);
    for (int c = 0; c < cols; ++c) {
      const double mean = h[2 * c] / (double)n;
      const double var = std::max(h[2 * c + 1] / (double)n - mean * mean, 0.0);
      double sd = std::sqrt(var);
      if (!(sd > 1e-12)) sd = 1.0;
      if (c < dba::kMlpIn) {
        stats[c] = (float)mean;
        stats[dba::kMlpIn + c] = (float)sd;
      } else {
        // targets: scaled by their root mean square (a zero-mean scale keeps "no step" at 0)
        const double rms = std::sqrt(h[2 * c + 1] / (double)n);
        stats[2 * dba::kMlpIn + (c - dba::kMlpIn)] = (float)(rms > 1e-12 ? rms : 1.0);
      }
    }
    MLP_CUDA(cudaMemcpy(m->params + dba::kTrainable, stats.data(), sizeof(float) * stats.size(), cudaMemcpyHostToDevice),
             "normalizer");
    return DBA_OK;
  });
}

dba_status dba_mlp_loss_grad(dba_mlp* m, const float* feats, const float* targets, int64_t n, double* loss,
                             float* grad) {
  return dba::guarded(m ? &m->err : nullptr, [&]() -> dba_status {
    if (!m || !feats || !targets || n <= 0 || n > (1 << 26)) return DBA_EINVAL;
    MLP_CUDA(dba::mlp_reserve(m, (int)n), "loss_grad");
    const int b = dba::blocks_for(n * dba::kMlpIn, 256);
    dba::gather_standardize_kernel<<<b, 256, 0, m->stream>>>(feats, nullptr, (int)n, m->params, m->x);
    dba::gather_targets_kernel<<<dba::blocks_for(n * dba::kMlpOut, 256), 256, 0, m->stream>>>(targets, nullptr, (int)n,
                                                                                              m->params, m->t);
    MLP_CUDA(dba::mlp_forward_backward(m, (int)n), "loss_grad");
    double h = 0.0;
    MLP_CUDA(cudaMemcpyAsync(&h, m->dloss, sizeof h, cudaMemcpyDeviceToHost, m->stream), "loss_grad");
    if (grad) MLP_CUDA(cudaMemcpyAsync(grad, m->grad, sizeof(float) * dba::kNParams, cudaMemcpyDeviceToHost, m->stream),
                       "loss_grad");
    MLP_CUDA(cudaStreamSynchronize(m->stream), "loss_grad");
    if (loss) *loss = h;
    return DBA_OK;
  });
}

dba_status dba_mlp_train(dba_mlp* m, const float* feats, const float* targets, int64_t n, int epochs, int batch,
                         float lr, uint64_t seed, double* last_loss) {
  return dba::guarded(m ? &m->err : nullptr, [&]() -> dba_status {
    if (!m || !feats || !targets || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0)) return DBA_EINVAL;
    MLP_CUDA(dba::mlp_reserve(m, batch), "train");
    int* perm_dev = nullptr;
    MLP_CUDA(cudaMalloc(&perm_dev, sizeof(int) * (size_t)n), "train");
    std::vector<int> perm(n);
    for (int64_t k = 0; k < n; ++k) perm[k] = (int)k;
    std::mt19937_64 rng(seed);
    double epoch_loss = 0.0;
    cudaError_t e = cudaSuccess;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
      std::shuffle(perm.begin(), perm.end(), rng);
      e = cudaMemcpyAsync(perm_dev, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, m->stream);
      double sum = 0.0;
      int nb = 0;
      for (int64_t s0 = 0; s0 + batch <= n && e == cudaSuccess; s0 += batch, ++nb) {
        dba::gather_standardize_kernel<<<dba::blocks_for((long long)batch * dba::kMlpIn, 256), 256, 0, m->stream>>>(
            feats, perm_dev + s0, batch, m->params, m->x);
        dba::gather_targets_kernel<<<dba::blocks_for((long long)batch * dba::kMlpOut, 256), 256, 0, m->stream>>>(
            targets, perm_dev + s0, batch, m->params, m->t);
        e = dba::mlp_forward_backward(m, batch);
        if (e != cudaSuccess) break;
        m->adam_t += 1;
        const float c1 = 1.f - std::pow(0.9f, (float)m->adam_t), c2 = 1.f - std::pow(0.999f, (float)m->adam_t);
        dba::adam_kernel<<<dba::blocks_for(dba::kTrainable, 256), 256, 0, m->stream>>>(
            m->params, m->grad, m->adam_m, m->adam_v, dba::kTrainable, lr, 0.9f, 0.999f, c1, c2);
        double h = 0.0;
        e = cudaMemcpyAsync(&h, m->dloss, sizeof h, cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        sum += h;
      }
      epoch_loss = nb ? sum / nb : 0.0;
    }
    cudaFree(perm_dev);
    if (e != cudaSuccess) return mlp_fail(m, e, "train");
    if (last_loss) *last_loss = epoch_loss;
    return DBA_OK;
  });
}

dba_status dba_mlp_predict(dba_mlp* m, const float* feats, int64_t n, float* out) {
  return dba::guarded(m ? &m->err : nullptr, [&]() -> dba_status {
    if (!m || !feats || !out || n <= 0) return DBA_EINVAL;
    std::vector<float> h(dba::kNParams);
    MLP_CUDA(cudaMemcpy(h.data(), m->params, sizeof(float) * h.size(), cudaMemcpyDeviceToHost), "predict");
    std::vector<unsigned char> blob;
    dba::mlp_make_blob(h.data(), blob);
    unsigned char* dblob = nullptr;
    int* derr = nullptr;
    MLP_CUDA(cudaMalloc(&dblob, blob.size()), "predict");
    MLP_CUDA(cudaMalloc(&derr, sizeof(int)), "predict");
    cudaError_t e = cudaMemcpyAsync(dblob, blob.data(), blob.size(), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), m->stream);
    dba::DevProblem none{};
    if (e == cudaSuccess)
      e = dba::launch_infer<float, false>(none, dba::Params{}, dblob, m->params, feats, n, out, derr, m->stream);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    cudaFree(dblob);
    cudaFree(derr);
    if (e != cudaSuccess) return mlp_fail(m, e, "predict");
    if (herr) {
      m->err = "dba_mlp_predict: a tensor-core wait timed out";
      return DBA_ETIMEOUT;
    }
    return DBA_OK;
  });
}

}  // extern "C"
