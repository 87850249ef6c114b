// Learned prior mean for the GP: an MLP 2 -> 64 -> 64 -> 1 (exact GELU),
// trained by full-batch Adam with the library's own kernels.
//
// One fused kernel per 64-row tile does the forward pass, the mean-squared
// error and the backward pass.  The three 64-wide products (the hidden
// layer forward, its input gradient and its weight gradient) run on the tensor
// cores as mma.sync m16n8k16 with BF16 operands and FP32 accumulation; the
// 2-wide input layer, the 1-wide output layer, GELU and the reductions are
// FP32.  Weight gradients of the tiles meet in FP32 atomics; a second kernel
// applies Adam to the FP32 master weights and clears the gradients.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "mdgp.h"
#include "md_ctx.h"

namespace {

constexpr int H = 64;                       // hidden width
constexpr int kRows = 64;                   // rows per tile
constexpr int kW1 = 0, kB1 = kW1 + H * 2, kW2 = kB1 + H, kB2 = kW2 + H * H, kW3 = kB2 + H, kB3 = kW3 + H;
constexpr int kNParams = kB3 + 1;           // 4417
constexpr int kLD = H + 8;                  // bf16 row stride in shared memory (bank spread)

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One warp: out[16 x 64] += A[16 x 64] * B[64 x 64] where A(m, k) and B(k, n)
// are bf16 accessors into shared memory; acc[nt][4] holds the 8 n-tiles in
// the m16n8 accumulator layout (rows g, g + 8; cols 2t, 2t + 1).
template <typename FA, typename FB>
__device__ __forceinline__ void warp_gemm_16x64x64(float (&acc)[8][4], FA A, FB B) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int k0 = ks * 16 + 2 * t;
    const uint32_t a0 = pack_bf16(A(g, k0), A(g, k0 + 1));
    const uint32_t a1 = pack_bf16(A(g + 8, k0), A(g + 8, k0 + 1));
    const uint32_t a2 = pack_bf16(A(g, k0 + 8), A(g, k0 + 9));
    const uint32_t a3 = pack_bf16(A(g + 8, k0 + 8), A(g + 8, k0 + 9));
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int n = nt * 8 + g;
      const uint32_t b0 = pack_bf16(B(k0, n), B(k0 + 1, n));
      const uint32_t b1 = pack_bf16(B(k0 + 8, n), B(k0 + 9, n));
      mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
    }
  }
}

// Forward (+ backward) for the rows [tile * 64, tile * 64 + 64) of the
// standardised data.  mode 0: forward only, writes out[]; mode 1: loss and
// gradients (scaled by 1 / n_total) accumulated into grad[] and loss[0];
// mode 2: loss only.
__global__ void __launch_bounds__(128) k_mlp_tile(const float* __restrict__ P, const float* __restrict__ X,
                                                  const float* __restrict__ y, int M, float inv_n, int mode,
                                                  float* __restrict__ out, float* __restrict__ grad,
                                                  float* __restrict__ loss) {
  __shared__ float sP[kNParams];
  __shared__ __nv_bfloat16 sA1[kRows][kLD];   // GELU(z1), bf16
  __shared__ __nv_bfloat16 sD2[kRows][kLD];   // dz2, bf16
  __shared__ __nv_bfloat16 sW2[H][kLD];       // W2 [out][in], bf16
  __shared__ float sX[kRows][2];
  __shared__ float sDout[kRows];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = lane >> 2, t = lane & 3;
  const int row0 = blockIdx.x * kRows;
  for (int i = tid; i < kNParams; i += blockDim.x) sP[i] = P[i];
  for (int i = tid; i < kRows * 2; i += blockDim.x) {
    const int r = i >> 1;
    sX[r][i & 1] = row0 + r < M ? X[(size_t)(row0 + r) * 2 + (i & 1)] : 0.0f;
  }
  __syncthreads();
  for (int i = tid; i < H * H; i += blockDim.x) sW2[i / H][i % H] = __float2bfloat16_rn(sP[kW2 + i]);
  // layer 1 (2 -> 64), FP32
  for (int i = tid; i < kRows * H; i += blockDim.x) {
    const int r = i / H, j = i % H;
    const float z = sP[kW1 + 2 * j] * sX[r][0] + sP[kW1 + 2 * j + 1] * sX[r][1] + sP[kB1 + j];
    sA1[r][j] = __float2bfloat16_rn(gelu_f(z));
  }
  __syncthreads();
  // layer 2 (64 -> 64) on the tensor cores: z2 = a1 W2^T
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
  const int rb = w * 16;
  warp_gemm_16x64x64(
      acc, [&](int m, int k) { return sA1[rb + m][k]; }, [&](int k, int n) { return sW2[n][k]; });
  // bias, GELU, output layer (64 -> 1)
  float z2[8][4], o_lo = 0.0f, o_hi = 0.0f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = nt * 8 + 2 * t + (c & 1);
      z2[nt][c] = acc[nt][c] + sP[kB2 + col];
      const float a = gelu_f(z2[nt][c]);
      if (c < 2) o_lo += a * sP[kW3 + col]; else o_hi += a * sP[kW3 + col];
    }
  }
  // reduce over the quad (t) that shares a row
  o_lo += __shfl_xor_sync(0xffffffffu, o_lo, 1);
  o_lo += __shfl_xor_sync(0xffffffffu, o_lo, 2);
  o_hi += __shfl_xor_sync(0xffffffffu, o_hi, 1);
  o_hi += __shfl_xor_sync(0xffffffffu, o_hi, 2);
  const int r_lo = rb + g, r_hi = rb + g + 8;
  const float out_lo = o_lo + sP[kB3], out_hi = o_hi + sP[kB3];
  if (mode == 0) {
    if (t == 0) {
      if (row0 + r_lo < M) out[row0 + r_lo] = out_lo;
      if (row0 + r_hi < M) out[row0 + r_hi] = out_hi;
    }
    return;
  }
  // loss and d_out = 2 (out - y) / n
  const bool v_lo = row0 + r_lo < M, v_hi = row0 + r_hi < M;
  const float res_lo = v_lo ? out_lo - y[row0 + r_lo] : 0.0f;
  const float res_hi = v_hi ? out_hi - y[row0 + r_hi] : 0.0f;
  if (t == 0) {
    sDout[r_lo] = 2.0f * res_lo * inv_n;
    sDout[r_hi] = 2.0f * res_hi * inv_n;
  }
  if (t == 0) atomicAdd(loss, (res_lo * res_lo + res_hi * res_hi) * inv_n);
  if (mode == 2) return;
  __syncwarp();
  const float d_lo = sDout[r_lo], d_hi = sDout[r_hi];
  // dW3 = sum_rows d_out a2 ; dz2 = d_out W3 * gelu'(z2) ; db2 = sum_rows dz2
  float gw3[8][2], gb2[8][2];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int col = nt * 8 + 2 * t + c;
      const float a_lo = gelu_f(z2[nt][c]), a_hi = gelu_f(z2[nt][c + 2]);
      gw3[nt][c] = d_lo * a_lo + d_hi * a_hi;
      const float dz_lo = d_lo * sP[kW3 + col] * gelu_grad_f(z2[nt][c]);
      const float dz_hi = d_hi * sP[kW3 + col] * gelu_grad_f(z2[nt][c + 2]);
      gb2[nt][c] = dz_lo + dz_hi;
      sD2[r_lo][col] = __float2bfloat16_rn(dz_lo);
      sD2[r_hi][col] = __float2bfloat16_rn(dz_hi);
    }
  }
  // reduce gw3 / gb2 over the 8 row groups (g) of the warp, then across warps
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        gw3[nt][c] += __shfl_xor_sync(0xffffffffu, gw3[nt][c], o);
        gb2[nt][c] += __shfl_xor_sync(0xffffffffu, gb2[nt][c], o);
      }
  if (g == 0) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = nt * 8 + 2 * t + c;
        atomicAdd(&grad[kW3 + col], gw3[nt][c]);
        atomicAdd(&grad[kB2 + col], gb2[nt][c]);
      }
  }
  if (t == 0) atomicAdd(&grad[kB3], d_lo + d_hi);
  __syncthreads();
  // dW2 += dz2^T a1 (warp w: output rows 16w.., K = the tile's rows)
  {
    float gacc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) gacc[nt][0] = gacc[nt][1] = gacc[nt][2] = gacc[nt][3] = 0.0f;
    warp_gemm_16x64x64(
        gacc, [&](int m, int k) { return sD2[k][rb + m]; }, [&](int k, int n) { return sA1[k][n]; });
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int orow = rb + g + (c >= 2 ? 8 : 0), col = nt * 8 + 2 * t + (c & 1);
        atomicAdd(&grad[kW2 + orow * H + col], gacc[nt][c]);
      }
  }
  // da1 = dz2 W2 (warp w: rows 16w..), dz1 = da1 * gelu'(z1)
  float dacc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) dacc[nt][0] = dacc[nt][1] = dacc[nt][2] = dacc[nt][3] = 0.0f;
  warp_gemm_16x64x64(
      dacc, [&](int m, int k) { return sD2[rb + m][k]; }, [&](int k, int n) { return sW2[k][n]; });
  float gw1[8][2][2], gb1[8][2];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int col = nt * 8 + 2 * t + c;
      // z1 recomputed (two FMAs) rather than kept in shared memory
      const float z1_lo = sP[kW1 + 2 * col] * sX[r_lo][0] + sP[kW1 + 2 * col + 1] * sX[r_lo][1] + sP[kB1 + col];
      const float z1_hi = sP[kW1 + 2 * col] * sX[r_hi][0] + sP[kW1 + 2 * col + 1] * sX[r_hi][1] + sP[kB1 + col];
      const float dz_lo = dacc[nt][c] * gelu_grad_f(z1_lo);
      const float dz_hi = dacc[nt][c + 2] * gelu_grad_f(z1_hi);
      gw1[nt][c][0] = dz_lo * sX[r_lo][0] + dz_hi * sX[r_hi][0];
      gw1[nt][c][1] = dz_lo * sX[r_lo][1] + dz_hi * sX[r_hi][1];
      gb1[nt][c] = dz_lo + dz_hi;
    }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        gw1[nt][c][0] += __shfl_xor_sync(0xffffffffu, gw1[nt][c][0], o);
        gw1[nt][c][1] += __shfl_xor_sync(0xffffffffu, gw1[nt][c][1], o);
        gb1[nt][c] += __shfl_xor_sync(0xffffffffu, gb1[nt][c], o);
      }
  if (g == 0) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = nt * 8 + 2 * t + c;
        atomicAdd(&grad[kW1 + 2 * col], gw1[nt][c][0]);
        atomicAdd(&grad[kW1 + 2 * col + 1], gw1[nt][c][1]);
        atomicAdd(&grad[kB1 + col], gb1[nt][c]);
      }
  }
}

// Adam (Kingma & Ba) on the FP32 master weights; clears the gradients.
__global__ void k_mlp_adam(float* P, float* G, float* Mo, float* V, int n, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * Mo[i] + (1.0f - b1) * g;
  const float v = b2 * V[i] + (1.0f - b2) * g * g;
  Mo[i] = m;
  V[i] = v;
  P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  G[i] = 0.0f;
}

}  // namespace

struct mdgp_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  float *dP = nullptr, *dG = nullptr, *dM = nullptr, *dV = nullptr, *dBest = nullptr;
  float *dX = nullptr, *dy = nullptr, *dout = nullptr, *dloss = nullptr;
  size_t cap = 0;
  double xm[2] = {0, 0}, xs[2] = {1, 1}, ym = 0, ys = 1;
  long long t = 0;
  long long launches = 0;
};

namespace {

int mlp_err(cudaError_t e) {
  if (e == cudaSuccess) return MDGP_OK;
  return e == cudaErrorMemoryAllocation ? MDGP_E_NOMEM : MDGP_E_CUDA;
}

#define MK(expr)                                     \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return mlp_err(e_);       \
  } while (0)

int mlp_rows(mdgp_mlp* m, size_t rows) {
  if (rows <= m->cap) return MDGP_OK;
  for (float** p : {&m->dX, &m->dy, &m->dout})
    if (*p) { cudaFree(*p); *p = nullptr; }
  MK(cudaMalloc(&m->dX, sizeof(float) * 2 * rows));
  MK(cudaMalloc(&m->dy, sizeof(float) * rows));
  MK(cudaMalloc(&m->dout, sizeof(float) * rows));
  m->cap = rows;
  return MDGP_OK;
}

// Upload standardised inputs (and outputs) of rows idx.
int mlp_upload(mdgp_mlp* m, const double* X, const double* y, const std::vector<int64_t>& idx) {
  const size_t n = idx.size();
  int st = mlp_rows(m, n);
  if (st) return st;
  std::vector<float> xs(2 * n), ys(n);
  for (size_t r = 0; r < n; ++r) {
    const int64_t i = idx[r];
    xs[2 * r] = (float)((X[2 * i] - m->xm[0]) / m->xs[0]);
    xs[2 * r + 1] = (float)((X[2 * i + 1] - m->xm[1]) / m->xs[1]);
    if (y) ys[r] = (float)((y[i] - m->ym) / m->ys);
  }
  MK(cudaMemcpyAsync(m->dX, xs.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice, m->stream));
  if (y) MK(cudaMemcpyAsync(m->dy, ys.data(), sizeof(float) * n, cudaMemcpyHostToDevice, m->stream));
  MK(cudaStreamSynchronize(m->stream));
  return MDGP_OK;
}

// Loss (standardised units) of the uploaded rows; accumulates gradients when grads.
int mlp_pass(mdgp_mlp* m, int64_t n, bool grads, double* loss) {
  MK(cudaMemsetAsync(m->dloss, 0, sizeof(float), m->stream));
  const unsigned tiles = (unsigned)((n + kRows - 1) / kRows);
  k_mlp_tile<<<tiles, 128, 0, m->stream>>>(m->dP, m->dX, m->dy, (int)n, 1.0f / (float)n, grads ? 1 : 0, m->dout,
                                           m->dG, m->dloss);
  m->launches++;
  MK(cudaGetLastError());
  if (loss) {
    float l = 0.0f;
    MK(cudaMemcpyAsync(&l, m->dloss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    MK(cudaStreamSynchronize(m->stream));
    *loss = l;
  }
  return MDGP_OK;
}

}  // namespace

extern "C" {

int mdgp_mlp_params_default(mdgp_mlp_params* p) {
  if (!p) return MDGP_E_ARG;
  std::memset(p, 0, sizeof(*p));
  p->epochs = 2000;
  p->eval_every = 20;
  p->lr = 1e-3;
  p->beta1 = 0.9;
  p->beta2 = 0.999;
  p->eps = 1e-8;
  p->holdout_frac = 0.2;
  p->seed = 1;
  return MDGP_OK;
}

int mdgp_mlp_create(mdgp_ctx* ctx, const float* init, uint64_t seed, mdgp_mlp** out) {
  if (!ctx || !out) return MDGP_E_ARG;
  *out = nullptr;
  cudaSetDevice(ctx->device);
  mdgp_mlp* m = new (std::nothrow) mdgp_mlp();
  if (!m) return MDGP_E_NOMEM;
  m->device = ctx->device;
  m->stream = ctx->stream;
  auto fail = [&](int st) { mdgp_mlp_free(m); return st; };
  for (float** p : {&m->dP, &m->dG, &m->dM, &m->dV, &m->dBest})
    if (cudaMalloc(p, sizeof(float) * kNParams) != cudaSuccess) return fail(MDGP_E_NOMEM);
  if (cudaMalloc(&m->dloss, sizeof(float)) != cudaSuccess) return fail(MDGP_E_NOMEM);
  std::vector<float> w(kNParams);
  if (init) {
    std::memcpy(w.data(), init, sizeof(float) * kNParams);
  } else {
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a 64-bit LCG (Knuth's MMIX constants)
    unsigned long long s = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    auto uni = [&]() {
      s = s * 6364136223846793005ULL + 1442695040888963407ULL;
      return (double)(s >> 11) * (1.0 / 9007199254740992.0);
    };
    const int fan[6] = {2, 2, H, H, H, H};
    const int off[7] = {kW1, kB1, kW2, kB2, kW3, kB3, kNParams};
    for (int part = 0; part < 6; ++part) {
      const double bound = 1.0 / std::sqrt((double)fan[part]);
      for (int i = off[part]; i < off[part + 1]; ++i) w[i] = (float)((2.0 * uni() - 1.0) * bound);
    }
  }
  if (cudaMemcpy(m->dP, w.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->dG, 0, sizeof(float) * kNParams) != cudaSuccess ||
      cudaMemset(m->dM, 0, sizeof(float) * kNParams) != cudaSuccess ||
      cudaMemset(m->dV, 0, sizeof(float) * kNParams) != cudaSuccess)
    return fail(MDGP_E_CUDA);
  *out = m;
  return MDGP_OK;
}

int mdgp_mlp_free(mdgp_mlp* m) {
  if (!m) return MDGP_E_ARG;
  cudaSetDevice(m->device);
  for (float** p : {&m->dP, &m->dG, &m->dM, &m->dV, &m->dBest, &m->dX, &m->dy, &m->dout, &m->dloss})
    if (*p) cudaFree(*p);
  delete m;
  return MDGP_OK;
}

int mdgp_mlp_num_params(void) { return kNParams; }

int mdgp_mlp_get(const mdgp_mlp* m, float* params, double* standardiser) {
  if (!m) return MDGP_E_ARG;
  cudaSetDevice(m->device);
  if (params && cudaMemcpy(params, m->dP, sizeof(float) * kNParams, cudaMemcpyDeviceToHost) != cudaSuccess)
    return MDGP_E_CUDA;
  if (standardiser) {
    standardiser[0] = m->xm[0]; standardiser[1] = m->xm[1];
    standardiser[2] = m->xs[0]; standardiser[3] = m->xs[1];
    standardiser[4] = m->ym; standardiser[5] = m->ys;
  }
  return MDGP_OK;
}

int mdgp_mlp_set(mdgp_mlp* m, const float* params, const double* standardiser) {
  if (!m) return MDGP_E_ARG;
  cudaSetDevice(m->device);
  if (params && cudaMemcpy(m->dP, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice) != cudaSuccess)
    return MDGP_E_CUDA;
  if (standardiser) {
    m->xm[0] = standardiser[0]; m->xm[1] = standardiser[1];
    m->xs[0] = standardiser[2]; m->xs[1] = standardiser[3];
    m->ym = standardiser[4]; m->ys = standardiser[5];
  }
  return MDGP_OK;
}

int mdgp_mlp_loss_grad(mdgp_mlp* m, const double* X, const double* y, int64_t n, double* loss, float* grads) {
  if (!m || !X || !y || n < 1) return MDGP_E_ARG;
  cudaSetDevice(m->device);
  std::vector<int64_t> idx((size_t)n);
  std::iota(idx.begin(), idx.end(), 0);
  int st = mlp_upload(m, X, y, idx);
  if (st) return st;
  MK(cudaMemsetAsync(m->dG, 0, sizeof(float) * kNParams, m->stream));
  if ((st = mlp_pass(m, n, true, loss))) return st;
  if (grads) {
    MK(cudaMemcpyAsync(grads, m->dG, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, m->stream));
    MK(cudaStreamSynchronize(m->stream));
  }
  return MDGP_OK;
}

int mdgp_mlp_adam_step(mdgp_mlp* m, const float* grads, const mdgp_mlp_params* p) {
  if (!m || !p) return MDGP_E_ARG;
  cudaSetDevice(m->device);
  if (grads) MK(cudaMemcpyAsync(m->dG, grads, sizeof(float) * kNParams, cudaMemcpyHostToDevice, m->stream));
  m->t += 1;
  const float c1 = (float)(1.0 - std::pow(p->beta1, (double)m->t));
  const float c2 = (float)(1.0 - std::pow(p->beta2, (double)m->t));
  k_mlp_adam<<<(kNParams + 255) / 256, 256, 0, m->stream>>>(m->dP, m->dG, m->dM, m->dV, kNParams, (float)p->lr,
                                                           (float)p->beta1, (float)p->beta2, (float)p->eps, c1, c2);
  m->launches++;
  MK(cudaGetLastError());
  MK(cudaStreamSynchronize(m->stream));
  return MDGP_OK;
}

int mdgp_mlp_train(mdgp_mlp* m, const double* X, const double* y, int64_t n, const mdgp_mlp_params* p,
                   double* train_loss, double* holdout_loss) {
  if (!m || !X || !y || !p || n < 2 || p->epochs < 0 || !(p->holdout_frac >= 0 && p->holdout_frac < 1))
    return MDGP_E_ARG;
  cudaSetDevice(m->device);
  // seeded split (Fisher-Yates with the same LCG as the initialisation)
  std::vector<int64_t> perm((size_t)n);
  std::iota(perm.begin(), perm.end(), 0);
  unsigned long long s = p->seed * 6364136223846793005ULL + 1442695040888963407ULL;
  for (int64_t i = n - 1; i > 0; --i) {
    s = s * 6364136223846793005ULL + 1442695040888963407ULL;
    const int64_t j = (int64_t)((s >> 33) % (unsigned long long)(i + 1));
    std::swap(perm[i], perm[j]);
  }
  int64_t nh = (int64_t)std::floor(p->holdout_frac * n);
  if (nh >= n) nh = n - 1;
  std::vector<int64_t> tr(perm.begin() + nh, perm.end()), ho(perm.begin(), perm.begin() + nh);
  // standardise with the training rows
  double sx[2] = {0, 0}, sxx[2] = {0, 0}, sy = 0, syy = 0;
  for (int64_t i : tr) {
    for (int d = 0; d < 2; ++d) { sx[d] += X[2 * i + d]; sxx[d] += X[2 * i + d] * X[2 * i + d]; }
    sy += y[i]; syy += y[i] * y[i];
  }
  const double nt = (double)tr.size();
  for (int d = 0; d < 2; ++d) {
    m->xm[d] = sx[d] / nt;
    const double var = sxx[d] / nt - m->xm[d] * m->xm[d];
    m->xs[d] = var > 0 ? std::sqrt(var) : 1.0;
  }
  m->ym = sy / nt;
  { const double var = syy / nt - m->ym * m->ym; m->ys = var > 0 ? std::sqrt(var) : 1.0; }
  // device copies: training rows first, holdout rows after
  std::vector<int64_t> all(tr);
  all.insert(all.end(), ho.begin(), ho.end());
  int st = mlp_upload(m, X, y, all);
  if (st) return st;
  MK(cudaMemsetAsync(m->dG, 0, sizeof(float) * kNParams, m->stream));
  MK(cudaMemsetAsync(m->dM, 0, sizeof(float) * kNParams, m->stream));
  MK(cudaMemsetAsync(m->dV, 0, sizeof(float) * kNParams, m->stream));
  m->t = 0;
  double best = INFINITY, last_train = 0.0;
  MK(cudaMemcpyAsync(m->dBest, m->dP, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice, m->stream));
  const float* Xho = m->dX + 2 * tr.size();
  const float* yho = m->dy + tr.size();
  for (int ep = 1; ep <= p->epochs; ++ep) {
    const bool eval = (ep % (p->eval_every > 0 ? p->eval_every : 1) == 0) || ep == p->epochs;
    if ((st = mlp_pass(m, (int64_t)tr.size(), true, eval ? &last_train : nullptr))) return st;
    m->t += 1;
    const float c1 = (float)(1.0 - std::pow(p->beta1, (double)m->t));
    const float c2 = (float)(1.0 - std::pow(p->beta2, (double)m->t));
    k_mlp_adam<<<(kNParams + 255) / 256, 256, 0, m->stream>>>(m->dP, m->dG, m->dM, m->dV, kNParams, (float)p->lr,
                                                             (float)p->beta1, (float)p->beta2, (float)p->eps, c1,
                                                             c2);
    m->launches++;
    if (eval && nh > 0) {
      // holdout loss (loss-only pass); keep the weights with the best one
      MK(cudaMemsetAsync(m->dloss, 0, sizeof(float), m->stream));
      k_mlp_tile<<<(unsigned)((nh + kRows - 1) / kRows), 128, 0, m->stream>>>(
          m->dP, Xho, yho, (int)nh, 1.0f / (float)nh, 2, m->dout, nullptr, m->dloss);
      m->launches++;
      float l = 0.0f;
      MK(cudaMemcpyAsync(&l, m->dloss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
      MK(cudaStreamSynchronize(m->stream));
      if (l < best) {
        best = l;
        MK(cudaMemcpyAsync(m->dBest, m->dP, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice, m->stream));
      }
    }
  }
  if (nh > 0 && best < INFINITY)
    MK(cudaMemcpyAsync(m->dP, m->dBest, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice, m->stream));
  if (train_loss) *train_loss = last_train;
  if (holdout_loss) *holdout_loss = nh > 0 ? best : NAN;
  MK(cudaStreamSynchronize(m->stream));
  return MDGP_OK;
}

int mdgp_mlp_predict(mdgp_mlp* m, const double* X, int64_t n, double* out) {
  if (!m || n < 0 || (n > 0 && (!X || !out))) return MDGP_E_ARG;
  if (n == 0) return MDGP_OK;
  cudaSetDevice(m->device);
  std::vector<int64_t> idx((size_t)n);
  std::iota(idx.begin(), idx.end(), 0);
  int st = mlp_upload(m, X, nullptr, idx);
  if (st) return st;
  if ((st = mlp_pass(m, n, false, nullptr))) return st;
  std::vector<float> o((size_t)n);
  MK(cudaMemcpyAsync(o.data(), m->dout, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream));
  MK(cudaStreamSynchronize(m->stream));
  for (int64_t i = 0; i < n; ++i) out[i] = (double)o[i] * m->ys + m->ym;
  return MDGP_OK;
}

}  // extern "C"
