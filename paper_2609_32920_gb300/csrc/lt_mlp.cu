// lt_mlp.cu -- training of the learned reservoir target (16 -> 64 -> 64 -> 1 ReLU MLP) on
// tensor cores: forward and backward GEMM tiles on mma.sync.m16n8k16 (BF16 operands, FP32
// accumulation), per-block gradient accumulation in shared memory, Adam update, and the
// feature/target standardisation statistics.
#include <cuda_runtime.h>

#include "lt_launch.h"
#include "lt_mlp.cuh"

namespace lt {

namespace {

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// A fragment of a transposed operand held sample-major in shared memory:
// element (row r, col s) = buf[s * ld + r] (rows 16mt.., cols = samples 16kc..).
__device__ __forceinline__ void afrag_T(const __nv_bfloat16* buf, int ld, int mt, int kc, uint32_t a[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = mt * 16 + g, r8 = r0 + 8, c0 = kc * 16 + 2 * t;
  auto pk = [&](int r, int c) {
    __nv_bfloat162 v;
    v.x = buf[c * ld + r];
    v.y = buf[(c + 1) * ld + r];
    return *reinterpret_cast<uint32_t*>(&v);
  };
  a[0] = pk(r0, c0);
  a[1] = pk(r8, c0);
  a[2] = pk(r0, c0 + 8);
  a[3] = pk(r8, c0 + 8);
}
// B fragment of a sample-major shared buffer: element (k = sample, n = column) =
// buf[k * ld + n].
__device__ __forceinline__ void bfrag_S(const __nv_bfloat16* buf, int ld, int kc, int nt, uint32_t& b0, uint32_t& b1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int k = kc * 16 + 2 * t, n = nt * 8 + g;
  __nv_bfloat162 v0, v1;
  v0.x = buf[k * ld + n];
  v0.y = buf[(k + 1) * ld + n];
  v1.x = buf[(k + 8) * ld + n];
  v1.y = buf[(k + 9) * ld + n];
  b0 = *reinterpret_cast<uint32_t*>(&v0);
  b1 = *reinterpret_cast<uint32_t*>(&v1);
}
// B fragment of W2^T for the backward product dz2 * W2^T: element (k = out j, n = in i) =
// W2[i][j] = w2t[j * 64 + i].
__device__ __forceinline__ void bfrag_w2back(const __nv_bfloat16* w2t, int kc, int nt, uint32_t& b0, uint32_t& b1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int k = kc * 16 + 2 * t, n = nt * 8 + g;
  __nv_bfloat162 v0, v1;
  v0.x = w2t[k * kMlpHid + n];
  v0.y = w2t[(k + 1) * kMlpHid + n];
  v1.x = w2t[(k + 8) * kMlpHid + n];
  v1.y = w2t[(k + 9) * kMlpHid + n];
  b0 = *reinterpret_cast<uint32_t*>(&v0);
  b1 = *reinterpret_cast<uint32_t*>(&v1);
}
// Store an accumulator-layout tile (rows 16mt.. of a 32-row sample-major buffer) as BF16.
__device__ __forceinline__ void store_hid(const Hid& H, int mt, __nv_bfloat16* buf) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c = nt * 8 + 2 * t;
    buf[(mt * 16 + g) * kMlpHid + c] = __float2bfloat16_rn(H.h[nt][0]);
    buf[(mt * 16 + g) * kMlpHid + c + 1] = __float2bfloat16_rn(H.h[nt][1]);
    buf[(mt * 16 + g + 8) * kMlpHid + c] = __float2bfloat16_rn(H.h[nt][2]);
    buf[(mt * 16 + g + 8) * kMlpHid + c + 1] = __float2bfloat16_rn(H.h[nt][3]);
  }
}

struct WarpBufs {
  __nv_bfloat16 x[32 * kMlpIn];     // standardized inputs, sample-major
  __nv_bfloat16 h1[32 * kMlpHid];   // relu(z1), later reused for dz1
  __nv_bfloat16 dz2[32 * kMlpHid];
};

constexpr int kTrainWarps = 4;

// One training pass over `n` samples: forward, loss, backward; gradients (of the mean
// squared error over the batch `n_batch`) accumulate into g[kMlpWeights] (FP32).
__global__ void __launch_bounds__(32 * kTrainWarps) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                          const float* __restrict__ T, int64_t n, float inv_batch,
                                                          float* __restrict__ g, float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& m = *reinterpret_cast<MlpSmem*>(smem_raw);
  float* gacc = reinterpret_cast<float*>(smem_raw + ((sizeof(MlpSmem) + 15) & ~size_t(15)));
  WarpBufs* wb = reinterpret_cast<WarpBufs*>(gacc + ((kMlpWeights + 3) & ~3));
  mlp_load_smem(m, P);
  for (int i = threadIdx.x; i < kMlpWeights; i += blockDim.x) gacc[i] = 0.0f;
  __syncthreads();
  const float tmean = P[kOffTMean], tinv = 1.0f / P[kOffTScale];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g8 = lane >> 2, t4 = lane & 3;
  WarpBufs& B = wb[warp];
  float lsum = 0.0f;
  const int64_t tiles = (n + 31) / 32;
  for (int64_t tile = (int64_t)blockIdx.x * kTrainWarps + warp; tile < tiles; tile += (int64_t)gridDim.x * kTrainWarps) {
    const int64_t s = tile * 32 + lane;
    const bool live = s < n;
    float f[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = live ? X[s * 16 + i] : m.mean[i];
    mlp_stage_features(m, f, B.x);
    const float tt = live ? (T[s] - tmean) * tinv : 0.0f;
    __syncwarp();
    Hid z1[2], z2[2];
    float dy_lane = 0.0f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      uint32_t a[4];
      afrag_from_tile(B.x, mt, a);
      float yg, yg8;
      mlp_tile_forward(m, a, z1[mt], z2[mt], yg, yg8);
      const int r = lane - 16 * mt;
      const float v0 = __shfl_sync(0xffffffffu, yg, 4 * (r & 7)), v8 = __shfl_sync(0xffffffffu, yg8, 4 * (r & 7));
      if (r >= 0 && r < 16) {
        const float y = r < 8 ? v0 : v8;
        const float e = live ? (y - tt) : 0.0f;
        lsum += e * e;
        dy_lane = 2.0f * e * inv_batch;
      }
    }
    // output layer: db3, dw3 and dz2 = dy w3 [z2 > 0]
    float db3 = dy_lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) db3 += __shfl_xor_sync(0xffffffffu, db3, o);
    if (lane == 0) atomicAdd(&gacc[kOffB3], db3);
    Hid dz2[2], h1[2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const float dyg = __shfl_sync(0xffffffffu, dy_lane, 16 * mt + g8);
      const float dyg8 = __shfl_sync(0xffffffffu, dy_lane, 16 * mt + g8 + 8);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int c = nt * 8 + 2 * t4;
        float w3a = m.w3[c], w3b = m.w3[c + 1];
        float z[4] = {z2[mt].h[nt][0], z2[mt].h[nt][1], z2[mt].h[nt][2], z2[mt].h[nt][3]};
        // dw3[c] += sum over rows of dy * h2
        float pa = dyg * bf16r(fmaxf(z[0], 0.0f)) + dyg8 * bf16r(fmaxf(z[2], 0.0f));
        float pb = dyg * bf16r(fmaxf(z[1], 0.0f)) + dyg8 * bf16r(fmaxf(z[3], 0.0f));
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
          pa += __shfl_xor_sync(0xffffffffu, pa, o);
          pb += __shfl_xor_sync(0xffffffffu, pb, o);
        }
        if (g8 == 0) {
          atomicAdd(&gacc[kOffW3 + c], pa);
          atomicAdd(&gacc[kOffW3 + c + 1], pb);
        }
        dz2[mt].h[nt][0] = z[0] > 0.0f ? dyg * w3a : 0.0f;
        dz2[mt].h[nt][1] = z[1] > 0.0f ? dyg * w3b : 0.0f;
        dz2[mt].h[nt][2] = z[2] > 0.0f ? dyg8 * w3a : 0.0f;
        dz2[mt].h[nt][3] = z[3] > 0.0f ? dyg8 * w3b : 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) h1[mt].h[nt][i] = fmaxf(z1[mt].h[nt][i], 0.0f);
      }
      store_hid(h1[mt], mt, B.h1);
      store_hid(dz2[mt], mt, B.dz2);
    }
    __syncwarp();
    // db2 = column sums of dz2 (from the BF16-staged copy, as the GEMMs see it)
    for (int c = lane; c < kMlpHid; c += 32) {
      float sacc = 0.0f;
      for (int r = 0; r < 32; ++r) sacc += __bfloat162float(B.dz2[r * kMlpHid + c]);
      atomicAdd(&gacc[kOffB2 + c], sacc);
    }
    // dW2 = h1^T dz2 : [64 x 32] x [32 x 64]
#pragma unroll 1
    for (int mi = 0; mi < 4; ++mi) {
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float d[4] = {0, 0, 0, 0};
#pragma unroll
        for (int kc = 0; kc < 2; ++kc) {
          uint32_t a[4], b0, b1;
          afrag_T(B.h1, kMlpHid, mi, kc, a);
          bfrag_S(B.dz2, kMlpHid, kc, nt, b0, b1);
          mma_bf16(d, a, b0, b1);
        }
        const int r = mi * 16 + g8, c = nt * 8 + 2 * t4;  // W2[r][c]
        atomicAdd(&gacc[kOffW2 + r * kMlpHid + c], d[0]);
        atomicAdd(&gacc[kOffW2 + r * kMlpHid + c + 1], d[1]);
        atomicAdd(&gacc[kOffW2 + (r + 8) * kMlpHid + c], d[2]);
        atomicAdd(&gacc[kOffW2 + (r + 8) * kMlpHid + c + 1], d[3]);
      }
    }
    // dz1 = (dz2 W2^T) [z1 > 0], staged into the h1 buffer
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      Hid dz1;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float d[4] = {0, 0, 0, 0};
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
          uint32_t a[4], b0, b1;
          afrag_from_hid(dz2[mt], kc, a);
          bfrag_w2back(m.w2t, kc, nt, b0, b1);
          mma_bf16(d, a, b0, b1);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) dz1.h[nt][i] = z1[mt].h[nt][i] > 0.0f ? d[i] : 0.0f;
      }
      store_hid(dz1, mt, B.h1);
    }
    __syncwarp();
    for (int c = lane; c < kMlpHid; c += 32) {
      float sacc = 0.0f;
      for (int r = 0; r < 32; ++r) sacc += __bfloat162float(B.h1[r * kMlpHid + c]);
      atomicAdd(&gacc[kOffB1 + c], sacc);
    }
    // dW1 = x^T dz1 : [16 x 32] x [32 x 64]
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float d[4] = {0, 0, 0, 0};
#pragma unroll
      for (int kc = 0; kc < 2; ++kc) {
        uint32_t a[4], b0, b1;
        afrag_T(B.x, kMlpIn, 0, kc, a);
        bfrag_S(B.h1, kMlpHid, kc, nt, b0, b1);
        mma_bf16(d, a, b0, b1);
      }
      const int r = g8, c = nt * 8 + 2 * t4;  // W1[r][c]
      atomicAdd(&gacc[kOffW1 + r * kMlpHid + c], d[0]);
      atomicAdd(&gacc[kOffW1 + r * kMlpHid + c + 1], d[1]);
      atomicAdd(&gacc[kOffW1 + (r + 8) * kMlpHid + c], d[2]);
      atomicAdd(&gacc[kOffW1 + (r + 8) * kMlpHid + c + 1], d[3]);
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0 && loss) atomicAdd(loss, lsum * inv_batch);
  __syncthreads();
  for (int i = threadIdx.x; i < kMlpWeights; i += blockDim.x)
    if (gacc[i] != 0.0f) atomicAdd(&g[i], gacc[i]);
}

// Adam (Kingma & Ba 2015) on the trainable block; step counts from 1.
__global__ void k_mlp_adam(float* __restrict__ P, float* __restrict__ Mm, float* __restrict__ Vv,
                           const float* __restrict__ g, int step, float lr, float b1, float b2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpWeights) return;
  const float gi = g[i];
  const float m = b1 * Mm[i] + (1.0f - b1) * gi;
  const float v = b2 * Vv[i] + (1.0f - b2) * gi * gi;
  Mm[i] = m;
  Vv[i] = v;
  const float mh = m / (1.0f - powf(b1, (float)step)), vh = v / (1.0f - powf(b2, (float)step));
  P[i] -= lr * mh / (sqrtf(vh) + eps);
}

// Mean and standard deviation of every feature and of the target, written into the
// parameter block (one block, FP64 sums; used once per training set).
__global__ void __launch_bounds__(1024) k_mlp_moments(const float* __restrict__ X, const float* __restrict__ T,
                                                      int64_t n, float* __restrict__ P) {
  __shared__ double sh[17][2];
  if (threadIdx.x < 34) (&sh[0][0])[threadIdx.x] = 0.0;
  __syncthreads();
  double loc[17][2] = {};
  for (int64_t s = threadIdx.x; s < n; s += blockDim.x) {
    for (int i = 0; i < 16; ++i) {
      const double v = X[s * 16 + i];
      loc[i][0] += v;
      loc[i][1] += v * v;
    }
    const double t = T[s];
    loc[16][0] += t;
    loc[16][1] += t * t;
  }
  for (int i = 0; i < 17; ++i) {
    atomicAdd(&sh[i][0], loc[i][0]);
    atomicAdd(&sh[i][1], loc[i][1]);
  }
  __syncthreads();
  const int i = threadIdx.x;
  if (i < 17) {
    const double mean = sh[i][0] / (double)n;
    const double var = sh[i][1] / (double)n - mean * mean;
    const double sd = sqrt(var > 1e-12 ? var : 1e-12);
    if (i < 16) {
      P[kOffMean + i] = (float)mean;
      P[kOffInvStd + i] = (float)(1.0 / sd);
    } else {
      P[kOffTMean] = (float)mean;
      P[kOffTScale] = (float)sd;
    }
  }
}

// Inference on arrays (for testing and diagnostics): standardized-target predictions.
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X, int64_t n,
                                                     float* __restrict__ out) {
  __shared__ MlpSmem m;
  __shared__ __align__(16) __nv_bfloat16 tiles[4][32 * kMlpIn];
  mlp_load_smem(m, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tiles_n = (n + 31) / 32;
  for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < tiles_n; tile += (int64_t)gridDim.x * 4) {
    const int64_t s = tile * 32 + lane;
    float f[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = s < n ? X[s * 16 + i] : m.mean[i];
    const float y = mlp_warp_infer(m, f, tiles[warp]);
    if (s < n) out[s] = y;
  }
}

}  // namespace

size_t mlp_grad_smem_bytes() {
  return ((sizeof(MlpSmem) + 15) & ~size_t(15)) + sizeof(float) * ((kMlpWeights + 3) & ~3) +
         sizeof(WarpBufs) * kTrainWarps;
}

cudaError_t launch_mlp_grad(const float* P, const float* X, const float* T, int64_t n, float inv_batch, float* g,
                            float* loss, int sms, cudaStream_t st) {
  const size_t smem = mlp_grad_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  int64_t tiles = (n + 31) / 32;
  int64_t blocks = (tiles + kTrainWarps - 1) / kTrainWarps;
  if (blocks > 2 * sms) blocks = 2 * sms;
  if (blocks < 1) blocks = 1;
  k_mlp_grad<<<(int)blocks, 32 * kTrainWarps, smem, st>>>(P, X, T, n, inv_batch, g, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* P, float* M, float* V, const float* g, int step, float lr, cudaStream_t st) {
  k_mlp_adam<<<(kMlpWeights + 255) / 256, 256, 0, st>>>(P, M, V, g, step, lr, 0.9f, 0.999f, 1e-8f);
  return cudaGetLastError();
}

cudaError_t launch_mlp_moments(const float* X, const float* T, int64_t n, float* P, cudaStream_t st) {
  k_mlp_moments<<<1, 1024, 0, st>>>(X, T, n, P);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* P, const float* X, int64_t n, float* out, int sms, cudaStream_t st) {
  int64_t tiles = (n + 31) / 32;
  int64_t blocks = (tiles + 3) / 4;
  if (blocks > 8 * sms) blocks = 8 * sms;
  if (blocks < 1) blocks = 1;
  k_mlp_forward<<<(int)blocks, 128, 0, st>>>(P, X, n, out);
  return cudaGetLastError();
}

}  // namespace lt
