// lt_mlp.cuh -- warp-level 16 -> 64 -> 64 -> 1 ReLU MLP on tensor cores (sm_103a).
//
// BF16 weights and activations, FP32 accumulation, mma.sync.m16n8k16 (32 samples per warp
// = two m16 tiles).  Used as the learned reservoir target of ResLRB: it predicts, from a
// sensor connection's features, the log of the adjoint weight the connection will see.
//
// Parameter block (FP32, LT_MLP_PARAMS floats, row-major):
//   W1 [16][64] | b1 [64] | W2 [64][64] | b2 [64] | W3 [64] | b3 | feature mean [16] |
//   feature 1/std [16] | target scale | target mean | pad
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lt {

constexpr int kMlpIn = 16, kMlpHid = 64;
constexpr int kOffW1 = 0, kOffB1 = 1024, kOffW2 = 1088, kOffB2 = 5184, kOffW3 = 5248, kOffB3 = 5312;
constexpr int kOffMean = 5313, kOffInvStd = 5329, kOffTScale = 5345, kOffTMean = 5346;
constexpr int kMlpParams = 5352;
constexpr int kMlpWeights = 5313;  // trainable parameters (W1..b3)

// Shared-memory image of the network: weights transposed to [out][in] in BF16 so that the
// two K-consecutive elements of a B fragment are one 32-bit word; biases in FP32.
struct MlpSmem {
  __nv_bfloat16 w1t[kMlpHid * kMlpIn];   // [64][16]
  __nv_bfloat16 w2t[kMlpHid * kMlpHid];  // [64][64]
  float b1[kMlpHid], b2[kMlpHid], w3[kMlpHid];
  float b3;
  float mean[kMlpIn], inv_std[kMlpIn];
  float tscale;
};

__device__ __forceinline__ void mlp_load_smem(MlpSmem& m, const float* __restrict__ P) {
  for (int i = threadIdx.x; i < kMlpHid * kMlpIn; i += blockDim.x) {
    int o = i / kMlpIn, k = i % kMlpIn;
    m.w1t[i] = __float2bfloat16_rn(P[kOffW1 + k * kMlpHid + o]);
  }
  for (int i = threadIdx.x; i < kMlpHid * kMlpHid; i += blockDim.x) {
    int o = i / kMlpHid, k = i % kMlpHid;
    m.w2t[i] = __float2bfloat16_rn(P[kOffW2 + k * kMlpHid + o]);
  }
  for (int i = threadIdx.x; i < kMlpHid; i += blockDim.x) {
    m.b1[i] = P[kOffB1 + i];
    m.b2[i] = P[kOffB2 + i];
    m.w3[i] = __bfloat162float(__float2bfloat16_rn(P[kOffW3 + i]));
  }
  for (int i = threadIdx.x; i < kMlpIn; i += blockDim.x) {
    m.mean[i] = P[kOffMean + i];
    m.inv_std[i] = P[kOffInvStd + i];
  }
  if (threadIdx.x == 0) {
    m.b3 = P[kOffB3];
    m.tscale = P[kOffTScale];
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low 16 bits), .y = hi
  return *reinterpret_cast<uint32_t*>(&v);
}

// D = A(16x16, row) * B(16x8, col) + C, BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragment of W^T stored [out][in]: element (k, n) = W[k][n] = wt[n * ld + k].
__device__ __forceinline__ void bfrag(const __nv_bfloat16* wt, int ld, int kc, int nt, uint32_t& b0, uint32_t& b1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* p = wt + (nt * 8 + g) * ld + kc * 16 + 2 * t;
  b0 = *reinterpret_cast<const uint32_t*>(p);
  b1 = *reinterpret_cast<const uint32_t*>(p + 8);
}

// Hidden activations of one m16 tile in accumulator layout: h[nt][0..3] holds rows
// (g, g, g+8, g+8) and columns (8nt+2t, 8nt+2t+1, 8nt+2t, 8nt+2t+1).
struct Hid {
  float h[8][4];
};

// A fragment for k-chunk kc (16 hidden units) built from accumulator tiles 2kc and 2kc+1.
__device__ __forceinline__ void afrag_from_hid(const Hid& H, int kc, uint32_t a[4]) {
  a[0] = pack_bf16(H.h[2 * kc][0], H.h[2 * kc][1]);
  a[1] = pack_bf16(H.h[2 * kc][2], H.h[2 * kc][3]);
  a[2] = pack_bf16(H.h[2 * kc + 1][0], H.h[2 * kc + 1][1]);
  a[3] = pack_bf16(H.h[2 * kc + 1][2], H.h[2 * kc + 1][3]);
}

// Forward pass of one m16 tile whose standardized BF16 inputs are given as an A fragment.
// Returns pre-activations z1, z2 (accumulator layout) when wanted and the tile's outputs in
// accumulator layout of column 0 (y[0] row g, y[1] row g+8; valid on lanes with t == 0).
__device__ __forceinline__ void mlp_tile_forward(const MlpSmem& m, const uint32_t ax[4], Hid& z1, Hid& z2,
                                                 float& y_g, float& y_g8) {
  const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float d[4] = {m.b1[nt * 8 + 2 * t], m.b1[nt * 8 + 2 * t + 1], m.b1[nt * 8 + 2 * t], m.b1[nt * 8 + 2 * t + 1]};
    uint32_t b0, b1;
    bfrag(m.w1t, kMlpIn, 0, nt, b0, b1);
    mma_bf16(d, ax, b0, b1);
#pragma unroll
    for (int i = 0; i < 4; ++i) z1.h[nt][i] = d[i];
  }
  Hid h1;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) h1.h[nt][i] = fmaxf(z1.h[nt][i], 0.0f);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float d[4] = {m.b2[nt * 8 + 2 * t], m.b2[nt * 8 + 2 * t + 1], m.b2[nt * 8 + 2 * t], m.b2[nt * 8 + 2 * t + 1]};
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      uint32_t a[4], b0, b1;
      afrag_from_hid(h1, kc, a);
      bfrag(m.w2t, kMlpHid, kc, nt, b0, b1);
      mma_bf16(d, a, b0, b1);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) z2.h[nt][i] = d[i];
  }
  // output layer (64 -> 1): per-thread partial dot products over its columns, then a
  // reduction across the four threads of a row group
  float yg = 0.0f, yg8 = 0.0f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float wa = m.w3[nt * 8 + 2 * t], wb = m.w3[nt * 8 + 2 * t + 1];
    yg += wa * __bfloat162float(__float2bfloat16_rn(fmaxf(z2.h[nt][0], 0.0f))) +
          wb * __bfloat162float(__float2bfloat16_rn(fmaxf(z2.h[nt][1], 0.0f)));
    yg8 += wa * __bfloat162float(__float2bfloat16_rn(fmaxf(z2.h[nt][2], 0.0f))) +
           wb * __bfloat162float(__float2bfloat16_rn(fmaxf(z2.h[nt][3], 0.0f)));
  }
  yg += __shfl_xor_sync(0xffffffffu, yg, 1);
  yg += __shfl_xor_sync(0xffffffffu, yg, 2);
  yg8 += __shfl_xor_sync(0xffffffffu, yg8, 1);
  yg8 += __shfl_xor_sync(0xffffffffu, yg8, 2);
  y_g = yg + m.b3;
  y_g8 = yg8 + m.b3;
}

// Standardize this lane's 16 raw features and stage them (BF16) in the warp's 32x16 tile.
__device__ __forceinline__ void mlp_stage_features(const MlpSmem& m, const float f[16], __nv_bfloat16* tile) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 16; ++i) tile[lane * 16 + i] = __float2bfloat16_rn((f[i] - m.mean[i]) * m.inv_std[i]);
}

// A fragment of m-tile mt (rows 16mt..16mt+15) from the staged 32x16 feature tile.
__device__ __forceinline__ void afrag_from_tile(const __nv_bfloat16* tile, int mt, uint32_t a[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* r0 = tile + (mt * 16 + g) * 16;
  const __nv_bfloat16* r8 = tile + (mt * 16 + g + 8) * 16;
  a[0] = *reinterpret_cast<const uint32_t*>(r0 + 2 * t);
  a[1] = *reinterpret_cast<const uint32_t*>(r8 + 2 * t);
  a[2] = *reinterpret_cast<const uint32_t*>(r0 + 2 * t + 8);
  a[3] = *reinterpret_cast<const uint32_t*>(r8 + 2 * t + 8);
}

// Standardize 16 raw features (src[i * stride]) and stage them (BF16) as row `row` of the
// warp's 32x16 tile.
__device__ __forceinline__ void mlp_stage_row(const MlpSmem& m, const float* src, int stride, __nv_bfloat16* tile,
                                              int row) {
#pragma unroll
  for (int i = 0; i < 16; ++i) tile[row * 16 + i] = __float2bfloat16_rn((src[i * stride] - m.mean[i]) * m.inv_std[i]);
}

// Whole-warp inference of the first `rows` (1..32, the same on every lane) rows of a staged
// tile: lane r receives the output of row r.  Up to 16 rows take one m16 tile.
__device__ __forceinline__ float mlp_warp_infer_rows(const MlpSmem& m, const __nv_bfloat16* tile, int rows) {
  const int lane = threadIdx.x & 31;
  float out = 0.0f;
  for (int mt = 0; mt < (rows > 16 ? 2 : 1); ++mt) {
    uint32_t a[4];
    afrag_from_tile(tile, mt, a);
    Hid z1, z2;
    float yg, yg8;
    mlp_tile_forward(m, a, z1, z2, yg, yg8);
    // the output of row r of this tile sits on lane 4(r mod 8)
    const int r = lane - 16 * mt;
    const int src = 4 * (r & 7);
    const float a0 = __shfl_sync(0xffffffffu, yg, src), a8 = __shfl_sync(0xffffffffu, yg8, src);
    if (r >= 0 && r < 16) out = (r < 8) ? a0 : a8;
  }
  return out;
}

// Whole-warp inference: every lane passes its raw features, every lane receives its own
// network output (must be called by all 32 lanes together).
__device__ __forceinline__ float mlp_warp_infer(const MlpSmem& m, const float f[16], __nv_bfloat16* tile) {
  const int lane = threadIdx.x & 31, g = lane >> 2;
  mlp_stage_features(m, f, tile);
  __syncwarp();
  float out = 0.0f;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    uint32_t a[4];
    afrag_from_tile(tile, mt, a);
    Hid z1, z2;
    float yg, yg8;
    mlp_tile_forward(m, a, z1, z2, yg, yg8);
    // the sample in row r of this tile is lane 16mt + r; its output sits on lane 4(r mod 8)
    const int r = lane - 16 * mt;
    const int src = 4 * (r & 7);
    const float a0 = __shfl_sync(0xffffffffu, yg, src), a8 = __shfl_sync(0xffffffffu, yg8, src);
    if (r >= 0 && r < 16) out = (r < 8) ? a0 : a8;
    (void)g;
  }
  __syncwarp();
  return out;
}

}  // namespace lt
