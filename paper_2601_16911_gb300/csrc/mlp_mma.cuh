// The surrogate sensor network 12 -> 64 -> 64 -> 2 (tanh-form GELU) on the tensor cores:
// BF16 operands, FP32 accumulation, one warp evaluates 32 samples (lane l owns sample l)
// with mma.sync m16n8k16 in two 16-row halves.  The weights arrive pre-packed in the
// per-lane B-fragment order (MlpPacked, built by mlp_pack_kernel), so a fragment is one
// 8-byte shared-memory load; the FP32 accumulators of one layer are converted in place
// into the A fragments of the next (the m16n8 accumulator layout of two adjacent column
// tiles is the m16k16 A layout), so hidden activations never leave registers.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace cvw {

constexpr int kMlpIn = 12, kMlpHidden = 64, kMlpOut = 2;
// Flat FP32 parameter layout: W1 (64,12), b1 (64), W2 (64,64), b2 (64), W3 (2,64), b3 (2).
constexpr int kMlpOffW1 = 0, kMlpOffB1 = 768, kMlpOffW2 = 832, kMlpOffB2 = 4928, kMlpOffW3 = 4992,
              kMlpOffB3 = 5120, kMlpParams = 5122;

// Packed weights: B fragments (two b32 registers of bf16 pairs per lane) and FP32 biases.
//   w1[nt][lane]      layer 1, K = 16 (inputs 12..15 zero), N tiles nt = 0..7
//   w2[kk][nt][lane]  layer 2, K steps kk = 0..3, N tiles nt = 0..7
//   w3[kk][lane]      layer 3, one N tile (outputs 2..7 zero)
struct MlpPacked {
  uint2 w1[8][32];
  uint2 w2[4][8][32];
  uint2 w3[4][32];
  float b1[64];
  float b2[64];
  float b3[4];
};
static_assert(sizeof(MlpPacked) % 16 == 0, "packed weights are copied as uint4");

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half), .y = hi
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// GELU, tanh form, with the hardware tanh approximation (its error, ~2^-11 relative, is
// below the bf16 rounding that follows).
__device__ __forceinline__ float gelu_fast(float x) {
  const float u = 0.7978845608028654f * fmaf(0.044715f * x * x, x, x);
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
  return 0.5f * x * (1.0f + t);
}

// One warp, 32 samples.  x: this lane's 12 inputs; xs: 32 x 16 bf16 warp scratch in shared
// memory (16-byte aligned); W: packed weights in shared memory.  Returns this lane's
// two outputs.  All 32 lanes must call it.
__device__ __forceinline__ void mlp_warp(const MlpPacked& W, const float (&x)[kMlpIn], __nv_bfloat16* xs, float& o0,
                                         float& o1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  {
    uint32_t* row = reinterpret_cast<uint32_t*>(xs + lane * 16);
#pragma unroll
    for (int j = 0; j < 6; ++j) row[j] = pack_bf16x2(x[2 * j], x[2 * j + 1]);
    row[6] = 0u;
    row[7] = 0u;
  }
  __syncwarp();
  const uint32_t* xw = reinterpret_cast<const uint32_t*>(xs);  // row r: words 8r .. 8r+7
  float out[2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = 16 * mt + g, r1 = r0 + 8;
    const uint32_t a_in[4] = {xw[8 * r0 + t], xw[8 * r1 + t], xw[8 * r0 + 4 + t], xw[8 * r1 + 4 + t]};
    // layer 1 -> GELU -> A fragments of layer 2
    uint32_t a1[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float bl = W.b1[8 * nt + 2 * t], bh = W.b1[8 * nt + 2 * t + 1];
      float c[4] = {bl, bh, bl, bh};
      mma_bf16_16816(c, a_in, W.w1[nt][lane]);
      const uint32_t lo = pack_bf16x2(gelu_fast(c[0]), gelu_fast(c[1]));
      const uint32_t hi = pack_bf16x2(gelu_fast(c[2]), gelu_fast(c[3]));
      a1[nt >> 1][(nt & 1) ? 2 : 0] = lo;
      a1[nt >> 1][(nt & 1) ? 3 : 1] = hi;
    }
    // layer 2 -> GELU -> A fragments of layer 3
    uint32_t a2[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float bl = W.b2[8 * nt + 2 * t], bh = W.b2[8 * nt + 2 * t + 1];
      float c[4] = {bl, bh, bl, bh};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma_bf16_16816(c, a1[kk], W.w2[kk][nt][lane]);
      const uint32_t lo = pack_bf16x2(gelu_fast(c[0]), gelu_fast(c[1]));
      const uint32_t hi = pack_bf16x2(gelu_fast(c[2]), gelu_fast(c[3]));
      a2[nt >> 1][(nt & 1) ? 2 : 0] = lo;
      a2[nt >> 1][(nt & 1) ? 3 : 1] = hi;
    }
    // layer 3: columns 2t, 2t+1 of rows g and g+8 (only t = 0 holds real outputs)
    const float bl = t == 0 ? W.b3[0] : 0.0f, bh = t == 0 ? W.b3[1] : 0.0f;
    float c[4] = {bl, bh, bl, bh};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) mma_bf16_16816(c, a2[kk], W.w3[kk][lane]);
#pragma unroll
    for (int i = 0; i < 4; ++i) out[mt][i] = c[i];
  }
  // sample l = 16 mt + r: row r < 8 sits in lane 4r (c0, c1), row r >= 8 in lane 4(r-8) (c2, c3)
  const int mt = lane >> 4, r = lane & 15, src = 4 * (r & 7);
  float v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float s0 = __shfl_sync(0xffffffffu, out[0][i], src);
    const float s1 = __shfl_sync(0xffffffffu, out[1][i], src);
    v[i] = mt ? s1 : s0;
  }
  o0 = r < 8 ? v[0] : v[2];
  o1 = r < 8 ? v[1] : v[3];
  __syncwarp();  // xs may be reused by the caller
}

}  // namespace cvw
