// Patch network f: 25 -> 64 -> 64 -> 1 (ReLU) on the tensor cores: warp-level
// mma.sync m16n8k16 with bfloat16 operands and FP32 accumulation, 16 patches per tile.
//
// The weights are bfloat16 already.  The inputs z and the first hidden layer h1 are FP32
// values; each is split into two bfloat16 terms, hi = bf16(v) and lo = bf16(v - hi), and both
// terms are multiplied by the weights (products of bfloat16 numbers are exact in FP32), so the
// layers see the FP32 operand to about 2^-17 relative instead of bfloat16's 2^-9.  Layer 3 (64
// -> 1) is a per-row dot product in FP32.
//
// Every evaluation of f in the library goes through nn_tile_f with the same instruction
// sequence, and each output row of an mma depends only on its own A row, so a patch gets
// bit-identical f wherever it sits in a tile: the inner chain's changes of F and the cached
// patch values agree exactly, which the exactness of the cumulative accept relies on.
//
// Fragment layouts (PTX ISA, mma.m16n8k16 with .bf16): lane = 4 g + t.
//   A (16 x 16, row): a0 = (A[g][2t], A[g][2t+1]), a1 = rows g+8, a2 = cols 2t+8.., a3 = both.
//   B (16 x 8, col):  b0 = (B[2t][g], B[2t+1][g]), b1 = (B[2t+8][g], B[2t+9][g]).
//   C (16 x 8):       c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1].
// The C fragments of n-tiles 2s and 2s+1 of one layer are exactly the A fragment of k-step s
// of the next layer, so h1 never leaves the registers.
#pragma once
#include <cstdint>
#include "hq_device.cuh"

namespace hq {

constexpr int TC_IN = 25, TC_H = 64, TC_K1 = 32;          // layer-1 K padded to two k-steps
constexpr int TC_W1 = 0, TC_B1 = TC_IN * TC_H, TC_W2 = TC_B1 + TC_H, TC_B2 = TC_W2 + TC_H * TC_H,
              TC_W3 = TC_B2 + TC_H, TC_B3 = TC_W3 + TC_H;
constexpr int TC_FRAGS = (2 + 4) * 8 * 32;                 // uint2 per CTA: W1 (2 k-steps), W2 (4)
constexpr int TC_FLOATS = 3 * TC_H + 4;                    // b1, b2, W3, b3 (padded)

struct NNFrags {
  const uint2* w1;  // [2][8][32]
  const uint2* w2;  // [4][8][32]
  const float* b1;
  const float* b2;
  const float* w3;
  float b3;
};

__device__ __forceinline__ uint32_t pack_bf16(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// Fragments of W1 (K padded with zeros) and W2 for every lane, and the FP32 vectors, from the
// bfloat16 weights; all threads of the CTA, ends with a barrier.
__device__ inline NNFrags nn_build_frags(const uint16_t* wb, uint2* frag, float* fl) {
  for (int e = threadIdx.x; e < TC_FRAGS; e += blockDim.x) {
    const int lane = e % 32, j = (e / 32) % 8, s = e / 256;  // s < 2: W1, else W2 step s - 2
    const int g = lane >> 2, t = lane & 3;
    uint16_t v[4];
    for (int q = 0; q < 4; ++q) {
      const int kk = 2 * t + (q & 1) + 8 * (q >> 1);  // k within the step
      const int n = 8 * j + g;
      if (s < 2) {
        const int k = 16 * s + kk;
        v[q] = k < TC_IN ? wb[TC_W1 + k * TC_H + n] : (uint16_t)0;
      } else {
        const int k = 16 * (s - 2) + kk;
        v[q] = wb[TC_W2 + k * TC_H + n];
      }
    }
    frag[e] = make_uint2(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]));
  }
  for (int e = threadIdx.x; e < TC_FLOATS; e += blockDim.x) {
    float x = 0.f;
    if (e < TC_H) x = bf16_to_float(wb[TC_B1 + e]);
    else if (e < 2 * TC_H) x = bf16_to_float(wb[TC_B2 + e - TC_H]);
    else if (e < 3 * TC_H) x = bf16_to_float(wb[TC_W3 + e - 2 * TC_H]);
    else if (e == 3 * TC_H) x = bf16_to_float(wb[TC_B3]);
    fl[e] = x;
  }
  __syncthreads();
  NNFrags f;
  f.w1 = frag;
  f.w2 = frag + 2 * 8 * 32;
  f.b1 = fl;
  f.b2 = fl + TC_H;
  f.w3 = fl + 2 * TC_H;
  f.b3 = fl[3 * TC_H];
  return f;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// v = hi + lo in bfloat16 (hi, lo packed by pairs: first element in the low half)
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const uint16_t h0 = float_to_bf16(v0), h1 = float_to_bf16(v1);
  const uint16_t l0 = float_to_bf16(v0 - bf16_to_float(h0)), l1 = float_to_bf16(v1 - bf16_to_float(h1));
  hi = pack_bf16(h0, h1);
  lo = pack_bf16(l0, l1);
}

// f of 16 patches by one warp.  zval(row, k) gives input k (0..24) of patch row (0..15) as a
// float; it is called for k < 25 only.  Returns f of row g in f_g and of row g + 8 in f_g8
// (g = lane / 4; every lane of the quad holds them).
template <class ZF>
__device__ __forceinline__ void nn_tile_f(const NNFrags& w, ZF zval, float& f_g, float& f_g8) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc1[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc1[j][e] = 0.f;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    uint32_t ahi[4], alo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = g + 8 * (q & 1);
      const int k = 16 * s + 2 * t + 8 * (q >> 1);
      const float v0 = k < TC_IN ? zval(row, k) : 0.f;
      const float v1 = k + 1 < TC_IN ? zval(row, k + 1) : 0.f;
      split2(v0, v1, ahi[q], alo[q]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint2 b = w.w1[(s * 8 + j) * 32 + lane];
      mma_bf16(acc1[j], ahi, b);
      mma_bf16(acc1[j], alo, b);
    }
  }
  float acc2[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc2[j][e] = 0.f;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    // h1 of n-tiles 2s, 2s+1 (bias, ReLU) as the A fragment of k-step s
    uint32_t ahi[4], alo[4];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int j = 2 * s + half;
      const float bb0 = w.b1[8 * j + 2 * t], bb1 = w.b1[8 * j + 2 * t + 1];
      split2(fmaxf(acc1[j][0] + bb0, 0.f), fmaxf(acc1[j][1] + bb1, 0.f), ahi[2 * half], alo[2 * half]);
      split2(fmaxf(acc1[j][2] + bb0, 0.f), fmaxf(acc1[j][3] + bb1, 0.f), ahi[2 * half + 1], alo[2 * half + 1]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint2 b = w.w2[(s * 8 + j) * 32 + lane];
      mma_bf16(acc2[j], ahi, b);
      mma_bf16(acc2[j], alo, b);
    }
  }
  float o0 = 0.f, o1 = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int u = 8 * j + 2 * t;
    const float bb0 = w.b2[u], bb1 = w.b2[u + 1], w0 = w.w3[u], w1 = w.w3[u + 1];
    o0 = fmaf(fmaxf(acc2[j][0] + bb0, 0.f), w0, o0);
    o0 = fmaf(fmaxf(acc2[j][1] + bb1, 0.f), w1, o0);
    o1 = fmaf(fmaxf(acc2[j][2] + bb0, 0.f), w0, o1);
    o1 = fmaf(fmaxf(acc2[j][3] + bb1, 0.f), w1, o1);
  }
  o0 += __shfl_xor_sync(HQ_FULL, o0, 1);
  o0 += __shfl_xor_sync(HQ_FULL, o0, 2);
  o1 += __shfl_xor_sync(HQ_FULL, o1, 1);
  o1 += __shfl_xor_sync(HQ_FULL, o1, 2);
  f_g = o0 + w.b3;
  f_g8 = o1 + w.b3;
}

}  // namespace hq

namespace hq {

// ------------------------------------------------------------------ training on the tensor cores
// Backward pass of the mean squared error (1/B) sum_a (F(X_a) - y_a)^2 for a minibatch, with
// F(X) = sum over the patches of f.  Every patch row of every sample gets the output gradient
// dout = 2 (F_a - y_a) / B; per tile of 16 rows a warp recomputes the forward pass and forms
//   d2 = relu'(a2) (dout W3),  d1 = relu'(a1) (d2 W2^T)           (tensor cores, K = 64)
// and the CTA then contracts over its 128 rows
//   gW2 = h1^T d2,  gW1 = z^T d1                                   (tensor cores, K = rows)
// with every operand split into bfloat16 hi + lo terms (products hi hi + hi lo + lo hi, FP32
// accumulation), so the gradient carries FP32-level precision.  The bias gradients and gW3 are
// column sums in FP32.  Every gradient entry has one owner, sums run in a fixed order, and the
// per-CTA partials are added in a fixed order by the Adam kernel: the result is deterministic.

constexpr int TR_ROWS = 128;        // rows per CTA chunk (8 warps x 16)
constexpr int TR_LD = TR_ROWS + 8;  // padded row of the transposed staging tiles (uint16)
constexpr int TR_FRAGS = TC_FRAGS + 4 * 8 * 32;  // + W2^T fragments

__host__ __device__ inline size_t nn_train_tc_smem_bytes() {
  return sizeof(uint2) * TR_FRAGS + sizeof(float) * (TC_FLOATS + 3 * 8 * TC_H + 8) +
         sizeof(uint16_t) * (size_t)TR_LD * (2 * TC_H + 2 * TC_H + 2 * TC_K1 + 2 * TC_H);
}

__device__ __forceinline__ void split1(float v, uint16_t& hi, uint16_t& lo) {
  hi = float_to_bf16(v);
  lo = float_to_bf16(v - bf16_to_float(hi));
}

__device__ __forceinline__ uint32_t ld32(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// C += A B over one k-step, A from a transposed tile AT[m][k] (rows m0.., cols k0..), B from a
// transposed tile BT[n][k]; three products hi hi, hi lo, lo hi.
__device__ __forceinline__ void mma_tiles3(float (&c)[4], const uint16_t* ah, const uint16_t* al, const uint16_t* bh,
                                           const uint16_t* bl, int m0, int n0, int k0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t Ah[4], Al[4];
  const int r0 = (m0 + g) * TR_LD + k0 + 2 * t, r1 = (m0 + g + 8) * TR_LD + k0 + 2 * t;
  Ah[0] = ld32(ah + r0); Ah[1] = ld32(ah + r1); Ah[2] = ld32(ah + r0 + 8); Ah[3] = ld32(ah + r1 + 8);
  Al[0] = ld32(al + r0); Al[1] = ld32(al + r1); Al[2] = ld32(al + r0 + 8); Al[3] = ld32(al + r1 + 8);
  const int q = (n0 + g) * TR_LD + k0 + 2 * t;
  const uint2 Bh = make_uint2(ld32(bh + q), ld32(bh + q + 8));
  const uint2 Bl = make_uint2(ld32(bl + q), ld32(bl + q + 8));
  mma_bf16(c, Ah, Bh);
  mma_bf16(c, Ah, Bl);
  mma_bf16(c, Al, Bh);
}

}  // namespace hq
