// hmat_mlp.cuh -- the rank predictor: a 3-layer MLP of width 64 with BF16
// weights and FP32 accumulation.
//
//   x (6 features) -> relu(W1 x + b1) (64) -> relu(W2 h1 + b2) (64)
//                  -> w3 . h2 + b3  = predicted log(1 + truncated rank)
//
// Features of a truncation of block (t, r) at tolerance eps:
//   log2 #t / 10, log2 #r / 10, log(dbar / (dist(t, r) + 1e-3 dbar)) / 4 with
//   dbar the mean diameter of t and r, dimension / 3,
//   l / 16 (l = rank of the sum before truncation), log10(eps) / 4.
// Parameters are one flat FP32 master array (layout below); the network is
// evaluated with the BF16-rounded copy of the masters.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#define HM_MLP_IN 6
#define HM_MLP_H 64
#define HM_MLP_W1 0                                  // [64][6]
#define HM_MLP_B1 (HM_MLP_W1 + HM_MLP_H * HM_MLP_IN)  // [64]
#define HM_MLP_W2 (HM_MLP_B1 + HM_MLP_H)              // [64][64]
#define HM_MLP_B2 (HM_MLP_W2 + HM_MLP_H * HM_MLP_H)   // [64]
#define HM_MLP_W3 (HM_MLP_B2 + HM_MLP_H)              // [64]
#define HM_MLP_B3 (HM_MLP_W3 + HM_MLP_H)              // [1]
#define HM_MLP_NPARAM (HM_MLP_B3 + 1)                 // 4673

namespace hm {

// One warp evaluates the network for one feature vector (lanes own two hidden
// units each); every lane returns the output.
static __device__ __forceinline__ float mlp_forward_warp(const __nv_bfloat16* W, const float* x) {
  int lane = threadIdx.x & 31;
  float h1[2], h2[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    int o = lane + 32 * u;
    float a = __bfloat162float(W[HM_MLP_B1 + o]);
#pragma unroll
    for (int i = 0; i < HM_MLP_IN; ++i) a += __bfloat162float(W[HM_MLP_W1 + o * HM_MLP_IN + i]) * x[i];
    h1[u] = a > 0.f ? a : 0.f;
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    int o = lane + 32 * u;
    float a = __bfloat162float(W[HM_MLP_B2 + o]);
    for (int i = 0; i < HM_MLP_H; ++i) {
      float hi = __shfl_sync(0xffffffffu, h1[i >> 5], i & 31);
      a += __bfloat162float(W[HM_MLP_W2 + o * HM_MLP_H + i]) * hi;
    }
    h2[u] = a > 0.f ? a : 0.f;
  }
  float part = __bfloat162float(W[HM_MLP_W3 + lane]) * h2[0] + __bfloat162float(W[HM_MLP_W3 + lane + 32]) * h2[1];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  return part + __bfloat162float(W[HM_MLP_B3]);
}

}  // namespace hm
