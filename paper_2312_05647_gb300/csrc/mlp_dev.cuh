// mlp_dev.cuh -- device pieces of the 4 -> 128 -> 128 -> 1 tanh perceptron
// shared by the training kernels (mlp.cu) and the delayed-acceptance screen
// (sampler.cu).  One CTA of 128 threads evaluates rows; thread j owns hidden
// unit j of both layers.  Every sum runs in one fixed order, so a row gives
// the same bits whichever kernel evaluates it.
#pragma once

#include <cstdint>

namespace mjp {
namespace mlp {

constexpr int D = 4, H = 128, NPAR = 17281;
constexpr int OW1 = 0, OB1 = 512, OW2 = 640, OB2 = 17024, OW3 = 17152, OB3 = 17280;
constexpr int W2S = H + 1;  // padded row stride of W2 in shared memory
constexpr uint32_t kInitStream = 0x4D4C5000u;
constexpr uint32_t kBatchStream = 0x4D4C5001u;

// Standardisation, in the order of the C ABI's norm vector.
struct Norm {
  double mux[4], sdx[4], muy, sdy;
};

// W2 (row i, column j at i*128 + j) into shared memory with row stride 129:
// thread j reading W2s[i*129 + j] over j, and thread i reading it over j, both
// touch 32 distinct banks.
__device__ __forceinline__ void stage_w2(const float* __restrict__ P, float* W2s) {
  const float4* src = reinterpret_cast<const float4*>(P + OW2);
  for (int e = threadIdx.x; e < H * H / 4; e += blockDim.x) {
    const float4 w = src[e];
    const int i = (e * 4) / H, c = (e * 4) % H;
    float* d = W2s + i * W2S + c;
    d[0] = w.x;
    d[1] = w.y;
    d[2] = w.z;
    d[3] = w.w;
  }
}

// Sum of v over the 32 lanes of a warp, butterfly order.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Standardised input component k of psi.
__device__ __forceinline__ float std_input(const Norm& nm, const double* psi, int k) {
  return (float)((psi[k] - nm.mux[k]) / nm.sdx[k]);
}

// Pre-activation of hidden unit j of layer 1: b1 + sum_k x_k W1[k][j], k ascending.
__device__ __forceinline__ float layer1(const float x[4], const float w1[4], float b1) {
  float z = b1;
#pragma unroll
  for (int k = 0; k < 4; ++k) z = fmaf(x[k], w1[k], z);
  return z;
}

}  // namespace mlp
}  // namespace mjp
