// Row-capacity MLP shared by the training kernels and the fused inference in
// the learned analysis pass: 8 features -> 32 -> 32 -> 16 classes, ReLU.
#pragma once

#include <cstdint>

#include "kk_device.cuh"

namespace kk {

constexpr int kMlpF = 8;
constexpr int kMlpH = 32;
constexpr int kMlpC = 16;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpF * kMlpH;
constexpr int kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + kMlpH * kMlpC;
constexpr int kMlpParams = kOffB3 + kMlpC;  // 1872

static_assert(kMlpParams == 1872, "parameter layout");

// Forward pass of one sample with parameters P (usually in shared memory).
__device__ __forceinline__ void mlp_forward(const float* P, const float (&x)[kMlpF],
                                            float (&h1)[kMlpH], float (&h2)[kMlpH],
                                            float (&z)[kMlpC]) {
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    float a = P[kOffB1 + j];
#pragma unroll
    for (int f = 0; f < kMlpF; ++f) a = fmaf(x[f], P[kOffW1 + f * kMlpH + j], a);
    h1[j] = fmaxf(a, 0.0f);
  }
#pragma unroll
  for (int k = 0; k < kMlpH; ++k) {
    float a = P[kOffB2 + k];
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) a = fmaf(h1[j], P[kOffW2 + j * kMlpH + k], a);
    h2[k] = fmaxf(a, 0.0f);
  }
#pragma unroll
  for (int c = 0; c < kMlpC; ++c) {
    float a = P[kOffB3 + c];
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) a = fmaf(h2[k], P[kOffW3 + k * kMlpC + c], a);
    z[c] = a;
  }
}

// Smallest class whose cumulative softmax probability reaches q (q <= 0: argmax).
__device__ __forceinline__ int mlp_class(const float (&z)[kMlpC], float q) {
  float mx = z[0];
  int am = 0;
#pragma unroll
  for (int c = 1; c < kMlpC; ++c)
    if (z[c] > mx) {
      mx = z[c];
      am = c;
    }
  if (q <= 0.0f) return am;
  float e[kMlpC], s = 0.0f;
#pragma unroll
  for (int c = 0; c < kMlpC; ++c) {
    e[c] = __expf(z[c] - mx);
    s += e[c];
  }
  const float target = q * s;
  float cum = 0.0f;
#pragma unroll
  for (int c = 0; c < kMlpC; ++c) {
    cum += e[c];
    if (cum >= target) return c;
  }
  return kMlpC - 1;
}

// Capacity class of a row count c: 0 if c <= 16, else ceil(log2(c / 16)), max 15.
__device__ __forceinline__ int capacity_class_of(long long c) {
  int t = 0;
  long long cap = 16;
  while (cap < c && t < kMlpC - 1) {
    cap <<= 1;
    ++t;
  }
  return t;
}

}  // namespace kk
