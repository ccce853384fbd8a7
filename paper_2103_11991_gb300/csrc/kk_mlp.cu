// Learned row-capacity predictor: row features, capacity labels, and the
// training kernels (forward, backward, Adam) and inference of the MLP
// declared in kk_learned.h.  Everything runs on the GPU in float32.
#include <cmath>
#include <cstdio>
#include <vector>

#include "kk_internal.h"
#include "kk_learned.h"
#include "kk_mlp.cuh"

namespace kk {
namespace {

constexpr int kFeatTeam = 8;

// Per B row: smallest and largest column (empty rows: INT_MAX, -1).
__global__ void k_brow_minmax(CsrView B, int2* __restrict__ mm) {
  const int tl = threadIdx.x % kFeatTeam;
  const unsigned mask = team_mask<kFeatTeam>();
  const long long team0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kFeatTeam;
  const long long nteams = (long long)gridDim.x * blockDim.x / kFeatTeam;
  const long long iters = (B.m + nteams - 1) / nteams;
  for (long long it = 0; it < iters; ++it) {
    const long long r = team0 + it * nteams;
    int lo = 0x7fffffff, hi = -1;
    if (r < B.m) {
      for (int q = B.rowptr[r] + tl; q < B.rowptr[r + 1]; q += kFeatTeam) {
        const int c = B.colind[q];
        lo = min(lo, c);
        hi = max(hi, c);
      }
    }
#pragma unroll
    for (int o = kFeatTeam / 2; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(mask, lo, o, kFeatTeam));
      hi = max(hi, __shfl_xor_sync(mask, hi, o, kFeatTeam));
    }
    if (r < B.m && tl == 0) mm[r] = make_int2(lo, hi);
  }
}

__global__ void k_row_features(CsrView A, CsrView B, const int2* __restrict__ mm,
                               float* __restrict__ feat) {
  const int tl = threadIdx.x % kFeatTeam;
  const unsigned mask = team_mask<kFeatTeam>();
  const long long team0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kFeatTeam;
  const long long nteams = (long long)gridDim.x * blockDim.x / kFeatTeam;
  const long long iters = (A.m + nteams - 1) / nteams;
  for (long long it = 0; it < iters; ++it) {
    const long long r = team0 + it * nteams;
    long long f = 0;
    int mx = 0, mn = 0x7fffffff, lo = 0x7fffffff, hi = -1, nza = 0;
    if (r < A.m) {
      const int pa = A.rowptr[r], pe = A.rowptr[r + 1];
      nza = pe - pa;
      for (int p = pa + tl; p < pe; p += kFeatTeam) {
        const int j = A.colind[p];
        const int len = B.rowptr[j + 1] - B.rowptr[j];
        f += len;
        mx = max(mx, len);
        mn = min(mn, len);
        if (len > 0) {
          const int2 v = mm[j];
          lo = min(lo, v.x);
          hi = max(hi, v.y);
        }
      }
    }
#pragma unroll
    for (int o = kFeatTeam / 2; o > 0; o >>= 1) {
      f += __shfl_xor_sync(mask, f, o, kFeatTeam);
      mx = max(mx, __shfl_xor_sync(mask, mx, o, kFeatTeam));
      mn = min(mn, __shfl_xor_sync(mask, mn, o, kFeatTeam));
      lo = min(lo, __shfl_xor_sync(mask, lo, o, kFeatTeam));
      hi = max(hi, __shfl_xor_sync(mask, hi, o, kFeatTeam));
    }
    if (r < A.m && tl == 0) {
      if (nza == 0) mn = 0;
      const double span = hi >= lo ? (double)hi - (double)lo + 1.0 : 0.0;
      const double mean = nza ? (double)f / nza : 0.0;
      const double v[kMlpF] = {(double)nza, (double)f, (double)mx, mean, (double)(mx - mn),
                               span, fmin((double)f, span), fmin(fmin((double)f, span), (double)B.n)};
      float* out = feat + r * kMlpF;
#pragma unroll
      for (int t = 0; t < kMlpF; ++t) out[t] = log2f(1.0f + (float)v[t]);
    }
  }
}

__global__ void k_capacity_classes(int32_t m, const int64_t* __restrict__ rp, int32_t* __restrict__ cls) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x)
    cls[i] = capacity_class_of(rp[i + 1] - rp[i]);
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_mlp_init(float* __restrict__ P, unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  int fan_in = 0;
  if (i < kOffB1) fan_in = kMlpF;
  else if (i >= kOffW2 && i < kOffB2) fan_in = kMlpH;
  else if (i >= kOffW3 && i < kOffB3) fan_in = kMlpH;
  if (fan_in == 0) {
    P[i] = 0.0f;
    return;
  }
  const unsigned long long r = splitmix64(seed * 0x9E3779B97F4A7C15ull + (unsigned long long)i);
  const float u = (float)((r >> 40) * (1.0 / 16777216.0));  // [0, 1)
  P[i] = (2.0f * u - 1.0f) * sqrtf(6.0f / (float)fan_in);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kMlpBlock = 128;

// Gradient of the mean loss over `count` samples; sample t of the batch is
// index (pa * (start + t) + pb) mod n of X / y.
__global__ void __launch_bounds__(kMlpBlock)
k_mlp_loss_grad(int32_t n, int32_t start, int32_t count, long long pa, long long pb,
                const float* __restrict__ X, const int32_t* __restrict__ y,
                const float* __restrict__ Pg, float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float P[kMlpParams];
  __shared__ float G[kMlpParams];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    P[i] = Pg[i];
    G[i] = 0.0f;
  }
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = t < count;
  const int lane = threadIdx.x & 31;
  float x[kMlpF];
  int label = 0;
  if (active) {
    const long long s = (pa * (long long)(start + t) + pb) % n;
#pragma unroll
    for (int f = 0; f < kMlpF; ++f) x[f] = X[s * kMlpF + f];
    label = y[s];
  } else {
#pragma unroll
    for (int f = 0; f < kMlpF; ++f) x[f] = 0.0f;
  }
  float h1[kMlpH], h2[kMlpH], z[kMlpC];
  mlp_forward(P, x, h1, h2, z);
  float mx = z[0];
#pragma unroll
  for (int c = 1; c < kMlpC; ++c) mx = fmaxf(mx, z[c]);
  float se = 0.0f;
#pragma unroll
  for (int c = 0; c < kMlpC; ++c) se += __expf(z[c] - mx);
  const float lse = mx + __logf(se);
  const float inv = active ? 1.0f / (float)count : 0.0f;
  float dz[kMlpC];
  float zl = 0.0f;
#pragma unroll
  for (int c = 0; c < kMlpC; ++c) {
    const float p = __expf(z[c] - lse);
    dz[c] = (p - (c == label ? 1.0f : 0.0f)) * inv;
    if (c == label) zl = z[c];
  }
  const float l = active ? (lse - zl) * inv : 0.0f;
  const float ls = warp_sum_f(l);
  if (lane == 0) atomicAdd(loss, ls);
  // W3, b3
#pragma unroll
  for (int c = 0; c < kMlpC; ++c) {
    const float g = warp_sum_f(dz[c]);
    if (lane == 0) atomicAdd(&G[kOffB3 + c], g);
  }
  float dh2[kMlpH];
#pragma unroll
  for (int k = 0; k < kMlpH; ++k) {
    float a = 0.0f;
#pragma unroll
    for (int c = 0; c < kMlpC; ++c) {
      const float g = warp_sum_f(h2[k] * dz[c]);
      if (lane == 0) atomicAdd(&G[kOffW3 + k * kMlpC + c], g);
      a = fmaf(P[kOffW3 + k * kMlpC + c], dz[c], a);
    }
    dh2[k] = h2[k] > 0.0f ? a : 0.0f;
  }
  // W2, b2
#pragma unroll
  for (int k = 0; k < kMlpH; ++k) {
    const float g = warp_sum_f(dh2[k]);
    if (lane == 0) atomicAdd(&G[kOffB2 + k], g);
  }
  float dh1[kMlpH];
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    float a = 0.0f;
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) {
      const float g = warp_sum_f(h1[j] * dh2[k]);
      if (lane == 0) atomicAdd(&G[kOffW2 + j * kMlpH + k], g);
      a = fmaf(P[kOffW2 + j * kMlpH + k], dh2[k], a);
    }
    dh1[j] = h1[j] > 0.0f ? a : 0.0f;
  }
  // W1, b1
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    const float g = warp_sum_f(dh1[j]);
    if (lane == 0) atomicAdd(&G[kOffB1 + j], g);
  }
#pragma unroll
  for (int f = 0; f < kMlpF; ++f) {
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
      const float g = warp_sum_f(x[f] * dh1[j]);
      if (lane == 0) atomicAdd(&G[kOffW1 + f * kMlpH + j], g);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) atomicAdd(&grad[i], G[i]);
}

__global__ void k_mlp_adam(const float* __restrict__ g, float* __restrict__ P, float* __restrict__ m1,
                           float* __restrict__ m2, float lr_t, float b1, float b2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.0f - b1) * gi;
  const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  P[i] -= lr_t * a / (sqrtf(b) + eps);
}

__global__ void __launch_bounds__(kMlpBlock)
k_mlp_predict(int32_t n, const float* __restrict__ X, const float* __restrict__ Pg, float q,
              int32_t* __restrict__ cls) {
  __shared__ float P[kMlpParams];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) P[i] = Pg[i];
  __syncthreads();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  float x[kMlpF];
#pragma unroll
  for (int f = 0; f < kMlpF; ++f) x[f] = X[t * kMlpF + f];
  float h1[kMlpH], h2[kMlpH], z[kMlpC];
  mlp_forward(P, x, h1, h2, z);
  cls[t] = mlp_class(z, q);
}

long long gcd_ll(long long a, long long b) {
  while (b) {
    const long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace

cudaError_t launch_row_features(cudaStream_t s, const CsrView& A, const CsrView& B, int2* mm,
                                float* feat, int num_sms) {
  if (B.m > 0) {
    long long g = ((long long)B.m * kFeatTeam + 255) / 256;
    if (g > num_sms * 8) g = num_sms * 8;
    k_brow_minmax<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(B, mm);
  }
  if (A.m > 0) {
    long long g = ((long long)A.m * kFeatTeam + 255) / 256;
    if (g > num_sms * 8) g = num_sms * 8;
    k_row_features<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(A, B, mm, feat);
  }
  return cudaGetLastError();
}

}  // namespace kk

using namespace kk;

extern "C" {

kk_status kk_capacity_classes(void* stream, int32_t m, const int64_t* c_rowptr, int32_t* cls) {
  if (m < 0 || (m > 0 && (!c_rowptr || !cls))) return KK_ERR_INVALID_ARG;
  if (m == 0) return KK_OK;
  int g = (m + 255) / 256;
  if (g > 4096) g = 4096;
  k_capacity_classes<<<g, 256, 0, static_cast<cudaStream_t>(stream)>>>(m, c_rowptr, cls);
  return cudaGetLastError() == cudaSuccess ? KK_OK : KK_ERR_CUDA;
}

kk_status kk_mlp_init(void* stream, float* params, uint64_t seed) {
  if (!params) return KK_ERR_INVALID_ARG;
  k_mlp_init<<<(kMlpParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, seed);
  return cudaGetLastError() == cudaSuccess ? KK_OK : KK_ERR_CUDA;
}

kk_status kk_mlp_loss_grad(void* stream, int32_t n, const float* X, const int32_t* y,
                           const float* params, float* grad, float* loss) {
  if (n <= 0 || !X || !y || !params || !grad || !loss) return KK_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s) != cudaSuccess) return KK_ERR_CUDA;
  if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return KK_ERR_CUDA;
  k_mlp_loss_grad<<<(n + kMlpBlock - 1) / kMlpBlock, kMlpBlock, 0, s>>>(n, 0, n, 1, 0, X, y, params,
                                                                        grad, loss);
  return cudaGetLastError() == cudaSuccess ? KK_OK : KK_ERR_CUDA;
}

kk_status kk_mlp_adam(void* stream, const float* grad, float* params, float* m1, float* m2,
                      int32_t step, float lr, float beta1, float beta2, float eps) {
  if (!grad || !params || !m1 || !m2 || step < 1) return KK_ERR_INVALID_ARG;
  const float lr_t = lr * sqrtf(1.0f - powf(beta2, (float)step)) / (1.0f - powf(beta1, (float)step));
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      grad, params, m1, m2, lr_t, beta1, beta2, eps);
  return cudaGetLastError() == cudaSuccess ? KK_OK : KK_ERR_CUDA;
}

kk_status kk_mlp_train(void* stream, int32_t n, const float* X, const int32_t* y, float* params,
                       int32_t epochs, int32_t batch, float lr, uint64_t seed, float* final_loss) {
  if (n <= 0 || !X || !y || !params || epochs < 0 || batch <= 0) return KK_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* buf = nullptr;  // grad | m1 | m2 | loss
  if (cudaMalloc(&buf, sizeof(float) * (3 * kMlpParams + 4)) != cudaSuccess) return KK_ERR_OOM;
  float* grad = buf;
  float* m1 = buf + kMlpParams;
  float* m2 = buf + 2 * kMlpParams;
  float* loss = buf + 3 * kMlpParams;
  kk_status st = KK_OK;
  if (cudaMemsetAsync(buf, 0, sizeof(float) * (3 * kMlpParams + 4), s) != cudaSuccess) st = KK_ERR_CUDA;
  unsigned long long rng = seed * 0x9E3779B97F4A7C15ull + 1;
  auto next = [&rng]() {
    rng += 0x9E3779B97F4A7C15ull;
    unsigned long long z = rng;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  int step = 0;
  for (int e = 0; e < epochs && st == KK_OK; ++e) {
    // seeded order: sample (a*t + b) mod n with gcd(a, n) = 1
    long long a = (long long)(next() % (unsigned long long)n) | 1;
    while (gcd_ll(a, n) != 1) a = (a + 2) % n == 0 ? 1 : (a + 2) % n;
    const long long b = (long long)(next() % (unsigned long long)n);
    for (int start = 0; start < n && st == KK_OK; start += batch) {
      const int count = n - start < batch ? n - start : batch;
      if (cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s) != cudaSuccess) st = KK_ERR_CUDA;
      k_mlp_loss_grad<<<(count + kMlpBlock - 1) / kMlpBlock, kMlpBlock, 0, s>>>(
          n, start, count, a, b, X, y, params, grad, loss);
      ++step;
      const float lr_t = lr * sqrtf(1.0f - powf(0.999f, (float)step)) / (1.0f - powf(0.9f, (float)step));
      k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(grad, params, m1, m2, lr_t, 0.9f, 0.999f, 1e-8f);
      if (cudaGetLastError() != cudaSuccess) st = KK_ERR_CUDA;
    }
  }
  if (st == KK_OK && final_loss) {
    cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s);
    cudaMemsetAsync(loss, 0, sizeof(float), s);
    k_mlp_loss_grad<<<(n + kMlpBlock - 1) / kMlpBlock, kMlpBlock, 0, s>>>(n, 0, n, 1, 0, X, y, params,
                                                                          grad, loss);
    if (cudaMemcpyAsync(final_loss, loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = KK_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) st = KK_ERR_CUDA;
  cudaFree(buf);
  return st;
}

kk_status kk_mlp_predict(void* stream, int32_t n, const float* X, const float* params, float quantile,
                         int32_t* cls) {
  if (n < 0 || (n > 0 && (!X || !params || !cls))) return KK_ERR_INVALID_ARG;
  if (n == 0) return KK_OK;
  k_mlp_predict<<<(n + kMlpBlock - 1) / kMlpBlock, kMlpBlock, 0, static_cast<cudaStream_t>(stream)>>>(
      n, X, params, quantile, cls);
  return cudaGetLastError() == cudaSuccess ? KK_OK : KK_ERR_CUDA;
}

}  // extern "C"
