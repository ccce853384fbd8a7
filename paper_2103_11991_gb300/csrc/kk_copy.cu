// Result download helper (include/kk_copy.h): a streaming copy kernel from
// device memory into page-locked host memory, written through the host
// buffer's device mapping.
#include <cstdint>

#include <cuda_runtime.h>

#include "kk_copy.h"

namespace {

__global__ void __launch_bounds__(512) k_copy_to_host(const int4* __restrict__ src, int4* __restrict__ dst,
                                                      long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

}  // namespace

extern "C" kk_status kk_copy_to_host(void* cuda_stream, void* dst_host, const void* src_device,
                                     size_t bytes) {
  if (bytes == 0) return KK_OK;
  if (!dst_host || !src_device) return KK_ERR_INVALID_ARG;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, dst_host) != cudaSuccess) {
    (void)cudaGetLastError();
    return KK_ERR_INVALID_ARG;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return KK_ERR_INVALID_ARG;
  cudaPointerAttributes as{};
  if (cudaPointerGetAttributes(&as, src_device) != cudaSuccess) {
    (void)cudaGetLastError();
    return KK_ERR_INVALID_ARG;
  }
  if (as.type != cudaMemoryTypeDevice) return KK_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const uintptr_t d = reinterpret_cast<uintptr_t>(at.devicePointer);
  const uintptr_t sp = reinterpret_cast<uintptr_t>(src_device);
  if ((d & 15u) || (sp & 15u) || (bytes & 15u)) {
    return cudaMemcpyAsync(dst_host, src_device, bytes, cudaMemcpyDeviceToHost, s) == cudaSuccess
               ? KK_OK
               : KK_ERR_CUDA;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return KK_ERR_CUDA;
  const long long n = (long long)(bytes / 16);
  long long grid = (n + 511) / 512;
  if (grid > sms) grid = sms;  // one CTA per SM saturates the host link
  k_copy_to_host<<<(int)grid, 512, 0, s>>>(static_cast<const int4*>(src_device),
                                           static_cast<int4*>(at.devicePointer), n);
  return cudaGetLastError() == cudaSuccess ? KK_OK : KK_ERR_CUDA;
}
