// Throughput probe: FP64 / FP32 FMA, integer multiply-add, shared-memory
// atomics.  Every access stays in bounds and no kernel waits on another.
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s %s\n",#x,cudaGetErrorString(e)); return 1;}}while(0)
constexpr int ITERS = 4096;
__global__ void k_dfma(double* out, double s) {
  double a0=threadIdx.x, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  for (int i=0;i<ITERS;i++){ a0=fma(a0,s,0.5); a1=fma(a1,s,0.5); a2=fma(a2,s,0.5); a3=fma(a3,s,0.5);
    a4=fma(a4,s,0.5); a5=fma(a5,s,0.5); a6=fma(a6,s,0.5); a7=fma(a7,s,0.5);}
  out[blockIdx.x*blockDim.x+threadIdx.x]=a0+a1+a2+a3+a4+a5+a6+a7;
}
__global__ void k_dadd(double* out, double s) {
  double a0=threadIdx.x, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  for (int i=0;i<ITERS;i++){ a0+=s; a1+=s; a2+=s; a3+=s; a4+=s; a5+=s; a6+=s; a7+=s;}
  out[blockIdx.x*blockDim.x+threadIdx.x]=a0+a1+a2+a3+a4+a5+a6+a7;
}
__global__ void k_ffma(float* out, float s) {
  float a0=threadIdx.x, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  for (int i=0;i<ITERS;i++){ a0=fmaf(a0,s,0.5f); a1=fmaf(a1,s,0.5f); a2=fmaf(a2,s,0.5f); a3=fmaf(a3,s,0.5f);
    a4=fmaf(a4,s,0.5f); a5=fmaf(a5,s,0.5f); a6=fmaf(a6,s,0.5f); a7=fmaf(a7,s,0.5f);}
  out[blockIdx.x*blockDim.x+threadIdx.x]=a0+a1+a2+a3+a4+a5+a6+a7;
}
__global__ void k_imad(unsigned* out, unsigned s) {
  unsigned a0=threadIdx.x, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  for (int i=0;i<ITERS;i++){ a0=a0*s+7u; a1=a1*s+7u; a2=a2*s+7u; a3=a3*s+7u; a4=a4*s+7u; a5=a5*s+7u; a6=a6*s+7u; a7=a7*s+7u;}
  out[blockIdx.x*blockDim.x+threadIdx.x]=a0^a1^a2^a3^a4^a5^a6^a7;
}
// shared memory: plain ld/add/st of double vs atomicAdd(double) vs atomicCAS(int); distinct slots per lane
__global__ void k_smem_plain(double* out, double s) {
  __shared__ double t[1024];
  for (int i=threadIdx.x;i<1024;i+=blockDim.x) t[i]=0;
  __syncthreads();
  unsigned idx = threadIdx.x;
  for (int i=0;i<ITERS/8;i++){ idx = (idx*97u + 13u) & 1023u; t[idx] += s; }
  __syncthreads();
  out[blockIdx.x*blockDim.x+threadIdx.x]=t[threadIdx.x & 1023];
}
__global__ void k_smem_atomic(double* out, double s) {
  __shared__ double t[1024];
  for (int i=threadIdx.x;i<1024;i+=blockDim.x) t[i]=0;
  __syncthreads();
  unsigned idx = threadIdx.x;
  for (int i=0;i<ITERS/8;i++){ idx = (idx*97u + 13u) & 1023u; atomicAdd(&t[idx], s); }
  __syncthreads();
  out[blockIdx.x*blockDim.x+threadIdx.x]=t[threadIdx.x & 1023];
}
__global__ void k_smem_cas(unsigned* out, unsigned s) {
  __shared__ unsigned t[1024];
  for (int i=threadIdx.x;i<1024;i+=blockDim.x) t[i]=0;
  __syncthreads();
  unsigned idx = threadIdx.x, acc=0;
  for (int i=0;i<ITERS/8;i++){ idx = (idx*97u + 13u) & 1023u; acc += atomicCAS(&t[idx], 0u, s+i); }
  __syncthreads();
  out[blockIdx.x*blockDim.x+threadIdx.x]=acc + t[threadIdx.x & 1023];
}
__global__ void k_smem_or(unsigned* out, unsigned s) {
  __shared__ unsigned t[1024];
  for (int i=threadIdx.x;i<1024;i+=blockDim.x) t[i]=0;
  __syncthreads();
  unsigned idx = threadIdx.x;
  for (int i=0;i<ITERS/8;i++){ idx = (idx*97u + 13u) & 1023u; atomicOr(&t[idx], 1u<<(i&31)); }
  __syncthreads();
  out[blockIdx.x*blockDim.x+threadIdx.x]=t[threadIdx.x & 1023];
}
template<class F> float timeit(F f, int reps){ cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b);
  f(); cudaDeviceSynchronize(); cudaEventRecord(a); for(int r=0;r<reps;r++) f(); cudaEventRecord(b); cudaEventSynchronize(b);
  float ms; cudaEventElapsedTime(&ms,a,b); return ms/reps; }
int main(){
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0));
  printf("name=%s sms=%d cc=%d.%d smem_optin=%zu l2=%d regsPerSM=%d maxThrSM=%d\n", p.name, p.multiProcessorCount, p.major, p.minor,
    p.sharedMemPerBlockOptin, p.l2CacheSize, p.regsPerMultiprocessor, p.maxThreadsPerMultiProcessor);
  int clk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0); printf("clockKHz=%d\n", clk);
  const int blocks = p.multiProcessorCount*8, threads=256; const size_t n=(size_t)blocks*threads;
  double* d; float* f; unsigned* u; CK(cudaMalloc(&d,n*8)); CK(cudaMalloc(&f,n*4)); CK(cudaMalloc(&u,n*4));
  double lanes = (double)n;
  float ms;
  ms = timeit([&]{k_dfma<<<blocks,threads>>>(d,0.999);}, 5); printf("DFMA  %.3f ms  %.3f TFLOP/s (2 flop/fma)\n", ms, lanes*ITERS*8*2/ms/1e9);
  ms = timeit([&]{k_dadd<<<blocks,threads>>>(d,0.5);}, 5); printf("DADD  %.3f ms  %.3f Tops/s\n", ms, lanes*ITERS*8/ms/1e9);
  ms = timeit([&]{k_ffma<<<blocks,threads>>>(f,0.999f);}, 5); printf("FFMA  %.3f ms  %.3f TFLOP/s\n", ms, lanes*ITERS*8*2/ms/1e9);
  ms = timeit([&]{k_imad<<<blocks,threads>>>(u,3u);}, 5); printf("IMAD  %.3f ms  %.3f Tops/s\n", ms, lanes*ITERS*8/ms/1e9);
  ms = timeit([&]{k_smem_plain<<<blocks,threads>>>(d,1.0);}, 5); printf("SMEM ld+dadd+st %.3f ms %.3f Gops/s\n", ms, lanes*(ITERS/8)/ms/1e6);
  ms = timeit([&]{k_smem_atomic<<<blocks,threads>>>(d,1.0);}, 5); printf("SMEM atomicAdd(f64) %.3f ms %.3f Gops/s\n", ms, lanes*(ITERS/8)/ms/1e6);
  ms = timeit([&]{k_smem_cas<<<blocks,threads>>>(u,1u);}, 5); printf("SMEM atomicCAS(u32) %.3f ms %.3f Gops/s\n", ms, lanes*(ITERS/8)/ms/1e6);
  ms = timeit([&]{k_smem_or<<<blocks,threads>>>(u,1u);}, 5); printf("SMEM atomicOr(u32) %.3f ms %.3f Gops/s\n", ms, lanes*(ITERS/8)/ms/1e6);
  CK(cudaDeviceSynchronize());
  printf("done\n"); return 0;
}
