// Pipe rates of one GPU for bench.py's count of the method's work: DFMA
// (and FFMA for comparison), double sqrt, reciprocal and exp, each as
// several independent chains per thread over 8 blocks of 256 threads per SM,
// timed with CUDA events. DFMA rate / function rate gives the
// DFMA-equivalent cost of each special function (bench.py FP64_COST).
// Not part of the library.
//
// Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o bench_pipe_rates bench_pipe_rates.cu && ./bench_pipe_rates
#include <cuda_runtime.h>

#include <cstdio>

#define CK(x)                                                                   \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      printf("CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__);  \
      return 1;                                                                 \
    }                                                                           \
  } while (0)

template <typename T>
__global__ void fma_k(T* out, int iters, T s)
{
  T a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
    a7 = a0 + 7;
  const T m = (T)0.9999;
  for (int i = 0; i < iters; i++) {
    a0 = a0 * m + s; a1 = a1 * m + s; a2 = a2 * m + s; a3 = a3 * m + s;
    a4 = a4 * m + s; a5 = a5 * m + s; a6 = a6 * m + s; a7 = a7 * m + s;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

__global__ void sqrt_k(double* out, int iters)
{
  double a0 = 1 + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  for (int i = 0; i < iters; i++) {
    a0 = sqrt(a0) + 1.5; a1 = sqrt(a1) + 1.5; a2 = sqrt(a2) + 1.5; a3 = sqrt(a3) + 1.5;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3;
}

__global__ void rcp_k(double* out, int iters)
{
  double a0 = 1 + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  for (int i = 0; i < iters; i++) {
    a0 = 1.0 / a0 + 1.5; a1 = 1.0 / a1 + 1.5; a2 = 1.0 / a2 + 1.5; a3 = 1.0 / a3 + 1.5;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3;
}

__global__ void exp_k(double* out, int iters)
{
  double a0 = -1e-3 * threadIdx.x, a1 = a0 - 0.1, a2 = a0 - 0.2, a3 = a0 - 0.3;
  for (int i = 0; i < iters; i++) {
    a0 = -exp(a0); a1 = -exp(a1); a2 = -exp(a2); a3 = -exp(a3);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3;
}

__global__ void expf_k(float* out, int iters)
{
  float a0 = -1e-3f * threadIdx.x, a1 = a0 - 0.1f, a2 = a0 - 0.2f, a3 = a0 - 0.3f;
  for (int i = 0; i < iters; i++) {
    a0 = -__expf(a0); a1 = -__expf(a1); a2 = -__expf(a2); a3 = -__expf(a3);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3;
}

int main()
{
  int dev;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, dev));
  printf("%s SMs=%d cc=%d.%d\n", p.name, p.multiProcessorCount, p.major, p.minor);
  const int blocks = p.multiProcessorCount * 8, threads = 256;
  const size_t n = (size_t)blocks * threads;
  double* d;
  float* f;
  CK(cudaMalloc(&d, n * sizeof(double)));
  CK(cudaMalloc(&f, n * sizeof(float)));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float ms;
  for (int rep = 0; rep < 2; rep++) {  // the first pass warms up
    int it = 1 << 14;
    CK(cudaEventRecord(e0));
    fma_k<double><<<blocks, threads>>>(d, it, 1e-7);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("DFMA: %.3f TFLOP/s\n", 2.0 * 8 * it * n / (ms * 1e-3) / 1e12);
    it = 1 << 16;
    CK(cudaEventRecord(e0));
    fma_k<float><<<blocks, threads>>>(f, it, 1e-7f);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("FFMA: %.3f TFLOP/s\n", 2.0 * 8 * it * n / (ms * 1e-3) / 1e12);
    it = 1 << 12;
    CK(cudaEventRecord(e0));
    sqrt_k<<<blocks, threads>>>(d, it);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("double sqrt: %.3f G/s\n", 4.0 * it * n / (ms * 1e-3) / 1e9);
    CK(cudaEventRecord(e0));
    rcp_k<<<blocks, threads>>>(d, it);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("double 1/x: %.3f G/s\n", 4.0 * it * n / (ms * 1e-3) / 1e9);
    CK(cudaEventRecord(e0));
    exp_k<<<blocks, threads>>>(d, it);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("double exp: %.3f G/s\n", 4.0 * it * n / (ms * 1e-3) / 1e9);
    it = 1 << 15;
    CK(cudaEventRecord(e0));
    expf_k<<<blocks, threads>>>(f, it);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("__expf: %.3f G/s\n", 4.0 * it * n / (ms * 1e-3) / 1e9);
  }
  CK(cudaFree(d));
  CK(cudaFree(f));
  return 0;
}
