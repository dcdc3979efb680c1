// Arithmetic-throughput probe: the FP64 (DFMA) and FP32 (FFMA) peaks that the
// solver's rooflines are measured against.  Each thread runs 8 independent
// fused multiply-add chains in registers; one store per thread keeps them live.
#include <algorithm>

#include "ssv_internal.cuh"

namespace ssv {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chain_kernel(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x * 1e-9) + (T)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(int iters, cudaStream_t st, double* tflops) {
  const int blocks = num_sms() * 8, threads = 256;
  T* buf = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&buf, sizeof(T) * blocks * threads, st));
  cudaEvent_t e0, e1;
  SSV_CUDA_TRY(cudaEventCreate(&e0));
  SSV_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    fma_chain_kernel<T><<<blocks, threads, 0, st>>>(buf, iters, (T)0.999999, (T)1e-7);
    count_launch();
    cudaEventRecord(e1, st);
    SSV_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SSV_CUDA_TRY(cudaFreeAsync(buf, st));
  SSV_CUDA_TRY(cudaStreamSynchronize(st));
  const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return SSV_OK;
}

}  // namespace

int peak_probe(int kind, cudaStream_t st, double* tflops) {
  if (kind == 0) return run<double>(2000, st, tflops);
  if (kind == 1) return run<float>(40000, st, tflops);
  return SSV_EINVAL;
}

}  // namespace ssv
