// Instrumentation: measured FMA throughput of the current GPU in FP64 or FP32, used to confirm the
// arithmetic peak that bounds the FP64 line passes (GB300: 2 FP64 FMA per clock per SM).
#include "internal.cuh"

namespace {

template <typename T>
__global__ void k_fma_chains(T* out, int iters, T a, T b) {
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = acc[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += acc[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run_probe(double* flops_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RFNSE_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RFNSE_ECUDA;
  const int blocks = sms * 8, threads = 256, iters = sizeof(T) == 8 ? 2048 : 8192, reps = 5;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = RFNSE_OK;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return RFNSE_ENOMEM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = RFNSE_ECUDA;
  if (st == RFNSE_OK) {
    rfnse::count_launch(1 + reps);
    k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e0);
    for (int r = 0; r < reps; ++r) k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = RFNSE_ECUDA;
    } else {
      *flops_per_s = 2.0 * 8.0 * iters * (double)blocks * threads * reps / (ms * 1e-3);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}

}  // namespace

extern "C" int rfnse_probe_fma(int fp64, double* flops_per_s) {
  if (!flops_per_s) return RFNSE_EINVAL;
  return fp64 ? run_probe<double>(flops_per_s) : run_probe<float>(flops_per_s);
}
