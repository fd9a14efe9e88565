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

// ---- the cooperative Arnoldi kernel alone ------------------------------------------------------

namespace {

__global__ void k_probe_fill(double2* v, long long n, long long ldv, int count) {
  for (int c = 0; c < count; ++c)
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      v[(size_t)c * ldv + i] = make_double2(sin(0.01 * (c + 1) * (double)(i % 9973) + 0.3),
                                            cos(0.0037 * (c + 1) * (double)(i % 7919)));
}

__global__ void k_probe_reset(rfnse::GmresState* gs, int j) {
  gs->j = j;
  gs->it = 0;
  gs->err = 0;
  gs->ref = 1.0;
  gs->tol = 0.0;
  gs->g[j] = 1.0;
}

}  // namespace

extern "C" int rfnse_probe_arnoldi(long long n, int j, int reps, double* us_per_step, int* blocks_out) {
  if (!us_per_step || n < 1 || n > (1LL << 28) || j < 0 || j > 62 || reps < 1 || reps > 1000) return RFNSE_EINVAL;
  using namespace rfnse;
  const int blocks = coop_blocks_for(n);
  GmresState* gs = nullptr;
  double2 *V = nullptr, *w = nullptr;
  double* partials = nullptr;
  GridBarrier* bar = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = nullptr;
  int st = RFNSE_OK;
  auto chk = [&](cudaError_t e, int code) {
    if (st == RFNSE_OK && e != cudaSuccess) st = code;
  };
  chk(cudaMalloc(&gs, sizeof(GmresState)), RFNSE_ENOMEM);
  chk(cudaMalloc(&V, sizeof(double2) * (size_t)(j + 1) * n), RFNSE_ENOMEM);
  chk(cudaMalloc(&w, sizeof(double2) * (size_t)n), RFNSE_ENOMEM);
  chk(cudaMalloc(&partials, sizeof(double) * 2 * (size_t)blocks), RFNSE_ENOMEM);
  chk(cudaMalloc(&bar, sizeof(GridBarrier)), RFNSE_ENOMEM);
  chk(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), RFNSE_ECUDA);
  chk(cudaEventCreate(&e0), RFNSE_ECUDA);
  chk(cudaEventCreate(&e1), RFNSE_ECUDA);
  if (st == RFNSE_OK) {
    chk(cudaMemsetAsync(gs, 0, sizeof(GmresState), s), RFNSE_ECUDA);
    chk(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s), RFNSE_ECUDA);
    count_launch(2);
    k_probe_fill<<<1024, 256, 0, s>>>(V, n, n, j + 1);
    k_probe_fill<<<1024, 256, 0, s>>>(w, n, n, 1);
    SolveCfg cfg{};
    cfg.m = kMaxM;
    cfg.max_it = 1 << 30;
    cfg.max_outer = 1;
    cfg.tol = 0.0;
    double total_ms = 0.0;
    for (int r = 0; r < reps + 2 && st == RFNSE_OK; ++r) {  // two untimed warm-up launches
      count_launch();
      k_probe_reset<<<1, 1, 0, s>>>(gs, j);
      chk(cudaEventRecord(e0, s), RFNSE_ECUDA);
      chk(launch_mgs_step(gs, V, n, w, n, partials, bar, cfg, 0, 0, blocks, s), RFNSE_ECUDA);
      chk(cudaEventRecord(e1, s), RFNSE_ECUDA);
      chk(cudaEventSynchronize(e1), RFNSE_ECUDA);
      float ms = 0.f;
      chk(cudaEventElapsedTime(&ms, e0, e1), RFNSE_ECUDA);
      if (r >= 2) total_ms += ms;
    }
    int err = 0;
    chk(cudaMemcpy(&err, &gs->err, sizeof(int), cudaMemcpyDeviceToHost), RFNSE_ECUDA);
    if (st == RFNSE_OK && err) st = RFNSE_ETIMEOUT;
    if (st == RFNSE_OK) {
      *us_per_step = 1e3 * total_ms / reps;
      if (blocks_out) *blocks_out = blocks;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(gs);
  cudaFree(V);
  cudaFree(w);
  cudaFree(partials);
  cudaFree(bar);
  if (st == RFNSE_ECUDA) cudaGetLastError();
  return st;
}
