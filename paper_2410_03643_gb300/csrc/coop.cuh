// Block and grid-wide reductions and the bounded grid barrier of the cooperative kernels (the Arnoldi
// kernel of control.cu and its lock-step batch version in lockstep.cu).
#pragma once
#include "internal.cuh"

namespace rfnse {

constexpr int kCtlThreads = 256;  // threads of the cooperative kernels
constexpr unsigned long long kMaxSpin = 1ull << 22;  // bounded barrier wait (~0.3 s), then err = 1

// Sum over the block (valid in thread 0); every thread of the block must call it.
__device__ __forceinline__ double block_sum_c(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;  // valid in thread 0
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The wait is bounded: after
// kMaxSpin polls the block records the failure in *err and continues.
__device__ __forceinline__ void grid_barrier_global(GridBarrier* b, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&b->count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      unsigned long long spins = 0;
      while (*vgen == g) {
        if (++spins > kMaxSpin) {
          *(volatile int*)err = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// A one-block grid needs only the block barrier (uniform branch); larger grids use the global protocol.
__device__ __forceinline__ void grid_barrier(GridBarrier* b, int* err) {
  if (gridDim.x == 1) {
    __syncthreads();
    return;
  }
  grid_barrier_global(b, err);
}

// The same value in every block: the partials summed in a fixed order.
__device__ __forceinline__ double fixed_sum(const double* part, int n, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += ((volatile const double*)part)[i];
  v = block_sum_c(v, sh);
  __shared__ double bc;
  if (threadIdx.x == 0) bc = v;
  __syncthreads();
  return bc;
}

// One modified Gram-Schmidt sweep over the elements k = start, start + stride, ... < N of this thread:
// w -= hprev vp (when vp is given; w written back), then acc += <a, w> with a = vi, or a = w itself
// when vi is null (the norm).  The real inner product of the complex storage, as FMA chains (GB300 issues
// two FP64 FMAs per SM and cycle).  Four elements are loaded before any is used, so each thread keeps
// four independent loads of every operand in flight; the products are accumulated in element order,
// the same order as one element at a time.
__device__ __forceinline__ double mgs_sweep(double2* __restrict__ w, const double2* __restrict__ vi,
                                            const double2* __restrict__ vp, double hprev, long long N,
                                            long long start, long long stride) {
  double acc = 0.0;
  long long k = start;
  for (; k + 3 * stride < N; k += 4 * stride) {
    double2 wv[4], pv[4], av[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) wv[u] = w[k + u * stride];
    if (vp) {
#pragma unroll
      for (int u = 0; u < 4; ++u) pv[u] = vp[k + u * stride];
    }
    if (vi) {
#pragma unroll
      for (int u = 0; u < 4; ++u) av[u] = vi[k + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (vp) {
        wv[u].x = fma(-hprev, pv[u].x, wv[u].x);
        wv[u].y = fma(-hprev, pv[u].y, wv[u].y);
        w[k + u * stride] = wv[u];
      }
      const double2 a = vi ? av[u] : wv[u];
      acc = fma(a.x, wv[u].x, acc);
      acc = fma(a.y, wv[u].y, acc);
    }
  }
  for (; k < N; k += stride) {
    double2 wv = w[k];
    if (vp) {
      const double2 pv = vp[k];
      wv.x = fma(-hprev, pv.x, wv.x);
      wv.y = fma(-hprev, pv.y, wv.y);
      w[k] = wv;
    }
    const double2 a = vi ? vi[k] : wv;
    acc = fma(a.x, wv.x, acc);
    acc = fma(a.y, wv.y, acc);
  }
  return acc;
}

}  // namespace rfnse
