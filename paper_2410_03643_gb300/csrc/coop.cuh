// Block and grid-wide reductions and the bounded grid barrier of the cooperative kernels (the Arnoldi
// kernel of control.cu and its lock-step batch version in lockstep.cu).
#pragma once
#include "internal.cuh"

namespace rfnse {

constexpr int kCtlThreads = 256;  // threads of the cooperative kernels
constexpr unsigned long long kMaxSpin = 1ull << 21;  // bounded barrier wait (~1 s of polls), then err = 1

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

// Grid-wide synchronisation of the cooperative kernels.  A launch counts its blocks' arrivals in
// `count`, which is zero when the launch starts: arrival c (0-based) of every block has happened once
// the count reaches (c + 1) * gridDim.x.  Each block adds its arrival with one release reduction (so
// the partial it wrote before is visible to whoever observes the count) and waits with acquire loads;
// the last block of the launch clears the count after every block has passed its last wait.  The
// wait is bounded: after kMaxSpin polls the block records the failure in *err and continues.
__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_volatile(const double* p) { return *(volatile const double*)p; }

__device__ __forceinline__ double warp_sum(double v) {  // valid in lane 0; shuffle tree (fixed order)
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Warp 0 only (all 32 lanes): wait until *count >= target.  Every lane polls with its own acquire
// load, so the loads that follow in any lane are ordered after the arrivals it observed.
__device__ __forceinline__ void warp_wait_count(const unsigned* count, unsigned target, int* err) {
  unsigned long long spins = 0;
  while (__any_sync(0xffffffffu, ld_acquire(count) < target)) {
    if (++spins > kMaxSpin) {
      if ((threadIdx.x & 31) == 0) *(volatile int*)err = 1;
      break;
    }
    if (spins > 4096) __nanosleep(64);
  }
}

// Block partial of v: the warps' shuffle sums in shared memory, added in warp order by lane 0 of
// warp 0 (valid there only).  Every thread of the block must call it; it ends with warp 0 alone
// active after one block barrier.
__device__ __forceinline__ double block_partial_w0(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double b = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) b += sh[q];
  return b;
}

// Warp 0: the sum of part[0 .. n) in a fixed order (lane l adds l, l + 32, ...; then the shuffle
// tree), valid in lane 0.  Volatile loads: the slots are rewritten between launches and sweeps.
__device__ __forceinline__ double warp_sum_partials(const double* part, int n) {
  double t = 0.0;
  for (int q = threadIdx.x & 31; q < n; q += 32) t += ld_volatile(part + q);
  return warp_sum(t);
}

// Grid-wide sum of v (one value per thread), the same in every block: block partials (slot
// blockIdx.x of part), arrival c of the launch (target (c + 1) * gridDim.x), fixed-order sum of the
// gridDim.x partials.  Two block barriers; the result is returned to every thread.
__device__ __forceinline__ double grid_sum(double v, double* part, unsigned* count, unsigned target, int* err,
                                           double* sh) {
  const double b = block_partial_w0(v, sh);
  if (threadIdx.x < 32) {
    double s = b;
    if (gridDim.x > 1) {
      if (threadIdx.x == 0) {
        part[blockIdx.x] = b;
        red_add_release(count, 1u);
      }
      warp_wait_count(count, target, err);
      s = warp_sum_partials(part, (int)gridDim.x);
    }
    if (threadIdx.x == 0) sh[32] = s;
  }
  __syncthreads();
  return sh[32];
}

// The grid's last sum of a launch: every block leaves its partial and counts itself in *done; the
// last block to arrive sums the partials in a fixed order (returns true, *out valid in all its
// threads) while the others return false and may leave.  The last block clears *done and *count.
__device__ __forceinline__ bool grid_sum_last(double v, double* part, unsigned* done, unsigned* count, double* sh,
                                              double* out) {
  __shared__ int s_last;
  const double b = block_partial_w0(v, sh);
  if (threadIdx.x < 32) {
    double s = b;
    int last = 1;
    if (gridDim.x > 1) {
      if (threadIdx.x == 0) {
        part[blockIdx.x] = b;
        last = atom_add_acq_rel(done, 1u) == gridDim.x - 1u;
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last) s = warp_sum_partials(part, (int)gridDim.x);
    }
    if (threadIdx.x == 0) {
      sh[32] = s;
      s_last = last;
      if (last) {  // every other block has passed its last wait: clear the counters for the next launch
        *done = 0u;
        *count = 0u;
      }
    }
  }
  __syncthreads();
  *out = sh[32];
  return s_last != 0;
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

// The end of Arnoldi step j, run by warp 0 of one block: h_{j+1,j} = sqrt(nrm2), the previous rotations
// on column j (hc: h_0j .. h_jj as computed by the sweeps, in shared memory), the new rotation, g, the
// convergence test and the state for the next column; returns (in lane 0) whether the cycle goes on to
// column j + 1.  The lanes first load the previous rotations and the scalars of the test together (one round trip to
// memory instead of one per dependent read); lane 0 does the arithmetic.
__device__ __forceinline__ int givens_finish_warp(GmresState* gs, int j, double nrm2, const double* hc, double2* w,
                                                  const SolveCfg& cfg) {
  __shared__ double rc[kMaxM], rs[kMaxM];
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < j; i += 32) {
    rc[i] = gs->cs[i];
    rs[i] = gs->sn[i];
  }
  double gj = 0.0, ref = 0.0, tol = 0.0;
  int it = 0, err = 0;
  if (lane == 0) {
    gj = gs->g[j];
    ref = gs->ref;
    tol = gs->tol;
    it = gs->it;
    err = *(volatile int*)&gs->err;
  }
  __syncwarp();
  if (lane != 0) return 0;
  double* Hc = gs->H + (size_t)j * (kMaxM + 1);
  const double hnext = sqrt(nrm2);
  double hi = hc[0];  // entry i of the column as the rotations reach it
  for (int i = 0; i < j; ++i) {  // previous rotations
    const double hi1 = hc[i + 1];
    Hc[i] = rc[i] * hi + rs[i] * hi1;
    hi = -rs[i] * hi + rc[i] * hi1;
  }
  const double rr = hypot(hi, hnext);
  const double c = hi / rr, sn = hnext / rr;
  gs->cs[j] = c;
  gs->sn[j] = sn;
  Hc[j] = rr;
  Hc[j + 1] = 0.0;
  const double gn = -sn * gj;
  gs->g[j + 1] = gn;
  gs->g[j] = c * gj;
  const double rel = fabs(gn) / ref;
  gs->relres = rel;
  const double inv_h = (hnext > 0.0) ? 1.0 / hnext : 0.0;
  gs->inv_h = inv_h;
  int done = 0;
  if (!isfinite(rel) || !isfinite(hnext)) done = 3;
  else if (rel < tol) done = 1;
  else if (hnext == 0.0) done = 2;
  gs->done = done;
  gs->it = it + 1;
  gs->j = j + 1;
  gs->src = w;
  gs->src_scale = inv_h;
  const int stop = done != 0 || it + 1 >= cfg.max_it || err;
  gs->no_restart = stop;
  return (!stop && j + 1 < cfg.m) ? 1 : 0;
}

}  // namespace rfnse
