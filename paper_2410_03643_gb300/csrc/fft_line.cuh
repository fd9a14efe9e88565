// In-shared-memory complex FFT of B lines of length L = 2^m (3 <= m <= 12), Stockham auto-sort
// formulation (Govindaraju et al., SC'08): radix-4 stages, plus one radix-2 stage when m is odd.
// nt threads work on one line; each handles nq = L/(4 nt) radix-4 butterflies per stage (1 or 2).
// A stage reads its butterfly inputs into registers, synchronises, writes its outputs, synchronises,
// so one buffer per line suffices.
//
// Shared-memory index of element i of a line: pad(i) = i + i/16 (one spare slot every 16 elements),
// which spreads the power-of-two strides of the Stockham write pattern over the banks.  Lines are
// line_stride() elements apart (odd, so lines adjacent in a tile fall on different banks).
//
// Forward transform: X_k = sum_j x_j exp(-2 pi i jk/L).  Inverse: conjugate twiddles, no 1/L.
// The twiddle table tw[k] = exp(-2 pi i k/L), k < L, is staged in shared memory by the caller.
#pragma once
#include "cplx.cuh"

namespace rfnse {

__host__ __device__ __forceinline__ int fft_pad(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int fft_line_stride(int L) { return L + (L >> 4) + 1; }

template <typename V>
__device__ __forceinline__ V tw_at(const V* tw, int idx, bool inv) {
  V w = tw[idx];
  if (inv) w.y = -w.y;
  return w;
}

// 4-point DFT in place (forward: W_4 = -i).
template <typename V>
__device__ __forceinline__ void dft4(V& a0, V& a1, V& a2, V& a3, bool inv) {
  V t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = csub(a1, a3);
  t3 = inv ? cmul_i(t3) : cmul_mi(t3);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

// One radix-4 Stockham stage on line x: L/4 butterflies, nq (<= 2) per thread.
template <typename V>
__device__ __forceinline__ void radix4_stage(V* x, int L, int Ns, const V* tw, int lt, int nt, int nq, bool inv) {
  const int nb = L >> 2;
  V v[2][4];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (q < nq) {
      const int j = lt + q * nt;
#pragma unroll
      for (int r = 0; r < 4; ++r) v[q][r] = x[fft_pad(j + r * nb)];
      const int k = j & (Ns - 1);
      if (Ns > 1) {
        const int step = (L / (Ns * 4)) * k;
#pragma unroll
        for (int r = 1; r < 4; ++r) v[q][r] = cmul(v[q][r], tw_at(tw, r * step, inv));
      }
      dft4(v[q][0], v[q][1], v[q][2], v[q][3], inv);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (q < nq) {
      const int j = lt + q * nt;
      const int k = j & (Ns - 1);
      const int base = ((j - k) << 2) + k;
#pragma unroll
      for (int r = 0; r < 4; ++r) x[fft_pad(base + r * Ns)] = v[q][r];
    }
  }
  __syncthreads();
}

// One radix-2 Stockham stage: L/2 butterflies, 2 nq per thread.
template <typename V>
__device__ __forceinline__ void radix2_stage(V* x, int L, int Ns, const V* tw, int lt, int nt, int nq, bool inv) {
  const int nb = L >> 1;
  V v[4][2];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < 2 * nq) {
      const int j = lt + q * nt;
      v[q][0] = x[fft_pad(j)];
      v[q][1] = x[fft_pad(j + nb)];
      const int k = j & (Ns - 1);
      if (Ns > 1) v[q][1] = cmul(v[q][1], tw_at(tw, (L / (Ns * 2)) * k, inv));
      const V a = cadd(v[q][0], v[q][1]);
      const V b = csub(v[q][0], v[q][1]);
      v[q][0] = a;
      v[q][1] = b;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < 2 * nq) {
      const int j = lt + q * nt;
      const int k = j & (Ns - 1);
      const int base = ((j - k) << 1) + k;
      x[fft_pad(base)] = v[q][0];
      x[fft_pad(base + Ns)] = v[q][1];
    }
  }
  __syncthreads();
}

// FFT of every line of the tile.  All threads of the block call this (it synchronises).
// Thread t works on line t / nt.
template <typename V>
__device__ __forceinline__ void fft_lines(V* buf, int Lp, int L, int log2L, int nt, const V* tw, bool inv) {
  const int line = threadIdx.x / nt;
  const int lt = threadIdx.x - line * nt;
  const int nq = (L >> 2) / nt;
  V* x = buf + (size_t)line * Lp;
  int Ns = 1;
  if (log2L & 1) {
    radix2_stage(x, L, Ns, tw, lt, nt, nq, inv);
    Ns = 2;
  }
  for (; Ns < L; Ns <<= 2) radix4_stage(x, L, Ns, tw, lt, nt, nq, inv);
}

}  // namespace rfnse
