// In-shared-memory complex FFT of B lines of length L = 2^m (3 <= m <= 12), Stockham auto-sort
// formulation (Govindaraju et al., SC'08): one radix-2 stage first when m is odd, then radix-4
// stages.  nt threads work on one line; each handles nq = L/(4 nt) radix-4 butterflies per stage (1 or
// 2).  A stage reads its butterfly inputs into registers, synchronises, writes its outputs,
// synchronises, so one buffer per line suffices.
//
// Shared-memory index of element i of a line: pad(i) = i + i/16 (one spare slot every 16 elements),
// which spreads the power-of-two strides of the Stockham write pattern over the banks.  Lines are
// line_stride() elements apart (odd, so lines adjacent in a tile fall on different banks).
//
// Forward transform: X_k = sum_j x_j exp(-2 pi i jk/L).  Inverse: conjugate twiddles, no 1/L.
//
// Twiddles are stored stage by stage so that the threads of a warp read consecutive entries: the
// radix-4 stage with sub-transform length Ns (> 1) uses W_{4Ns}^{r k}, r = 1..3, k = 0..Ns-1, stored
// at seg[(r-1) Ns + k]; the segments follow each other in stage order (see twiddle_table_index).
//
// Options for the circulant-embedding products, whose input is zero in its upper half and whose
// output is needed only in its lower half: `zero_upper` skips the loads of the zero half in the
// first stage; `half_out` computes and stores only the lower-half outputs of the last stage.
#pragma once
#include "cplx.cuh"

namespace rfnse {

__host__ __device__ __forceinline__ int fft_pad(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int fft_line_stride(int L) { return L + (L >> 4) + 1; }

// Position of twiddle W_{4Ns}^{r k} (1 <= r <= 3, 0 <= k < Ns) in the per-stage table of a length-L
// transform (stage order as executed: radix-2 first for odd log2 L, then Ns = Ns0, 4 Ns0, ...).
__host__ __device__ __forceinline__ int twiddle_table_index(int log2L, int Ns, int r, int k) {
  // segments exist for radix-4 stages with Ns > 1; their sizes 3 Ns sum over earlier stages
  int off = 0;
  for (int s = (log2L & 1) ? 2 : 4; s < Ns; s <<= 2) off += 3 * s;
  return off + (r - 1) * Ns + k;
}

template <typename V>
__device__ __forceinline__ V tw_conj(V w, bool inv) {
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
//   first_zero_upper: inputs r = 2, 3 (indices >= L/2) are known to be zero (first stage only)
//   last_half_out:    only outputs r = 0, 1 (indices < L/2) are needed (last stage only)
template <typename V>
__device__ __forceinline__ void radix4_stage(V* x, int L, int Ns, const V* seg, int lt, int nt, int nq, bool inv,
                                             bool first_zero_upper, bool last_half_out) {
  const int nb = L >> 2;
  V v[2][4];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (q < nq) {
      const int j = lt + q * nt;
      const int k = j & (Ns - 1);
      if (first_zero_upper) {  // Ns == 1: no twiddles; a2 = a3 = 0
        const V a0 = x[fft_pad(j)], a1 = x[fft_pad(j + nb)];
        const V b1 = inv ? cmul_i(a1) : cmul_mi(a1);
        v[q][0] = cadd(a0, a1);
        v[q][2] = csub(a0, a1);
        v[q][1] = cadd(a0, b1);
        v[q][3] = csub(a0, b1);
        continue;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) v[q][r] = x[fft_pad(j + r * nb)];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < 4; ++r) v[q][r] = cmul(v[q][r], tw_conj(seg[(r - 1) * Ns + k], inv));
      }
      if (last_half_out) {     // outputs 0 and 1 of the 4-point DFT
        const V t0 = cadd(v[q][0], v[q][2]), t1 = csub(v[q][0], v[q][2]);
        const V t2 = cadd(v[q][1], v[q][3]);
        V t3 = csub(v[q][1], v[q][3]);
        t3 = inv ? cmul_i(t3) : cmul_mi(t3);
        v[q][0] = cadd(t0, t2);
        v[q][1] = cadd(t1, t3);
      } else {
        dft4(v[q][0], v[q][1], v[q][2], v[q][3], inv);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (q < nq) {
      const int j = lt + q * nt;
      const int k = j & (Ns - 1);
      const int base = ((j - k) << 2) + k;
      x[fft_pad(base)] = v[q][0];
      x[fft_pad(base + Ns)] = v[q][1];
      if (!last_half_out) {
        x[fft_pad(base + 2 * Ns)] = v[q][2];
        x[fft_pad(base + 3 * Ns)] = v[q][3];
      }
    }
  }
  __syncthreads();
}

// The radix-2 first stage (Ns = 1, no twiddles): L/2 butterflies, 2 nq per thread.
template <typename V>
__device__ __forceinline__ void radix2_first_stage(V* x, int L, int lt, int nt, int nq, bool zero_upper) {
  const int nb = L >> 1;
  V v[4][2];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < 2 * nq) {
      const int j = lt + q * nt;
      const V a = x[fft_pad(j)];
      if (zero_upper) {
        v[q][0] = a;
        v[q][1] = a;
      } else {
        const V b = x[fft_pad(j + nb)];
        v[q][0] = cadd(a, b);
        v[q][1] = csub(a, b);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < 2 * nq) {
      const int j = lt + q * nt;
      x[fft_pad(2 * j)] = v[q][0];
      x[fft_pad(2 * j + 1)] = v[q][1];
    }
  }
  __syncthreads();
}

// FFT of every line of the tile.  All threads of the block call this (it synchronises).
// Thread t works on line t / nt.  tw: the per-stage twiddle table of length L.
template <typename V>
__device__ __forceinline__ void fft_lines(V* buf, int Lp, int L, int log2L, int nt, const V* tw, bool inv,
                                          bool zero_upper = false, bool half_out = false) {
  const int line = threadIdx.x / nt;
  const int lt = threadIdx.x - line * nt;
  const int nq = (L >> 2) / nt;
  V* x = buf + (size_t)line * Lp;
  int Ns = 1;
  bool first = true;
  const V* seg = tw;
  if (log2L & 1) {
    radix2_first_stage(x, L, lt, nt, nq, zero_upper);
    Ns = 2;
    first = false;
  }
  for (; Ns < L; Ns <<= 2) {
    const bool last = (Ns << 2) == L;
    radix4_stage(x, L, Ns, seg, lt, nt, nq, inv, first && zero_upper, last && half_out);
    if (Ns > 1) seg += 3 * Ns;
    first = false;
  }
}

}  // namespace rfnse
