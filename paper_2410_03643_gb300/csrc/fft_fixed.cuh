// In-shared-memory complex FFT of B lines whose length L = 2^LOG2L is fixed at compile time: a
// Stockham auto-sort FFT with radix-RMAX stages (RMAX = 16 or 8, the butterflies held in registers:
// two or one and a half radix-4 levels per shared-memory round trip) and one smaller last stage when
// LOG2L is not a multiple of log2 RMAX.  T = L/RMAX threads work on one line (one radix-RMAX
// butterfly each per full stage).  All index arithmetic is compile-time apart from the thread's
// lane in its line.  Same buffer layout, padding and conventions as fft_line.cuh:
// X_k = sum_j x_j exp(-2 pi i jk/L) forward, conjugate twiddles and no 1/L inverse; `ZU` (zero upper
// half of the input) and `HO` (only the lower half of the output) prune the circulant-embedding
// products.
//
// Twiddles: stage s with sub-transform length Ns > 1 and radix R uses W_{R Ns}^{r k}, r = 1..R-1,
// k = 0..Ns-1, stored at off_s + (r-1) Ns + k, the stages in execution order (the table has L - 1
// entries: sum_s (R_s - 1) Ns_s telescopes).  fixed_twiddle_entry maps a table position back to its
// (R, Ns, r, k) for the table builder.
#pragma once
#include "cplx.cuh"
#include "fft_line.cuh"

namespace rfnse {

// The lengths the FP32 line passes compile with a fixed FFT (2^8 .. 2^11: grids n = 127 .. 1023),
// radix 2^kFixedLogR = 8 (measured faster than radix 16 in the passes: 128 rather than 64 threads per
// line hide the latency of the passes' pointwise work).  The set-up builds the FP32 twiddle table in
// this layout for these lengths.
__host__ __device__ constexpr bool fixed_fft_length(int log2L) { return log2L >= 8 && log2L <= 11; }
constexpr int kFixedLogR = 3;
// The double-float Toeplitz passes (toep_df.cu) use radix 4 (L/4 threads per line): their butterflies
// hold four times the registers of FP32 ones, and the extra threads measured faster on both workloads.
constexpr int kFixedLogRDF = 2;

template <int LOG2L, int LOGR>
struct FixedPlan {
  static constexpr int L = 1 << LOG2L;
  static constexpr int NFULL = LOG2L / LOGR;               // full-radix stages
  static constexpr int LOGLAST = LOG2L - NFULL * LOGR;     // radix of the last stage (0: none)
  static constexpr int T = (LOG2L >= LOGR) ? (L >> LOGR) : 1;   // threads per line
};

// Stage decomposition for the table builder (runtime): the radix exponent and Ns of table entry idx.
__host__ __device__ inline void fixed_twiddle_entry(int log2L, int logR, int idx, int& R, int& Ns, int& r, int& k) {
  const int nfull = log2L / logR;
  const int loglast = log2L - nfull * logR;
  const int nst = nfull + (loglast ? 1 : 0);
  int ns = 1;
  for (int s = 0; s < nst; ++s) {
    const int lr = (s < nfull) ? logR : loglast;
    const int rad = 1 << lr;
    if (ns > 1) {
      const int sz = (rad - 1) * ns;
      if (idx < sz) {
        R = rad;
        Ns = ns;
        r = idx / ns + 1;
        k = idx - (r - 1) * ns;
        return;
      }
      idx -= sz;
    }
    ns <<= lr;
  }
  R = 1;  // past the end (entry L - 1 of a length-L table): unused
  Ns = 1;
  r = 0;
  k = 0;
}

// ---- register DFTs (natural order in and out) -------------------------------------------------
template <bool INV, typename V>
__device__ __forceinline__ V mul_mi(V a) {  // forward W_4 = -i; inverse +i
  return INV ? cmul_i(a) : cmul_mi(a);
}

// Butterfly additions: t + d, t - d, and t +- (-i d) (forward; +i d inverse).  For FP32 each is one
// packed pair instruction (cplx.cuh f2_*): the rotation by -i swaps the parts of d and takes its sign
// from a multiplier of +-1 in a fused multiply-add, which rounds as the addition does.
template <typename V> __device__ __forceinline__ V badd(V t, V d) { return cadd(t, d); }
template <typename V> __device__ __forceinline__ V bsub(V t, V d) { return csub(t, d); }
template <bool INV, typename V> __device__ __forceinline__ V badd_rot(V t, V d) { return cadd(t, mul_mi<INV>(d)); }
template <bool INV, typename V> __device__ __forceinline__ V bsub_rot(V t, V d) { return csub(t, mul_mi<INV>(d)); }
template <> __device__ __forceinline__ float2 badd<float2>(float2 t, float2 d) { return f2_add(t, d); }
template <> __device__ __forceinline__ float2 bsub<float2>(float2 t, float2 d) { return f2_sub(t, d); }
template <> __device__ __forceinline__ float2 badd_rot<false, float2>(float2 t, float2 d) {  // (t.x + d.y, t.y - d.x)
  return f2_fma(make_float2(d.y, d.x), make_float2(1.f, -1.f), t);
}
template <> __device__ __forceinline__ float2 bsub_rot<false, float2>(float2 t, float2 d) {  // (t.x - d.y, t.y + d.x)
  return f2_fma(make_float2(d.y, d.x), make_float2(-1.f, 1.f), t);
}
template <> __device__ __forceinline__ float2 badd_rot<true, float2>(float2 t, float2 d) {  // (t.x - d.y, t.y + d.x)
  return f2_fma(make_float2(d.y, d.x), make_float2(-1.f, 1.f), t);
}
template <> __device__ __forceinline__ float2 bsub_rot<true, float2>(float2 t, float2 d) {  // (t.x + d.y, t.y - d.x)
  return f2_fma(make_float2(d.y, d.x), make_float2(1.f, -1.f), t);
}

template <bool INV, typename V>
__device__ __forceinline__ void dft2(V& a0, V& a1) {
  const V t = a0;
  a0 = badd(t, a1);
  a1 = bsub(t, a1);
}

template <bool INV, typename V>
__device__ __forceinline__ void dft4r(V& a0, V& a1, V& a2, V& a3) {
  const V t0 = badd(a0, a2), t1 = bsub(a0, a2), t2 = badd(a1, a3);
  const V d = bsub(a1, a3);
  a0 = badd(t0, t2);
  a2 = bsub(t0, t2);
  a1 = badd_rot<INV>(t1, d);
  a3 = bsub_rot<INV>(t1, d);
}

// W_16^e (forward) as constants: cos/sin of multiples of pi/8
template <typename R>
struct W16c {
  static constexpr double c1 = 0.92387953251128675613;  // cos(pi/8)
  static constexpr double s1 = 0.38268343236508977173;  // sin(pi/8)
  static constexpr double h = 0.70710678118654752440;   // cos(pi/4)
};

template <bool INV, typename V, typename R>
__device__ __forceinline__ V w16(V a, int e) {  // a * W_16^e, e in 0..9 (compile-time after unrolling)
  const R c1 = (R)W16c<R>::c1, s1 = (R)W16c<R>::s1, h = (R)W16c<R>::h;
  R wr = 1, wi = 0;
  switch (e & 15) {
    case 0: return a;
    case 1: wr = c1; wi = -s1; break;
    case 2: wr = h; wi = -h; break;
    case 3: wr = s1; wi = -c1; break;
    case 4: return mul_mi<INV>(a);
    case 6: wr = -h; wi = -h; break;
    case 9: wr = -c1; wi = s1; break;
    default: {  // not used by the 4 x 4 decomposition
      wr = 0; wi = 0; break;
    }
  }
  if (INV) wi = -wi;
  return cmul(a, cvec<R>::make(wr, wi));
}

// 16-point DFT: n = 4 n1 + n2, k = k1 + 4 k2.  After the three steps X[k1 + 4 k2] is in v[4 k1 + k2];
// the stage stores through perm16.
template <bool INV, bool ZU, typename V, typename R>
__device__ __forceinline__ void dft16(V (&v)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    if (ZU) {  // v[n2 + 8], v[n2 + 12] are zero
      const V a0 = v[n2], a1 = v[n2 + 4];
      v[n2] = badd(a0, a1);
      v[n2 + 8] = bsub(a0, a1);
      v[n2 + 4] = badd_rot<INV>(a0, a1);
      v[n2 + 12] = bsub_rot<INV>(a0, a1);
    } else {
      dft4r<INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    }
  }
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) v[n2 + 4 * k1] = w16<INV, V, R>(v[n2 + 4 * k1], n2 * k1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4r<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
}
__host__ __device__ constexpr int perm16(int r) { return 4 * (r & 3) + (r >> 2); }

// 8-point DFT: n = 4 n1 + n2 (n1 < 2), k = k1 + 2 k2; X[k1 + 2 k2] ends in v[4 k1 + k2].
template <bool INV, bool ZU, typename V, typename R>
__device__ __forceinline__ void dft8(V (&v)[8]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    if (ZU) {
      v[n2 + 4] = v[n2];
    } else {
      dft2<INV>(v[n2], v[n2 + 4]);
    }
  }
  const R h = (R)W16c<R>::h;
  // v[n2 + 4] *= W_8^{n2}
  v[5] = cmul(v[5], cvec<R>::make(h, INV ? h : -h));
  v[6] = mul_mi<INV>(v[6]);
  v[7] = cmul(v[7], cvec<R>::make(-h, INV ? h : -h));
  dft4r<INV>(v[0], v[1], v[2], v[3]);
  dft4r<INV>(v[4], v[5], v[6], v[7]);
}
__host__ __device__ constexpr int perm8(int r) { return 4 * (r & 1) + (r >> 1); }

template <int RAD>
__host__ __device__ constexpr int permr(int r) {
  return RAD == 16 ? perm16(r) : (RAD == 8 ? perm8(r) : r);
}

template <bool INV, bool ZU, int RAD, typename V, typename R>
__device__ __forceinline__ void dft_r(V (&v)[RAD]) {
  if constexpr (RAD == 16) {
    dft16<INV, ZU, V, R>(v);
  } else if constexpr (RAD == 8) {
    dft8<INV, ZU, V, R>(v);
  } else if constexpr (RAD == 4) {
    if (ZU) {
      const V a0 = v[0], a1 = v[1];
      v[0] = badd(a0, a1);
      v[2] = bsub(a0, a1);
      v[1] = badd_rot<INV>(a0, a1);
      v[3] = bsub_rot<INV>(a0, a1);
    } else {
      dft4r<INV>(v[0], v[1], v[2], v[3]);
    }
  } else {
    if (ZU) v[1] = v[0];
    else dft2<INV>(v[0], v[1]);
  }
}

// Padded offset of element i + d from that of element i, d a compile-time step: every stage reads
// j + r NB (NB a multiple of 16) and writes base + r NS with base a multiple of RAD NS plus k < NS, and
// for these (i mod 16) + (d mod 16) < 16, so fft_pad(i + d) = fft_pad(i) + d + (d >> 4) and the r-th
// access of a butterfly is a constant offset from its first.
__host__ __device__ constexpr int pad_step(int d) { return d + (d >> 4); }

// One Stockham stage of radix RAD on sub-transforms of length NS: L/RAD butterflies, Q per thread.
template <int L, int RAD, int NS, int T, bool INV, bool ZU, bool HO, typename V, typename R>
__device__ __forceinline__ void fixed_stage(V* x, const V* seg, int lt) {
  constexpr int NB = L / RAD;
  constexpr int Q = (NB >= T) ? NB / T : 1;
  V v[Q][RAD];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = lt + q * T;
    if (j < NB) {
      const int k = j & (NS - 1);
      const V* xj = x + fft_pad(j);
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        if (ZU && 2 * r >= RAD) v[q][r] = cvec<R>::make((R)0, (R)0);
        else v[q][r] = xj[pad_step(r * NB)];
      }
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          V w = seg[(r - 1) * NS + k];
          if (INV) w = cconj(w);
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dft_r<INV, ZU, RAD, V, R>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = lt + q * T;
    if (j < NB) {
      const int k = j & (NS - 1);
      V* xb = x + fft_pad((j - k) * RAD + k);
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        if (HO && 2 * r >= RAD) continue;
        xb[pad_step(r * NS)] = v[q][permr<RAD>(r)];
      }
    }
  }
  __syncthreads();
}

template <int L, int LOGR, int S, int NST, int NFULL, int LOGLAST, int NS, int T, bool INV, bool ZU, bool HO,
          typename V, typename R>
__device__ __forceinline__ void fixed_stages(V* x, const V* seg, int lt) {
  if constexpr (S < NST) {
    constexpr int LR = (S < NFULL) ? LOGR : LOGLAST;
    constexpr int RAD = 1 << LR;
    fixed_stage<L, RAD, NS, T, INV, ZU && S == 0, HO && S == NST - 1, V, R>(x, seg, lt);
    const V* next = (NS > 1) ? seg + (RAD - 1) * NS : seg;
    fixed_stages<L, LOGR, S + 1, NST, NFULL, LOGLAST, NS * RAD, T, INV, ZU, HO, V, R>(x, next, lt);
  }
}

// FFT of every line of the tile (B lines, line stride Lp).  Threads beyond B * T wait at the barriers.
template <int LOG2L, int LOGR, bool INV, bool ZU, bool HO, typename V>
__device__ __forceinline__ void fft_lines_fixed(V* buf, int Lp, int B, const V* tw) {
  using R = typename creal<V>::type;
  using P = FixedPlan<LOG2L, LOGR>;
  constexpr int NST = P::NFULL + (P::LOGLAST ? 1 : 0);
  const int line = threadIdx.x / P::T;
  const int lt = threadIdx.x - line * P::T;
  V* x = buf + (size_t)(line < B ? line : 0) * Lp;
  // threads without a line (blockDim > B T) run the stages on line 0 with their loads and stores
  // disabled by an out-of-range lane
  const int lane = line < B ? lt : (1 << 30);
  fixed_stages<P::L, LOGR, 0, NST, P::NFULL, P::LOGLAST, 1, P::T, INV, ZU, HO, V, R>(x, tw, lane);
}

}  // namespace rfnse
