// Line passes: every transform of the method acts along one grid axis at a time.  A pass kernel
// stages B lines of one axis in shared memory, transforms them there, and fuses the pointwise
// work that follows.  Operations (compile-time flags, applied in this order):
//
//   F_INSCALE  multiply the loaded (FP64) input by a device scalar and write the scaled vector out
//              (this is v_{j+1} = w / h_{j+1,j} of the Arnoldi process, folded into the first pass)
//   F_DST      y = S x, S the orthonormal DST-I matrix [S]_{jk} = sqrt(2/(n+1)) sin(pi jk/(n+1))
//              (paper Sec. 4, eq. 'taudiagonal'; normalisation sqrt(2/(n+1))).  Computed from the odd
//              extension of x, a complex FFT of length L = 2(n+1): (S x)_k = i Y_k / sqrt(2(n+1)).
//   F_LAM      multiply by 1/(omega + i Lambda(k)), Lambda(k) = sum_a mu_a lambda^{(a)}_{k_a}, and
//              apply S again: the sub-solve with omega I + tau(T_d) in the DST basis (eq. 'taupre',
//              '2Dtau').  Only on the last axis, when every other axis is already in the DST basis, so
//              the mode index of an element is its grid index; the factor comes from a per-mode table.
//   F_DSCALE   z = 2 omega / ((omega+1) - i D) * y: the sub-solve with omega I + D_d and the factor
//              2 omega of F~^{-1} (eq. 'taupre'), from a per-point table.  Stores z (or adds it).
//   F_TOEP_X   t = mu_a T_0^{(a)} z by circulant embedding (length-L FFT, multiply by the scaled
//              circulant eigenvalues, inverse FFT) and acc = add + a z + b (t - D z)  (first axis)
//   F_TOEP_ACC t = mu_a T_0^{(a)} z and acc = acc + b t                                  (other axes)
//   F_CIRC     (with F_DST) the circulant comparator of Sec. 5: the transform is the unnormalised
//              length-n DFT instead of S (forward, or inverse when inv_dft is set; with F_LAM forward,
//              multiply, inverse), computed by Bluestein's chirp-z identity from one circular
//              convolution of length L, i.e. two FFTs; no output scale (it is folded into lamfac).
//   Without F_DST, F_DSCALE stores the loaded input itself (times dfac if given): the identity
//   preconditioner of plain GMRES.
//   F_DOT0     (with a Toeplitz flag, result stored in FP64) the block's partial sum of the real inner
//              product <v_0, w> of the stored result w with dot_v0, written to dot_part[block]: the
//              first modified Gram-Schmidt dot product of the Arnoldi step, so that the Arnoldi kernel
//              starts from their fixed-order sum instead of a sweep of its own.
//
// With a = 1, b = i the Toeplitz passes give w = R z for the complex form R = I + i(T_d - D) of the
// real block matrix R_d of eq. 'positiveBlockForm' (u = y + iz  <->  x = [z; y]).
//
// All per-point arithmetic runs in the compute precision R (FP32 kernels issue no FP64 work except
// the FP64 loads/stores their operands require).  Complex data are interleaved (re, im); x is the
// fastest axis.  Lines along x are contiguous; a tile of a strided axis is B lines adjacent in the
// fastest coordinate, so every global access of a tile row is B consecutive complex values.
#pragma once
#include <cstdint>
#include "cplx.cuh"
#include "fft_line.cuh"
#include "fft_fixed.cuh"
#include "internal.cuh"

namespace rfnse {

enum : int {
  F_INSCALE = 1,
  F_DST = 2,
  F_LAM = 4,
  F_DSCALE = 8,
  F_TOEP_X = 16,
  F_TOEP_ACC = 32,
  F_CIRC = 64,
  F_DOT0 = 128,
};

struct PassParams {
  const void* in;          // input vector (storage TIN)
  void* out;               // DST / z output (storage TOUT); may be null when not needed
  double2* copy_out;       // F_INSCALE: the scaled input is written here
  const double* in_scale;  // F_INSCALE: device scalar
  const void* acc_in;      // F_TOEP_X: optional additive vector; F_TOEP_ACC: accumulator (storage TACCI)
  void* acc_out;           // Toeplitz result (storage TACCO)
  const void* Dr;          // diagonal D in the compute precision (physical positions)
  const void* dfac;        // per-point factor 2w((w+1) + iD)/((w+1)^2 + D^2), compute precision
  const void* lamfac;      // per-mode factor i dst_scale / (w + i Lambda), compute precision
  const void* tw;          // twiddle table exp(-2 pi i k/L), k < L, compute precision
  const void* circ;        // circulant eigenvalues of this axis times mu_a / L (length L), compute precision
  double dst_scale;        // 1/sqrt(2(n+1))
  double2 ca, cb;          // epilogue scalars a and b
  float dst_scale_f;       // the same in FP32 (set by launch_pass): FP32 kernels convert nothing
  float2 ca_f, cb_f;
  int n, L, log2L, nt, B;  // axis extent, FFT length, log2 L, threads per line, lines per block
  int log2B;               // B = 2^log2B
  long long stride;        // element stride of the axis
  long long nlines;        // N / n
  long long tiles_inner;   // strided axes: ceil(stride / B)
  int z_add;               // F_DSCALE: out += z instead of out = z
  // device-side control: when gdyn is set, F_INSCALE takes its source vector and factor from the
  // GMRES state and writes V[j] = vbase + j ldv, and F_DSCALE writes Z[j] = zbase + j ldv (if zbase)
  const GmresState* gdyn;
  double2* vbase;
  void* zbase;
  long long ldv;
  const int* skip;         // when set and nonzero, the launch does nothing
  int in_dyn_z;            // with gdyn: the input is Z[j] = zbase + j ldv (storage TIN)
  // F_CIRC: chirp exp(i pi j^2/n) (length n) and Bluestein filter spectrum (length L, 1/L folded in),
  // compute precision; inv_dft: the (first) transform is the inverse DFT
  const void* chirp;
  const void* bspec;
  int inv_dft;
  // double-float Toeplitz passes: ca and cb as codes when they are 0, +-1 or +-i (products become
  // swaps and sign changes), -1 otherwise
  int ca_code, cb_code;
  // F_DOT0: v_0 (FP64, grid order) and the per-block partials (one per block of the launch)
  const double2* dot_v0;
  double* dot_part;
  // double-float Toeplitz passes: when set, each block's share of ||result||^2
  double* nrm_part;
  // double-float Toeplitz passes of a product along several axes: the input split into double-float
  // once, written by the first pass and read by the others (float4 per point: re.hi, im.hi, re.lo,
  // im.lo); null when not used
  const void* dfz_in;
  void* dfz_out;
};

// Sum of v over the block, written by thread 0 to *out; every thread of the block must call it.  The
// block size is a power of two (every pass tile is), at most 1024; below 32 the one warp is partial
// and its tree starts at half its width.  Warp shuffles, then the warps in order: a fixed order.
__device__ __forceinline__ void block_sum_store(double v, double* out) {
  __shared__ double red[32];
  const unsigned nt = blockDim.x;
  const unsigned mask = nt >= 32u ? 0xffffffffu : ((1u << nt) - 1u);
  for (int o = nt >= 32u ? 16 : (int)(nt >> 1); o > 0; o >>= 1) v += __shfl_down_sync(mask, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)((blockDim.x + 31) >> 5); ++q) t += red[q];
    *out = t;
  }
}

template <typename R> __device__ __forceinline__ cv<R> ld_c(const void* p, long long i);
template <> __device__ __forceinline__ double2 ld_c<double>(const void* p, long long i) {
  return reinterpret_cast<const double2*>(p)[i];
}
template <> __device__ __forceinline__ float2 ld_c<float>(const void* p, long long i) {
  return reinterpret_cast<const float2*>(p)[i];
}

// FP32 passes whose FFT length passes fixed_fft_length (fft_fixed.cuh) are compiled with the length
// fixed (radix-8 register butterflies; k_line_pass_fixed below, or for the Bluestein passes of the
// circulant comparator this kernel with the twiddles read from the global per-stage table through L1);
// all other passes use the runtime-length radix-4 FFT of fft_line.cuh with the table in shared memory.
template <int LOG2L, bool INV, bool ZU, bool HO, typename V>
__device__ __forceinline__ void fft_any(V* buf, int Lp, int L, int log2L, int nt, int B, const V* tw) {
  if constexpr (LOG2L > 0) {
    fft_lines_fixed<LOG2L, kFixedLogR, INV, ZU, HO>(buf, Lp, B, tw);
  } else {
    fft_lines(buf, Lp, L, log2L, nt, tw, INV, ZU, HO);
  }
}

// Unnormalised length-n DFT of every line of the tile by Bluestein's identity: element j of a line is
// at position 1 + j (as everywhere in the passes); forward X_k = sum_j x_j exp(-2 pi i jk/n) =
// conj(b_k) sum_j (x_j conj(b_j)) bt_{k-j}, inverse with b and conj(bt) (whose spectrum is conj(bspec):
// bt is symmetric).  The circular convolution of length L >= 2n - 1 is exact for the needed range; its
// input is zero from position n + 1 = L/2 on and only positions 1..n are read back, so the two FFTs
// are the pruned ones of the Toeplitz products.  All threads of the block call this.
template <typename R, int LOG2L>
__device__ __forceinline__ void bluestein_lines(cv<R>* buf, int Lp, int L, int log2L, int nt, const cv<R>* tws,
                                                int n, int B, const void* chirp, const void* bspec, bool inv) {
  using V = cv<R>;
  const V zero = cvec<R>::make((R)0, (R)0);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const V* ch = reinterpret_cast<const V*>(chirp);
  const V* bs = reinterpret_cast<const V*>(bspec);
  for (int e = tid; e < B * L; e += nthr) {
    const int l = e >> log2L, k = e & (L - 1);
    V& v = buf[(size_t)l * Lp + fft_pad(k)];
    if (k >= 1 && k <= n) {
      V b = ch[k - 1];
      if (!inv) b.y = -b.y;
      v = cmul(v, b);
    } else {
      v = zero;
    }
  }
  __syncthreads();
  fft_any<LOG2L, false, true, false>(buf, Lp, L, log2L, nt, B, tws);   // zero upper half in
  for (int e = tid; e < B * L; e += nthr) {
    const int l = e >> log2L, k = e & (L - 1);
    V s = bs[k];
    if (inv) s.y = -s.y;
    V& v = buf[(size_t)l * Lp + fft_pad(k)];
    v = cmul(v, s);
  }
  __syncthreads();
  fft_any<LOG2L, true, false, true>(buf, Lp, L, log2L, nt, B, tws);    // lower half out
  for (int e = tid; e < B * n; e += nthr) {
    const int l = e / n, j = e - l * n;
    V b = ch[j];
    if (!inv) b.y = -b.y;
    V& v = buf[(size_t)l * Lp + fft_pad(1 + j)];
    v = cmul(v, b);
  }
  __syncthreads();
}

constexpr int kPassMaxThreads = 512;  // the line-pass kernels' launch bound
constexpr size_t kPassMaxSmem = 200 * 1024;  // the dynamic shared memory the pass kernels opt in to

// A batched launch over several instances' tiles (the lock-step batch, lockstep.cu): block b works on
// tile b - start[i] of instance i, start[i] <= b < start[i + 1], with that instance's parameters.
struct PassWork {
  const PassParams* plist;  // one per instance
  const long long* start;   // n + 1 prefix sums of the instances' tile counts
  int n;
};

// The work item of this block: its instance's parameters copied to shared memory and its tile there.
__device__ __forceinline__ void pass_work_item(const PassWork& w, PassParams& ps, long long& tile) {
  __shared__ int inst;
  if (threadIdx.x == 0) {
    const long long b = blockIdx.x;
    int lo = 0, hi = w.n - 1;
    while (lo < hi) {  // the last instance whose range starts at or before b
      const int mid = (lo + hi + 1) >> 1;
      if (w.start[mid] <= b) lo = mid;
      else hi = mid - 1;
    }
    inst = lo;
    tile = b - w.start[lo];
  }
  __syncthreads();
  const int* src = reinterpret_cast<const int*>(w.plist + inst);
  int* dst = reinterpret_cast<int*>(&ps);
  for (int i = threadIdx.x; i < (int)(sizeof(PassParams) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// The elements e = tid, tid + nthr, ... < B n of a tile, visited in that order without a division or a
// 64-bit multiply per element: (line l, position pos) and the global index g are stepped.  Strided
// axes: e = pos B + l, and nthr is a multiple of B, so l is fixed and pos, g advance by constant
// steps.  x-lines: g = line0 n + e is contiguous; with several lines per tile, pos wraps into the
// next line (nthr / n + 1 wraps at most per step).
struct TileWalk {
  int l, pos;         // line of the tile and position along it
  long long g;        // global index of the element
  bool valid;         // its line exists in the grid
  int n, B, dpos;     // axis extent, lines per tile, position step (strided axes)
  long long dg;       // global step
  bool xax;
  long long line0, nlines;
  __device__ __forceinline__ TileWalk(const PassParams& p, bool xax_, int tid, int nthr, long long line0_,
                                      long long hi, long long lo0)
      : n(p.n), B(p.B), xax(xax_), line0(line0_), nlines(p.nlines) {
    if (xax) {
      l = (B == 1) ? 0 : tid / n;
      pos = tid - l * n;
      g = line0 * n + tid;
      dg = nthr;
      dpos = nthr;
      valid = line0 + l < nlines;
    } else {
      l = tid & (B - 1);
      pos = tid >> p.log2B;
      dpos = nthr >> p.log2B;
      g = lo0 + l + (long long)pos * p.stride + hi * p.stride * n;
      dg = (long long)dpos * p.stride;
      valid = lo0 + l < p.stride;
    }
  }
  __device__ __forceinline__ bool more() const { return xax ? (pos < n && l < B) : pos < n; }
  __device__ __forceinline__ void next() {
    pos += dpos;
    g += dg;
    if (xax && B > 1) {
      while (pos >= n) {
        pos -= n;
        ++l;
      }
      valid = line0 + l < nlines;
    }
  }
};

template <typename R, typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS, int LOG2L>
__device__ __forceinline__ void line_pass_body(const PassParams& p, const long long tile) {
  using V = cv<R>;
  if (p.skip && *p.skip) return;  // uniform: the whole launch is a no-op
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = p.L, n = p.n, Nh = L >> 1, B = p.B;
  const int Lp = fft_line_stride(L);
  V* buf = reinterpret_cast<V*>(smem_raw);
  V* zsave = buf + (size_t)B * Lp + (LOG2L > 0 ? 0 : L);
  // twiddles: staged in shared memory for the runtime-length FFT, read from the table otherwise
  const V* tws = (LOG2L > 0) ? reinterpret_cast<const V*>(p.tw) : buf + (size_t)B * Lp;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const bool xax = (p.stride == 1);
  const V zero = cvec<R>::make((R)0, (R)0);

  if (LOG2L == 0)
    for (int i = tid; i < L; i += nthr) (buf + (size_t)B * Lp)[i] = ld_c<R>(p.tw, i);

  long long line0 = 0, hi = 0, lo0 = 0;
  if (xax) {
    line0 = tile * B;
  } else {
    hi = tile / p.tiles_inner;
    lo0 = (tile - hi * p.tiles_inner) * B;
  }
  auto at = [&](int l, int i) -> V& { return buf[(size_t)l * Lp + fft_pad(i)]; };

  // ---- load -----------------------------------------------------------------------------------
  const TIN* in = reinterpret_cast<const TIN*>(p.in);
  if (p.gdyn && p.in_dyn_z) in = reinterpret_cast<const TIN*>(p.zbase) + (long long)p.gdyn->j * p.ldv;
  double sc = 1.0;
  const double2* src = reinterpret_cast<const double2*>(p.in);
  double2* cpy = p.copy_out;
  if (FLAGS & F_INSCALE) {
    if (p.gdyn) {
      src = p.gdyn->src;
      sc = p.gdyn->src_scale;
      cpy = p.vbase + (long long)p.gdyn->j * p.ldv;
    } else {
      sc = *p.in_scale;
    }
  }
  for (TileWalk it(p, xax, tid, nthr, line0, hi, lo0); it.more(); it.next()) {
    const int l = it.l, pos = it.pos;
    const bool valid = it.valid;
    const long long g = it.g;
    V v = zero;
    if (valid) {
      if (FLAGS & F_INSCALE) {
        double2 vd = src[g];
        vd.x *= sc;
        vd.y *= sc;
        cpy[g] = vd;
        v = to_c<R>(vd);
      } else {
        v = to_c<R>(in[g]);
      }
    }
    at(l, 1 + pos) = v;
    if (FLAGS & F_DST) {
      if (!(FLAGS & F_CIRC)) at(l, L - 1 - pos) = cneg(v);   // odd extension y_{2(n+1)-j} = -x_j
    } else if (FLAGS & F_TOEP_X) {
      zsave[l * n + pos] = v;
    }
  }
  for (int l = tid; l < B; l += nthr) {
    at(l, 0) = zero;
    at(l, Nh) = zero;
  }
  if (!(FLAGS & F_DST) || (FLAGS & F_CIRC)) {      // zero padding of the circulant embedding
    for (int e = tid; e < B * Nh; e += nthr) at(e >> (p.log2L - 1), Nh + (e & (Nh - 1))) = zero;  // Nh .. L-1
  }
  __syncthreads();

  const R dsc = sizeof(R) == 4 ? (R)p.dst_scale_f : (R)p.dst_scale;

  // ---- circulant comparator: DFTs by Bluestein ------------------------------------------------
  if ((FLAGS & F_DST) && (FLAGS & F_CIRC)) {
    bluestein_lines<R, LOG2L>(buf, Lp, L, p.log2L, p.nt, tws, n, B, p.chirp, p.bspec,
                              (FLAGS & F_LAM) ? false : p.inv_dft != 0);
    if (FLAGS & F_LAM) {
      for (TileWalk it(p, xax, tid, nthr, line0, hi, lo0); it.more(); it.next()) {
        const int l = it.l, pos = it.pos;
        const bool valid = it.valid;
        const long long g = it.g;
        const V f = valid ? ld_c<R>(p.lamfac, g) : zero;   // mode index = grid index on this axis
        at(l, 1 + pos) = cmul(at(l, 1 + pos), f);
      }
      __syncthreads();
      bluestein_lines<R, LOG2L>(buf, Lp, L, p.log2L, p.nt, tws, n, B, p.chirp, p.bspec, true);
    }
  }

  // ---- sine transforms ------------------------------------------------------------------------
  if ((FLAGS & F_DST) && !(FLAGS & F_CIRC)) {
    fft_any<LOG2L, false, false, false>(buf, Lp, L, p.log2L, p.nt, B, tws);
    if (FLAGS & F_LAM) {
      for (TileWalk it(p, xax, tid, nthr, line0, hi, lo0); it.more(); it.next()) {
        const int l = it.l, pos = it.pos;
        const bool valid = it.valid;
        const long long g = it.g;
        const int k = pos + 1;                     // sine mode k = 1..n along this axis
        const V f = valid ? ld_c<R>(p.lamfac, g) : zero;
        at(l, k) = cmul(at(l, k), f);
        at(l, L - k) = cmul(at(l, L - k), f);
      }
      for (int l = tid; l < B; l += nthr) {
        at(l, 0) = zero;
        at(l, Nh) = zero;
      }
      __syncthreads();
      fft_any<LOG2L, false, false, false>(buf, Lp, L, p.log2L, p.nt, B, tws);
    }
  }

  // ---- DST output / D sub-solve ---------------------------------------------------------------
  if ((FLAGS & F_DST) && !(FLAGS & F_DSCALE)) {
    TOUT* out = reinterpret_cast<TOUT*>(p.out);
    for (TileWalk it(p, xax, tid, nthr, line0, hi, lo0); it.more(); it.next()) {
      const int l = it.l, pos = it.pos;
      const bool valid = it.valid;
      const long long g = it.g;
      if (valid) st_c(out + g, (FLAGS & F_CIRC) ? at(l, 1 + pos) : cmul_i(cscale(at(l, 1 + pos), dsc)));
    }
  }
  if (FLAGS & F_DSCALE) {
    TOUT* out = reinterpret_cast<TOUT*>(p.out);
    if (p.gdyn && p.zbase) out = reinterpret_cast<TOUT*>(p.zbase) + (long long)p.gdyn->j * p.ldv;
    for (TileWalk it(p, xax, tid, nthr, line0, hi, lo0); it.more(); it.next()) {
      const int l = it.l, pos = it.pos;
      const bool valid = it.valid;
      const long long g = it.g;
      V z = zero;
      if (valid) {
        z = at(l, 1 + pos);                                   // identity preconditioner: the input
        if ((FLAGS & F_DST) && !(FLAGS & F_CIRC)) z = cmul_i(cscale(z, dsc));
        if (p.dfac) z = cmul(z, ld_c<R>(p.dfac, g));
        if (out) {
          if (p.z_add) st_c(out + g, cadd(to_c<R>(out[g]), z));
          else st_c(out + g, z);
        }
      }
      if (FLAGS & (F_TOEP_X | F_TOEP_ACC)) {
        at(l, 1 + pos) = z;
        if (FLAGS & F_TOEP_X) zsave[l * n + pos] = z;
      }
    }
    if (FLAGS & (F_TOEP_X | F_TOEP_ACC)) {
      for (int e = tid; e < B * Nh; e += nthr) at(e >> (p.log2L - 1), Nh + (e & (Nh - 1))) = zero;  // Nh .. L-1
      for (int l = tid; l < B; l += nthr) {
        at(l, 0) = zero;
        at(l, Nh) = zero;
      }
    }
    __syncthreads();
  }

  // ---- Toeplitz product by circulant embedding ------------------------------------------------
  if (FLAGS & (F_TOEP_X | F_TOEP_ACC)) {
    // the embedded vector is zero from position L/2 on, and only positions 1..n < L/2 are read back
    fft_any<LOG2L, false, true, false>(buf, Lp, L, p.log2L, p.nt, B, tws);   // zero upper half in
    const R* circ = reinterpret_cast<const R*>(p.circ);
    for (int e = tid; e < B * L; e += nthr) {
      const int l = e >> p.log2L;
      const int k = e & (L - 1);
      at(l, k) = cscale(at(l, k), circ[k]);
    }
    __syncthreads();
    fft_any<LOG2L, true, false, true>(buf, Lp, L, p.log2L, p.nt, B, tws);    // lower half out
    const V ca = sizeof(R) == 4 ? cvec<R>::make((R)p.ca_f.x, (R)p.ca_f.y) : cvec<R>::make((R)p.ca.x, (R)p.ca.y);
    const V cb = sizeof(R) == 4 ? cvec<R>::make((R)p.cb_f.x, (R)p.cb_f.y) : cvec<R>::make((R)p.cb.x, (R)p.cb.y);
    const TACCI* accin = reinterpret_cast<const TACCI*>(p.acc_in);
    TACCO* accout = reinterpret_cast<TACCO*>(p.acc_out);
    const R* Dr = reinterpret_cast<const R*>(p.Dr);
    [[maybe_unused]] double dot = 0.0;
    for (TileWalk it(p, xax, tid, nthr, line0, hi, lo0); it.more(); it.next()) {
      const int l = it.l, pos = it.pos;
      const bool valid = it.valid;
      const long long g = it.g;
      if (!valid) continue;
      V t = at(l, 1 + pos);
      V acc = accin ? to_c<R>(accin[g]) : zero;
      if (FLAGS & F_TOEP_X) {
        const V z = zsave[l * n + pos];
        const R Dj = Dr ? Dr[g] : (R)0;
        t = csub(t, cscale(z, Dj));
        acc = cadd(acc, cmul(ca, z));
      }
      acc = cadd(acc, cmul(cb, t));
      st_c(accout + g, acc);
      if constexpr ((FLAGS & F_DOT0) != 0) {  // on the stored FP64 value
        const double2 wv = make_double2((double)acc.x, (double)acc.y), v0 = p.dot_v0[g];
        dot = fma(v0.x, wv.x, dot);
        dot = fma(v0.y, wv.y, dot);
      }
    }
    if constexpr ((FLAGS & F_DOT0) != 0) block_sum_store(dot, p.dot_part + tile);
  }
}

template <typename R, typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS, int LOG2L>
__global__ void __launch_bounds__(kPassMaxThreads) k_line_pass(const PassParams p) {
  line_pass_body<R, TIN, TOUT, TACCI, TACCO, FLAGS, LOG2L>(p, blockIdx.x);
}

template <typename R, typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS, int LOG2L>
__global__ void __launch_bounds__(kPassMaxThreads) k_line_pass_wl(const PassWork w) {
  __shared__ PassParams ps;
  __shared__ long long tile;
  pass_work_item(w, ps, tile);
  line_pass_body<R, TIN, TOUT, TACCI, TACCO, FLAGS, LOG2L>(ps, tile);
}

// FP32 passes whose FFT length is fixed at compile time (fixed_fft_length), every operation of
// k_line_pass but the circulant comparator's Bluestein DFTs.  Same tiles and geometry (B lines,
// T = L/8 threads per line, B T threads), so with n = L/2 - 1 a thread owns at most QN = L/(2T) points
// of the tile and QL = L/T of its B L spectrum positions: the per-point loops are unrolled over these
// slots.  Every global operand (input, D, dfac, lamfac, accumulator, z_add target, circulant
// eigenvalues, twiddles) is loaded into registers in one batch at the start, so the pass waits on
// global memory once rather than once per loop iteration and FFT stage; the twiddles are then staged in
// shared memory, and z stays in registers between the sub-solve and the Toeplitz epilogue.
template <typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS, int LOG2L>
__device__ __forceinline__ void line_pass_fixed_body(const PassParams& p, const long long tile) {
  static_assert(!(FLAGS & F_CIRC), "the circulant comparator's passes run in k_line_pass");
  static_assert(LOG2L > 0, "fixed FFT length only");
  static_assert(!(FLAGS & F_DOT0) || sizeof(TACCO) == sizeof(double2), "F_DOT0 needs an FP64 result");
  using R = float;
  using V = float2;
  using P = FixedPlan<LOG2L, kFixedLogR>;
  constexpr int L = P::L, Nh = L / 2, T = P::T;
  constexpr int QN = (Nh + T - 1) / T;
  constexpr int QL = L / T;
  constexpr bool TOEP = (FLAGS & (F_TOEP_X | F_TOEP_ACC)) != 0;
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n = Nh - 1;  // the grids have n + 1 = L / 2 points per axis (a power of two)
  const int B = p.B;
  const int Lp = fft_line_stride(L);
  V* buf = reinterpret_cast<V*>(smem_raw);
  V* tws = buf + (size_t)B * Lp;  // the L - 1 entries of the per-stage twiddle table
  const int tid = threadIdx.x, nthr = B * T;
  const bool xax = (p.stride == 1);
  const V zero = make_float2(0.f, 0.f);

  long long line0 = 0, hi = 0, lo0 = 0;
  if (xax) {
    line0 = tile * B;
  } else {
    hi = tile / p.tiles_inner;
    lo0 = (tile - hi * p.tiles_inner) * B;
  }
  // slot q of this thread: tile element e = tid + q B T -> line l, position pos, global index g
  int sl[QN], sp[QN];
  long long sg[QN];
  bool sin_[QN], sok[QN];  // in the tile (e < B n); also in the grid
#pragma unroll
  for (int q = 0; q < QN; ++q) {
    const int e = tid + q * nthr;
    int l = 0, pos = 0;
    if (xax) {
      if (B == 1) pos = e;
      else { l = e / n; pos = e - l * n; }
    } else {
      pos = e >> p.log2B;
      l = e & (B - 1);
    }
    bool valid;
    long long g;
    if (xax) {
      const long long ln = line0 + l;
      valid = ln < p.nlines;
      g = ln * n + pos;
    } else {
      const long long lo = lo0 + l;
      valid = lo < p.stride;
      g = lo + (long long)pos * p.stride + hi * p.stride * n;
    }
    sin_[q] = e < B * n;
    sok[q] = sin_[q] && valid;
    sl[q] = l;
    sp[q] = pos;
    sg[q] = g;
  }
  auto at = [&](int l, int i) -> V& { return buf[(size_t)l * Lp + fft_pad(i)]; };

  // ---- every global operand, one batch ---------------------------------------------------------
  V twr[QL];
  {
    const V* twg = reinterpret_cast<const V*>(p.tw);
#pragma unroll
    for (int q = 0; q < QL; ++q) {
      const int i = tid + q * nthr;
      if (i < L - 1) twr[q] = __ldg(twg + i);
    }
  }
  [[maybe_unused]] R cq[QL];
  if constexpr (TOEP) {
    const R* circ = reinterpret_cast<const R*>(p.circ);
#pragma unroll
    for (int q = 0; q < QL; ++q) cq[q] = __ldg(circ + ((tid + q * nthr) & (L - 1)));
  }
  V xq[QN];
  {
    const TIN* in = reinterpret_cast<const TIN*>(p.in);
    if (p.gdyn && p.in_dyn_z) in = reinterpret_cast<const TIN*>(p.zbase) + (long long)p.gdyn->j * p.ldv;
    const double2* src = reinterpret_cast<const double2*>(p.in);
    double2* cpy = p.copy_out;
    double sc = 1.0;
    if constexpr ((FLAGS & F_INSCALE) != 0) {
      if (p.gdyn) {
        src = p.gdyn->src;
        sc = p.gdyn->src_scale;
        cpy = p.vbase + (long long)p.gdyn->j * p.ldv;
      } else {
        sc = *p.in_scale;
      }
    }
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      xq[q] = zero;
      if (sok[q]) {
        if constexpr ((FLAGS & F_INSCALE) != 0) {
          double2 vd = __ldg(src + sg[q]);
          vd.x *= sc;
          vd.y *= sc;
          cpy[sg[q]] = vd;
          xq[q] = to_c<R>(vd);
        } else {
          xq[q] = to_c<R>(__ldg(in + sg[q]));
        }
      }
    }
  }
  [[maybe_unused]] V fq[QN], lq[QN], aq[QN], oq[QN];
  [[maybe_unused]] R dq[QN];
  [[maybe_unused]] TOUT* zout = reinterpret_cast<TOUT*>(p.out);
  if constexpr ((FLAGS & F_DSCALE) != 0) {
    if (p.gdyn && p.zbase) zout = reinterpret_cast<TOUT*>(p.zbase) + (long long)p.gdyn->j * p.ldv;
    const V* dfac = reinterpret_cast<const V*>(p.dfac);
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      fq[q] = (dfac && sok[q]) ? __ldg(dfac + sg[q]) : make_float2(1.f, 0.f);
      oq[q] = (zout && p.z_add && sok[q]) ? to_c<R>(zout[sg[q]]) : zero;
    }
  }
  if constexpr ((FLAGS & F_LAM) != 0) {
    const V* lam = reinterpret_cast<const V*>(p.lamfac);
#pragma unroll
    for (int q = 0; q < QN; ++q) lq[q] = sok[q] ? __ldg(lam + sg[q]) : zero;   // mode index = grid index
  }
  if constexpr (TOEP) {
    const TACCI* accin = reinterpret_cast<const TACCI*>(p.acc_in);
    const R* Dr = reinterpret_cast<const R*>(p.Dr);
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      aq[q] = (accin && sok[q]) ? to_c<R>(__ldg(accin + sg[q])) : zero;
      if constexpr ((FLAGS & F_TOEP_X) != 0) dq[q] = (Dr && sok[q]) ? __ldg(Dr + sg[q]) : 0.f;
    }
  }

  // ---- tile and twiddles into shared memory ------------------------------------------------------
#pragma unroll
  for (int q = 0; q < QL; ++q) {
    const int i = tid + q * nthr;
    if (i < L - 1) tws[i] = twr[q];
  }
#pragma unroll
  for (int q = 0; q < QN; ++q) {
    if (!sin_[q]) continue;
    at(sl[q], 1 + sp[q]) = xq[q];
    if constexpr ((FLAGS & F_DST) != 0) at(sl[q], L - 1 - sp[q]) = cneg(xq[q]);   // odd extension
  }
  for (int l = tid; l < B; l += nthr) {
    at(l, 0) = zero;
    at(l, Nh) = zero;
  }
  if constexpr ((FLAGS & F_DST) == 0) {  // zero padding of the circulant embedding
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      const int e = tid + q * nthr;
      if (e < B * Nh) at(e >> (LOG2L - 1), Nh + (e & (Nh - 1))) = zero;  // positions Nh .. L-1
    }
  }
  __syncthreads();
  const R dsc = p.dst_scale_f;

  // ---- sine transforms ------------------------------------------------------------------------
  if constexpr ((FLAGS & F_DST) != 0) {
    fft_lines_fixed<LOG2L, kFixedLogR, false, false, false>(buf, Lp, B, tws);
    if constexpr ((FLAGS & F_LAM) != 0) {
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        if (!sin_[q]) continue;
        const int k = sp[q] + 1;  // sine mode k = 1..n along this axis
        at(sl[q], k) = cmul(at(sl[q], k), lq[q]);
        at(sl[q], L - k) = cmul(at(sl[q], L - k), lq[q]);
      }
      for (int l = tid; l < B; l += nthr) {
        at(l, 0) = zero;
        at(l, Nh) = zero;
      }
      __syncthreads();
      fft_lines_fixed<LOG2L, kFixedLogR, false, false, false>(buf, Lp, B, tws);
    }
  }

  // ---- DST output / D sub-solve ---------------------------------------------------------------
  V zq[QN];
#pragma unroll
  for (int q = 0; q < QN; ++q) zq[q] = xq[q];
  if constexpr ((FLAGS & F_DST) != 0 && (FLAGS & F_DSCALE) == 0) {
    TOUT* out = reinterpret_cast<TOUT*>(p.out);
#pragma unroll
    for (int q = 0; q < QN; ++q)
      if (sok[q]) st_c(out + sg[q], cmul_i(cscale(at(sl[q], 1 + sp[q]), dsc)));
  }
  if constexpr ((FLAGS & F_DSCALE) != 0) {
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      V z = zero;
      if (sok[q]) {
        z = xq[q];  // identity preconditioner: the input
        if constexpr ((FLAGS & F_DST) != 0) z = cmul_i(cscale(at(sl[q], 1 + sp[q]), dsc));
        z = cmul(z, fq[q]);
        if (zout) st_c(zout + sg[q], p.z_add ? cadd(oq[q], z) : z);
      }
      zq[q] = z;
      if constexpr (TOEP) {
        if (sin_[q]) at(sl[q], 1 + sp[q]) = z;
      }
    }
    if constexpr (TOEP) {
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        const int e = tid + q * nthr;
        if (e < B * Nh) at(e >> (LOG2L - 1), Nh + (e & (Nh - 1))) = zero;  // positions Nh .. L-1
      }
      for (int l = tid; l < B; l += nthr) {
        at(l, 0) = zero;
        at(l, Nh) = zero;
      }
    }
    __syncthreads();
  }

  // ---- Toeplitz product by circulant embedding ------------------------------------------------
  if constexpr (TOEP) {
    fft_lines_fixed<LOG2L, kFixedLogR, false, true, false>(buf, Lp, B, tws);   // zero upper half in
#pragma unroll
    for (int q = 0; q < QL; ++q) {
      const int e = tid + q * nthr;
      V& v = at(e >> LOG2L, e & (L - 1));
      v = cscale(v, cq[q]);
    }
    // v_0 for the partials of <v_0, w>: loaded here so that the inverse FFT hides the wait
    [[maybe_unused]] double2 v0q[QN];
    if constexpr ((FLAGS & F_DOT0) != 0) {
#pragma unroll
      for (int q = 0; q < QN; ++q) v0q[q] = sok[q] ? __ldg(p.dot_v0 + sg[q]) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    fft_lines_fixed<LOG2L, kFixedLogR, true, false, true>(buf, Lp, B, tws);    // lower half out
    const V ca = p.ca_f, cb = p.cb_f;
    TACCO* accout = reinterpret_cast<TACCO*>(p.acc_out);
    [[maybe_unused]] double dot = 0.0;
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      if (!sok[q]) continue;
      V t = at(sl[q], 1 + sp[q]);
      V acc = aq[q];
      if constexpr ((FLAGS & F_TOEP_X) != 0) {
        t = csub(t, cscale(zq[q], dq[q]));
        acc = cadd(acc, cmul(ca, zq[q]));
      }
      acc = cadd(acc, cmul(cb, t));
      st_c(accout + sg[q], acc);
      if constexpr ((FLAGS & F_DOT0) != 0) {  // on the stored FP64 value
        dot = fma(v0q[q].x, (double)acc.x, dot);
        dot = fma(v0q[q].y, (double)acc.y, dot);
      }
    }
    if constexpr ((FLAGS & F_DOT0) != 0) block_sum_store(dot, p.dot_part + tile);
  }
}

template <typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS, int LOG2L>
__global__ void __launch_bounds__(kPassMaxThreads) k_line_pass_fixed(const PassParams p) {
  line_pass_fixed_body<TIN, TOUT, TACCI, TACCO, FLAGS, LOG2L>(p, blockIdx.x);
}

template <typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS, int LOG2L>
__global__ void __launch_bounds__(kPassMaxThreads) k_line_pass_fixed_wl(const PassWork w) {
  __shared__ PassParams ps;
  __shared__ long long tile;
  pass_work_item(w, ps, tile);
  line_pass_fixed_body<TIN, TOUT, TACCI, TACCO, FLAGS, LOG2L>(ps, tile);
}

// Threads per line (one or two radix-4 butterflies each) and lines per block for FFT length L.
inline void pass_geometry(int L, bool xax, long long lines_avail, int& nt, int& B) {
  nt = L / 4;
  if (nt > 256) nt = L / 8;
  int target = xax ? 256 : 512;
  if (nt > target) target = nt;
  B = target / nt;
  if (B < 1) B = 1;
  while (B > 1 && B > lines_avail) B >>= 1;  // keep B a power of two
}

// The fixed-length FFT: L / 2^logR threads per line; blocks of up to 128 threads along x and 256
// along a strided axis (B lines adjacent in x, so B >= 2 keeps 16-byte runs per row), with fewer lines
// per block while that leaves fewer than two blocks per SM (152 SMs).  Measured on the 2-D 511^2 and
// 3-D 255^3 workloads against 1..4 lines per block on each axis.
inline void pass_geometry_fixed(int L, bool xax, long long lines_avail, long long nlines, int& nt, int& B,
                                int logR = kFixedLogR) {
  nt = L >> logR;
  B = (xax ? 128 : 256) / nt;
  if (B < 1) B = 1;
  while (B > 1 && B * nt > kPassMaxThreads) B >>= 1;
  while (B > 1 && B > lines_avail) B >>= 1;
  auto blocks = [&](int b) -> long long {
    return xax ? (nlines + b - 1) / b : ((lines_avail + b - 1) / b) * (nlines / lines_avail);
  };
  const int bmin = xax ? 1 : 2;
  while (B > bmin && blocks(B) < 2 * 152) B >>= 1;
}

template <typename R, typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS>
struct PassKernels {
  using Fn = void (*)(const PassParams);
  // prefetch: the fixed-length FP32 passes run k_line_pass_fixed (not for the Bluestein passes)
  static Fn get(int log2L, bool prefetch) {
    if constexpr (sizeof(R) == 4 && (FLAGS & F_CIRC) == 0) {
      if (prefetch) {
        switch (log2L) {
          case 8: return k_line_pass_fixed<TIN, TOUT, TACCI, TACCO, FLAGS, 8>;
          case 9: return k_line_pass_fixed<TIN, TOUT, TACCI, TACCO, FLAGS, 9>;
          case 10: return k_line_pass_fixed<TIN, TOUT, TACCI, TACCO, FLAGS, 10>;
          case 11: return k_line_pass_fixed<TIN, TOUT, TACCI, TACCO, FLAGS, 11>;
          default: break;
        }
      }
    }
    if constexpr (sizeof(R) == 4) {
      switch (log2L) {
        case 8: return k_line_pass<R, TIN, TOUT, TACCI, TACCO, FLAGS, 8>;
        case 9: return k_line_pass<R, TIN, TOUT, TACCI, TACCO, FLAGS, 9>;
        case 10: return k_line_pass<R, TIN, TOUT, TACCI, TACCO, FLAGS, 10>;
        case 11: return k_line_pass<R, TIN, TOUT, TACCI, TACCO, FLAGS, 11>;
        default: break;
      }
    }
    return k_line_pass<R, TIN, TOUT, TACCI, TACCO, FLAGS, 0>;
  }
  // the batched (work-list) kernels of the same configurations
  using FnW = void (*)(const PassWork);
  static FnW get_wl(int log2L, bool prefetch) {
    if constexpr (sizeof(R) == 4 && (FLAGS & F_CIRC) == 0) {
      if (prefetch) {
        switch (log2L) {
          case 8: return k_line_pass_fixed_wl<TIN, TOUT, TACCI, TACCO, FLAGS, 8>;
          case 9: return k_line_pass_fixed_wl<TIN, TOUT, TACCI, TACCO, FLAGS, 9>;
          case 10: return k_line_pass_fixed_wl<TIN, TOUT, TACCI, TACCO, FLAGS, 10>;
          case 11: return k_line_pass_fixed_wl<TIN, TOUT, TACCI, TACCO, FLAGS, 11>;
          default: break;
        }
      }
    }
    if constexpr (sizeof(R) == 4) {
      switch (log2L) {
        case 8: return k_line_pass_wl<R, TIN, TOUT, TACCI, TACCO, FLAGS, 8>;
        case 9: return k_line_pass_wl<R, TIN, TOUT, TACCI, TACCO, FLAGS, 9>;
        case 10: return k_line_pass_wl<R, TIN, TOUT, TACCI, TACCO, FLAGS, 10>;
        case 11: return k_line_pass_wl<R, TIN, TOUT, TACCI, TACCO, FLAGS, 11>;
        default: break;
      }
    }
    return k_line_pass_wl<R, TIN, TOUT, TACCI, TACCO, FLAGS, 0>;
  }
  static cudaError_t allow_smem_wl() {
    cudaError_t e = cudaSuccess;
    for (int lg = 0; lg <= 12; ++lg) {
      if (lg != 0 && !(sizeof(R) == 4 && fixed_fft_length(lg))) continue;
      for (int pf = 0; pf < 2; ++pf) {
        const cudaError_t r = cudaFuncSetAttribute(get_wl(lg, pf != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kPassMaxSmem);
        if (e == cudaSuccess) e = r;
      }
    }
    return e;
  }
  // dynamic shared memory above 48 KB for every variant, once per process (thread-safe static init)
  static cudaError_t allow_smem() {
    cudaError_t e = cudaSuccess;
    for (int lg = 0; lg <= 12; ++lg) {
      if (lg != 0 && !(sizeof(R) == 4 && fixed_fft_length(lg))) continue;
      for (int pf = 0; pf < 2; ++pf) {
        const cudaError_t r = cudaFuncSetAttribute(get(lg, pf != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kPassMaxSmem);
        if (e == cudaSuccess) e = r;
      }
    }
    return e;
  }
};

// Algorithmic work of one launch: 5 L log2 L flops per complex FFT of length L per line, and
// bytes with every operand read once and every result written once.
template <typename R, typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS>
void pass_work(const PassParams& p, double& flops, double& bytes) {
  const double lines = (double)p.nlines, N = lines * p.n;
  int nfft = 0;
  if (FLAGS & F_DST) nfft += (FLAGS & F_CIRC) ? 2 : 1;
  if (FLAGS & F_LAM) nfft += (FLAGS & F_CIRC) ? 2 : 1;
  if (FLAGS & (F_TOEP_X | F_TOEP_ACC)) nfft += 2;
  flops = lines * nfft * 5.0 * p.L * p.log2L;
  bytes = N * sizeof(TIN);
  if (FLAGS & F_INSCALE) bytes += N * sizeof(double2);
  if ((FLAGS & F_DST) && p.out) bytes += N * sizeof(TOUT) * (p.z_add ? 2 : 1);
  if (FLAGS & F_LAM) bytes += N * sizeof(cv<R>);
  if ((FLAGS & F_DSCALE) && p.dfac) bytes += N * sizeof(cv<R>);
  if ((FLAGS & F_TOEP_X) && p.Dr) bytes += N * sizeof(R);
  if (FLAGS & (F_TOEP_X | F_TOEP_ACC)) bytes += N * sizeof(TACCO) + (p.acc_in ? N * sizeof(TACCI) : 0.0);
  if (FLAGS & F_DOT0) {
    bytes += N * sizeof(double2);
    flops += 4.0 * N;
  }
}

// Key of a pass configuration for the autotuner: everything that selects the kernel and its geometry
// (flags, compute precision, operand storage, axis).
template <typename R, typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS>
unsigned long long pass_key(const rfnse_ctx* c, const PassParams& p) {
  int axis = 0;
  for (int a = 0; a < c->d; ++a)
    if (c->stride[a] == p.stride && c->n[a] == p.n) axis = a;
  unsigned long long k = (unsigned long long)FLAGS;
  k |= (unsigned long long)(sizeof(R) == 4) << 8;
  k |= (unsigned long long)(sizeof(TIN) == 16) << 9;
  k |= (unsigned long long)(sizeof(TOUT) == 16) << 10;
  k |= (unsigned long long)(sizeof(TACCI) == 16) << 11;
  k |= (unsigned long long)(sizeof(TACCO) == 16) << 12;
  k |= (unsigned long long)axis << 13;
  return k;
}

// The geometry a pass gets without tuning: lines per block and threads per line from pass_geometry /
// pass_geometry_fixed, and on grids of up to about four waves the prefetching kernel (k_line_pass_fixed,
// ~105 registers, faster there: 2-D 511^2 fused x-pass 18.0 -> 15.2 us), otherwise k_line_pass with its
// higher occupancy (3-D 255^3: equal or slightly faster).
template <int FLAGS>
PassGeom default_pass_geometry(const PassParams& p, bool fixed) {
  const bool xax = (p.stride == 1);
  PassGeom g{};
  if (fixed) pass_geometry_fixed(p.L, xax, xax ? p.nlines : p.stride, p.nlines, g.nt, g.B);
  else pass_geometry(p.L, xax, xax ? p.nlines : p.stride, g.nt, g.B);
  const long long grid_est =
      xax ? (p.nlines + g.B - 1) / g.B : ((p.stride + g.B - 1) / g.B) * (p.nlines / p.stride);
  g.variant = (fixed && !(FLAGS & F_CIRC) && grid_est <= 4 * 152) ? 1 : 0;
  return g;
}

// Launch one pass with an explicit geometry g (lines per block B, threads per line nt, kernel variant:
// 1 = the prefetching fixed-length kernel).  A geometry the kernels cannot run (threads beyond the
// launch bound, a thread count the FFT does not support, shared memory beyond the opt-in limit) is
// refused before any launch: inside a stream capture a failed launch would invalidate the capture.
template <typename R, typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS>
cudaError_t launch_pass_geom(rfnse_ctx* c, PassParams p, cudaStream_t s, const PassGeom& g) {
  using V = cv<R>;
  const bool xax = (p.stride == 1);
  const bool fixed = sizeof(R) == 4 && fixed_fft_length(p.log2L);
  p.B = g.B;
  p.nt = g.nt;
  const bool prefetch = fixed && !(FLAGS & F_CIRC) && g.variant == 1;
  if (p.B < 1 || (p.B & (p.B - 1)) != 0 || p.B * p.nt > kPassMaxThreads || p.B * p.nt < 1)
    return cudaErrorInvalidConfiguration;
  if (fixed ? (p.nt != (p.L >> kFixedLogR)) : (p.nt != p.L / 4 && p.nt != p.L / 8))
    return cudaErrorInvalidConfiguration;
  if (p.L != 2 * (p.n + 1)) return cudaErrorInvalidConfiguration;  // the kernels index with n = L/2 - 1
  p.dst_scale_f = (float)p.dst_scale;
  p.ca_f = make_float2((float)p.ca.x, (float)p.ca.y);
  p.cb_f = make_float2((float)p.cb.x, (float)p.cb.y);
  p.log2B = 0;
  while ((1 << p.log2B) < p.B) ++p.log2B;
  long long grid;
  if (xax) {
    grid = (p.nlines + p.B - 1) / p.B;
    p.tiles_inner = 1;
  } else {
    p.tiles_inner = (p.stride + p.B - 1) / p.B;
    const long long nhi = p.nlines / p.stride;
    grid = p.tiles_inner * nhi;
  }
  // tile; twiddles staged in shared memory (all but the fixed-length passes of k_line_pass, which read
  // them through L1); z of the x-Toeplitz pass saved in shared memory (k_line_pass only)
  size_t smem = ((size_t)p.B * fft_line_stride(p.L) + ((fixed && !prefetch) ? 0 : p.L)) * sizeof(V);
  if ((FLAGS & F_TOEP_X) && !prefetch) smem += (size_t)p.B * p.n * sizeof(V);
  if (smem > kPassMaxSmem) return cudaErrorInvalidConfiguration;
  using K = PassKernels<R, TIN, TOUT, TACCI, TACCO, FLAGS>;
  const auto kern = K::get(fixed ? p.log2L : 0, prefetch);
  static const cudaError_t attr_err = K::allow_smem();
  if (attr_err != cudaSuccess) return attr_err;
  if constexpr ((FLAGS & F_DOT0) != 0) {  // too many partials for the Arnoldi kernel to sum: plain pass
    if (grid > kDot0MaxBlocks || grid <= 0) {
      c->dot0_blocks = 0;
      return launch_pass_geom<R, TIN, TOUT, TACCI, TACCO, FLAGS & ~F_DOT0>(c, p, s, g);
    }
    c->dot0_blocks = (int)grid;
  }
  if (grid <= 0) return cudaSuccess;
  const int kind = FLAGS | (sizeof(R) == 4 ? 256 : 0);
  const bool prof = c->prof_kind != 0 && ((c->prof_kind | F_INSCALE | F_DOT0) == (kind | F_INSCALE | F_DOT0));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof) {
    while (c->prof_used + 2 > c->prof_events.size()) {
      cudaEvent_t ev;
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return e;
      c->prof_events.push_back(ev);
    }
    e0 = c->prof_events[c->prof_used];
    e1 = c->prof_events[c->prof_used + 1];
    c->prof_used += 2;
    cudaEventRecord(e0, s);
  }
  if (c->debug) {  // the tiles must cover the grid's lines exactly once
    const long long covered = xax ? grid * p.B : p.tiles_inner * p.B * (p.nlines / p.stride);
    const long long spare = xax ? (grid - 1) * p.B : (p.tiles_inner - 1) * p.B * (p.nlines / p.stride);
    if (p.nlines * p.n != c->N || covered < p.nlines || spare >= p.nlines ||
        (!xax && p.nlines % p.stride != 0)) {
      c->err = "debug check: line-pass geometry does not cover the grid";
      return cudaErrorInvalidConfiguration;
    }
  }
  {
    NvtxRange range("rfnse pass");
    kern<<<(unsigned)grid, p.B * p.nt, smem, s>>>(p);
  }
  count_launch();
  if (prof) {
    cudaEventRecord(e1, s);
    double fl, by;
    pass_work<R, TIN, TOUT, TACCI, TACCO, FLAGS>(p, fl, by);
    c->prof_flops += fl;
    c->prof_bytes += by;
  }
  cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
  if (c->debug && cudaStreamIsCapturing(s, &cap_st) == cudaSuccess && cap_st == cudaStreamCaptureStatusNone) {
    char what[96];
    std::snprintf(what, sizeof what, "line pass (flags %d, %s, axis stride %lld)", FLAGS,
                  sizeof(R) == 4 ? "FP32" : "FP64", p.stride);
    const void* outs[3] = {(FLAGS & (F_DST | F_DSCALE)) ? p.out : nullptr,
                           (FLAGS & (F_TOEP_X | F_TOEP_ACC)) ? p.acc_out : nullptr,
                           (FLAGS & F_INSCALE) ? (const void*)p.copy_out : nullptr};
    const int elems[3] = {(int)sizeof(TOUT), (int)sizeof(TACCO), 16};
    if (p.gdyn) outs[0] = outs[2] = nullptr;  // device-resolved operands: not known on the host
    return debug_after_pass(c, s, what, outs, elems, 3, c->N);
  }
  return cudaGetLastError();
}

// The geometries the autotuner tries for a pass: every power-of-two tile that fits the launch bound,
// the lines available and the shared memory; both FFT thread schedules of the runtime-length FFT (one
// or two radix-4 butterflies per thread); both kernels of the fixed-length FP32 FFT.
template <int FLAGS>
std::vector<PassGeom> pass_candidates(const PassParams& p, bool fixed, size_t elem) {
  std::vector<PassGeom> out;
  const bool xax = (p.stride == 1);
  const long long avail = xax ? p.nlines : p.stride;
  std::vector<int> nts;
  if (fixed) nts.push_back(p.L >> kFixedLogR);
  else {
    if (p.L / 4 <= kPassMaxThreads) nts.push_back(p.L / 4);
    if (p.L / 8 >= 1) nts.push_back(p.L / 8);
  }
  for (int nt : nts)
    for (int B = 1; B * nt <= kPassMaxThreads && B <= 64; B <<= 1) {
      if (B > 1 && B > avail) break;
      for (int variant = 0; variant < ((fixed && !(FLAGS & F_CIRC)) ? 2 : 1); ++variant) {
        const bool pf = variant == 1;
        size_t smem = ((size_t)B * fft_line_stride(p.L) + ((fixed && !pf) ? 0 : p.L)) * elem;
        if ((FLAGS & F_TOEP_X) && !pf) smem += (size_t)B * p.n * elem;
        if (smem > kPassMaxSmem) continue;
        out.push_back(PassGeom{B, nt, variant});
      }
    }
  return out;
}

// A pass of one instance recorded for a lock-step batch: its key, parameters and geometry, and the
// launcher of the batched kernel for a group of instances that run the same pass with the same FFT
// length.  grids receives every member's tile count; *dot0 whether the partials of <v_0, w> were
// written (F_DOT0 passes; 0 when some member's grid is too large for the Arnoldi kernel to sum).
struct ParamRecord {
  unsigned long long key = 0;
  PassParams p{};
  PassGeom geom{};
  bool df = false;  // double-float residual pass (toep_df.cu)
  std::function<cudaError_t(std::vector<PassParams>&, const PassGeom&, TableArena&, cudaStream_t,
                            std::vector<long long>&, int*)>
      group;
};

// The geometry of a batched launch over instances with the same FFT length on this axis: the default
// tile for the combined number of lines (on strided axes at most the smallest stride), the prefetching
// kernel while the combined grid stays within about four waves.
template <int FLAGS>
PassGeom group_pass_geometry(const std::vector<PassParams>& ps, bool fixed) {
  const PassParams& p0 = ps[0];
  const bool xax = (p0.stride == 1);
  long long avail = xax ? 0 : (1LL << 62), lines = 0;
  for (const PassParams& p : ps) {
    lines += p.nlines;
    if (xax) avail += p.nlines;
    else if (p.stride < avail) avail = p.stride;
  }
  PassGeom g{};
  if (fixed) pass_geometry_fixed(p0.L, xax, avail, lines, g.nt, g.B);
  else pass_geometry(p0.L, xax, avail, g.nt, g.B);
  long long grid = 0;
  for (const PassParams& p : ps)
    grid += xax ? (p.nlines + g.B - 1) / g.B : ((p.stride + g.B - 1) / g.B) * (p.nlines / p.stride);
  g.variant = (fixed && !(FLAGS & F_CIRC) && grid <= 4 * 152) ? 1 : 0;
  return g;
}

// One batched launch of a pass over a group of instances (same configuration and FFT length): block b
// runs tile b - start[i] of member i.  The members' parameter blocks and tile offsets go into the
// arena.  Geometry gin (gin.B = 0: group_pass_geometry), checked as in launch_pass_geom.
template <typename R, typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS>
cudaError_t launch_pass_group(std::vector<PassParams>& ps, const PassGeom& gin, TableArena& ar, cudaStream_t s,
                              std::vector<long long>& grids, int* dot0) {
  using V = cv<R>;
  if (ps.empty()) return cudaSuccess;
  const int L = ps[0].L;
  const bool fixed = sizeof(R) == 4 && fixed_fft_length(ps[0].log2L);
  const PassGeom g = gin.B > 0 ? gin : group_pass_geometry<FLAGS>(ps, fixed);  // B = 0: the default
  const bool prefetch = fixed && !(FLAGS & F_CIRC) && g.variant == 1;
  if (g.B < 1 || (g.B & (g.B - 1)) != 0 || g.B * g.nt > kPassMaxThreads || g.B * g.nt < 1)
    return cudaErrorInvalidConfiguration;
  if (fixed ? (g.nt != (L >> kFixedLogR)) : (g.nt != L / 4 && g.nt != L / 8)) return cudaErrorInvalidConfiguration;
  for (const PassParams& q : ps)
    if (q.L != L || q.L != 2 * (q.n + 1)) return cudaErrorInvalidConfiguration;  // n = L/2 - 1 in the kernels
  std::vector<long long> start(ps.size() + 1, 0);
  grids.assign(ps.size(), 0);
  bool dot_fits = true;
  for (size_t i = 0; i < ps.size(); ++i) {
    PassParams& p = ps[i];
    if (p.L != L) return cudaErrorInvalidValue;
    p.B = g.B;
    p.nt = g.nt;
    p.dst_scale_f = (float)p.dst_scale;
    p.ca_f = make_float2((float)p.ca.x, (float)p.ca.y);
    p.cb_f = make_float2((float)p.cb.x, (float)p.cb.y);
    p.log2B = 0;
    while ((1 << p.log2B) < p.B) ++p.log2B;
    long long grid;
    if (p.stride == 1) {
      grid = (p.nlines + p.B - 1) / p.B;
      p.tiles_inner = 1;
    } else {
      p.tiles_inner = (p.stride + p.B - 1) / p.B;
      grid = p.tiles_inner * (p.nlines / p.stride);
    }
    grids[i] = grid;
    start[i + 1] = start[i] + grid;
    if (grid > kDot0MaxBlocks) dot_fits = false;
  }
  if constexpr ((FLAGS & F_DOT0) != 0) {
    if (!dot_fits) {
      if (dot0) *dot0 = 0;
      return launch_pass_group<R, TIN, TOUT, TACCI, TACCO, FLAGS & ~F_DOT0>(ps, g, ar, s, grids, nullptr);
    }
    if (dot0) *dot0 = 1;
  }
  size_t smem = ((size_t)g.B * fft_line_stride(L) + ((fixed && !prefetch) ? 0 : L)) * sizeof(V);
  if ((FLAGS & F_TOEP_X) && !prefetch) smem += (size_t)g.B * ps[0].n * sizeof(V);
  if (smem > kPassMaxSmem) return cudaErrorInvalidConfiguration;
  if (start.back() <= 0) return cudaSuccess;
  using K = PassKernels<R, TIN, TOUT, TACCI, TACCO, FLAGS>;
  static const cudaError_t attr_err = K::allow_smem_wl();
  if (attr_err != cudaSuccess) return attr_err;
  const void* dp = ar.put(ps.data(), sizeof(PassParams) * ps.size());
  const void* ds = ar.put(start.data(), sizeof(long long) * start.size());
  if (!dp || !ds) return cudaErrorMemoryAllocation;
  PassWork w{static_cast<const PassParams*>(dp), static_cast<const long long*>(ds), (int)ps.size()};
  {
    NvtxRange range("rfnse pass group");
    K::get_wl(fixed ? ps[0].log2L : 0, prefetch)<<<(unsigned)start.back(), g.B * g.nt, smem, s>>>(w);
  }
  count_launch();
  return cudaGetLastError();
}

template <typename R, typename TIN, typename TOUT, typename TACCI, typename TACCO, int FLAGS>
cudaError_t launch_pass(rfnse_ctx* c, PassParams p, cudaStream_t s) {
  const bool fixed = sizeof(R) == 4 && fixed_fft_length(p.log2L);
  PassGeom g = default_pass_geometry<FLAGS>(p, fixed);
  if (c->param_rec) {  // a lock-step batch records the pass instead of launching it
    ParamRecord r;
    r.key = pass_key<R, TIN, TOUT, TACCI, TACCO, FLAGS>(c, p);
    r.p = p;
    r.geom = g;
    r.group = [](std::vector<PassParams>& ps, const PassGeom& gg, TableArena& ar, cudaStream_t st,
                 std::vector<long long>& grids, int* dot0) {
      return launch_pass_group<R, TIN, TOUT, TACCI, TACCO, FLAGS>(ps, gg, ar, st, grids, dot0);
    };
    c->param_rec->push_back(std::move(r));
    return cudaSuccess;
  }
  if (c->tune_rec || !c->tune.empty()) {
    const unsigned long long key = pass_key<R, TIN, TOUT, TACCI, TACCO, FLAGS>(c, p);
    if (c->tune_rec) {  // rfnse_autotune is recording the solver's pass configurations
      bool seen = false;
      for (const TuneRecord& r : *c->tune_rec) seen = seen || r.key == key;
      if (!seen) {
        TuneRecord r;
        r.key = key;
        r.dflt = g;
        r.cands = pass_candidates<FLAGS>(p, fixed, sizeof(cv<R>));
        r.launch = [c, p, s](const PassGeom& gg) { return launch_pass_geom<R, TIN, TOUT, TACCI, TACCO, FLAGS>(c, p, s, gg); };
        c->tune_rec->push_back(std::move(r));
      }
    } else {
      const auto it = c->tune.find(key);
      if (it != c->tune.end()) {
        g = it->second;
        c->tuned_launches += 1;
      }
    }
  }
  return launch_pass_geom<R, TIN, TOUT, TACCI, TACCO, FLAGS>(c, p, s, g);
}

}  // namespace rfnse
