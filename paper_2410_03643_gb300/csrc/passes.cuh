// Line passes: every transform of the method acts along one grid axis at a time.  A pass kernel
// stages B lines of one axis in shared memory, transforms them there, and fuses the pointwise
// work that follows.  Operations (compile-time flags, applied in this order):
//
//   F_INSCALE  multiply the loaded (FP64) input by a device scalar and write the scaled vector out
//              (this is v_{j+1} = w / h_{j+1,j} of the Arnoldi process, folded into the first pass)
//   F_DST      y = S x, S the orthonormal DST-I matrix [S]_{jk} = sqrt(2/(n+1)) sin(pi jk/(n+1))
//              (paper Sec. 4, eq. 'taudiagonal'; normalisation sqrt(2/(n+1))).  Computed from the odd
//              extension of x, a complex FFT of length L = 2(n+1): (S x)_k = i Y_k / sqrt(2(n+1)).
//   F_LAM      divide by (omega + i Lambda(k)), Lambda(k) = sum_a mu_a lambda^{(a)}_{k_a}, and apply S
//              again: the sub-solve with omega I + tau(T_d) in the DST basis (eq. 'taupre', '2Dtau').
//              Only on the last axis, when every other axis is already in the DST basis.
//   F_DSCALE   z = 2 omega / ((omega+1) - i D) * y: the sub-solve with omega I + D_d and the factor
//              2 omega of F~^{-1} (eq. 'taupre').  Stores z (or adds it to the output).
//   F_TOEP_X   t = mu_a T_0^{(a)} z by circulant embedding (length-L FFT, multiply by the circulant
//              eigenvalues, inverse FFT) and acc = add + a z + b (t - D z)          (first axis)
//   F_TOEP_ACC t = mu_a T_0^{(a)} z and acc = acc + b t                                   (other axes)
//
// With a = 1, b = i the Toeplitz passes give w = R z for the complex form R = I + i(T_d - D) of the
// real block matrix R_d of eq. 'positiveBlockForm' (u = y + iz  <->  x = [z; y]).
//
// Complex data are interleaved (re, im); x is the fastest axis.  Lines along x are contiguous; a
// tile of a strided axis is B lines adjacent in the fastest coordinate, so every global access of a
// tile row is B consecutive complex values.
#pragma once
#include <cstdint>
#include "cplx.cuh"
#include "fft_line.cuh"
#include "internal.cuh"

namespace rfnse {

enum : int {
  F_INSCALE = 1,
  F_DST = 2,
  F_LAM = 4,
  F_DSCALE = 8,
  F_TOEP_X = 16,
  F_TOEP_ACC = 32,
};

struct PassParams {
  const void* in;          // input vector (storage type TIN)
  void* out;               // DST / z output (storage type TOUT); may be null when not needed
  double2* copy_out;       // F_INSCALE: the scaled input is written here
  const double* in_scale;  // F_INSCALE: device scalar
  const double2* acc_in;   // F_TOEP_X: optional additive vector; F_TOEP_ACC: accumulator input
  double2* acc_out;        // Toeplitz result
  const double* D;         // diagonal D (physical positions)
  const void* tw;          // twiddle table exp(-2 pi i k/L), k < L, in the compute precision
  const double* lam[3];    // tau eigenvalues lambda^{(a)}_k of T_0 per axis (k = 1..n_a at index k-1)
  const double* circ;      // circulant eigenvalues of the embedded T_0 of this axis (length L)
  double mu[3];            // mu_a per axis (including the first-step factor 1/2)
  double omega;
  double toep_scale;       // mu_axis / L
  double dst_scale;        // 1/sqrt(2(n+1))
  double2 ca, cb;          // epilogue scalars a and b
  int n_ax[3];
  int d, axis;
  int n, L, log2L, nt, B;  // axis extent, FFT length, log2 L, threads per line, lines per block
  long long stride;        // element stride of the axis
  long long nlines;        // N / n
  long long tiles_inner;   // strided axes: ceil(stride / B)
  int z_add;               // F_DSCALE: out += z instead of out = z
};

template <typename R, typename TIN, typename TOUT, int FLAGS>
__global__ void __launch_bounds__(512) k_line_pass(const PassParams p) {
  using V = cv<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int L = p.L, n = p.n, Nh = L >> 1, Lp = L + 1, B = p.B;
  V* zsave = buf + (size_t)B * Lp;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const bool xax = (p.stride == 1);
  const V zero = cvec<R>::make((R)0, (R)0);

  long long line0 = 0, hi = 0, lo0 = 0;
  if (xax) {
    line0 = (long long)blockIdx.x * B;
  } else {
    hi = (long long)blockIdx.x / p.tiles_inner;
    lo0 = ((long long)blockIdx.x - hi * p.tiles_inner) * B;
  }
  // element e of the tile -> (line l, position pos), ordered for coalesced global access
  auto map = [&](int e, int& l, int& pos) {
    if (xax) { l = e / n; pos = e - l * n; }
    else { pos = e / B; l = e - pos * B; }
  };
  auto gidx = [&](int l, int pos, bool& valid) -> long long {
    if (xax) {
      const long long ln = line0 + l;
      valid = ln < p.nlines;
      return ln * n + pos;
    }
    const long long lo = lo0 + l;
    valid = lo < p.stride;
    return lo + (long long)pos * p.stride + hi * p.stride * n;
  };

  // ---- load ---------------------------------------------------------------------------------
  const TIN* in = reinterpret_cast<const TIN*>(p.in);
  double sc = 1.0;
  if (FLAGS & F_INSCALE) sc = *p.in_scale;
  for (int e = tid; e < B * n; e += nthr) {
    int l, pos;
    map(e, l, pos);
    bool valid;
    const long long g = gidx(l, pos, valid);
    V v = zero;
    if (valid) {
      if (FLAGS & F_INSCALE) {
        double2 vd = reinterpret_cast<const double2*>(p.in)[g];
        vd.x *= sc;
        vd.y *= sc;
        p.copy_out[g] = vd;
        v = to_c<R>(vd);
      } else {
        v = to_c<R>(in[g]);
      }
    }
    buf[l * Lp + 1 + pos] = v;
    if (FLAGS & F_DST) {
      buf[l * Lp + L - 1 - pos] = cneg(v);      // odd extension y_{2(n+1)-j} = -x_j
    } else if (FLAGS & F_TOEP_X) {
      zsave[l * n + pos] = v;
    }
  }
  for (int l = tid; l < B; l += nthr) {
    buf[l * Lp] = zero;
    buf[l * Lp + Nh] = zero;
  }
  if (!(FLAGS & F_DST)) {                        // zero padding of the circulant embedding
    for (int e = tid; e < B * (Nh - 1); e += nthr) {
      const int l = e / (Nh - 1);
      buf[l * Lp + Nh + 1 + (e - l * (Nh - 1))] = zero;
    }
  }
  __syncthreads();

  const V* tw = reinterpret_cast<const V*>(p.tw);
  const R dsc = (R)p.dst_scale;

  // ---- sine transforms -----------------------------------------------------------------------
  if (FLAGS & F_DST) {
    fft_lines(buf, Lp, L, p.log2L, p.nt, tw, false);
    if (FLAGS & F_LAM) {
      for (int e = tid; e < B * n; e += nthr) {
        const int l = e / n;
        const int k = e - l * n + 1;                 // sine mode k = 1..n along this axis
        double lam = p.mu[p.axis] * p.lam[p.axis][k - 1];
        if (p.d > 1) {
          long long lo = xax ? 0 : lo0 + l;          // position in the faster (transformed) axes
          for (int b = 0; b < p.axis; ++b) {
            const long long kb = lo % p.n_ax[b];
            lo /= p.n_ax[b];
            lam += p.mu[b] * p.lam[b][kb];
          }
        }
        // i * dst_scale / (omega + i lam) = dst_scale (lam + i omega) / (omega^2 + lam^2)
        const double den = p.omega * p.omega + lam * lam;
        const V f = cvec<R>::make((R)(p.dst_scale * lam / den), (R)(p.dst_scale * p.omega / den));
        buf[l * Lp + k] = cmul(buf[l * Lp + k], f);
        buf[l * Lp + L - k] = cmul(buf[l * Lp + L - k], f);
      }
      for (int l = tid; l < B; l += nthr) {
        buf[l * Lp] = zero;
        buf[l * Lp + Nh] = zero;
      }
      __syncthreads();
      fft_lines(buf, Lp, L, p.log2L, p.nt, tw, false);
    }
  }

  // ---- DST output / D sub-solve ---------------------------------------------------------------
  if ((FLAGS & F_DST) && !(FLAGS & F_DSCALE)) {
    TOUT* out = reinterpret_cast<TOUT*>(p.out);
    for (int e = tid; e < B * n; e += nthr) {
      int l, pos;
      map(e, l, pos);
      bool valid;
      const long long g = gidx(l, pos, valid);
      if (valid) st_c(out + g, cmul_i(cscale(buf[l * Lp + 1 + pos], dsc)));
    }
  }
  if (FLAGS & F_DSCALE) {
    TOUT* out = reinterpret_cast<TOUT*>(p.out);
    const double w1 = p.omega + 1.0, two_w = 2.0 * p.omega;
    for (int e = tid; e < B * n; e += nthr) {
      int l, pos;
      map(e, l, pos);
      bool valid;
      const long long g = gidx(l, pos, valid);
      V y = cmul_i(cscale(buf[l * Lp + 1 + pos], dsc));
      V z = zero;
      if (valid) {
        const double Dj = p.D[g];
        const double den = w1 * w1 + Dj * Dj;
        // 2w / ((w+1) - i D) = 2w ((w+1) + i D) / ((w+1)^2 + D^2)
        const V f = cvec<R>::make((R)(two_w * w1 / den), (R)(two_w * Dj / den));
        z = cmul(y, f);
        if (out) {
          if (p.z_add) {
            const TOUT old = out[g];
            st_c(out + g, cadd(to_c<R>(old), z));
          } else {
            st_c(out + g, z);
          }
        }
      }
      if (FLAGS & (F_TOEP_X | F_TOEP_ACC)) {
        buf[l * Lp + 1 + pos] = z;
        if (FLAGS & F_TOEP_X) zsave[l * n + pos] = z;
      }
    }
    if (FLAGS & (F_TOEP_X | F_TOEP_ACC)) {
      for (int e = tid; e < B * (Nh - 1); e += nthr) {
        const int l = e / (Nh - 1);
        buf[l * Lp + Nh + 1 + (e - l * (Nh - 1))] = zero;
      }
      for (int l = tid; l < B; l += nthr) {
        buf[l * Lp] = zero;
        buf[l * Lp + Nh] = zero;
      }
    }
    __syncthreads();
  }

  // ---- Toeplitz product by circulant embedding -------------------------------------------------
  if (FLAGS & (F_TOEP_X | F_TOEP_ACC)) {
    fft_lines(buf, Lp, L, p.log2L, p.nt, tw, false);
    const R ts = (R)p.toep_scale;
    for (int e = tid; e < B * L; e += nthr) {
      const int l = e / L;
      const int k = e - l * L;
      buf[l * Lp + k] = cscale(buf[l * Lp + k], (R)__ldg(p.circ + k) * ts);
    }
    __syncthreads();
    fft_lines(buf, Lp, L, p.log2L, p.nt, tw, true);
    for (int e = tid; e < B * n; e += nthr) {
      int l, pos;
      map(e, l, pos);
      bool valid;
      const long long g = gidx(l, pos, valid);
      if (!valid) continue;
      const V tv = buf[l * Lp + 1 + pos];
      double2 t = make_double2((double)tv.x, (double)tv.y);
      double2 acc = p.acc_in ? p.acc_in[g] : make_double2(0.0, 0.0);
      if (FLAGS & F_TOEP_X) {
        const V zv = zsave[l * n + pos];
        const double2 z = make_double2((double)zv.x, (double)zv.y);
        const double Dj = p.D ? p.D[g] : 0.0;
        t.x -= Dj * z.x;
        t.y -= Dj * z.y;
        acc = cadd(acc, cmul(p.ca, z));
      }
      acc = cadd(acc, cmul(p.cb, t));
      p.acc_out[g] = acc;
    }
  }
}

// Threads per line and lines per block for an FFT length L.
inline void pass_geometry(int L, long long nlines_or_stride, int& nt, int& B) {
  nt = L / 8;
  int target = 256;
  if (nt > target) target = nt;
  B = target / nt;
  if (B < 1) B = 1;
  if (B > nlines_or_stride) B = (int)nlines_or_stride;
  if (B < 1) B = 1;
}

// Algorithmic work of one launch: 5 L log2 L flops per complex FFT of length L per line, and
// bytes with every operand read once and every result written once.
template <typename R, typename TIN, typename TOUT, int FLAGS>
void pass_work(const PassParams& p, double& flops, double& bytes) {
  const double lines = (double)p.nlines, N = lines * p.n;
  int nfft = 0;
  if (FLAGS & F_DST) ++nfft;
  if (FLAGS & F_LAM) ++nfft;
  if (FLAGS & (F_TOEP_X | F_TOEP_ACC)) nfft += 2;
  flops = lines * nfft * 5.0 * p.L * p.log2L;
  bytes = N * sizeof(TIN);
  if (FLAGS & F_INSCALE) bytes += N * sizeof(double2);
  if ((FLAGS & F_DST) && p.out) bytes += N * sizeof(TOUT) * (p.z_add ? 2 : 1);
  if (FLAGS & (F_DSCALE | F_TOEP_X)) bytes += N * sizeof(double);
  if (FLAGS & (F_TOEP_X | F_TOEP_ACC)) bytes += N * sizeof(double2) * (p.acc_in ? 2 : 1);
}

template <typename R, typename TIN, typename TOUT, int FLAGS>
cudaError_t launch_pass(rfnse_ctx* c, PassParams p, cudaStream_t s) {
  using V = cv<R>;
  const bool xax = (p.stride == 1);
  pass_geometry(p.L, xax ? p.nlines : p.stride, p.nt, p.B);
  long long grid;
  if (xax) {
    grid = (p.nlines + p.B - 1) / p.B;
    p.tiles_inner = 1;
  } else {
    p.tiles_inner = (p.stride + p.B - 1) / p.B;
    const long long nhi = p.nlines / p.stride;
    grid = p.tiles_inner * nhi;
  }
  size_t smem = (size_t)p.B * (p.L + 1) * sizeof(V);
  if (FLAGS & F_TOEP_X) smem += (size_t)p.B * p.n * sizeof(V);
  auto kern = k_line_pass<R, TIN, TOUT, FLAGS>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (grid <= 0) return cudaSuccess;
  const int kind = FLAGS | (sizeof(R) == 4 ? 256 : 0);
  const bool prof = c->prof_kind != 0 && ((c->prof_kind | F_INSCALE) == (kind | F_INSCALE));
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
  kern<<<(unsigned)grid, p.B * p.nt, smem, s>>>(p);
  count_launch();
  if (prof) {
    cudaEventRecord(e1, s);
    double fl, by;
    pass_work<R, TIN, TOUT, FLAGS>(p, fl, by);
    c->prof_flops += fl;
    c->prof_bytes += by;
  }
  return cudaGetLastError();
}

}  // namespace rfnse
