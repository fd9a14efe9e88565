// Set-up kernels, run once per context: FCD coefficients (paper Sec. 2.1), tau eigenvalues
// (Sec. 4), circulant eigenvalues of the Toeplitz embedding and FFT twiddles.
#include "internal.cuh"
#include "fft_fixed.cuh"

namespace rfnse {

// c_0 = Gamma(alpha+1)/Gamma(alpha/2+1)^2 and c_{k+1} = c_k (k - alpha/2)/(alpha/2 + k + 1), the ratio
// of consecutive terms of eq. 'coefficients' (Gamma(z+1) = z Gamma(z)).  Sequential: one thread.
__global__ void k_coefficients(double* c, int nmax, double alpha) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double half = 0.5 * alpha;
  const double g = tgamma(half + 1.0);
  double ck = tgamma(alpha + 1.0) / (g * g);
  c[0] = ck;
  for (int k = 0; k + 1 < nmax; ++k) {
    ck = ck * ((double)k - half) / (half + (double)k + 1.0);
    c[k + 1] = ck;
  }
}

// For one axis with n points and L = 2(n+1):
//   circ[k] = c_0 + 2 sum_{m=1}^{n-1} c_m cos(2 pi m k / L),  k = 0..L-1:
//     eigenvalues of the symmetric circulant of order L whose first column is
//     (c_0, c_1, .., c_{n-1}, 0, 0, 0, c_{n-1}, .., c_1), which holds T_0 (eq. 'equ2') in its
//     leading n x n block;
//   lam[k-1] = circ[k], k = 1..n: the eigenvalues of tau(T_0) = T_0 - HC(T_0) (eq. 'taudefine',
//     'taudiagonal'), i.e. c_0 + 2 sum_m c_m cos(pi m k/(n+1)).
//   tw: the per-stage twiddle table of a length-L FFT, FP64 in the layout of fft_line.cuh, FP32 in
//     that of fft_fixed.cuh for the lengths the FP32 passes compile with a fixed FFT.
// k_axis_eigen computes circ and lam, k_axis_tables the twiddles.
// The eigenvalue sums, one block of kEigThreads per k: thread t takes m = n - 1 - t, n - 1 - t - T, ...
// (each thread's terms in decreasing m), then a fixed-order block reduction (warp shuffles, then the
// warps in order), so every table entry is reproducible.
constexpr int kEigThreads = 128;
__global__ void __launch_bounds__(kEigThreads) k_axis_eigen(const double* __restrict__ c, int n, int L,
                                                           double* __restrict__ lam, double* __restrict__ circ) {
  __shared__ double red[kEigThreads / 32];
  const int k = blockIdx.x;
  const int period = L;  // cos(2 pi m k / L) has period L in (m k)
  double s = 0.0;
  for (int m = n - 1 - (int)threadIdx.x; m >= 1; m -= kEigThreads) {
    const long long mk = ((long long)m * k) % period;
    s += c[m] * cospi(2.0 * (double)mk / (double)L);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int w = 0; w < kEigThreads / 32; ++w) t += red[w];
  const double v = c[0] + 2.0 * t;
  circ[k] = v;
  if (k >= 1 && k <= n) lam[k - 1] = v;
}

__global__ void k_axis_tables(const double* __restrict__ c, int n, int L, double* __restrict__ lam,
                              double* __restrict__ circ, double2* __restrict__ tw64, float2* __restrict__ tw32) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  // twiddle entry k of the per-stage table of fft_line.cuh: stage Ns holds W_{4Ns}^{r kk},
  // r = 1..3, kk = 0..Ns-1, at (r-1) Ns + kk of its segment
  int log2L = 0;
  while ((1 << log2L) < L) ++log2L;
  int t = k, Ns = (log2L & 1) ? 2 : 4;
  while (Ns < L && t >= 3 * Ns) {
    t -= 3 * Ns;
    Ns <<= 2;
  }
  double sn = 0.0, cs = 1.0;
  if (Ns < L) {
    const int r = t / Ns + 1, kk = t - (r - 1) * Ns;
    // exp(-2 pi i r kk / (4 Ns)) = exp(-i pi (r kk)/(2 Ns)); the argument is an exact binary fraction
    sincospi((double)(r * kk) / (double)(2 * Ns), &sn, &cs);
  }
  tw64[k] = make_double2(cs, -sn);
  if (fixed_fft_length(log2L)) {  // the FP32 passes of these lengths use the fixed-length FFT's layout
    int R, ns, r, kk;
    fixed_twiddle_entry(log2L, kFixedLogR, k, R, ns, r, kk);
    double s2 = 0.0, c2 = 1.0;
    if (R > 1) sincospi(2.0 * (double)(r * kk) / (double)(R * ns), &s2, &c2);
    tw32[k] = make_float2((float)c2, (float)-s2);
  } else {
    tw32[k] = make_float2((float)cs, (float)-sn);
  }
}

// Strang-circulant comparator (Sec. 5, F_C), one axis with n points (n odd) and L = 2(n+1):
//   lamC[k] = c_0 + 2 sum_{m=1}^{(n-1)/2} c_m cos(2 pi m k/n), k < n: the eigenvalues of Strang's
//     circulant of T_0 (first column c_0..c_{(n-1)/2}, c_{(n-1)/2}..c_1);
//   chirp[j] = exp(i pi j^2/n), j < n (argument reduced mod 2n);
//   bspec[k] = (1/L) sum_j bt_j exp(-2 pi i jk/L), the spectrum of the Bluestein filter
//     bt_j = chirp[j] (0 <= j < n), bt_{L-j} = chirp[j] (0 < j < n), 0 otherwise, which is symmetric,
//     so bspec[k] = (1/L)(chirp[0] + 2 sum_{m=1}^{n-1} chirp[m] cos(2 pi m k/L)).
// With these a length-n DFT is X_k = conj(b_k) sum_j (x_j conj(b_j)) bt_{k-j} (jk = (j^2 + k^2 -
// (k-j)^2)/2): one length-L circular convolution, i.e. two FFTs of length L.
__device__ __forceinline__ double2 chirp_at(long long j, int n) {
  const long long q = (j * j) % (2LL * n);
  double sn, cs;
  sincospi((double)q / (double)n, &sn, &cs);
  return make_double2(cs, sn);
}

__global__ void k_circ_tables(const double* __restrict__ c, int n, int L, double* __restrict__ lamC,
                              double2* __restrict__ chirp64, float2* __restrict__ chirp32,
                              double2* __restrict__ bspec64, float2* __restrict__ bspec32) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  if (k < n) {
    double s = 0.0;
    for (int m = (n - 1) / 2; m >= 1; --m) {
      const long long mk = ((long long)m * k) % n;
      s += c[m] * cospi(2.0 * (double)mk / (double)n);
    }
    lamC[k] = c[0] + 2.0 * s;
    const double2 b = chirp_at(k, n);
    chirp64[k] = b;
    chirp32[k] = make_float2((float)b.x, (float)b.y);
  }
  double re = 0.0, im = 0.0;
  for (int m = n - 1; m >= 1; --m) {
    const double2 b = chirp_at(m, n);
    const long long mk = ((long long)m * k) % L;
    const double cw = cospi(2.0 * (double)mk / (double)L);
    re += b.x * cw;
    im += b.y * cw;
  }
  const double2 b0 = chirp_at(0, n);
  const double2 v = make_double2((b0.x + 2.0 * re) / L, (b0.y + 2.0 * im) / L);
  bspec64[k] = v;
  bspec32[k] = make_float2((float)v.x, (float)v.y);
}

// Per-mode factor of the (omega I + tau(T_d)) sub-solve in the DST basis (eq. 'taupre', '2Dtau'):
//   lamfac[g] = i dst_scale / (omega + i Lambda),  Lambda = sum_a mu_a lambda_a(k_a),
// where (k_0, k_1, k_2) are the (0-based) mode indices of grid index g, x fastest.  i dst_scale is
// the output scale of the DST-I computed from an FFT (folded in so the pass multiplies once).
// circ = 1 (the circulant comparator, DFT basis): lamfac[g] = dst_scale / (omega + i Lambda), with
// dst_scale = 1/(n_0 n_1 n_2), the scale of the unnormalised forward and inverse DFTs.
__global__ void k_lamfac(const double* __restrict__ lam0, const double* __restrict__ lam1,
                         const double* __restrict__ lam2, int n0, int n1, int n2, double mu0, double mu1,
                         double mu2, double omega, double dst_scale, int circ, double2* __restrict__ f64,
                         float2* __restrict__ f32, long long N) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    long long r = g;
    const int k0 = (int)(r % n0);
    r /= n0;
    const int k1 = (int)(r % n1);
    r /= n1;
    const int k2 = (int)r;
    double lam = mu0 * lam0[k0];
    if (lam1) lam += mu1 * lam1[k1];
    if (lam2) lam += mu2 * lam2[k2];
    // i s/(w + i lam) = s (lam + i w)/(w^2 + lam^2);  s/(w + i lam) = s (w - i lam)/(w^2 + lam^2)
    const double den = omega * omega + lam * lam;
    const double2 f = circ ? make_double2(dst_scale * omega / den, -dst_scale * lam / den)
                           : make_double2(dst_scale * lam / den, dst_scale * omega / den);
    f64[g] = f;
    f32[g] = make_float2((float)f.x, (float)f.y);
  }
}

__global__ void k_scale_circ(const double* __restrict__ circ, int L, double scale, double* __restrict__ c64,
                             float* __restrict__ c32) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  const double v = circ[k] * scale;
  c64[k] = v;
  c32[k] = (float)v;
}

void launch_setup_lamfac(const double* lam0, const double* lam1, const double* lam2, int n0, int n1, int n2,
                         double mu0, double mu1, double mu2, double omega, double dst_scale, int circ,
                         double2* f64, float2* f32, long long N, cudaStream_t s) {
  long long blocks = (N + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launch();
  k_lamfac<<<(unsigned)blocks, 256, 0, s>>>(lam0, lam1, lam2, n0, n1, n2, mu0, mu1, mu2, omega, dst_scale, circ,
                                           f64, f32, N);
}

void launch_setup_circ(const double* c, int n, int L, double* lamC, double2* chirp64, float2* chirp32,
                       double2* bspec64, float2* bspec32, cudaStream_t s) {
  count_launch();
  k_circ_tables<<<(L + 127) / 128, 128, 0, s>>>(c, n, L, lamC, chirp64, chirp32, bspec64, bspec32);
}

void launch_scale_circ(const double* circ, int L, double scale, double* c64, float* c32, cudaStream_t s) {
  count_launch();
  k_scale_circ<<<(L + 127) / 128, 128, 0, s>>>(circ, L, scale, c64, c32);
}

void launch_setup_coefficients(double* c, int nmax, double alpha, cudaStream_t s) {
  count_launch();
  k_coefficients<<<1, 1, 0, s>>>(c, nmax, alpha);
}

void launch_setup_axis(const double* c, int n, int L, double* lam, double* circ, double2* tw64, float2* tw32,
                       cudaStream_t s) {
  count_launch(2);
  k_axis_eigen<<<L, kEigThreads, 0, s>>>(c, n, L, lam, circ);
  k_axis_tables<<<(L + 127) / 128, 128, 0, s>>>(c, n, L, lam, circ, tw64, tw32);
}

}  // namespace rfnse
