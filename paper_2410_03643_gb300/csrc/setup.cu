// Set-up kernels, run once per context: FCD coefficients (paper Sec. 2.1), tau eigenvalues
// (Sec. 4), circulant eigenvalues of the Toeplitz embedding and FFT twiddles.
#include "internal.cuh"

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
//   tw[k] = exp(-2 pi i k / L).
__global__ void k_axis_tables(const double* __restrict__ c, int n, int L, double* __restrict__ lam,
                              double* __restrict__ circ, double2* __restrict__ tw64, float2* __restrict__ tw32) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  const int period = L;  // cos(2 pi m k / L) has period L in (m k)
  double s = 0.0;
  for (int m = n - 1; m >= 1; --m) {
    const long long mk = ((long long)m * k) % period;
    s += c[m] * cospi(2.0 * (double)mk / (double)L);
  }
  const double v = c[0] + 2.0 * s;
  circ[k] = v;
  if (k >= 1 && k <= n) lam[k - 1] = v;
  double sn, cs;
  sincospi(2.0 * (double)k / (double)L, &sn, &cs);
  tw64[k] = make_double2(cs, -sn);
  tw32[k] = make_float2((float)cs, (float)-sn);
}

void launch_setup_coefficients(double* c, int nmax, double alpha, cudaStream_t s) {
  count_launch();
  k_coefficients<<<1, 1, 0, s>>>(c, nmax, alpha);
}

void launch_setup_axis(const double* c, int n, int L, double* lam, double* circ, double2* tw64, float2* tw32,
                       cudaStream_t s) {
  count_launch();
  k_axis_tables<<<(L + 127) / 128, 128, 0, s>>>(c, n, L, lam, circ, tw64, tw32);
}

}  // namespace rfnse
