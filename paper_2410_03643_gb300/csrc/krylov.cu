// Norms, cycle start, back-substitution, solution updates and pointwise kernels of the GMRES solve
// (paper Sec. 5, "PGMRES") as the host-driven loops use them; the Arnoldi step itself (modified
// Gram-Schmidt, Givens) is the cooperative kernel of control.cu in both loop forms.  Krylov vectors
// are complex FP64 with the real inner product <a, b> = Re(a^H b), which is the Euclidean inner
// product of the real block vectors [Im; Re] of Sec. 3.
#include <cmath>
#include <string>
#include "internal.cuh"
#include "cplx.cuh"
#include "dfloat.cuh"

namespace rfnse {

std::atomic<long long> g_kernel_launches{0};

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
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

// Store this block's partial; return true in every thread of the last block to arrive, which then
// owns the final fixed-order sum.
__device__ __forceinline__ bool arrive_last(double part, double* partials, unsigned* counter) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = part;
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

__device__ __forceinline__ double final_sum(const double* partials, unsigned* counter, double* sh) {
  __threadfence();
  double v = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += ((volatile const double*)partials)[i];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) *counter = 0u;
  return v;
}

// beta = ||x||, 1/beta, g = beta e_1; clears the column state of a new cycle.
__global__ void __launch_bounds__(kRedThreads) k_norm(const double2* __restrict__ x, GmresState* gs, long long N,
                                                      double* partials, unsigned* counter) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    acc += v.x * v.x + v.y * v.y;
  }
  const double part = block_sum(acc, sh);
  if (arrive_last(part, partials, counter)) {
    const double s = final_sum(partials, counter, sh);
    if (threadIdx.x == 0) {
      const double b = sqrt(s);
      gs->beta = b;
      gs->inv_beta = (b > 0.0) ? 1.0 / b : 0.0;
      gs->g[0] = b;
      for (int i = 1; i <= kMaxM; ++i) gs->g[i] = 0.0;
      gs->done = isfinite(b) ? 0 : 3;
    }
  }
}

__global__ void k_start_cycle(GmresState* gs, double ref, double tol) {
  gs->ref = (ref > 0.0) ? ref : gs->beta;
  gs->tol = tol;
  gs->relres = gs->beta / gs->ref;
  gs->j = 0;  // the cooperative Arnoldi kernel takes the column index from the state
  gs->it = 0;
  gs->err = 0;
}

// y = R^{-1} g on the leading k x k triangle (single thread; k <= 64).
__global__ void k_backsolve(GmresState* gs, int k) {
  const int ld = kMaxM + 1;
  for (int i = k - 1; i >= 0; --i) {
    double s = gs->g[i];
    for (int jj = i + 1; jj < k; ++jj) s -= gs->H[(size_t)jj * ld + i] * gs->y[jj];
    gs->y[i] = s / gs->H[(size_t)i * ld + i];
  }
}

// out = sum_{i<k} y_i V_i
__global__ void k_combine(const double2* __restrict__ V, long long ldv, const GmresState* gs, int k,
                          double2* __restrict__ out, long long N) {
  __shared__ double y[kMaxM];
  for (int t = threadIdx.x; t < k; t += blockDim.x) y[t] = gs->y[t];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double2 a = make_double2(0.0, 0.0);
    for (int q = 0; q < k; ++q) {
      const double2 v = V[(size_t)q * ldv + i];
      a.x += y[q] * v.x;
      a.y += y[q] * v.y;
    }
    out[i] = a;
  }
}

// x += sum_{i<k} y_i Z_i  (Z in FP32, accumulation in FP64)
__global__ void k_combine_f32_add(const float2* __restrict__ Z, long long ldz, const GmresState* gs, int k,
                                  double2* __restrict__ x, long long N) {
  __shared__ double y[kMaxM];
  for (int t = threadIdx.x; t < k; t += blockDim.x) y[t] = gs->y[t];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double2 a = x[i];
    for (int q = 0; q < k; ++q) {
      const float2 v = Z[(size_t)q * ldz + i];
      a.x += y[q] * df_f2d(v.x);  // exact, without an FP64-pipe conversion
      a.y += y[q] * df_f2d(v.y);
    }
    x[i] = a;
  }
}

// D = rho dt |u|^2, or rho dt |(u + u2)/2|^2 when u2 is given.
__global__ void k_diag(const double2* __restrict__ u, const double2* __restrict__ u2, double* __restrict__ D,
                       double rho_dt, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double2 v = u[i];
    if (u2) {
      const double2 b = u2[i];
      v.x = 0.5 * (v.x + b.x);
      v.y = 0.5 * (v.y + b.y);
    }
    D[i] = rho_dt * (v.x * v.x + v.y * v.y);
  }
}

// f = -i b
__global__ void k_neg_i(const double2* __restrict__ b, double2* __restrict__ f, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = b[i];
    f[i] = make_double2(v.y, -v.x);
  }
}

// D in FP32 and the per-point factor of the (omega I + D_d) sub-solve with the 2 omega of F~^{-1}
// (eq. 'taupre'): 2w/((w+1) - iD) = 2w((w+1) + iD)/((w+1)^2 + D^2), in FP64 and FP32.
__global__ void k_prep_D(const double* __restrict__ D, float* __restrict__ D32, double2* __restrict__ dfac64,
                         float2* __restrict__ dfac32, double omega, long long N) {
  const double w1 = omega + 1.0, two_w = 2.0 * omega;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double d = D[i];
    const double s = two_w / (w1 * w1 + d * d);
    const double2 f = make_double2(s * w1, s * d);
    D32[i] = (float)d;
    dfac64[i] = f;
    dfac32[i] = make_float2((float)f.x, (float)f.y);
  }
}

// From the final FP64 residual r = f - x - i(T - D)x of a solve: Tx = s (D x - i (f - x - r)).
// (s = 2 turns the first step's (T/2) x into T x.)
__global__ void k_tu_from_residual(const double* __restrict__ D, const double2* __restrict__ f,
                                   const double2* __restrict__ x, const double2* __restrict__ r,
                                   double2* __restrict__ Tu, double s, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 fv = f[i], xv = x[i], rv = r[i];
    const double d = D[i];
    const double qx = fv.x - xv.x - rv.x, qy = fv.y - xv.y - rv.y;
    Tu[i] = make_double2(s * (d * xv.x + qy), s * (d * xv.y - qx));
  }
}

// One steady step's pointwise set-up in the mixed form, with T u^{n-1} cached: D = rho dt |u^n|^2
// (as k_diag), the right-hand side f = u^{n-1} - i (T u^{n-1} - D u^{n-1}) (paper Sec. 2, the block
// form's f = -i b with b = (T - D + iI) u^{n-1}) and the tables of k_prep_D, in one sweep.  With
// dfac64 null (the mixed form's solves read only the FP32 tables) the FP32 factor is computed in
// FP32: the FP64 division per point made this sweep FP64-bound (GB300 issues two FP64 FMAs per SM and
// cycle), and the preconditioner needs the factor only to FP32 accuracy.
__global__ void k_step_prep(const double2* __restrict__ uc, const double2* __restrict__ up,
                            const double2* __restrict__ Tup, double* __restrict__ D, double2* __restrict__ f,
                            float* __restrict__ D32, double2* __restrict__ dfac64, float2* __restrict__ dfac32,
                            double rho_dt, double omega, long long N, double* __restrict__ nrm_part) {
  __shared__ double sh[32];
  const double w1 = omega + 1.0, two_w = 2.0 * omega;
  const float w1f = (float)w1, two_wf = (float)two_w;
  double nacc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = uc[i], uv = up[i], tv = Tup[i];
    const double d = rho_dt * (v.x * v.x + v.y * v.y);
    D[i] = d;
    const double px = tv.x - d * uv.x, py = tv.y - d * uv.y;
    const double2 fv = make_double2(uv.x + py, uv.y - px);
    f[i] = fv;
    nacc = fma(fv.x, fv.x, nacc);
    nacc = fma(fv.y, fv.y, nacc);
    const float df = (float)d;
    D32[i] = df;
    if (dfac64) {
      const double s = two_w / (w1 * w1 + d * d);
      const double2 fac = make_double2(s * w1, s * d);
      dfac64[i] = fac;
      dfac32[i] = make_float2((float)fac.x, (float)fac.y);
    } else {
      const float sf = two_wf / fmaf(df, df, w1f * w1f);
      dfac32[i] = make_float2(sf * w1f, sf * df);
    }
  }
  if (nrm_part) {  // this block's share of ||f||^2 for the solve's norm kernel (uniform branch)
    nacc = block_sum(nacc, sh);
    if (threadIdx.x == 0) nrm_part[blockIdx.x] = nacc;
  }
}

__global__ void k_zero(double2* __restrict__ x, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    x[i] = make_double2(0.0, 0.0);
}

// Count the non-finite components of n complex values (FP32 or FP64 storage) into *count.
__global__ void k_count_nonfinite(const void* __restrict__ p, long long n, int is_double, int* count) {
  int bad = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (is_double) {
      const double2 v = reinterpret_cast<const double2*>(p)[i];
      bad += !isfinite(v.x) || !isfinite(v.y);
    } else {
      const float2 v = reinterpret_cast<const float2*>(p)[i];
      bad += !isfinite(v.x) || !isfinite(v.y);
    }
  }
  if (bad) atomicAdd(count, bad);
}

cudaError_t debug_after_pass(rfnse_ctx* c, cudaStream_t s, const char* what, const void* const* outs,
                             const int* elems, int nout, long long count) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    c->err = std::string("debug check after ") + what + ": " + cudaGetErrorString(e);
    return e;
  }
  if (!c->dbg_count || !c->dbg_first.empty()) return cudaSuccess;
  for (int k = 0; k < nout; ++k) {
    if (!outs[k]) continue;
    int h = 0;
    e = cudaMemsetAsync(c->dbg_count, 0, sizeof(int), s);
    if (e == cudaSuccess) {
      k_count_nonfinite<<<152 * 4, 256, 0, s>>>(outs[k], count, elems[k] == 16, c->dbg_count);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, c->dbg_count, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (h > 0) {
      c->dbg_first = std::string(what) + ": " + std::to_string(h) + " non-finite values in output " + std::to_string(k);
      return cudaSuccess;
    }
  }
  return cudaSuccess;
}

static inline unsigned ew_blocks(long long N) {
  long long b = (N + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

void launch_norm(const double2* x, GmresState* gs, long long N, int blocks, double* partials, unsigned* counter,
                 cudaStream_t s) {
  count_launch();
  k_norm<<<blocks, kRedThreads, 0, s>>>(x, gs, N, partials, counter);
}
void launch_start_cycle(GmresState* gs, double ref, double tol, cudaStream_t s) {
  count_launch();
  k_start_cycle<<<1, 1, 0, s>>>(gs, ref, tol);
}
void launch_backsolve(GmresState* gs, int k, cudaStream_t s) {
  count_launch();
  k_backsolve<<<1, 1, 0, s>>>(gs, k);
}
void launch_combine(const double2* V, long long ldv, const GmresState* gs, int k, double2* out, long long N,
                    cudaStream_t s) {
  count_launch();
  k_combine<<<ew_blocks(N), 256, 0, s>>>(V, ldv, gs, k, out, N);
}
void launch_combine_f32_add(const float2* Z, long long ldz, const GmresState* gs, int k, double2* x, long long N,
                            cudaStream_t s) {
  count_launch();
  k_combine_f32_add<<<ew_blocks(N), 256, 0, s>>>(Z, ldz, gs, k, x, N);
}
void launch_diag(const double2* u, const double2* u2, double* D, double rho_dt, long long N, cudaStream_t s) {
  count_launch();
  k_diag<<<ew_blocks(N), 256, 0, s>>>(u, u2, D, rho_dt, N);
}
void launch_neg_i(const double2* b, double2* f, long long N, cudaStream_t s) {
  count_launch();
  k_neg_i<<<ew_blocks(N), 256, 0, s>>>(b, f, N);
}
void launch_prep_D(const double* D, float* D32, double2* dfac64, float2* dfac32, double omega, long long N,
                   cudaStream_t s) {
  count_launch();
  k_prep_D<<<ew_blocks(N), 256, 0, s>>>(D, D32, dfac64, dfac32, omega, N);
}
void launch_tu_from_residual(const double* D, const double2* f, const double2* x, const double2* r, double2* Tu,
                             double scale, long long N, cudaStream_t s) {
  count_launch();
  k_tu_from_residual<<<ew_blocks(N), 256, 0, s>>>(D, f, x, r, Tu, scale, N);
}
int step_prep_blocks(long long N) { return (int)ew_blocks(N); }
void launch_step_prep(rfnse_ctx* c, const double2* uc, const double2* up, const double2* Tup, cudaStream_t s,
                      double* nrm_part) {
  count_launch();
  k_step_prep<<<ew_blocks(c->N), 256, 0, s>>>(uc, up, Tup, c->D, c->f, c->D32,
                                              c->p.precision == 1 ? nullptr : c->dfac64, c->dfac32,
                                              c->p.rho * c->p.dt, c->p.omega, c->N, nrm_part);
}
void launch_zero(double2* x, long long N, cudaStream_t s) { k_zero<<<ew_blocks(N), 256, 0, s>>>(x, N); }

__global__ void k_differs(const double2* __restrict__ a, const double2* __restrict__ b, long long N, int* flag) {
  int d = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 u = a[i], v = b[i];
    d |= (__double_as_longlong(u.x) != __double_as_longlong(v.x)) | (__double_as_longlong(u.y) != __double_as_longlong(v.y));
  }
  if (__syncthreads_or(d) && threadIdx.x == 0) atomicExch(flag, 1);
}
__global__ void k_clear_flag(int* flag) { *flag = 0; }
void launch_differs(const double2* a, const double2* b, long long N, int* flag, cudaStream_t s) {
  count_launch(2);
  k_clear_flag<<<1, 1, 0, s>>>(flag);
  k_differs<<<ew_blocks(N), 256, 0, s>>>(a, b, N, flag);
}

}  // namespace rfnse
