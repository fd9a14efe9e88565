// Device-side control of the GMRES solve (paper Sec. 5, "PGMRES"): the Arnoldi step with modified
// Gram-Schmidt, Givens rotations and the convergence test in one cooperative kernel, and the small
// kernels that start a solve or a cycle and decide, on the device, whether the next Arnoldi step,
// restart or refinement cycle runs.  With a CUDA graph whose conditional WHILE nodes read the
// handles these kernels set, a whole solve runs without the host.
#include <cooperative_groups.h>
#include <cmath>
#include "internal.cuh"
#include "coop.cuh"
#include "dfloat.cuh"

namespace rfnse {

// Arnoldi step j = gs->j: w holds A M^{-1} v_j.  Modified Gram-Schmidt (for i = 0..j:
// h_ij = <v_i, w>, w -= h_ij v_i; one sweep per i fusing the previous subtraction with the next dot),
// h_{j+1,j} = ||w||, the Givens update of column j and the convergence test; then the state for the
// next column (src = w, scale = 1/h_{j+1,j}, j + 1) and, if set_cond, the inner-loop condition.
// With pre_n > 0 the product pass that wrote w has also left pre_n block partials of h_0j = <v_0, w>:
// every block sums them in a fixed order and the first sweep (and its grid-wide sum) is skipped.
// Each sweep's grid-wide sum is one counted arrival (grid_sum); the norm's sum is taken by the last
// block to arrive, which finishes the step while the others leave.  A thread's elements are the same
// in every sweep, so w needs no grid-wide ordering between sweeps.
__global__ void __launch_bounds__(kCtlThreads) k_mgs_step(GmresState* gs, const double2* __restrict__ V,
                                                         long long ldv, double2* __restrict__ w, long long N,
                                                         double* partials, GridBarrier* bar, SolveCfg cfg,
                                                         cudaGraphConditionalHandle h_inner, int set_cond,
                                                         const double* __restrict__ pre_part, int pre_n) {
  __shared__ double sh[33];
  __shared__ double hc[kMaxM + 1];  // column j of H before the rotations (h_0j .. h_jj)
  const int j = gs->j;
  const int nb = gridDim.x;
  const long long start = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)nb * blockDim.x;
  double hprev = 0.0;
  int i0 = 0;
  if (pre_n > 0) {
    double v = 0.0;
    for (int b = threadIdx.x; b < pre_n; b += blockDim.x) v += pre_part[b];
    v = block_sum_c(v, sh);
    if (threadIdx.x == 0) sh[32] = v;
    __syncthreads();
    hprev = sh[32];
    i0 = 1;
  }
  if (threadIdx.x == 0) hc[0] = hprev;
  for (int i = i0; i <= j; ++i) {
    const double2* vp = (i > 0) ? V + (size_t)(i - 1) * ldv : nullptr;
    const double acc = mgs_sweep(w, V + (size_t)i * ldv, vp, hprev, N, start, stride);
    hprev = grid_sum(acc, partials + (size_t)(i & 1) * nb, &bar->count, (unsigned)(i - i0 + 1) * (unsigned)nb,
                     &gs->err, sh);
    if (threadIdx.x == 0) hc[i] = hprev;
  }
  // the norm sweep: w -= h_jj v_j, ||w||^2
  const double acc = mgs_sweep(w, nullptr, V + (size_t)j * ldv, hprev, N, start, stride);
  double nrm2;
  if (!grid_sum_last(acc, partials + (size_t)((j + 1) & 1) * nb, &bar->done, &bar->count, sh, &nrm2)) return;
  if (threadIdx.x < 32) {
    const int cont = givens_finish_warp(gs, j, nrm2, hc, w, cfg);
    if (threadIdx.x == 0 && set_cond) cudaGraphSetConditional(h_inner, cont ? 1u : 0u);
  }
}

// The same Arnoldi step on one thread-block cluster of CL CTAs (small grids: a sweep moves a few MB
// from L2, and the grid-wide barrier of k_mgs_step, global atomics and polling, costs more than the
// sweep).  Each CTA leaves its partial of a sweep in its own shared memory; after the cluster barrier
// (hardware, no polling) every CTA reads the CL partials through distributed shared memory in rank
// order, so all hold the same sum.  The other SMs stay free for concurrent work.
constexpr int kClThreads = 1024;
__global__ void __launch_bounds__(kClThreads) k_mgs_cluster(GmresState* gs, const double2* __restrict__ V,
                                                            long long ldv, double2* __restrict__ w, long long N,
                                                            SolveCfg cfg, cudaGraphConditionalHandle h_inner,
                                                            int set_cond, const double* __restrict__ pre_part,
                                                            int pre_n) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int nr = (int)cl.num_blocks();
  __shared__ double sh[32];
  __shared__ double part[2];  // this CTA's partial of the current sweep (by sweep parity)
  __shared__ double bc;
  __shared__ double hc[kMaxM + 1];  // column j of H before the rotations (h_0j .. h_jj)
  const int j = gs->j;
  double hprev = 0.0, nrm2 = 0.0;
  int i0 = 0;
  if (pre_n > 0) {
    hprev = fixed_sum(pre_part, pre_n, sh);
    i0 = 1;
  }
  if (threadIdx.x == 0) hc[0] = hprev;
  for (int i = i0; i <= j + 1; ++i) {
    const double2* vi = (i <= j) ? V + (size_t)i * ldv : nullptr;
    const double2* vp = (i > 0) ? V + (size_t)(i - 1) * ldv : nullptr;
    double acc = mgs_sweep(w, vi, vp, hprev, N, (long long)rank * blockDim.x + threadIdx.x,
                           (long long)nr * blockDim.x);
    acc = block_sum_c(acc, sh);
    if (threadIdx.x == 0) part[i & 1] = acc;
    cl.sync();  // the partials of sweep i are complete (and w's updates visible in the cluster)
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int r = 0; r < nr; ++r) t += *cl.map_shared_rank(&part[i & 1], r);
      bc = t;
    }
    __syncthreads();
    const double sum = bc;
    __syncthreads();
    if (i <= j) {
      hprev = sum;
      if (threadIdx.x == 0) hc[i] = sum;
    } else {
      nrm2 = sum;
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
  if (rank == 0 && threadIdx.x < 32) {
    const int cont = givens_finish_warp(gs, j, nrm2, hc, w, cfg);
    if (threadIdx.x == 0 && set_cond) cudaGraphSetConditional(h_inner, cont ? 1u : 0u);
  }
}

// ||x|| into gs (beta, 1/beta, g = beta e_1), fixed-order reduction; then, by mode:
//   mode 0 (solve start): fnorm = beta, src = x (= f), it = outer = j = err = 0; outer condition = beta > 0
//   mode 1 (FP64 restart): skipped when gs->no_restart (outer condition 0); else relres = beta/fnorm,
//          converged -> done = 1; outer condition = not converged
//   mode 2 (mixed refinement): outer += 1; relres = beta/fnorm; outer condition = beta/fnorm >= tol and
//          outer < max_outer and it < max_it
// In modes 1, 2 the new cycle starts from src = x (= r) with scale 1/beta.
// When x's producer left block partials of ||x||^2 (mode 0: pa, na; mode 2: pa, na if the residual
// came from the recurrence, else pb, nb), block 0 sums them in a fixed order and the other blocks
// return; a count of 0 falls back to the sweep.
__global__ void __launch_bounds__(kCtlThreads) k_norm_ctl(const double2* __restrict__ x, GmresState* gs, long long N,
                                                         double* partials, unsigned* counter, GridBarrier* bar,
                                                         SolveCfg cfg, int mode, cudaGraphConditionalHandle h_outer,
                                                         int set_cond, const double* __restrict__ pa, int na,
                                                         const double* __restrict__ pb, int nb) {
  __shared__ double sh[32];
  __shared__ bool last;
  if (mode == 1 && gs->no_restart) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && set_cond) cudaGraphSetConditional(h_outer, 0u);
    return;
  }
  const double* pp = nullptr;
  int pn = 0;
  if (mode == 0) {
    pp = pa;
    pn = na;
  } else if (mode == 2) {
    const bool upd = gs->upd != 0;  // uniform
    pp = upd ? pa : pb;
    pn = upd ? na : nb;
  }
  double s = 0.0;
  if (pn > 0) {
    if (blockIdx.x != 0) return;
    for (int i = threadIdx.x; i < pn; i += blockDim.x) s += pp[i];
    s = block_sum_c(s, sh);
    if (threadIdx.x != 0) return;
  } else {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
      const double2 v = x[i];
      acc = fma(v.x, v.x, acc);
      acc = fma(v.y, v.y, acc);
    }
    acc = block_sum_c(acc, sh);
    if (threadIdx.x == 0) {
      partials[blockIdx.x] = acc;
      __threadfence();
      last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += ((volatile const double*)partials)[i];
    s = block_sum_c(s, sh);
    if (threadIdx.x != 0) return;
    *counter = 0u;
  }
  const double b = sqrt(s);
  gs->beta = b;
  gs->inv_beta = (b > 0.0) ? 1.0 / b : 0.0;
  gs->g[0] = b;
  for (int i = 1; i <= kMaxM; ++i) gs->g[i] = 0.0;
  gs->src = x;
  gs->src_scale = gs->inv_beta;
  gs->j = 0;
  unsigned cont;
  if (mode == 0) {
    gs->fnorm = b;
    gs->upd = 0;
    gs->upd_err = 0.0;
    gs->it = 0;
    gs->outer = 0;
    gs->err = 0;
    gs->no_restart = 0;
    gs->done = isfinite(b) ? 0 : 3;
    gs->relres = (b > 0.0) ? 1.0 : 0.0;
    bar->count = 0u;
    bar->done = 0u;
    cont = (b > 0.0 && isfinite(b)) ? 1u : 0u;
  } else {
    gs->outer += 1;
    const double rel = b / gs->fnorm;
    const double margin = (mode == 2 && gs->upd) ? gs->upd_err : 0.0;  // recurrence residual: its error bound
    gs->relres = rel;
    if (!isfinite(b)) {
      gs->done = 3;
      cont = 0u;
    } else if (rel + margin < cfg.tol) {
      gs->done = 1;
      cont = 0u;
    } else {
      gs->done = 0;
      cont = (mode == 1) ? 1u : ((gs->outer < cfg.max_outer && gs->it < cfg.max_it && !gs->err) ? 1u : 0u);
    }
  }
  if (set_cond) cudaGraphSetConditional(h_outer, cont);
}

// Start of an Arnoldi cycle: reference norm and tolerance of the relative residual test, j = 0, and
// the inner-loop condition set to run.  FP64 form: ref = ||f||, tol = tol.  Mixed form: ref = beta
// (the outer residual), tol = max(eta_min, 0.1 tol ||f|| / beta).
// The outer condition is cleared here and set again only by the residual kernel at the end of the
// cycle, so the outer loop can only stop early if that kernel does not run.
__global__ void k_cycle_begin(GmresState* gs, SolveCfg cfg, cudaGraphConditionalHandle h_inner,
                              cudaGraphConditionalHandle h_outer, int set_cond) {
  if (cfg.mixed) {
    gs->ref = gs->beta;
    gs->tol = fmax(cfg.eta_min, 0.1 * cfg.tol * gs->fnorm / gs->beta);
  } else {
    gs->ref = gs->fnorm;
    gs->tol = cfg.tol;
  }
  gs->j = 0;
  gs->done = 0;
  gs->no_restart = 0;
  if (set_cond) {
    cudaGraphSetConditional(h_outer, 0u);
    cudaGraphSetConditional(h_inner, 1u);
  }
}

// y = R^{-1} g on the leading k x k triangle, k = gs->j (single thread).
__global__ void k_backsolve_dev(GmresState* gs) {
  const int k = gs->j;
  const int ld = kMaxM + 1;
  for (int i = k - 1; i >= 0; --i) {
    double s = gs->g[i];
    for (int jj = i + 1; jj < k; ++jj) s -= gs->H[(size_t)jj * ld + i] * gs->y[jj];
    gs->y[i] = s / gs->H[(size_t)i * ld + i];
  }
}

// out = sum_{i<k} y_i V_i, k = gs->j
__global__ void k_combine_dev(const double2* __restrict__ V, long long ldv, const GmresState* gs,
                              double2* __restrict__ out, long long N) {
  __shared__ double y[kMaxM];
  const int k = gs->j;
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

// Mixed form, end of a refinement cycle: the residual recurrence.  The flexible Arnoldi relation
// R Z_k = V_{k+1} Hbar_k (products R z_j in FP32, basis and Hessenberg matrix in FP64) gives
//   r_new = r_old - R Z_k y = V_{k+1} (beta e_1 - Hbar_k y) = V_{k+1} Q_k^T (g_k e_k),
// i.e. the Givens rotations undone on the last residual estimate g_k, up to the FP32 error of the
// products, about kUpdErr ||Z_k y|| <= kUpdErr beta (||R^{-1}|| <= 1: R = I + i(T - D), T - D real
// symmetric).  Used only when beta <= kUpdRatio tol ||f||, so that this error stays a small fraction
// of tol ||f||; it is also added to the stopping test.  k < 0: k = gs->j and the decision is taken
// here; otherwise upd and err come from the host.
__device__ __forceinline__ void resid_coeffs_body(GmresState* gs, int k_in, int upd_in, double err_in, double tol) {
  const int k = k_in >= 0 ? k_in : gs->j;
  int upd;
  double err;
  if (k_in >= 0) {
    upd = upd_in;
    err = err_in;
  } else {
    upd = (gs->outer >= 1 && gs->beta <= kUpdRatio * tol * gs->fnorm) ? 1 : 0;
    err = kUpdErr * gs->beta / gs->fnorm;
  }
  gs->upd = upd;
  gs->upd_err = upd ? err : 0.0;
  if (!upd) return;
  double t = gs->g[k];
  for (int i = k - 1; i >= 0; --i) {
    gs->q[i + 1] = gs->cs[i] * t;
    t = -gs->sn[i] * t;
  }
  gs->q[0] = t;
}
__global__ void k_resid_coeffs(GmresState* gs, int k_in, int upd_in, double err_in, double tol) {
  resid_coeffs_body(gs, k_in, upd_in, err_in, tol);
}

// Mixed form, end of a refinement cycle of k = gs->j flexible Arnoldi steps, in one launch (in place of
// the back-substitution, the solution update and the recurrence's coefficients as three): thread 0 of
// every block solves R y = g on the leading k x k triangle into shared memory (the operations of
// k_backsolve_dev, in its order), block 0 stores y and takes the recurrence's decision and
// coefficients (k_resid_coeffs), and every block adds its share of sum_q y_q Z_q to x.
__global__ void k_cycle_end_mixed(const float2* __restrict__ Z, long long ldz, GmresState* gs,
                                  double2* __restrict__ x, long long N, double tol) {
  __shared__ double y[kMaxM];
  const int k = gs->j;
  if (threadIdx.x == 0) {
    const int ld = kMaxM + 1;
    for (int i = k - 1; i >= 0; --i) {
      double s = gs->g[i];
      for (int jj = i + 1; jj < k; ++jj) s -= gs->H[(size_t)jj * ld + i] * y[jj];
      y[i] = s / gs->H[(size_t)i * ld + i];
    }
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int t = threadIdx.x; t < k; t += blockDim.x) gs->y[t] = y[t];
    if (threadIdx.x == 0) resid_coeffs_body(gs, -1, -1, 0.0, tol);
  }
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

// r = sum_{i<k} q_i V_i + q_k inv_h w when gs->upd, k = gs->j if k_in < 0; with nrm_part, each
// block also leaves its share of ||r||^2 there for the norm kernel.
__global__ void k_resid_update(const double2* __restrict__ V, long long ldv, const double2* __restrict__ w,
                               const GmresState* gs, int k_in, double2* __restrict__ r, long long N,
                               double* __restrict__ nrm_part) {
  if (!gs->upd) return;  // uniform
  __shared__ double q[kMaxM + 1];
  __shared__ double sh[32];
  double nacc = 0.0;
  const int k = k_in >= 0 ? k_in : gs->j;
  for (int t = threadIdx.x; t <= k; t += blockDim.x) q[t] = gs->q[t];
  __syncthreads();
  const double cw = (q[k] == 0.0) ? 0.0 : q[k] * gs->inv_h;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 wv = w[i];
    double2 a = make_double2(cw * wv.x, cw * wv.y);
    for (int j = 0; j < k; ++j) {
      const double2 v = V[(size_t)j * ldv + i];
      a.x += q[j] * v.x;
      a.y += q[j] * v.y;
    }
    r[i] = a;
    nacc = fma(a.x, a.x, nacc);
    nacc = fma(a.y, a.y, nacc);
  }
  if (nrm_part) {
    nacc = block_sum_c(nacc, sh);
    if (threadIdx.x == 0) nrm_part[blockIdx.x] = nacc;
  }
}

// x += sum_{i<k} y_i Z_i (Z in FP32), k = gs->j
__global__ void k_combine_f32_add_dev(const float2* __restrict__ Z, long long ldz, const GmresState* gs,
                                      double2* __restrict__ x, long long N) {
  __shared__ double y[kMaxM];
  const int k = gs->j;
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

// Mixed form, inside a captured time step: T x from the solve's final residual r = f - x - i(T - D)x,
// Tx = D x - i (f - x - r); when the solve did no refinement cycle (f = 0, x = 0) Tx = 0.
__global__ void k_tu_from_residual_dev(const GmresState* gs, const double* __restrict__ D,
                                       const double2* __restrict__ f, const double2* __restrict__ x,
                                       const double2* __restrict__ r, double2* __restrict__ Tu, long long N) {
  const bool have = gs->outer > 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    if (!have) {
      Tu[i] = make_double2(0.0, 0.0);
      continue;
    }
    const double2 fv = f[i], xv = x[i], rv = r[i];
    const double d = D[i];
    const double qx = fv.x - xv.x - rv.x, qy = fv.y - xv.y - rv.y;
    Tu[i] = make_double2(d * xv.x + qy, d * xv.y - qx);
  }
}

// Copy the host-read prefix of every instance's GMRES state into one array.
__global__ void k_gather_peeks(GmresState* const* gs, GmresPeek* out, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = *reinterpret_cast<const GmresPeek*>(gs[i]);
}

void launch_tu_from_residual_dev(const GmresState* gs, const double* D, const double2* f, const double2* x,
                                 const double2* r, double2* Tu, long long N, cudaStream_t s);
void launch_gather_peeks(GmresState* const* gs, GmresPeek* out, int count, cudaStream_t s);

static inline unsigned ew_blocks_c(long long N) {
  long long b = (N + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

int coop_blocks_max(long long N) {
  if (N <= 4096) return 1;
  int dev = 0, sms = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mgs_step, kCtlThreads, 0);
  if (per_sm > 4) per_sm = 4;
  long long b = (long long)sms * (per_sm < 1 ? 1 : per_sm);
  const long long need = (N + kCtlThreads - 1) / kCtlThreads;
  if (b > need) b = need;
  return (int)(b < 1 ? 1 : b);
}

// A column of the GMRES state for timing the Arnoldi kernel (rfnse_autotune): j, no convergence test
// that stops (ref 1, tol 0), counters cleared.
__global__ void k_set_column(GmresState* gs, int j) {
  gs->j = j;
  gs->done = 0;
  gs->it = 0;
  gs->err = 0;
  gs->ref = 1.0;
  gs->tol = 0.0;
}
void launch_set_column(GmresState* gs, int j, cudaStream_t s) {
  count_launch();
  k_set_column<<<1, 1, 0, s>>>(gs, j);
}

int coop_blocks_for(long long N) {
  int dev = 0, sms = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mgs_step, kCtlThreads, 0);
  // Small grids (up to a few 10^5 points) are bound by the barriers between the MGS passes: one block
  // per SM is faster and leaves room for other instances' kernels; large grids stream their vectors
  // and take two blocks per SM (measured on the 2-D 511^2, batched and 3-D 255^3 workloads).
  if (N <= 4096) return 1;  // a few points per thread: block barriers only, no grid-wide protocol
  const int use = (N >= (1LL << 22)) ? 2 : 1;
  long long b = (long long)sms * (per_sm < use ? per_sm : use);
  const long long need = (N + kCtlThreads - 1) / kCtlThreads;
  if (b > need) b = need;
  if (b < 1) b = 1;
  return (int)b;
}

// blocks < 0: one cluster of -blocks CTAs (k_mgs_cluster)
static cudaError_t launch_mgs_cluster(GmresState* gs, const double2* V, long long ldv, double2* w, long long N,
                                      const SolveCfg& cfg, cudaGraphConditionalHandle h_inner, int set_cond,
                                      int csize, cudaStream_t s, const double* pre_part, int pre_n) {
  static const cudaError_t attr = cudaFuncSetAttribute(k_mgs_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (attr != cudaSuccess) return attr;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)csize);
  lc.blockDim = dim3(kClThreads);
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&lc, k_mgs_cluster, gs, V, ldv, w, N, cfg, h_inner, set_cond, pre_part, pre_n);
}

// Whether one cluster of csize CTAs of the cluster Arnoldi kernel can be resident on this device.
bool mgs_cluster_fits(int csize) {
  if (cudaFuncSetAttribute(k_mgs_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)csize);
  lc.blockDim = dim3(kClThreads);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_mgs_cluster, &lc) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters >= 1;
}

cudaError_t launch_mgs_step(GmresState* gs, const double2* V, long long ldv, double2* w, long long N,
                            double* partials, GridBarrier* bar, const SolveCfg& cfg,
                            cudaGraphConditionalHandle h_inner, int set_cond, int blocks, cudaStream_t s,
                            const double* pre_part, int pre_n) {
  if (blocks < 0) return launch_mgs_cluster(gs, V, ldv, w, N, cfg, h_inner, set_cond, -blocks, s, pre_part, pre_n);
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)blocks);
  lc.blockDim = dim3(kCtlThreads);
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&lc, k_mgs_step, gs, V, ldv, w, N, partials, bar, cfg, h_inner, set_cond, pre_part,
                            pre_n);
}

void launch_norm_ctl(const double2* x, GmresState* gs, long long N, int blocks, double* partials, unsigned* counter,
                     GridBarrier* bar, const SolveCfg& cfg, int mode, cudaGraphConditionalHandle h_outer,
                     int set_cond, cudaStream_t s, const double* pa, int na, const double* pb, int nb) {
  count_launch();
  // one block when every outcome has partials to sum
  const bool partial_only = (mode == 0 && na > 0) || (mode == 2 && na > 0 && nb > 0);
  k_norm_ctl<<<partial_only ? 1 : blocks, kCtlThreads, 0, s>>>(x, gs, N, partials, counter, bar, cfg, mode, h_outer,
                                                               set_cond, pa, na, pb, nb);
}
void launch_cycle_begin(GmresState* gs, const SolveCfg& cfg, cudaGraphConditionalHandle h_inner,
                        cudaGraphConditionalHandle h_outer, int set_cond, cudaStream_t s) {
  count_launch();
  k_cycle_begin<<<1, 1, 0, s>>>(gs, cfg, h_inner, h_outer, set_cond);
}
void launch_tu_from_residual_dev(const GmresState* gs, const double* D, const double2* f, const double2* x,
                                 const double2* r, double2* Tu, long long N, cudaStream_t s) {
  count_launch();
  k_tu_from_residual_dev<<<ew_blocks_c(N), 256, 0, s>>>(gs, D, f, x, r, Tu, N);
}
void launch_gather_peeks(GmresState* const* gs, GmresPeek* out, int count, cudaStream_t s) {
  count_launch();
  k_gather_peeks<<<(count + 127) / 128, 128, 0, s>>>(gs, out, count);
}
void launch_backsolve_dev(GmresState* gs, cudaStream_t s) {
  count_launch();
  k_backsolve_dev<<<1, 1, 0, s>>>(gs);
}
void launch_combine_dev(const double2* V, long long ldv, const GmresState* gs, double2* out, long long N,
                        cudaStream_t s) {
  count_launch();
  k_combine_dev<<<ew_blocks_c(N), 256, 0, s>>>(V, ldv, gs, out, N);
}
void launch_combine_f32_add_dev(const float2* Z, long long ldz, const GmresState* gs, double2* x, long long N,
                                cudaStream_t s) {
  count_launch();
  k_combine_f32_add_dev<<<ew_blocks_c(N), 256, 0, s>>>(Z, ldz, gs, x, N);
}
void launch_cycle_end_mixed(const float2* Z, long long ldz, GmresState* gs, double2* x, long long N, double tol,
                            cudaStream_t s) {
  count_launch();
  k_cycle_end_mixed<<<ew_blocks_c(N), 256, 0, s>>>(Z, ldz, gs, x, N, tol);
}
void launch_resid_coeffs(GmresState* gs, int k, int upd, double err, double tol, cudaStream_t s) {
  count_launch();
  k_resid_coeffs<<<1, 1, 0, s>>>(gs, k, upd, err, tol);
}
int resid_update_blocks(long long N) { return (int)ew_blocks_c(N); }
void launch_resid_update(const double2* V, long long ldv, const double2* w, const GmresState* gs, int k,
                         double2* r, long long N, cudaStream_t s, double* nrm_part) {
  count_launch();
  k_resid_update<<<ew_blocks_c(N), 256, 0, s>>>(V, ldv, w, gs, k, r, N, nrm_part);
}

// Self-test of the bounded wait: the single block of this launch arrives and then waits for the
// arrival of a second block, which does not exist (a release that nothing performs); the wait must
// give up after kMaxSpin polls, record the failure and return.
__global__ void k_selftest_wait(GridBarrier* b, int* err) {
  if (threadIdx.x == 0) red_add_release(&b->count, 1u);
  warp_wait_count(&b->count, 2u, err);
}

}  // namespace rfnse

extern "C" int rfnse_selftest_bounded_wait(void* stream, int* err, double* ms) {
  using namespace rfnse;
  if (!err) return RFNSE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  GridBarrier* b = nullptr;
  int* d_err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = RFNSE_OK;
  const GridBarrier init = {0u, 0u};
  if (cudaMalloc(&b, sizeof(GridBarrier)) != cudaSuccess || cudaMalloc(&d_err, sizeof(int)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = RFNSE_ENOMEM;
  } else if (cudaMemcpyAsync(b, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess ||
             cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess) {
    st = RFNSE_ECUDA;
  } else {
    cudaEventRecord(e0, s);
    k_selftest_wait<<<1, 32, 0, s>>>(b, d_err);
    count_launch();
    cudaEventRecord(e1, s);
    int h = 0;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                                                 cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = RFNSE_ECUDA;
    } else {
      *err = h;
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      if (ms) *ms = t;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(b);
  cudaFree(d_err);
  return st;
}
