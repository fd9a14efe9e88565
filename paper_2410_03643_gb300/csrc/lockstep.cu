// Kernels of the lock-step batch (lockstep.cuh): the per-instance set-up, solve-start, cycle and
// Arnoldi bookkeeping of the GMRES solves of many instances, each launch covering all of them.
// Every instance's arithmetic is that of its single-instance solve (control.cu, krylov.cu): the same
// modified Gram-Schmidt sweeps with fixed-order reductions, Givens rotations, convergence tests,
// refinement decisions and residual recurrence; only the partition of an instance's vectors over
// blocks (and so the order of its partial sums) differs.
#include <cmath>
#include "internal.cuh"
#include "coop.cuh"
#include "dfloat.cuh"
#include "lockstep.cuh"

namespace rfnse {

long long lock_ew_blocks(long long N) {
  long long b = (N + kLockEwThreads - 1) / kLockEwThreads;
  if (b > 2048) b = 2048;  // at most kNormPartMax partials per instance
  if (b < 1) b = 1;
  return b;
}

// The instance of this block in a batched element-wise launch and the block's index within it.
__device__ __forceinline__ int ew_item(const LockInst* __restrict__ li, int n, long long& local) {
  __shared__ int inst_s;
  __shared__ long long local_s;
  if (threadIdx.x == 0) {
    const long long b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (li[mid].blk0 <= b) lo = mid;
      else hi = mid - 1;
    }
    inst_s = lo;
    local_s = b - li[lo].blk0;
  }
  __syncthreads();
  local = local_s;
  return inst_s;
}

// Steady step set-up of every instance (the mixed form's k_step_prep): D = rho dt |u^n|^2,
// f = u^{n-1} - i (T u^{n-1} - D u^{n-1}), the FP32 (omega I + D) sub-solve tables, x = 0, and the
// block partials of ||f||^2.
__global__ void __launch_bounds__(kLockEwThreads) k_ls_step_prep(const LockInst* __restrict__ li, int n,
                                                                  unsigned long long* counts) {
  __shared__ double sh[32];
  if (blockIdx.x == 0 && threadIdx.x == 0) counts[0] = counts[1] = 0ull;  // this step's loop counts
  long long lb;
  const LockInst& I = li[ew_item(li, n, lb)];
  const long long N = I.N, nb = I.nblk;
  const double rho_dt = I.rho_dt;
  const float w1f = (float)(I.omega + 1.0), two_wf = (float)(2.0 * I.omega);
  const double2* __restrict__ uc = I.u_cur;
  const double2* __restrict__ up = I.u_prev;
  const double2* __restrict__ tp = I.Tu_prev;
  double nacc = 0.0;
  for (long long i = lb * blockDim.x + threadIdx.x; i < N; i += nb * blockDim.x) {
    const double2 v = uc[i], uv = up[i], tv = tp[i];
    const double d = rho_dt * (v.x * v.x + v.y * v.y);
    I.D[i] = d;
    const double px = tv.x - d * uv.x, py = tv.y - d * uv.y;
    const double2 fv = make_double2(uv.x + py, uv.y - px);
    I.f[i] = fv;
    nacc = fma(fv.x, fv.x, nacc);
    nacc = fma(fv.y, fv.y, nacc);
    const float df = (float)d;
    const float sf = two_wf / fmaf(df, df, w1f * w1f);  // FP32: the batch's solves read the FP32 tables only
    I.D32[i] = df;
    I.dfac32[i] = make_float2(sf * w1f, sf * df);
    I.x[i] = make_double2(0.0, 0.0);
  }
  nacc = block_sum_c(nacc, sh);
  if (threadIdx.x == 0) I.nrm_f[lb] = nacc;
}

// The last block of the launch to arrive (every block calls it once, thread 0 returns the answer).
__device__ __forceinline__ bool last_to_arrive(unsigned* done_all) {
  __threadfence();
  const bool last = atomicAdd(done_all, 1u) == gridDim.x - 1;
  if (last) {
    __threadfence();
    *done_all = 0u;
  }
  return last;
}

// Solve start of every instance (control.cu k_norm_ctl, mode 0): ||f|| from the set-up's partials in
// a fixed order, g = beta e_1, counters cleared; the instance needs a cycle when beta > 0.  The last
// block sets the outer loop's condition (any instance needs a cycle) and clears the batch's barrier.
__global__ void __launch_bounds__(kCtlThreads) k_ls_norm_start(const LockInst* __restrict__ li, int n,
                                                               GridBarrier* bar, unsigned* done_all,
                                                               cudaGraphConditionalHandle h_outer) {
  __shared__ double sh[32];
  const LockInst& I = li[blockIdx.x];
  double s = 0.0;
  for (long long i = threadIdx.x; i < I.nblk; i += blockDim.x) s += I.nrm_f[i];
  s = block_sum_c(s, sh);
  if (threadIdx.x != 0) return;
  GmresState* gs = I.gs;
  const double b = sqrt(s);
  gs->beta = b;
  gs->inv_beta = (b > 0.0) ? 1.0 / b : 0.0;
  gs->g[0] = b;
  for (int i = 1; i <= kMaxM; ++i) gs->g[i] = 0.0;
  gs->src = I.f;
  gs->src_scale = gs->inv_beta;
  gs->j = 0;
  gs->fnorm = b;
  gs->upd = 0;
  gs->upd_err = 0.0;
  gs->it = 0;
  gs->outer = 0;
  gs->err = 0;
  gs->no_restart = 0;
  gs->done = isfinite(b) ? 0 : 3;
  gs->relres = (b > 0.0) ? 1.0 : 0.0;
  const int cont = (b > 0.0 && isfinite(b)) ? 1 : 0;
  LockFlags* fl = I.fl;
  fl->act = cont;
  fl->oskip = !cont;
  fl->iskip = 1;
  fl->dfskip = 1;
  fl->arrive = 0u;
  if (last_to_arrive(done_all)) {
    bar->count = 0u;
    int any = 0;
    for (int k = 0; k < n; ++k) any |= ((volatile LockFlags*)li[k].fl)->act;
    cudaGraphSetConditional(h_outer, any ? 1u : 0u);
  }
}

// Start of a refinement cycle of every instance that is still active (control.cu k_cycle_begin, mixed
// form): reference norm beta, inner tolerance max(eta_min, 0.1 tol ||f|| / beta), j = 0.  One thread per
// instance.  Sets the inner condition (any instance iterates) and clears the outer one, which the
// residual kernel at the end of the cycle sets again.
__global__ void k_ls_cycle_begin(const LockInst* __restrict__ li, int n, unsigned long long* counts,
                                 cudaGraphConditionalHandle h_inner, cudaGraphConditionalHandle h_outer) {
  const int k = threadIdx.x;
  int run = 0;
  if (k < n) {
    const LockInst& I = li[k];
    GmresState* gs = I.gs;
    if (I.fl->act) {
      gs->ref = gs->beta;
      gs->tol = fmax(I.cfg.eta_min, 0.1 * I.cfg.tol * gs->fnorm / gs->beta);
      gs->j = 0;
      gs->done = 0;
      gs->no_restart = 0;
      I.fl->iskip = 0;
      run = 1;
    } else {
      I.fl->iskip = 1;
    }
  }
  const int any = __syncthreads_or(run);
  if (k == 0) {
    cudaGraphSetConditional(h_outer, 0u);
    cudaGraphSetConditional(h_inner, any ? 1u : 0u);
    counts[1] += 1ull;
  }
}

// One Arnoldi step of every instance still iterating in its cycle (control.cu k_mgs_step): modified
// Gram-Schmidt of w against v_0..v_j in j + 1 sweeps (h_0j from the product pass's partials when it
// left them), h_{j+1,j} = ||w||, Givens update and convergence test.  The instances' blocks partition
// the grid (cb0, ncb); sweep i of every instance runs between the same two grid-wide barriers, the
// instances with fewer columns idle through the later ones.  The last block of the grid sets the inner
// condition: any instance continues.
__global__ void __launch_bounds__(kCtlThreads) k_ls_mgs(const LockInst* __restrict__ li, int n, GridBarrier* bar,
                                                        unsigned* done_all, unsigned long long* counts,
                                                        cudaGraphConditionalHandle h_inner) {
  __shared__ double sh[33];
  __shared__ double hc[kMaxM + 1];  // this instance's column j of H before the rotations
  __shared__ int s_inst, s_jmax, s_first;
  if (threadIdx.x == 0) {
    const int b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (li[mid].cb0 <= b) lo = mid;
      else hi = mid - 1;
    }
    s_inst = lo;
    // read before this block's first arrival: the finishing blocks write j and iskip only after the
    // last one, which no block passes before every block has made these reads
    int jm = -1, first = 1;
    for (int k = 0; k < n; ++k)
      if (!li[k].fl->iskip) {
        jm = max(jm, li[k].gs->j);
        if (li[k].dot_n <= 0) first = 0;  // this instance sweeps its first dot product itself
      }
    s_jmax = jm;
    s_first = first;
  }
  __syncthreads();
  const LockInst& I = li[s_inst];
  const int jmax = s_jmax;
  const int lb = blockIdx.x - I.cb0, nb = I.ncb;
  GmresState* gs = I.gs;
  const bool active = !I.fl->iskip;
  const int j = active ? gs->j : -1;
  const long long N = I.N;
  double2* __restrict__ w = I.w;
  double hprev = 0.0, nrm2 = 0.0;
  int i0 = 0;
  if (active && I.dot_n > 0) {  // h_0j from the partials the product pass left (same sum in every block)
    hprev = fixed_sum(I.dot_part, I.dot_n, sh);
    i0 = 1;
  }
  if (threadIdx.x == 0) hc[0] = hprev;
  // Sweep i of every instance between two counted arrivals of the whole grid (coop.cuh); each
  // instance sums only its own blocks' partials.
  unsigned arrivals = 0;
  for (int i = s_first; i <= jmax + 1; ++i) {  // sweep 0 only when some instance needs it
    const bool mine = active && i >= i0 && i <= j + 1;  // uniform in the block
    double acc = 0.0;
    if (mine) {
      const double2* vi = (i <= j) ? I.V + (size_t)i * N : nullptr;
      const double2* vp = (i > 0) ? I.V + (size_t)(i - 1) * N : nullptr;
      acc = mgs_sweep(w, vi, vp, hprev, N, (long long)lb * blockDim.x + threadIdx.x, (long long)nb * blockDim.x);
    }
    const double b = block_partial_w0(acc, sh);
    double* buf = I.cpart + (size_t)(i & 1) * nb;
    ++arrivals;
    if (threadIdx.x < 32) {
      if (threadIdx.x == 0) {
        if (mine) buf[lb] = b;
        red_add_release(&bar->count, 1u);
      }
      warp_wait_count(&bar->count, arrivals * gridDim.x, &gs->err);
      const double t = mine ? warp_sum_partials(buf, nb) : 0.0;
      if (threadIdx.x == 0) sh[32] = t;
    }
    __syncthreads();
    if (mine) {
      const double t = sh[32];
      if (i <= j) {
        hprev = t;
        if (threadIdx.x == 0) hc[i] = t;
      } else {
        nrm2 = t;
      }
    }
  }
  if (active && lb == 0 && threadIdx.x < 32) {  // Givens update and test of this instance
    const int cont = givens_finish_warp(gs, j, nrm2, hc, w, I.cfg);
    if (threadIdx.x == 0) I.fl->iskip = cont ? 0 : 1;
  }
  __shared__ bool last;
  if (threadIdx.x == 0) last = last_to_arrive(done_all);
  __syncthreads();
  if (last && threadIdx.x == 0) {
    bar->count = 0u;  // every block has passed its last wait: clear the arrivals for the next launch
    int any = 0;
    for (int k = 0; k < n; ++k) any |= !((volatile LockFlags*)li[k].fl)->iskip;
    cudaGraphSetConditional(h_inner, any ? 1u : 0u);
    counts[0] += 1ull;
  }
}

// y = R^{-1} g on the leading j x j triangle of every instance still in its solve (one thread each).
__global__ void k_ls_backsolve(const LockInst* __restrict__ li, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || li[k].fl->oskip) return;
  GmresState* gs = li[k].gs;
  const int m = gs->j;
  const int ld = kMaxM + 1;
  for (int i = m - 1; i >= 0; --i) {
    double s = gs->g[i];
    for (int jj = i + 1; jj < m; ++jj) s -= gs->H[(size_t)jj * ld + i] * gs->y[jj];
    gs->y[i] = s / gs->H[(size_t)i * ld + i];
  }
}

// x += sum_{q<j} y_q Z_q (Z in FP32) for every instance still in its solve.
__global__ void __launch_bounds__(kLockEwThreads) k_ls_combine_add(const LockInst* __restrict__ li, int n) {
  __shared__ double y[kMaxM];
  long long lb;
  const LockInst& I = li[ew_item(li, n, lb)];
  if (I.fl->oskip) return;  // uniform
  const GmresState* gs = I.gs;
  const int k = gs->j;
  for (int t = threadIdx.x; t < k; t += blockDim.x) y[t] = gs->y[t];
  __syncthreads();
  const long long N = I.N, nb = I.nblk;
  for (long long i = lb * blockDim.x + threadIdx.x; i < N; i += nb * blockDim.x) {
    double2 a = I.x[i];
    for (int q = 0; q < k; ++q) {
      const float2 v = I.Z32[(size_t)q * N + i];
      a.x += y[q] * df_f2d(v.x);  // exact, without an FP64-pipe conversion
      a.y += y[q] * df_f2d(v.y);
    }
    I.x[i] = a;
  }
}

// End of a refinement cycle (control.cu k_resid_coeffs, decision on the device): the new residual
// from the Arnoldi basis when the cycle's starting residual beta <= kUpdRatio tol ||f||, with its
// coefficients q = Q^T g_k e_k; otherwise the double-float product runs (dfskip = 0).  One thread each.
__global__ void k_ls_resid_coeffs(const LockInst* __restrict__ li, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const LockInst& I = li[k];
  if (I.fl->oskip) {
    I.fl->dfskip = 1;
    return;
  }
  GmresState* gs = I.gs;
  const int m = gs->j;
  const int upd = (gs->outer >= 1 && gs->beta <= kUpdRatio * I.cfg.tol * gs->fnorm) ? 1 : 0;
  gs->upd = upd;
  gs->upd_err = upd ? kUpdErr * gs->beta / gs->fnorm : 0.0;
  I.fl->dfskip = upd;
  if (!upd) return;
  double t = gs->g[m];
  for (int i = m - 1; i >= 0; --i) {
    gs->q[i + 1] = gs->cs[i] * t;
    t = -gs->sn[i] * t;
  }
  gs->q[0] = t;
}

// r = sum_{i<j} q_i V_i + q_j inv_h w for every instance whose residual comes from the recurrence,
// with the block partials of ||r||^2 (control.cu k_resid_update).
__global__ void __launch_bounds__(kLockEwThreads) k_ls_resid_update(const LockInst* __restrict__ li, int n) {
  __shared__ double q[kMaxM + 1];
  __shared__ double sh[32];
  long long lb;
  const LockInst& I = li[ew_item(li, n, lb)];
  const GmresState* gs = I.gs;
  if (I.fl->oskip || !gs->upd) return;  // uniform
  const int k = gs->j;
  for (int t = threadIdx.x; t <= k; t += blockDim.x) q[t] = gs->q[t];
  __syncthreads();
  const double cw = (q[k] == 0.0) ? 0.0 : q[k] * gs->inv_h;
  const long long N = I.N, nb = I.nblk;
  double nacc = 0.0;
  for (long long i = lb * blockDim.x + threadIdx.x; i < N; i += nb * blockDim.x) {
    const double2 wv = I.w[i];
    double2 a = make_double2(cw * wv.x, cw * wv.y);
    for (int jj = 0; jj < k; ++jj) {
      const double2 v = I.V[(size_t)jj * N + i];
      a.x += q[jj] * v.x;
      a.y += q[jj] * v.y;
    }
    I.r[i] = a;
    nacc = fma(a.x, a.x, nacc);
    nacc = fma(a.y, a.y, nacc);
  }
  nacc = block_sum_c(nacc, sh);
  if (threadIdx.x == 0) I.nrm_upd[lb] = nacc;
}

// The residual norm at the end of a cycle and the refinement decision of every instance still in its
// solve (control.cu k_norm_ctl, mode 2), one block each: ||r|| from the partials of whichever kernel
// formed r (or a sweep of r), outer += 1, converged when ||r||/||f|| (+ the recurrence's error bound)
// < tol; the next cycle starts from r.  The last block sets the outer condition: any instance continues.
__global__ void __launch_bounds__(kCtlThreads) k_ls_norm_resid(const LockInst* __restrict__ li, int n,
                                                               unsigned* done_all,
                                                               cudaGraphConditionalHandle h_outer) {
  __shared__ double sh[32];
  const LockInst& I = li[blockIdx.x];
  GmresState* gs = I.gs;
  if (!I.fl->oskip) {  // uniform
    const bool upd = gs->upd != 0;
    double s = 0.0;
    if (upd || I.nb_df > 0) {
      const double* pp = upd ? I.nrm_upd : I.nrm_df;
      const long long pn = upd ? I.nblk : I.nb_df;
      for (long long i = threadIdx.x; i < pn; i += blockDim.x) s += pp[i];
    } else {
      for (long long i = threadIdx.x; i < I.N; i += blockDim.x) {
        const double2 v = I.r[i];
        s = fma(v.x, v.x, s);
        s = fma(v.y, v.y, s);
      }
    }
    s = block_sum_c(s, sh);
    if (threadIdx.x == 0) {
      const SolveCfg cfg = I.cfg;
      const double b = sqrt(s);
      gs->beta = b;
      gs->inv_beta = (b > 0.0) ? 1.0 / b : 0.0;
      gs->g[0] = b;
      for (int i = 1; i <= kMaxM; ++i) gs->g[i] = 0.0;
      gs->src = I.r;
      gs->src_scale = gs->inv_beta;
      gs->j = 0;
      gs->outer += 1;
      const double rel = b / gs->fnorm;
      const double margin = upd ? gs->upd_err : 0.0;
      gs->relres = rel;
      int cont;
      if (!isfinite(b)) {
        gs->done = 3;
        cont = 0;
      } else if (rel + margin < cfg.tol) {
        gs->done = 1;
        cont = 0;
      } else {
        gs->done = 0;
        cont = (gs->outer < cfg.max_outer && gs->it < cfg.max_it && !gs->err) ? 1 : 0;
      }
      I.fl->act = cont;
      I.fl->oskip = !cont;
    }
  }
  if (threadIdx.x == 0 && last_to_arrive(done_all)) {
    int any = 0;
    for (int k = 0; k < n; ++k) any |= ((volatile LockFlags*)li[k].fl)->act;
    cudaGraphSetConditional(h_outer, any ? 1u : 0u);
  }
}

// T x of every instance from its final residual r = f - x - i(T - D)x: Tx = D x - i (f - x - r)
// (control.cu k_tu_from_residual_dev); zero when the solve ran no cycle (f = 0).
__global__ void __launch_bounds__(kLockEwThreads) k_ls_tu(const LockInst* __restrict__ li, int n) {
  long long lb;
  const LockInst& I = li[ew_item(li, n, lb)];
  const bool have = I.gs->outer > 0;
  const long long N = I.N, nb = I.nblk;
  for (long long i = lb * blockDim.x + threadIdx.x; i < N; i += nb * blockDim.x) {
    if (!have) {
      I.Tu_next[i] = make_double2(0.0, 0.0);
      continue;
    }
    const double2 fv = I.f[i], xv = I.x[i], rv = I.r[i];
    const double d = I.D[i];
    const double qx = fv.x - xv.x - rv.x, qy = fv.y - xv.y - rv.y;
    I.Tu_next[i] = make_double2(d * xv.x + qy, d * xv.y - qx);
  }
}

// ---- launchers ----------------------------------------------------------------------------------

static unsigned ctl_threads(int n) { return (unsigned)(((n + 31) / 32) * 32); }

void launch_ls_step_prep(const LockInst* li, int n, long long blocks, unsigned long long* counts, cudaStream_t s) {
  count_launch();
  k_ls_step_prep<<<(unsigned)blocks, kLockEwThreads, 0, s>>>(li, n, counts);
}
void launch_ls_norm_start(const LockInst* li, int n, GridBarrier* bar, unsigned* done_all,
                          cudaGraphConditionalHandle h_outer, cudaStream_t s) {
  count_launch();
  k_ls_norm_start<<<n, kCtlThreads, 0, s>>>(li, n, bar, done_all, h_outer);
}
void launch_ls_cycle_begin(const LockInst* li, int n, unsigned long long* counts, cudaGraphConditionalHandle h_inner,
                           cudaGraphConditionalHandle h_outer, cudaStream_t s) {
  count_launch();
  k_ls_cycle_begin<<<1, ctl_threads(n), 0, s>>>(li, n, counts, h_inner, h_outer);
}
int ls_mgs_max_blocks() {
  int dev = 0, sms = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ls_mgs, kCtlThreads, 0);
  return sms * (per_sm < 2 ? per_sm : 2);
}
cudaError_t launch_ls_mgs(const LockInst* li, int n, int blocks, GridBarrier* bar, unsigned* done_all,
                          unsigned long long* counts, cudaGraphConditionalHandle h_inner, cudaStream_t s) {
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
  return cudaLaunchKernelEx(&lc, k_ls_mgs, li, n, bar, done_all, counts, h_inner);
}
void launch_ls_backsolve(const LockInst* li, int n, cudaStream_t s) {
  count_launch();
  k_ls_backsolve<<<(n + 127) / 128, 128, 0, s>>>(li, n);
}
void launch_ls_combine_add(const LockInst* li, int n, long long blocks, cudaStream_t s) {
  count_launch();
  k_ls_combine_add<<<(unsigned)blocks, kLockEwThreads, 0, s>>>(li, n);
}
void launch_ls_resid_coeffs(const LockInst* li, int n, cudaStream_t s) {
  count_launch();
  k_ls_resid_coeffs<<<(n + 127) / 128, 128, 0, s>>>(li, n);
}
void launch_ls_resid_update(const LockInst* li, int n, long long blocks, cudaStream_t s) {
  count_launch();
  k_ls_resid_update<<<(unsigned)blocks, kLockEwThreads, 0, s>>>(li, n);
}
void launch_ls_norm_resid(const LockInst* li, int n, unsigned* done_all, cudaGraphConditionalHandle h_outer,
                          cudaStream_t s) {
  count_launch();
  k_ls_norm_resid<<<n, kCtlThreads, 0, s>>>(li, n, done_all, h_outer);
}
void launch_ls_tu(const LockInst* li, int n, long long blocks, cudaStream_t s) {
  count_launch();
  k_ls_tu<<<(unsigned)blocks, kLockEwThreads, 0, s>>>(li, n);
}

}  // namespace rfnse
