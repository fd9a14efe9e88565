// Reverse pass (discrete adjoint) of the time stepper: the gradient of a real loss of u^N with
// respect to u^0 and rho.  The paper has no adjoint; this is the exact derivative of its discrete
// scheme (Sec. 2.1 eq. 'discretizedCNLSMaxForm', Sec. 2.2 eq. 'discretizedRFSE2DMaxForm', and the
// first step read as a predictor-corrector Crank-Nicolson step).
//
// Gradient convention: g = dL/dRe(u) + i dL/dIm(u), so dL = Re(g^H du).
// Step n >= 1, M_n u^{n+1} = N_n u^{n-1}, M_n = D_n - T + iI, N_n = T - D_n + iI, D_n = rho dt |u^n|^2.
// M_n is complex symmetric (T real symmetric, D_n real diagonal), so M_n^{-H} g = conj(M_n^{-1} conj g):
//   lambda   = conj(M_n^{-1} conj(g_{n+1}))     -- the same tau-preconditioned GMRES solve
//   g_{n-1}  = (T - D_n - iI) lambda             -- N_n^H lambda (the first contribution to g_{n-1})
//   s_j      = -Re(conj(lambda_j)(u^{n+1}_j + u^{n-1}_j))
//   g_n     += 2 rho dt s u^n,   dL/drho += dt sum_j |u^n_j|^2 s_j
// First step: T -> T/2, D = rho (dt/2)|u~|^2, u~ = (u^0 + u^1*)/2 for the corrector (u^1* the
// predictor) and u~ = u^0 for the predictor; the corrector's u~-gradient rho dt s u~ is split evenly
// between u^0 and u^1*.
//
// Memory: a taped forward run keeps u^0, its final pair and the pair (u^{kC-1}, u^{kC}) at every
// multiple kC < N of the checkpoint interval C; the reverse pass recomputes each segment's states
// from its checkpoint (one extra forward step per step) and then runs the segment's adjoint steps.
#include <cmath>
#include "internal.cuh"
#include "cplx.cuh"
#include "solve.cuh"

namespace rfnse {

constexpr int kAdjThreads = 256;
constexpr int kAdjMaxBlocks = 152 * 8;

static inline int adj_blocks(long long N) {
  long long b = (N + kAdjThreads - 1) / kAdjThreads;
  if (b > kAdjMaxBlocks) b = kAdjMaxBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

__device__ __forceinline__ double adj_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;  // valid in thread 0
}

// f = -i conj(g): the block right-hand side of M u = conj(g) (f = -i b, Sec. 3).
__global__ void k_adj_rhs(const double2* __restrict__ g, double2* __restrict__ f, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = g[i];
    f[i] = make_double2(-v.y, -v.x);
  }
}

// lambda = conj(x).  If ga: s = -Re(conj(lambda)(ua + ub)), w = ud (or (ud + ud2)/2),
// ga += ca s w, gb = cb s w (if gb), and the block's sum of |w|^2 s goes to partials[block].
__global__ void __launch_bounds__(kAdjThreads) k_adj_point(const double2* __restrict__ x,
                                                           const double2* __restrict__ ua,
                                                           const double2* __restrict__ ub,
                                                           const double2* __restrict__ ud,
                                                           const double2* __restrict__ ud2, double2* __restrict__ lam,
                                                           double2* __restrict__ ga, double ca,
                                                           double2* __restrict__ gb, double cb,
                                                           double* __restrict__ partials, long long N) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 xv = x[i];
    const double2 l = make_double2(xv.x, -xv.y);
    lam[i] = l;
    if (!ga) continue;
    const double2 a = ua[i], b = ub[i];
    const double s = -(l.x * (a.x + b.x) + l.y * (a.y + b.y));
    double2 w = ud[i];
    if (ud2) {
      const double2 w2 = ud2[i];
      w.x = 0.5 * (w.x + w2.x);
      w.y = 0.5 * (w.y + w2.y);
    }
    double2 gv = ga[i];
    gv.x += ca * s * w.x;
    gv.y += ca * s * w.y;
    ga[i] = gv;
    if (gb) gb[i] = make_double2(cb * s * w.x, cb * s * w.y);
    acc += (w.x * w.x + w.y * w.y) * s;
  }
  if (!ga) return;
  acc = adj_block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// sum += scale * (partials[0] + ... + partials[nb-1]), summed in a fixed order (one block).
__global__ void __launch_bounds__(kAdjThreads) k_adj_rho(const double* __restrict__ partials, int nb, double scale,
                                                         double* __restrict__ sum) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v += partials[i];
  v = adj_block_sum(v, sh);
  if (threadIdx.x == 0) *sum += scale * v;
}

static void launch_adj_rhs(const double2* g, double2* f, long long N, cudaStream_t s) {
  count_launch();
  k_adj_rhs<<<adj_blocks(N), kAdjThreads, 0, s>>>(g, f, N);
}

// lambda = conj(x) plus, with ga, the s-terms; with rho_scale != 0 also dL/drho += rho_scale * sum.
static void launch_adj_point(rfnse_ctx* c, const double2* x, const double2* ua, const double2* ub,
                             const double2* ud, const double2* ud2, double2* lam, double2* ga, double ca,
                             double2* gb, double cb, double rho_scale) {
  const int nb = adj_blocks(c->N);
  count_launch();
  k_adj_point<<<nb, kAdjThreads, 0, c->stream>>>(x, ua, ub, ud, ud2, lam, ga, ca, gb, cb, c->adj_red, c->N);
  if (ga) {
    count_launch();
    k_adj_rho<<<1, kAdjThreads, 0, c->stream>>>(c->adj_red, nb, rho_scale, c->adj_red + kAdjMaxBlocks);
  }
}

// lambda = M^{-H} g for M = D - T + iI (mu_a / 2 when half): solve M u = conj(g), lambda = conj(u).
static rfnse_status adjoint_solve(rfnse_ctx* c, const double* D, const double2* g, int half, int* iters,
                                  double* relres) {
  launch_adj_rhs(g, c->f, c->N, c->stream);
  return solve_block(c, D, c->f, c->x, half, iters, relres);
}

// ---- tape ---------------------------------------------------------------------------------------
// Vectors of the tape (N complex each): 0 = u^0, 1-2 = final pair, then P checkpoint pairs, then
// C - 1 segment states, the predictor, three gradient vectors, lambda and the predictor's gradient.
struct TapeLayout {
  int P, C;
  size_t ckpt(int k, int which) const { return 3 + 2 * (size_t)(k - 1) + which; }  // k = 1..P
  size_t seg(int j) const { return 3 + 2 * (size_t)P + j; }                           // j = 0..C-2
  size_t pred() const { return 3 + 2 * (size_t)P + (C - 1); }
  size_t ring(int i) const { return pred() + 1 + i; }
  size_t lam() const { return pred() + 4; }
  size_t gpred() const { return pred() + 5; }
  size_t total() const { return pred() + 6; }
};

static TapeLayout layout_for(int nsteps, int every) {
  TapeLayout t;
  t.C = every;
  t.P = nsteps >= 1 ? (nsteps - 1) / every : 0;
  return t;
}

static double2* tv(rfnse_ctx* c, size_t i) { return c->tape + i * (size_t)c->N; }

}  // namespace rfnse

using namespace rfnse;

extern "C" {

int rfnse_tape_forward(rfnse_ctx* c, const void* u0, int nsteps, int every, void* uN, int* iters, int on_device) {
  NvtxRange range("rfnse tape forward");
  if (!c) return RFNSE_EINVAL;
  if (!u0 || nsteps < 0 || every < 1) {
    c->err = "rfnse_tape_forward: u0 required, nsteps >= 0, every >= 1";
    return RFNSE_EINVAL;
  }
  const long long N = c->N;
  const size_t bytes = sizeof(double2) * (size_t)N;
  const TapeLayout t = layout_for(nsteps, every);
  c->tape_steps = -1;
  if (c->tape_vecs < t.total()) {
    RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->tape);
    c->tape = nullptr;
    c->tape_vecs = 0;
    const cudaError_t e = dev_alloc((void**)&c->tape, bytes * t.total());
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->tape = nullptr;
      c->err = std::string("tape allocation: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? RFNSE_ENOMEM : RFNSE_ECUDA;
    }
    c->tape_vecs = t.total();
  }
  if (!c->adj_red) {
    const cudaError_t e = dev_alloc((void**)&c->adj_red, sizeof(double) * (kAdjMaxBlocks + 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->adj_red = nullptr;
      c->err = std::string("allocation: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? RFNSE_ENOMEM : RFNSE_ECUDA;
    }
  }
  RFNSE_CUDA_TRY(c, cudaMemcpyAsync(tv(c, 0), u0, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    c->stream));
  int st = rfnse_set_state(c, nullptr, tv(c, 0), 0, 1);
  if (st) return st;
  int worst = RFNSE_OK;
  for (int s = 1; s <= nsteps; ++s) {
    int it = 0;
    double rr = 0.0;
    const rfnse_status r = time_step(c, &it, &rr);
    if (r != RFNSE_OK && r != RFNSE_ENOCONV) return r;
    if (r == RFNSE_ENOCONV) worst = RFNSE_ENOCONV;
    if (iters) iters[s - 1] = it;
    if (s < nsteps && s % every == 0) {
      const int k = s / every;
      RFNSE_CUDA_TRY(c, cudaMemcpyAsync(tv(c, t.ckpt(k, 0)), c->u[c->iprev], bytes, cudaMemcpyDeviceToDevice,
                                        c->stream));
      RFNSE_CUDA_TRY(c, cudaMemcpyAsync(tv(c, t.ckpt(k, 1)), c->u[c->icur], bytes, cudaMemcpyDeviceToDevice,
                                        c->stream));
    }
  }
  if (nsteps >= 1)
    RFNSE_CUDA_TRY(c, cudaMemcpyAsync(tv(c, 1), c->u[c->iprev], bytes, cudaMemcpyDeviceToDevice, c->stream));
  RFNSE_CUDA_TRY(c, cudaMemcpyAsync(tv(c, 2), c->u[c->icur], bytes, cudaMemcpyDeviceToDevice, c->stream));
  if (uN)
    RFNSE_CUDA_TRY(c, cudaMemcpyAsync(uN, c->u[c->icur], bytes,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->tape_steps = nsteps;
  c->tape_every = every;
  return worst;
}

int rfnse_tape_backward(rfnse_ctx* c, const void* gN, void* g0, double* grho, int* iters, int on_device) {
  NvtxRange range("rfnse reverse pass");
  if (!c) return RFNSE_EINVAL;
  if (!gN || !g0 || c->tape_steps < 0) {
    c->err = "rfnse_tape_backward: needs gN, g0 and a taped run (rfnse_tape_forward)";
    return RFNSE_EINVAL;
  }
  const long long N = c->N;
  const size_t bytes = sizeof(double2) * (size_t)N;
  const int NS = c->tape_steps, C = c->tape_every;
  const TapeLayout t = layout_for(NS, C);
  const double rho = c->p.rho, dt = c->p.dt;
  const cudaMemcpyKind in_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind out_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  int total_it = 0, worst = RFNSE_OK;
  auto G = [&](int k) { return tv(c, t.ring(k % 3)); };
  double2* lam = tv(c, t.lam());
  double2* gpred = tv(c, t.gpred());
  double2* pred = tv(c, t.pred());

  RFNSE_CUDA_TRY(c, cudaMemcpyAsync(G(NS), gN, bytes, in_kind, c->stream));
  RFNSE_CUDA_TRY(c, cudaMemsetAsync(c->adj_red + kAdjMaxBlocks, 0, sizeof(double), c->stream));
  if (NS >= 1) launch_zero(G(NS - 1), N, c->stream);

  auto check = [&](rfnse_status r, int it) -> bool {
    total_it += it;
    if (r == RFNSE_ENOCONV) worst = RFNSE_ENOCONV;
    return r == RFNSE_OK || r == RFNSE_ENOCONV;
  };

  const int S = NS >= 1 ? (NS + C - 1) / C : 0;
  for (int k = S - 1; k >= 0; --k) {
    const int s0 = k * C;
    const int e = (k + 1) * C < NS ? (k + 1) * C : NS;
    // the states of this segment: u^{s0-1}, u^{s0} (checkpoint or u^0), u^{s0+1}..u^{e-1}
    // (recomputed), u^e (next checkpoint or the final state)
    auto U = [&](int m) -> const double2* {
      if (m == 0) return tv(c, 0);
      if (m == NS) return tv(c, 2);
      if (m == NS - 1) return tv(c, 1);
      if (m % C == 0) return tv(c, t.ckpt(m / C, 1));
      if ((m + 1) % C == 0) return tv(c, t.ckpt((m + 1) / C, 0));
      return tv(c, t.seg(m - s0 - 1));
    };
    int nrec = e - s0 - 1;
    if (k == 0 && c->p.first_step == 1 && nrec < 1) nrec = 1;  // the predictor
    if (nrec > 0) {
      int r = (s0 == 0) ? rfnse_set_state(c, nullptr, tv(c, 0), 0, 1)
                        : rfnse_set_state(c, U(s0 - 1), U(s0), s0, 1);
      if (r) return r;
      c->keep_pred = (s0 == 0 && c->p.first_step == 1) ? pred : nullptr;
      for (int m = s0 + 1; m <= s0 + nrec; ++m) {
        int it = 0;
        double rr = 0.0;
        const rfnse_status st = time_step(c, &it, &rr);
        c->keep_pred = nullptr;
        if (!check(st, 0)) return st;
        if (m < e)
          RFNSE_CUDA_TRY(c, cudaMemcpyAsync(tv(c, t.seg(m - s0 - 1)), c->u[c->icur], bytes, cudaMemcpyDeviceToDevice,
                                            c->stream));
      }
    }
    // adjoint steps n = e-1 .. max(s0, 1): (u^{n-1}, u^n) -> u^{n+1}
    for (int n = e - 1; n >= (s0 > 1 ? s0 : 1); --n) {
      const double2 *uo = U(n - 1), *uc = U(n), *un = U(n + 1);
      launch_diag(uc, nullptr, c->D, rho * dt, N, c->stream);
      int it = 0;
      double rr = 0.0;
      const rfnse_status st = adjoint_solve(c, c->D, G(n + 1), 0, &it, &rr);
      if (!check(st, it)) return st;
      launch_adj_point(c, c->x, un, uo, uc, nullptr, lam, G(n), 2.0 * rho * dt, nullptr, 0.0, dt);
      RFNSE_CUDA_TRY(c, run_matvec_fp64(c, lam, c->D, G(n - 1), nullptr, make_double2(0.0, -1.0),
                                        make_double2(1.0, 0.0), 0, nullptr));
    }
    if (k == 0) {  // first step (T/2); the gradient of u^0 accumulates in G(0)
      const double2* u0 = U(0);
      const double2* u1 = U(1);
      const double2* gsrc = G(1);
      const double2* u1p = u1;
      if (c->p.first_step == 1) {
        launch_diag(u0, pred, c->D, rho * dt * 0.5, N, c->stream);
        int it = 0;
        double rr = 0.0;
        const rfnse_status st = adjoint_solve(c, c->D, G(1), 1, &it, &rr);
        if (!check(st, it)) return st;
        launch_adj_point(c, c->x, u1, u0, u0, pred, lam, G(0), 0.5 * rho * dt, gpred, 0.5 * rho * dt, 0.5 * dt);
        RFNSE_CUDA_TRY(c, run_matvec_fp64(c, lam, c->D, G(0), G(0), make_double2(0.0, -1.0), make_double2(1.0, 0.0),
                                          1, nullptr));
        gsrc = gpred;
        u1p = pred;
      }
      launch_diag(u0, nullptr, c->D, rho * dt * 0.5, N, c->stream);
      int it = 0;
      double rr = 0.0;
      const rfnse_status st = adjoint_solve(c, c->D, gsrc, 1, &it, &rr);
      if (!check(st, it)) return st;
      launch_adj_point(c, c->x, u1p, u0, u0, nullptr, lam, G(0), rho * dt, nullptr, 0.0, 0.5 * dt);
      RFNSE_CUDA_TRY(c, run_matvec_fp64(c, lam, c->D, G(0), G(0), make_double2(0.0, -1.0), make_double2(1.0, 0.0), 1,
                                        nullptr));
    }
  }
  RFNSE_CUDA_TRY(c, cudaMemcpyAsync(g0, G(0), bytes, out_kind, c->stream));
  double acc = 0.0;
  RFNSE_CUDA_TRY(c, cudaMemcpyAsync(&acc, c->adj_red + kAdjMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (grho) *grho = acc;
  if (iters) *iters = total_it;
  // leave the context at the taped run's final state
  const int r = NS >= 1 ? rfnse_set_state(c, tv(c, 1), tv(c, 2), NS, 1) : rfnse_set_state(c, nullptr, tv(c, 2), 0, 1);
  if (r) return r;
  return worst;
}

int rfnse_adjoint_solve(rfnse_ctx* c, const double* D, const void* g, void* lam, int half, int* iters,
                        double* relres) {
  if (!c || !D || !g || !lam || g == lam) return RFNSE_EINVAL;
  if (!c->adj_red) {
    const cudaError_t e = dev_alloc((void**)&c->adj_red, sizeof(double) * (kAdjMaxBlocks + 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->adj_red = nullptr;
      c->err = std::string("allocation: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? RFNSE_ENOMEM : RFNSE_ECUDA;
    }
  }
  int it = 0;
  double rr = 0.0;
  const rfnse_status st = adjoint_solve(c, D, (const double2*)g, half ? 1 : 0, &it, &rr);
  if (st != RFNSE_OK && st != RFNSE_ENOCONV) return st;
  launch_adj_point(c, c->x, nullptr, nullptr, nullptr, nullptr, (double2*)lam, nullptr, 0.0, nullptr, 0.0, 0.0);
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return st;
}

}  // extern "C"
