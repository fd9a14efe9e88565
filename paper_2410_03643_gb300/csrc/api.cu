// C ABI (include/rfnse.h): context life cycle, state, time stepping and building blocks.
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>
#include "internal.cuh"
#include "fft_fixed.cuh"
#include "solve.cuh"

using namespace rfnse;

namespace {
bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
}  // namespace

namespace rfnse {

const char* validate_problem(const rfnse_params* p) {
  if (!p) return "params is NULL";
  if (p->d < 1 || p->d > 3) return "d must be 1, 2 or 3";
  for (int a = 0; a < p->d; ++a) {
    if (p->n[a] < 3 || p->n[a] > 2047 || !is_pow2((long long)p->n[a] + 1))
      return "n[a] + 1 must be a power of two between 4 and 2048";
    if (!(p->hi[a] > p->lo[a]) || !std::isfinite(p->hi[a] - p->lo[a])) return "need hi[a] > lo[a]";
  }
  if (!(p->alpha > 1.0 && p->alpha <= 2.0)) return "alpha must satisfy 1 < alpha <= 2";
  if (!(p->rho >= 0.0) || !std::isfinite(p->rho)) return "rho must be finite and >= 0";
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return "dt must be finite and > 0";
  if (!(p->omega > 0.0) || !std::isfinite(p->omega)) return "omega must be finite and > 0";
  return nullptr;
}

}  // namespace rfnse

namespace {
// Allocations still allowed before every later one fails (-1: no limit); rfnse_test_fail_allocations.
std::atomic<long long> g_alloc_budget{-1};

bool take_alloc_budget() {
  long long b = g_alloc_budget.load();
  while (b >= 0) {
    if (b == 0) return false;
    if (g_alloc_budget.compare_exchange_weak(b, b - 1)) return true;
  }
  return true;
}
}  // namespace

namespace rfnse {

cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (!take_alloc_budget()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t host_alloc_pinned(void** p, size_t bytes) {
  *p = nullptr;
  if (!take_alloc_budget()) return cudaErrorMemoryAllocation;
  return cudaMallocHost(p, bytes);
}

}  // namespace rfnse

namespace {

int ilog2(long long v) {
  int r = 0;
  while ((1LL << r) < v) ++r;
  return r;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return dev_alloc((void**)p, count * sizeof(T));
}

void free_ctx(rfnse_ctx* c) {
  if (!c) return;
  cudaFree(c->c);
  for (int a = 0; a < 3; ++a) {
    cudaFree(c->lam[a]);
    cudaFree(c->circ[a]);
    cudaFree(c->tw64[a]);
    cudaFree(c->tw32[a]);
    cudaFree(c->u[a]);
  }
  cudaFree(c->D);
  cudaFree(c->f);
  cudaFree(c->x);
  cudaFree(c->w);
  cudaFree(c->r);
  cudaFree(c->t1);
  cudaFree(c->t2);
  cudaFree(c->zb);
  cudaFree(c->V);
  cudaFree(c->Z32);
  cudaFree(c->t1f);
  cudaFree(c->t2f);
  cudaFree(c->wp32);
  for (int i = 0; i < 3; ++i) cudaFree(c->Tu[i]);
  cudaFree(c->D32);
  cudaFree(c->dfac64);
  cudaFree(c->dfac32);
  for (int h = 0; h < 2; ++h) {
    cudaFree(c->lamfac64[h]);
    cudaFree(c->lamfac32[h]);
    for (int a = 0; a < 3; ++a) {
      cudaFree(c->circ64s[h][a]);
      cudaFree(c->circ32s[h][a]);
    }
  }
  cudaFree(c->partials);
  cudaFree(c->counter);
  cudaFree(c->dbg_count);
  cudaFree(c->cmp_flag);
  cudaFree(c->gs);
  if (c->peek) cudaFreeHost(c->peek);
  for (cudaEvent_t ev : c->prof_events) cudaEventDestroy(ev);
  for (int a = 0; a < 2; ++a)
    for (int h = 0; h < 2; ++h) {
      if (c->graph_exec[a][h]) cudaGraphExecDestroy(c->graph_exec[a][h]);
      if (c->graph[a][h]) cudaGraphDestroy(c->graph[a][h]);
    }
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->cap_stream2) cudaStreamDestroy(c->cap_stream2);
  cudaFree(c->bar);
  cudaFree(c->coop_partials);
  cudaFree(c->dot_part);
  cudaFree(c->nrm_part);
  cudaFree(c->tape);
  cudaFree(c->adj_red);
  for (int a = 0; a < 3; ++a) {
    cudaFree(c->twdf[a]);
    for (int h = 0; h < 2; ++h) cudaFree(c->circdf[h][a]);
  }
  for (int a = 0; a < 3; ++a) {
    cudaFree(c->lamC[a]);
    cudaFree(c->chirp64[a]);
    cudaFree(c->chirp32[a]);
    cudaFree(c->bspec64[a]);
    cudaFree(c->bspec32[a]);
  }
  for (int h = 0; h < 2; ++h) {
    cudaFree(c->lamfacC64[h]);
    cudaFree(c->lamfacC32[h]);
  }
  delete c;
}

const char* validate(const rfnse_params* p) {
  if (const char* why = validate_problem(p)) return why;
  if (p->restart < 1 || p->restart > kMaxM) return "restart must be in 1..256";
  if (p->max_it < 1) return "max_it must be >= 1";
  if (!(p->tol > 0.0)) return "tol must be > 0";
  if (p->precision != 0 && p->precision != 1) return "precision must be 0 (FP64) or 1 (mixed)";
  if (p->first_step != 0 && p->first_step != 1) return "first_step must be 0 or 1";
  if (p->precond < 0 || p->precond > 2) return "precond must be 0 (tau), 1 (Strang circulant) or 2 (none)";
  return nullptr;
}

thread_local std::string g_create_error;

}  // namespace

extern "C" {

void rfnse_default_params(rfnse_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->d = 1;
  p->n[0] = p->n[1] = p->n[2] = 255;
  for (int a = 0; a < 3; ++a) {
    p->lo[a] = -20.0;
    p->hi[a] = 20.0;
  }
  p->alpha = 1.5;
  p->rho = 2.0;
  p->dt = 0.01;
  p->omega = 1.0;
  p->restart = 20;
  p->max_it = 2000;
  p->tol = 1e-10;
  p->precision = 0;
  p->first_step = 1;
  p->inner_tol = 1e-6;
  p->max_outer = 30;
  p->device_loop = 1;
  p->precond = 0;
}

int rfnse_create(const rfnse_params* p, void* stream, rfnse_ctx** out) {
  if (!out) return RFNSE_EINVAL;
  *out = nullptr;
  if (const char* why = validate(p)) {
    g_create_error = why;
    return RFNSE_EINVAL;
  }
  rfnse_ctx* c = new (std::nothrow) rfnse_ctx();
  if (!c) return RFNSE_ENOMEM;
  c->p = *p;
  c->stream = (cudaStream_t)stream;
  c->d = p->d;
  c->N = 1;
  int nmax = 0;
  for (int a = 0; a < 3; ++a) {
    c->n[a] = (a < c->d) ? p->n[a] : 1;
    c->stride[a] = c->N;
    c->N *= c->n[a];
    if (a < c->d) {
      c->L[a] = 2 * (c->n[a] + 1);
      c->log2L[a] = ilog2(c->L[a]);
      c->h[a] = (p->hi[a] - p->lo[a]) / (c->n[a] + 1);
      c->mu[a] = p->dt / std::pow(c->h[a], p->alpha);
      if (c->n[a] > nmax) nmax = c->n[a];
    } else {
      c->L[a] = 0;
      c->log2L[a] = 0;
      c->h[a] = 0.0;
      c->mu[a] = 0.0;
    }
  }
  const long long N = c->N;
  const int m = p->restart;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess && r != cudaSuccess) e = r;
  };
  chk(dalloc(&c->c, nmax));
  for (int a = 0; a < c->d; ++a) {
    chk(dalloc(&c->lam[a], c->n[a]));
    chk(dalloc(&c->circ[a], c->L[a]));
    chk(dalloc(&c->tw64[a], c->L[a]));
    chk(dalloc(&c->tw32[a], c->L[a]));
  }
  for (int i = 0; i < 3; ++i) chk(dalloc(&c->u[i], N));
  chk(dalloc(&c->D, N));
  chk(dalloc(&c->f, N));
  chk(dalloc(&c->x, N));
  chk(dalloc(&c->w, N));
  chk(dalloc(&c->r, N));
  chk(dalloc(&c->t1, N));
  chk(dalloc(&c->t2, N));
  chk(dalloc(&c->zb, N));
  chk(dalloc(&c->V, (size_t)(m + 1) * N));
  chk(dalloc(&c->t1f, N));
  chk(dalloc(&c->t2f, N));
  if (p->precision == 1) chk(dalloc(&c->Z32, (size_t)m * N));
  chk(dalloc(&c->wp32, N));
  if (p->precision == 1)
    for (int i = 0; i < 3; ++i) chk(dalloc(&c->Tu[i], N));
  chk(dalloc(&c->D32, N));
  chk(dalloc(&c->dfac64, N));
  chk(dalloc(&c->dfac32, N));
  for (int h = 0; h < 2; ++h) {
    chk(dalloc(&c->lamfac64[h], N));
    chk(dalloc(&c->lamfac32[h], N));
    for (int a = 0; a < c->d; ++a) {
      chk(dalloc(&c->circ64s[h][a], c->L[a]));
      chk(dalloc(&c->circ32s[h][a], c->L[a]));
    }
  }
  if (p->precond == 1) {
    for (int a = 0; a < c->d; ++a) {
      chk(dalloc(&c->lamC[a], c->n[a]));
      chk(dalloc(&c->chirp64[a], c->n[a]));
      chk(dalloc(&c->chirp32[a], c->n[a]));
      chk(dalloc(&c->bspec64[a], c->L[a]));
      chk(dalloc(&c->bspec32[a], c->L[a]));
    }
    for (int h = 0; h < 2; ++h) {
      chk(dalloc(&c->lamfacC64[h], N));
      chk(dalloc(&c->lamfacC32[h], N));
    }
  }
  if (p->precision == 1) {  // double-float Toeplitz passes of the residual when every axis has a fixed FFT
    bool all = true;
    for (int a = 0; a < c->d; ++a) all = all && fixed_fft_length(c->log2L[a]);
    if (all) {
      for (int a = 0; a < c->d; ++a) {
        chk(dev_alloc(&c->twdf[a], 16 * (size_t)c->L[a]));
        for (int h = 0; h < 2; ++h) chk(dev_alloc(&c->circdf[h][a], 8 * (size_t)c->L[a]));
      }
    }
  }
  c->red_blocks = choose_reduce_blocks(N);
  {
    const char* dbg = std::getenv("RFNSE_DEBUG");
    c->debug = dbg && dbg[0] == '1';
  }
  c->use_graphs = p->device_loop != 0 && !c->debug;  // debug checks synchronise after every pass
  if (c->debug) chk(dalloc(&c->dbg_count, 1));
  chk(dalloc(&c->cmp_flag, 2));
  c->coop_blocks = coop_blocks_for(N);
  chk(dalloc(&c->bar, 1));
  chk(dalloc(&c->coop_partials, 2 * (size_t)coop_blocks_max(N)));  // room for any grid the tuner picks
  chk(dalloc(&c->dot_part, (size_t)kDot0MaxBlocks));
  chk(dalloc(&c->nrm_part, 3 * (size_t)kNormPartMax));
  if (e == cudaSuccess) chk(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  if (e == cudaSuccess) chk(cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking));
  chk(dalloc(&c->partials, 1024));
  chk(dalloc(&c->counter, 1));
  chk(dalloc(&c->gs, 1));
  if (e == cudaSuccess) chk(host_alloc_pinned((void**)&c->peek, sizeof(GmresPeek)));
  if (e != cudaSuccess) {
    g_create_error = std::string("allocation failed: ") + cudaGetErrorString(e);
    cudaGetLastError();
    free_ctx(c);
    return (e == cudaErrorMemoryAllocation) ? RFNSE_ENOMEM : RFNSE_ECUDA;
  }
  chk(cudaMemsetAsync(c->counter, 0, sizeof(unsigned), c->stream));
  chk(cudaMemsetAsync(c->gs, 0, sizeof(GmresState), c->stream));
  chk(cudaMemsetAsync(c->bar, 0, sizeof(GridBarrier), c->stream));
  chk(cudaMemsetAsync(c->u[0], 0, sizeof(double2) * N, c->stream));
  chk(cudaMemsetAsync(c->u[1], 0, sizeof(double2) * N, c->stream));
  launch_setup_coefficients(c->c, nmax, p->alpha, c->stream);
  for (int a = 0; a < c->d; ++a) {
    launch_setup_axis(c->c, c->n[a], c->L[a], c->lam[a], c->circ[a], c->tw64[a], c->tw32[a], c->stream);
    if (p->precond == 1)
      launch_setup_circ(c->c, c->n[a], c->L[a], c->lamC[a], c->chirp64[a], c->chirp32[a], c->bspec64[a],
                        c->bspec32[a], c->stream);
  }
  for (int h = 0; h < 2; ++h) {  // h = 1: the first step's mu_a / 2
    const double hf = h ? 0.5 : 1.0;
    launch_setup_lamfac(c->lam[0], c->lam[1], c->lam[2], c->n[0], c->n[1], c->n[2], hf * c->mu[0], hf * c->mu[1],
                        hf * c->mu[2], p->omega, 1.0 / std::sqrt((double)c->L[c->d - 1]), 0, c->lamfac64[h],
                        c->lamfac32[h], N, c->stream);
    if (p->precond == 1)
      launch_setup_lamfac(c->lamC[0], c->lamC[1], c->lamC[2], c->n[0], c->n[1], c->n[2], hf * c->mu[0],
                          hf * c->mu[1], hf * c->mu[2], p->omega, 1.0 / (double)N, 1, c->lamfacC64[h],
                          c->lamfacC32[h], N, c->stream);
    for (int a = 0; a < c->d; ++a)
      launch_scale_circ(c->circ[a], c->L[a], hf * c->mu[a] / c->L[a], c->circ64s[h][a], c->circ32s[h][a],
                        c->stream);
  }
  if (c->twdf[0])
    for (int a = 0; a < c->d; ++a)
      launch_setup_df(c->log2L[a], c->circ64s[0][a], c->circ64s[1][a], c->twdf[a], c->circdf[0][a],
                      c->circdf[1][a], c->stream);
  chk(cudaGetLastError());
  chk(cudaStreamSynchronize(c->stream));
  if (e != cudaSuccess) {
    g_create_error = std::string("set-up failed: ") + cudaGetErrorString(e);
    free_ctx(c);
    return RFNSE_ECUDA;
  }
  *out = c;
  return RFNSE_OK;
}

void rfnse_destroy(rfnse_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
}

const char* rfnse_last_error(const rfnse_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

long long rfnse_size(const rfnse_ctx* ctx) { return ctx ? ctx->N : 0; }

int rfnse_set_state(rfnse_ctx* c, const void* u_prev, const void* u_cur, int step, int on_device) {
  if (!c) return RFNSE_EINVAL;
  if (!u_cur || step < 0 || (step > 0 && !u_prev)) {
    c->err = "rfnse_set_state: u_cur required; u_prev required when step > 0";
    return RFNSE_EINVAL;
  }
  const size_t bytes = sizeof(double2) * (size_t)c->N;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // A caller that continues its own run through host buffers loads the state the last step left
  // (u^{n-1}, u^n): the history slots whose contents come back unchanged keep their cached T u (mixed
  // form), so the next right-hand side needs no Toeplitz product.  The uploads land in the free slot
  // and a work vector and are compared bit by bit with the slots on the device.
  const int p = c->iprev, q = c->icur, f = 3 - p - q;
  if (step > 0 && c->step > 0 && c->cmp_flag && (c->tu_valid[p] || c->tu_valid[q])) {
    RFNSE_CUDA_TRY(c, cudaMemcpyAsync(c->u[f], u_prev, bytes, kind, c->stream));
    RFNSE_CUDA_TRY(c, cudaMemcpyAsync(c->t2, u_cur, bytes, kind, c->stream));
    launch_differs(c->u[f], c->u[p], c->N, c->cmp_flag, c->stream);
    launch_differs(c->t2, c->u[q], c->N, c->cmp_flag + 1, c->stream);
    int differs[2] = {1, 1};
    RFNSE_CUDA_TRY(c, cudaMemcpyAsync(differs, c->cmp_flag, sizeof(differs), cudaMemcpyDeviceToHost, c->stream));
    RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int np = differs[0] ? f : p;  // u^{n-1}: the uploaded copy, or the identical slot
    int nq = q;                         // u^n: the identical slot, or the uploaded copy moved into a slot
    if (differs[1]) {                   // other than u^{n-1}'s
      nq = (np == f) ? q : f;
      RFNSE_CUDA_TRY(c, cudaMemcpyAsync(c->u[nq], c->t2, bytes, cudaMemcpyDeviceToDevice, c->stream));
      RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    const bool keep_p = !differs[0] && c->tu_valid[p], keep_q = !differs[1] && c->tu_valid[q];
    for (int i = 0; i < 3; ++i) c->tu_valid[i] = false;
    c->tu_valid[np] = keep_p;  // keep_p implies np == p, keep_q implies nq == q
    c->tu_valid[nq] = keep_q;
    c->iprev = np;
    c->icur = nq;
    c->step = step;
    return RFNSE_OK;
  }
  c->iprev = 0;
  c->icur = 1;
  for (int i = 0; i < 3; ++i) c->tu_valid[i] = false;
  if (step > 0) RFNSE_CUDA_TRY(c, cudaMemcpyAsync(c->u[c->iprev], u_prev, bytes, kind, c->stream));
  RFNSE_CUDA_TRY(c, cudaMemcpyAsync(c->u[c->icur], u_cur, bytes, kind, c->stream));
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->step = step;
  return RFNSE_OK;
}

int rfnse_get_state(rfnse_ctx* c, void* u_prev, void* u_cur, int* step, int on_device) {
  if (!c) return RFNSE_EINVAL;
  const size_t bytes = sizeof(double2) * (size_t)c->N;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (u_prev && c->step > 0) RFNSE_CUDA_TRY(c, cudaMemcpyAsync(u_prev, c->u[c->iprev], bytes, kind, c->stream));
  if (u_cur) RFNSE_CUDA_TRY(c, cudaMemcpyAsync(u_cur, c->u[c->icur], bytes, kind, c->stream));
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (step) *step = c->step;
  return RFNSE_OK;
}

int rfnse_run(rfnse_ctx* c, int nsteps, void* traj, int* iters, double* relres, int on_device) {
  if (!c || nsteps < 0) return RFNSE_EINVAL;
  const size_t bytes = sizeof(double2) * (size_t)c->N;
  int worst = RFNSE_OK;
  for (int s = 0; s < nsteps; ++s) {
    int it = 0;
    double rr = 0.0;
    NvtxRange range("rfnse step");
    rfnse_status st = time_step(c, &it, &rr);
    if (c->debug && !c->dbg_first.empty() && (st == RFNSE_OK || st == RFNSE_ENOCONV || st == RFNSE_ENUMERIC)) {
      c->err = "debug check: first non-finite output after " + c->dbg_first;
      c->dbg_first.clear();
      st = RFNSE_ENUMERIC;
    }
    if (st != RFNSE_OK && st != RFNSE_ENOCONV) return st;
    if (st == RFNSE_ENOCONV) worst = RFNSE_ENOCONV;
    if (iters) iters[s] = it;
    if (relres) relres[s] = rr;
    if (traj) {
      char* dst = (char*)traj + (size_t)s * bytes;
      RFNSE_CUDA_TRY(c, cudaMemcpyAsync(dst, c->u[c->icur], bytes,
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    }
  }
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return worst;
}

int rfnse_apply_A(rfnse_ctx* c, const void* u, void* out, const double* D, int half) {
  if (!c || !u || !out || !D || u == out) return RFNSE_EINVAL;
  RFNSE_CUDA_TRY(c, run_apply_A(c, (const double2*)u, (double2*)out, D, half ? 1 : 0));
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RFNSE_OK;
}

int rfnse_apply_prec(rfnse_ctx* c, const void* v, void* z, const double* D, int half, int precision) {
  if (!c || !v || !z || !D || v == z || (precision != 0 && precision != 1)) return RFNSE_EINVAL;
  RFNSE_CUDA_TRY(c, run_apply_prec(c, (const double2*)v, (double2*)z, D, half ? 1 : 0, precision));
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RFNSE_OK;
}

int rfnse_dst(rfnse_ctx* c, int axis, const void* in, void* out, int precision) {
  if (!c || !in || !out || in == out || axis < 0 || axis >= c->d || (precision != 0 && precision != 1))
    return RFNSE_EINVAL;
  RFNSE_CUDA_TRY(c, run_dst(c, axis, (const double2*)in, (double2*)out, precision));
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RFNSE_OK;
}

int rfnse_toeplitz(rfnse_ctx* c, int axis, const void* in, void* out, int half) {
  if (!c || !in || !out || in == out || axis < 0 || axis >= c->d) return RFNSE_EINVAL;
  RFNSE_CUDA_TRY(c, run_toeplitz(c, axis, (const double2*)in, (double2*)out, half ? 1 : 0));
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RFNSE_OK;
}

int rfnse_solve(rfnse_ctx* c, const double* D, const void* b, void* u, int half, int* iters, double* relres) {
  if (!c || !D || !b || !u || b == u) return RFNSE_EINVAL;
  launch_neg_i((const double2*)b, c->f, c->N, c->stream);  // f = -i b  (Sec. 3: f = [-p; q])
  int it = 0;
  double rr = 0.0;
  const rfnse_status st = solve_block(c, D, c->f, (double2*)u, half ? 1 : 0, &it, &rr);
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return st;
}

int rfnse_tban_solve(rfnse_ctx* c, const double* D, const void* b, void* u, int half, int* iters, double* relres) {
  if (!c || !D || !b || !u || b == u) return RFNSE_EINVAL;
  launch_neg_i((const double2*)b, c->f, c->N, c->stream);  // f = -i b  (Sec. 3: f = [-p; q])
  int it = 0;
  double rr = 0.0;
  const rfnse_status st = tban_solve(c, D, c->f, (double2*)u, half ? 1 : 0, &it, &rr);
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return st;
}

int rfnse_get_coefficients(rfnse_ctx* c, double* cc, double* lam) {
  if (!c) return RFNSE_EINVAL;
  int nmax = 0;
  for (int a = 0; a < c->d; ++a) nmax = c->n[a] > nmax ? c->n[a] : nmax;
  if (cc) RFNSE_CUDA_TRY(c, cudaMemcpyAsync(cc, c->c, sizeof(double) * nmax, cudaMemcpyDeviceToHost, c->stream));
  if (lam) {
    size_t off = 0;
    for (int a = 0; a < c->d; ++a) {
      RFNSE_CUDA_TRY(c, cudaMemcpyAsync(lam + off, c->lam[a], sizeof(double) * c->n[a], cudaMemcpyDeviceToHost,
                                        c->stream));
      off += c->n[a];
    }
  }
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RFNSE_OK;
}

long long rfnse_launch_count(void) { return g_kernel_launches.load(); }

int rfnse_autotune(rfnse_ctx* c, int reps, int force, int* n_configs, int* n_changed, double* est_speedup) {
  if (!c || reps < 1 || reps > 1000) return RFNSE_EINVAL;
  return autotune(c, reps, force, n_configs, n_changed, est_speedup);
}

long long rfnse_tuned_launches(const rfnse_ctx* c) { return c ? c->tuned_launches : 0; }

int rfnse_set_arnoldi_grid(rfnse_ctx* c, int blocks) {
  if (!c) return RFNSE_EINVAL;
  int g = blocks;
  if (g == 0) g = coop_blocks_for(c->N);
  else if (g > 0 && (c->N <= 4096 ? g != 1 : g > coop_blocks_max(c->N))) g = 0;
  else if (g < 0 && (g != -8 && g != -16)) g = 0;
  else if (g < 0 && !mgs_cluster_fits(-g)) g = 0;
  if (g == 0) {
    c->err = "rfnse_set_arnoldi_grid: blocks must be 1..co-resident maximum, -8 or -16 (a cluster that fits)";
    return RFNSE_EINVAL;
  }
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->coop_blocks = g;
  for (int a = 0; a < 2; ++a)  // the cached solve graphs hold the old launch: capture them again
    for (int h = 0; h < 2; ++h) {
      if (c->graph_exec[a][h]) cudaGraphExecDestroy(c->graph_exec[a][h]);
      if (c->graph[a][h]) cudaGraphDestroy(c->graph[a][h]);
      c->graph_exec[a][h] = nullptr;
      c->graph[a][h] = nullptr;
    }
  return RFNSE_OK;
}

int rfnse_arnoldi_grid(const rfnse_ctx* c) { return c ? c->coop_blocks : 0; }

int rfnse_test_fail_allocations(long long after) {
  g_alloc_budget.store(after < 0 ? -1 : after);
  return RFNSE_OK;
}

int rfnse_profile(rfnse_ctx* c, int kind) {
  if (!c || kind < 0) return RFNSE_EINVAL;
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->prof_kind = kind;
  c->prof_used = 0;
  c->prof_flops = 0.0;
  c->prof_bytes = 0.0;
  return RFNSE_OK;
}

int rfnse_profile_read(rfnse_ctx* c, int* launches, double* ms, double* flops, double* bytes) {
  if (!c) return RFNSE_EINVAL;
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  double total = 0.0;
  for (size_t i = 0; i + 1 < c->prof_used; i += 2) {
    float t = 0.f;
    RFNSE_CUDA_TRY(c, cudaEventElapsedTime(&t, c->prof_events[i], c->prof_events[i + 1]));
    total += t;
  }
  if (launches) *launches = (int)(c->prof_used / 2);
  if (ms) *ms = total;
  if (flops) *flops = c->prof_flops;
  if (bytes) *bytes = c->prof_bytes;
  return RFNSE_OK;
}

}  // extern "C"
