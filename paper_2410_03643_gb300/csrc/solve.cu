// Solver drivers: the preconditioner and matrix sequences of line passes, right-preconditioned
// GMRES (FP64), the mixed-precision FGMRES with FP64 iterative refinement, and the time steps.
//
// Two ways to drive a solve:
//   * device loop (default): the whole solve is one CUDA graph whose conditional WHILE nodes (outer
//     restart / refinement cycles, inner Arnoldi steps) are decided by the kernels themselves; the host
//     launches the graph and reads the statistics once;
//   * host loop: the host reads the Arnoldi state after every step and launches the next kernels.
// Both run the same algorithm on the same kernels' arithmetic.
#include <algorithm>
#include <cmath>
#include <limits>
#include <mutex>
#include <tuple>
#include "internal.cuh"
#include "passes.cuh"
#include "solve.cuh"
#include "precon.cuh"

namespace rfnse {

RFNSE_PRECON_VARIANTS(RFNSE_PRECON_EXTERN, 1)
RFNSE_PRECON_VARIANTS(RFNSE_PRECON_EXTERN, 2)

// The preconditioner the context was created with (rfnse_params::precond), then the product.
template <typename R, typename TIN, typename TMP, typename TZ, typename TW, bool INSC, bool MATVEC>
cudaError_t run_precon(rfnse_ctx* c, const TIN* v, const double* in_scale, double2* copy_v, TZ* z, int z_add,
                       const double* D, double2* w, TW* wtmp, const double2* w_add, double2 a, double2 b, int half,
                       TMP* t1, TMP* t2, const Dyn& dyn = Dyn()) {
  switch (c->p.precond) {
    case 1:
      return run_precon_pc<1, R, TIN, TMP, TZ, TW, INSC, MATVEC>(c, v, in_scale, copy_v, z, z_add, D, w, wtmp,
                                                                  w_add, a, b, half, t1, t2, dyn);
    case 2:
      return run_precon_pc<2, R, TIN, TMP, TZ, TW, INSC, MATVEC>(c, v, in_scale, copy_v, z, z_add, D, w, wtmp,
                                                                  w_add, a, b, half, t1, t2, dyn);
    default:
      return run_precon_pc<0, R, TIN, TMP, TZ, TW, INSC, MATVEC>(c, v, in_scale, copy_v, z, z_add, D, w, wtmp,
                                                                  w_add, a, b, half, t1, t2, dyn);
  }
}

// The per-point factors of the (omega I + D) sub-solve for diagonal D (recomputed when D changes).
cudaError_t prepare_D(rfnse_ctx* c, const double* D) {
  launch_prep_D(D, c->D32, c->dfac64, c->dfac32, c->p.omega, c->N, c->stream);
  return cudaGetLastError();
}

// w = add + a z + b (T - D) z in FP64 (the Toeplitz products by circulant embedding).  In the mixed
// form the FFTs of the embedding run in double-float (toep_df.cu) when every axis has a fixed FFT.
cudaError_t run_matvec_fp64(rfnse_ctx* c, const double2* z, const double* D, double2* w, const double2* add,
                            double2 a, double2 b, int half, const int* skip, double* nrm_part) {
  cudaStream_t s = c->stream;
  cudaError_t e;
  const int h = half ? 1 : 0;
  c->nrm_df_blocks = 0;
  if (c->p.precision == 1 && toeplitz_df_available(c)) {
    // the last pass may leave the partials of ||w||^2 (c->nrm_df_blocks of them).  With several axes the
    // first pass splits z into double-float once, into the FP64 work vector t1 (16 bytes per point,
    // unused by the mixed form while a product runs), and the others read the split copy
    const bool multi = c->d > 1;
    void* zdf = multi ? (void*)c->t1 : nullptr;
    if ((e = run_toeplitz_df(c, 0, h, true, z, D, add, w, a, b, skip, multi ? nullptr : nrm_part, nullptr, zdf)) !=
        cudaSuccess)
      return e;
    for (int a2 = 1; a2 < c->d; ++a2)
      if ((e = run_toeplitz_df(c, a2, h, false, z, nullptr, w, w, a, b, skip, a2 == c->d - 1 ? nrm_part : nullptr,
                               zdf, nullptr)) != cudaSuccess)
        return e;
    return cudaSuccess;
  }
  {
    PassParams p = base_params<double>(c, 0, h);
    p.in = z; p.Dr = D; p.acc_in = add; p.acc_out = w; p.ca = a; p.cb = b; p.skip = skip;
    if ((e = launch_pass<double, double2, double2, double2, double2, F_TOEP_X>(c, p, s)) != cudaSuccess) return e;
  }
  for (int a2 = 1; a2 < c->d; ++a2) {
    PassParams p = base_params<double>(c, a2, h);
    p.in = z; p.acc_in = w; p.acc_out = w; p.cb = b; p.skip = skip;
    if ((e = launch_pass<double, double2, double2, double2, double2, F_TOEP_ACC>(c, p, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t run_dst(rfnse_ctx* c, int axis, const double2* in, double2* out, int precision) {
  if (precision) {
    PassParams p = base_params<float>(c, axis, 0);
    p.in = in; p.out = out;
    return launch_pass<float, double2, double2, double2, double2, F_DST>(c, p, c->stream);
  }
  PassParams p = base_params<double>(c, axis, 0);
  p.in = in; p.out = out;
  return launch_pass<double, double2, double2, double2, double2, F_DST>(c, p, c->stream);
}

cudaError_t run_toeplitz(rfnse_ctx* c, int axis, const double2* in, double2* out, int half) {
  PassParams p = base_params<double>(c, axis, half ? 1 : 0);
  p.in = in; p.acc_in = nullptr; p.acc_out = out; p.cb = kOne;
  return launch_pass<double, double2, double2, double2, double2, F_TOEP_ACC>(c, p, c->stream);
}

cudaError_t run_apply_prec(rfnse_ctx* c, const double2* v, double2* z, const double* D, int half, int precision) {
  cudaError_t e = prepare_D(c, D);
  if (e != cudaSuccess) return e;
  if (precision) {
    if (!c->t1f) return cudaErrorInvalidValue;
    return run_precon<float, double2, float2, double2, float2, false, false>(
        c, v, nullptr, nullptr, z, 0, D, nullptr, nullptr, nullptr, kOne, kI, half, c->t1f, c->t2f);
  }
  return run_precon<double, double2, double2, double2, double2, false, false>(
      c, v, nullptr, nullptr, z, 0, D, nullptr, nullptr, nullptr, kOne, kI, half, c->t1, c->t2);
}

cudaError_t run_apply_A(rfnse_ctx* c, const double2* u, double2* out, const double* D, int half) {
  // (D - T + iI) u = i u - (T - D) u
  return run_matvec_fp64(c, u, D, out, nullptr, kI, kMinusOne, half, nullptr);
}

// ---------------------------------------------------------------------------------------------

static rfnse_status peek(rfnse_ctx* c, GmresPeek* out) {
  RFNSE_CUDA_TRY(c, cudaMemcpyAsync(c->peek, c->gs, sizeof(GmresPeek), cudaMemcpyDeviceToHost, c->stream));
  RFNSE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *out = *c->peek;
  return RFNSE_OK;
}

// ---- host loop -------------------------------------------------------------------------------

static SolveCfg make_cfg(const rfnse_ctx* c, int mixed) {
  SolveCfg cfg{};
  cfg.m = c->p.restart;
  cfg.max_it = c->p.max_it;
  cfg.max_outer = mixed ? (c->p.max_outer > 0 ? c->p.max_outer : 30) : (1 << 30);
  cfg.mixed = mixed;
  cfg.tol = c->p.tol;
  cfg.eta_min = c->p.inner_tol > 0 ? c->p.inner_tol : 1e-6;
  return cfg;
}

SolveCfg solve_cfg(const rfnse_ctx* c, int mixed) { return make_cfg(c, mixed); }

// The line passes of one Arnoldi step of the mixed form with device-resolved operands (as the solve
// graphs launch them), recorded for a lock-step batch (c->param_rec set) with the given skip flag.
cudaError_t record_mixed_arnoldi_passes(rfnse_ctx* c, const int* skip) {
  Dyn dyn;
  dyn.gs = c->gs;
  dyn.vbase = c->V;
  dyn.zbase = c->Z32;
  dyn.ldv = c->N;
  dyn.skip = skip;
  dyn.dot0 = true;
  return run_precon<float, double2, float2, float2, float2, true, true>(
      c, nullptr, nullptr, nullptr, c->Z32, 0, c->D, c->w, c->wp32, nullptr, kOne, kI, 0, c->t1f, c->t2f, dyn);
}

// Host-driven Arnoldi steps: operands from the host, but the last product pass leaves the partials of
// <v_0, w> for the Arnoldi kernel as in the device loop.
static Dyn dot0_dyn(rfnse_ctx* c) {
  Dyn d;
  d.vbase = c->V;
  d.dot0 = true;
  return d;
}

// Modified Gram-Schmidt of w against V_0..V_j, then h_{j+1,j}, Givens and the convergence test: the
// cooperative kernel of the device loop, launched on its own (gs->j = j).  Timed per launch under
// rfnse_profile(RFNSE_K_ARNOLDI).
static cudaError_t arnoldi_orthogonalise(rfnse_ctx* c, int j) {
  const long long N = c->N;
  const SolveCfg cfg = make_cfg(c, c->p.precision == 1 ? 1 : 0);
  const bool prof = c->prof_kind == RFNSE_K_ARNOLDI;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof) {
    while (c->prof_used + 2 > c->prof_events.size()) {
      cudaEvent_t ev;
      const cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return e;
      c->prof_events.push_back(ev);
    }
    e0 = c->prof_events[c->prof_used];
    e1 = c->prof_events[c->prof_used + 1];
    c->prof_used += 2;
    cudaEventRecord(e0, c->stream);
  }
  const cudaError_t e = launch_mgs_step(c->gs, c->V, N, c->w, N, c->coop_partials, c->bar, cfg, 0, 0,
                                        c->coop_blocks, c->stream, c->dot_part, c->dot0_blocks);
  if (prof) {
    cudaEventRecord(e1, c->stream);
    c->prof_flops += (8.0 * (j + 1) + 4.0) * (double)N;  // dot and update per basis vector, the norm
    c->prof_bytes += 16.0 * (j + 3) * (double)N;         // V_0..V_j and w read once, w written once
  }
  return e;
}

// Right-preconditioned GMRES(m) for R x = f, x0 = 0 (paper Sec. 5 protocol), all FP64.
static rfnse_status gmres_fp64(rfnse_ctx* c, const double* D, const double2* f, double2* x, int half, int* iters,
                               double* relres) {
  const long long N = c->N;
  const Dyn dot0 = dot0_dyn(c);
  const int m = c->p.restart;
  const double tol = c->p.tol;
  GmresPeek pk;
  launch_zero(x, N, c->stream);
  launch_norm(f, c->gs, N, c->red_blocks, c->partials, c->counter, c->stream);
  rfnse_status st = peek(c, &pk);
  if (st) return st;
  const double fnorm = pk.beta;
  *iters = 0;
  *relres = 0.0;
  if (!std::isfinite(fnorm)) { c->err = "non-finite right-hand side"; return RFNSE_ENUMERIC; }
  if (fnorm == 0.0) return RFNSE_OK;
  launch_start_cycle(c->gs, fnorm, tol, c->stream);
  const double2* r = f;
  double beta = fnorm;
  int it = 0;
  for (;;) {
    if (beta / fnorm < tol) { *relres = beta / fnorm; break; }
    const double2* src = r;
    const double* scale = &c->gs->inv_beta;
    int k = 0;
    int done = 0;
    double rel = beta / fnorm;
    for (int j = 0; j < m; ++j) {
      RFNSE_CUDA_TRY(c, (run_precon<double, double2, double2, double2, double2, true, true>(
                            c, src, scale, c->V + (size_t)j * N, c->zb, 0, D, c->w, c->w, nullptr, kOne, kI, half,
                            c->t1, c->t2, dot0)));
      RFNSE_CUDA_TRY(c, arnoldi_orthogonalise(c, j));
      if ((st = peek(c, &pk))) return st;
      if (pk.err) { c->err = "a bounded device-side wait gave up"; return RFNSE_ETIMEOUT; }
      ++it;
      k = j + 1;
      rel = pk.relres;
      done = pk.done;
      if (done == 3) { c->err = "non-finite value in the Arnoldi process"; return RFNSE_ENUMERIC; }
      if (done || it >= c->p.max_it) break;
      src = c->w;
      scale = &c->gs->inv_h;
    }
    launch_backsolve(c->gs, k, c->stream);
    launch_combine(c->V, N, c->gs, k, c->r, N, c->stream);
    RFNSE_CUDA_TRY(c, (run_precon<double, double2, double2, double2, double2, false, false>(
                          c, c->r, nullptr, nullptr, x, 1, D, nullptr, nullptr, nullptr, kOne, kI, half, c->t1,
                          c->t2)));
    *relres = rel;
    if (done) break;
    if (it >= c->p.max_it) {
      *iters = it;
      c->err = "GMRES reached max_it";
      return RFNSE_ENOCONV;
    }
    // restart: true residual r = f - R x
    RFNSE_CUDA_TRY(c, run_matvec_fp64(c, x, D, c->r, f, kMinusOne, kMinusI, half, nullptr));
    launch_norm(c->r, c->gs, N, c->red_blocks, c->partials, c->counter, c->stream);
    if ((st = peek(c, &pk))) return st;
    beta = pk.beta;
    if (!std::isfinite(beta)) { c->err = "non-finite residual"; return RFNSE_ENUMERIC; }
    launch_start_cycle(c->gs, fnorm, tol, c->stream);
    r = c->r;
    *relres = beta / fnorm;
  }
  *iters = it;
  return RFNSE_OK;
}

// Mixed form: FP64 outer iterative refinement r = f - R x; each correction from an FGMRES inner solve
// whose preconditioner and matrix products run in FP32 while the Arnoldi basis, Gram-Schmidt,
// Givens and the solution update stay FP64.  Stops on the true FP64 relative residual.
static rfnse_status solve_mixed(rfnse_ctx* c, const double* D, const double2* f, double2* x, int half, int* iters,
                                double* relres, int* outer_out) {
  const long long N = c->N;
  const Dyn dot0 = dot0_dyn(c);
  const int m = c->p.restart;
  const double tol = c->p.tol;
  const double eta_min = c->p.inner_tol > 0 ? c->p.inner_tol : 1e-6;
  const int max_outer = c->p.max_outer > 0 ? c->p.max_outer : 30;
  GmresPeek pk;
  c->resid_current = false;
  launch_zero(x, N, c->stream);
  launch_norm(f, c->gs, N, c->red_blocks, c->partials, c->counter, c->stream);
  rfnse_status st = peek(c, &pk);
  if (st) return st;
  const double fnorm = pk.beta;
  *iters = 0;
  *relres = 0.0;
  *outer_out = 0;
  if (!std::isfinite(fnorm)) { c->err = "non-finite right-hand side"; return RFNSE_ENUMERIC; }
  if (fnorm == 0.0) return RFNSE_OK;
  const double2* r = f;
  double beta = fnorm;
  double margin = 0.0;  // error bound of a residual formed by the recurrence
  int it = 0, outer = 0;
  for (;;) {
    *relres = beta / fnorm;
    if (beta / fnorm + margin < tol) break;
    if (outer >= max_outer || it >= c->p.max_it) {
      *iters = it;
      *outer_out = outer;
      c->err = "mixed-precision refinement did not reach tol";
      return RFNSE_ENOCONV;
    }
    const double eta = std::max(eta_min, 0.1 * tol * fnorm / beta);
    launch_start_cycle(c->gs, beta, eta, c->stream);
    const double2* src = r;
    const double* scale = &c->gs->inv_beta;
    int k = 0;
    for (int j = 0; j < m && it < c->p.max_it; ++j) {
      RFNSE_CUDA_TRY(c, (run_precon<float, double2, float2, float2, float2, true, true>(
                            c, src, scale, c->V + (size_t)j * N, c->Z32 + (size_t)j * N, 0, D, c->w, c->wp32,
                            nullptr, kOne, kI, half, c->t1f, c->t2f, dot0)));
      RFNSE_CUDA_TRY(c, arnoldi_orthogonalise(c, j));
      if ((st = peek(c, &pk))) return st;
      if (pk.err) { c->err = "a bounded device-side wait gave up"; return RFNSE_ETIMEOUT; }
      ++it;
      k = j + 1;
      if (pk.done == 3) { c->err = "non-finite value in the Arnoldi process"; return RFNSE_ENUMERIC; }
      if (pk.done) break;
      src = c->w;
      scale = &c->gs->inv_h;
    }
    launch_backsolve(c->gs, k, c->stream);
    launch_combine_f32_add(c->Z32, N, c->gs, k, x, N, c->stream);
    // the new residual: FP64 product after the first cycle and while beta is large, else the
    // recurrence from the Arnoldi basis (k_resid_coeffs)
    const int upd = (outer >= 1 && beta <= kUpdRatio * tol * fnorm) ? 1 : 0;
    margin = upd ? kUpdErr * beta / fnorm : 0.0;
    ++outer;
    if (upd) {
      launch_resid_coeffs(c->gs, k, 1, margin, tol, c->stream);
      launch_resid_update(c->V, N, c->w, c->gs, k, c->r, N, c->stream);
    } else {
      launch_resid_coeffs(c->gs, k, 0, 0.0, tol, c->stream);
      RFNSE_CUDA_TRY(c, run_matvec_fp64(c, x, D, c->r, f, kMinusOne, kMinusI, half, nullptr));
    }
    launch_norm(c->r, c->gs, N, c->red_blocks, c->partials, c->counter, c->stream);
    if ((st = peek(c, &pk))) return st;
    beta = pk.beta;
    if (!std::isfinite(beta)) { c->err = "non-finite residual"; return RFNSE_ENUMERIC; }
    r = c->r;
    c->resid_current = true;
  }
  *iters = it;
  *outer_out = outer;
  return RFNSE_OK;
}

// ---- device loop: the solve as one CUDA graph ------------------------------------------------

// Add a conditional WHILE node at the current capture position of stream s and make it the capture's
// dependency; returns its body graph.
cudaError_t add_while_node(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &edges, &nd);
  if (e != cudaSuccess) return e;
  if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, edges, nd, &np)) != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// One Arnoldi step with operands resolved on the device: z = M^{-1} v_j, w = R z, then MGS/Givens.
static cudaError_t arnoldi_step_dev(rfnse_ctx* c, int half, const SolveCfg& cfg, cudaGraphConditionalHandle hi,
                                    int set_cond) {
  const long long N = c->N;
  cudaError_t e;
  Dyn dyn;
  dyn.gs = c->gs;
  dyn.vbase = c->V;
  dyn.ldv = N;
  dyn.dot0 = true;
  if (cfg.mixed) {
    dyn.zbase = c->Z32;
    e = run_precon<float, double2, float2, float2, float2, true, true>(
        c, nullptr, nullptr, nullptr, c->Z32, 0, c->D, c->w, c->wp32, nullptr, kOne, kI, half, c->t1f, c->t2f, dyn);
  } else {
    e = run_precon<double, double2, double2, double2, double2, true, true>(
        c, nullptr, nullptr, nullptr, c->zb, 0, c->D, c->w, c->w, nullptr, kOne, kI, half, c->t1, c->t2, dyn);
  }
  if (e != cudaSuccess) return e;
  return launch_mgs_step(c->gs, c->V, N, c->w, N, c->coop_partials, c->bar, cfg, hi, set_cond, c->coop_blocks,
                         c->stream, c->dot_part, c->dot0_blocks);
}

// Record the solve of R x = f (c->f, c->x, c->D fixed) for one precision and half flag at the current
// capture position of stream s, which is capturing into graph g: x = 0, ||f||, then the outer WHILE
// node.  The loop bodies are captured on the context's private body stream.
cudaError_t capture_solve(rfnse_ctx* c, int mixed, int half, cudaGraph_t g, cudaStream_t s, const double* f_part,
                          int f_n) {
  const long long N = c->N;
  const SolveCfg cfg = make_cfg(c, mixed);
  cudaStream_t user = c->stream;
  cudaStream_t bs = c->cap_stream;
  cudaGraph_t obody = nullptr, ibody = nullptr;
  cudaGraphConditionalHandle ho = 0, hi = 0;
  cudaError_t e;
  auto fail = [&](cudaError_t err) {
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(bs, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(bs, &junk);
    }
    c->stream = user;
    return err;
  };
  if ((e = cudaGraphConditionalHandleCreate(&ho, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return fail(e);
  // solve start: x = 0, beta = ||f||, outer condition
  c->stream = s;
  launch_zero(c->x, N, s);
  launch_norm_ctl(c->f, c->gs, N, c->red_blocks, c->partials, c->counter, c->bar, cfg, 0, ho, 1, s, f_part, f_n);
  if ((e = add_while_node(s, ho, &obody)) != cudaSuccess) return fail(e);
  // outer body: cycle start, inner loop, solution update, residual and the outer condition
  c->stream = bs;
  if ((e = cudaGraphConditionalHandleCreate(&hi, obody, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
    return fail(e);
  if ((e = cudaStreamBeginCaptureToGraph(bs, obody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
      cudaSuccess)
    return fail(e);
  launch_cycle_begin(c->gs, cfg, hi, ho, 1, bs);
  if ((e = add_while_node(bs, hi, &ibody)) != cudaSuccess) return fail(e);
  if (mixed) {
    launch_cycle_end_mixed(c->Z32, N, c->gs, c->x, N, cfg.tol, bs);
    // the residual (product or recurrence, whichever runs) leaves the partials of ||r||^2
    double* part_df = c->nrm_part + kNormPartMax;
    double* part_upd = c->nrm_part + 2 * kNormPartMax;
    if ((e = run_matvec_fp64(c, c->x, c->D, c->r, c->f, kMinusOne, kMinusI, half, &c->gs->upd, part_df)) !=
        cudaSuccess)
      return fail(e);
    launch_resid_update(c->V, N, c->w, c->gs, -1, c->r, N, bs, part_upd);
    launch_norm_ctl(c->r, c->gs, N, c->red_blocks, c->partials, c->counter, c->bar, cfg, 2, ho, 1, bs, part_upd,
                    resid_update_blocks(N), part_df, c->nrm_df_blocks);
  } else {
    launch_backsolve_dev(c->gs, bs);
    launch_combine_dev(c->V, N, c->gs, c->r, N, bs);
    if ((e = run_precon<double, double2, double2, double2, double2, false, false>(
             c, c->r, nullptr, nullptr, c->x, 1, c->D, nullptr, nullptr, nullptr, kOne, kI, half, c->t1, c->t2)) !=
        cudaSuccess)
      return fail(e);
    if ((e = run_matvec_fp64(c, c->x, c->D, c->r, c->f, kMinusOne, kMinusI, half, &c->gs->no_restart)) !=
        cudaSuccess)
      return fail(e);
    launch_norm_ctl(c->r, c->gs, N, c->red_blocks, c->partials, c->counter, c->bar, cfg, 1, ho, 1, bs);
  }
  if ((e = cudaStreamEndCapture(bs, &obody)) != cudaSuccess) return fail(e);
  // inner body: one Arnoldi step
  if ((e = cudaStreamBeginCaptureToGraph(bs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
      cudaSuccess)
    return fail(e);
  if ((e = arnoldi_step_dev(c, half, cfg, hi, 1)) != cudaSuccess) return fail(e);
  if ((e = cudaStreamEndCapture(bs, &ibody)) != cudaSuccess) return fail(e);
  c->stream = user;
  return cudaSuccess;
}

// The solve alone as an instantiated graph, cached per (precision, half).
static cudaError_t build_solve_graph(rfnse_ctx* c, int mixed, int half) {
  cudaStream_t s = c->cap_stream2;
  cudaGraph_t top = nullptr;
  const long long launches_before = g_kernel_launches.load();  // capture records, it does not launch
  cudaError_t e = cudaGraphCreate(&top, 0);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(s, top, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    e = capture_solve(c, mixed, half, top, s);
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &out);
    if (e == cudaSuccess) e = e2;
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, top, 0);
  g_kernel_launches.store(launches_before);
  if (e != cudaSuccess) {
    if (top) cudaGraphDestroy(top);
    cudaGetLastError();
    return e;
  }
  c->graph[mixed][half] = top;
  c->graph_exec[mixed][half] = exec;
  return cudaSuccess;
}

// Solve R x = f on the device loop; f, x may be any buffers (copied to / from the graph's own).
static rfnse_status solve_graph(rfnse_ctx* c, const double* D, const double2* f, double2* x, int half, int* iters,
                                double* relres, int* outer_out) {
  const int mixed = c->p.precision == 1 ? 1 : 0;
  const int h = half ? 1 : 0;
  const long long N = c->N;
  if (!c->graph_exec[mixed][h]) RFNSE_CUDA_TRY(c, build_solve_graph(c, mixed, h));
  if (D != c->D) RFNSE_CUDA_TRY(c, cudaMemcpyAsync(c->D, D, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
  if (f != c->f) RFNSE_CUDA_TRY(c, cudaMemcpyAsync(c->f, f, sizeof(double2) * N, cudaMemcpyDeviceToDevice, c->stream));
  if (!c->tables_ready || D != c->D) RFNSE_CUDA_TRY(c, prepare_D(c, c->D));
  c->tables_ready = false;
  RFNSE_CUDA_TRY(c, cudaGraphLaunch(c->graph_exec[mixed][h], c->stream));
  if (x != c->x) RFNSE_CUDA_TRY(c, cudaMemcpyAsync(x, c->x, sizeof(double2) * N, cudaMemcpyDeviceToDevice, c->stream));
  GmresPeek pk;
  rfnse_status st = peek(c, &pk);
  if (st) return st;
  *iters = pk.it;
  *relres = pk.relres;
  *outer_out = pk.outer;
  {  // kernels the graph executed: 2 at the start, per Arnoldi step its passes and the MGS kernel,
     // per cycle the cycle start, back-substitution, update and residual kernels
    const int d = c->d;
    const long long step_k = (d == 1 ? 1 : 3 * d - 2) + 1;
    const long long cycle_k = mixed ? 1 + 1 + d + 1 + 1 : 1 + 1 + 1 + (d == 1 ? 1 : 2 * d - 1) + d + 1;
    const long long cycles = mixed ? pk.outer : (pk.it > 0 ? pk.outer + 1 : 0);
    count_launch(2 + step_k * pk.it + cycle_k * cycles);
  }
  c->resid_current = mixed && pk.outer > 0;
  if (pk.err) { c->err = "a bounded device-side wait gave up"; return RFNSE_ETIMEOUT; }
  if (pk.done == 3) { c->err = "non-finite value in the solve"; return RFNSE_ENUMERIC; }
  if (pk.beta == 0.0 && pk.it == 0) { *relres = 0.0; return RFNSE_OK; }
  if (pk.done == 1 || pk.done == 2) return RFNSE_OK;
  c->err = mixed ? "mixed-precision refinement did not reach tol" : "GMRES reached max_it";
  return RFNSE_ENOCONV;
}

rfnse_status solve_block(rfnse_ctx* c, const double* D, const double2* f, double2* x, int half, int* iters,
                         double* relres) {
  NvtxRange range("rfnse solve");
  int outer = 0;
  rfnse_status st;
  if (c->use_graphs) {
    st = solve_graph(c, D, f, x, half, iters, relres, &outer);
  } else {
    if (!c->tables_ready || D != c->D) RFNSE_CUDA_TRY(c, prepare_D(c, D));
    c->tables_ready = false;
    if (c->p.precision == 1) {
      st = solve_mixed(c, D, f, x, half, iters, relres, &outer);
    } else {
      st = gmres_fp64(c, D, f, x, half, iters, relres);
      outer = 1;
    }
  }
  c->last_outer = outer;
  return st;
}

// ---------------------------------------------------------------------------------------------
// The TBAN iteration (Sec. 3, Method 3.1) in its stationary form F x^{k+1} = G x^k + f, i.e.
// x^{k+1} = x^k + P^{-1}(f - R x^k), from x^0 = 0, with the context's preconditioner P as F (the
// sine-transform F~: tau(T_d) in place of T_d; or the circulant F_C; or none, which is Richardson).
// FP64 throughout; stops when ||f - R x|| / ||f|| < tol or after max_it iterations.
rfnse_status tban_solve(rfnse_ctx* c, const double* D, const double2* f, double2* x, int half, int* iters,
                        double* relres) {
  const long long N = c->N;
  GmresPeek pk;
  *iters = 0;
  *relres = 0.0;
  RFNSE_CUDA_TRY(c, prepare_D(c, D));
  launch_zero(x, N, c->stream);
  launch_norm(f, c->gs, N, c->red_blocks, c->partials, c->counter, c->stream);
  rfnse_status st = peek(c, &pk);
  if (st) return st;
  const double fnorm = pk.beta;
  if (!std::isfinite(fnorm)) { c->err = "non-finite right-hand side"; return RFNSE_ENUMERIC; }
  if (fnorm == 0.0) return RFNSE_OK;
  const double2* r = f;
  double rel = 1.0;
  int k = 0;
  while (k < c->p.max_it) {
    RFNSE_CUDA_TRY(c, (run_precon<double, double2, double2, double2, double2, false, false>(
                          c, r, nullptr, nullptr, x, 1, D, nullptr, nullptr, nullptr, kOne, kI, half, c->t1, c->t2)));
    RFNSE_CUDA_TRY(c, run_matvec_fp64(c, x, D, c->r, f, kMinusOne, kMinusI, half, nullptr));
    launch_norm(c->r, c->gs, N, c->red_blocks, c->partials, c->counter, c->stream);
    if ((st = peek(c, &pk))) return st;
    r = c->r;
    ++k;
    rel = pk.beta / fnorm;
    if (!std::isfinite(rel)) { c->err = "non-finite residual"; return RFNSE_ENUMERIC; }
    if (rel < c->p.tol) break;
  }
  *iters = k;
  *relres = rel;
  if (rel < c->p.tol) return RFNSE_OK;
  c->err = "the TBAN iteration reached max_it";
  return RFNSE_ENOCONV;
}

// ---------------------------------------------------------------------------------------------
// Time steps (paper Sec. 2.1/2.2): (D - T + iI) u^{n+1} = (T - D + iI) u^{n-1}, solved in the
// block form R x = f with f = -i b = u^{n-1} - i (T - D) u^{n-1}.
//
// Mixed form: the final FP64 residual of each solve gives T u^{n+1} pointwise (kept in c->Tu), so
// the right-hand side of step n+2, which needs T u^{n+1}, costs no Toeplitz product.
static void keep_Tu(rfnse_ctx* c, rfnse_status st, const double* D, const double2* f, int inext, double scale) {
  if (c->Tu[inext] && st == RFNSE_OK && c->p.precision == 1 && c->resid_current) {
    launch_tu_from_residual(D, f, c->u[inext], c->r, c->Tu[inext], scale, c->N, c->stream);
    c->tu_valid[inext] = true;
  }
}

rfnse_status time_step(rfnse_ctx* c, int* iters, double* relres) {
  const long long N = c->N;
  const int inext = 3 - c->iprev - c->icur;
  double2* un = c->u[inext];
  rfnse_status st = RFNSE_OK, st2;
  int it = 0;
  c->tu_valid[inext] = false;
  if (c->step == 0) {
    const double2* u0 = c->u[c->icur];
    const double rdt = c->p.rho * c->p.dt * 0.5;
    launch_diag(u0, nullptr, c->D, rdt, N, c->stream);
    RFNSE_CUDA_TRY(c, run_matvec_fp64(c, u0, c->D, c->f, nullptr, kOne, kMinusI, 1, nullptr));
    st = solve_block(c, c->D, c->f, un, 1, &it, relres);
    if (st != RFNSE_OK && st != RFNSE_ENOCONV) return st;
    if (c->p.first_step == 1) {
      int it2 = 0;
      if (c->keep_pred)  // the reverse pass reads the predictor
        RFNSE_CUDA_TRY(c, cudaMemcpyAsync(c->keep_pred, un, sizeof(double2) * N, cudaMemcpyDeviceToDevice, c->stream));
      launch_diag(u0, un, c->D, rdt, N, c->stream);
      RFNSE_CUDA_TRY(c, run_matvec_fp64(c, u0, c->D, c->f, nullptr, kOne, kMinusI, 1, nullptr));
      st2 = solve_block(c, c->D, c->f, un, 1, &it2, relres);
      if (st2 != RFNSE_OK && st2 != RFNSE_ENOCONV) return st2;
      if (st2 != RFNSE_OK) st = st2;
      it += it2;
    }
    keep_Tu(c, st, c->D, c->f, inext, 2.0);  // the first step's system has T/2
  } else {
    const double2* up = c->u[c->iprev];
    const double2* uc = c->u[c->icur];
    if (c->tu_valid[c->iprev]) {  // mixed form: D, f and the sub-solve tables in one sweep
      launch_step_prep(c, uc, up, c->Tu[c->iprev], c->stream);
      c->tables_ready = true;
    } else {
      launch_diag(uc, nullptr, c->D, c->p.rho * c->p.dt, N, c->stream);
      RFNSE_CUDA_TRY(c, run_matvec_fp64(c, up, c->D, c->f, nullptr, kOne, kMinusI, 0, nullptr));
    }
    st = solve_block(c, c->D, c->f, un, 0, &it, relres);
    if (st != RFNSE_OK && st != RFNSE_ENOCONV) return st;
    keep_Tu(c, st, c->D, c->f, inext, 1.0);
  }
  c->iprev = c->icur;
  c->icur = inext;
  c->step += 1;
  *iters = it;
  return st;
}

// ---------------------------------------------------------------------------------------------
// Autotuner of the line passes (rfnse_autotune).  The tuner runs the passes of one Arnoldi step and of
// the solver's other products once in recording mode, so that every pass configuration the solves
// launch is seen with its real operands; then it times each configuration under every candidate
// geometry (tile of B lines, threads per line, kernel variant) with CUDA events and keeps the fastest
// in the context.  Choices are shared between contexts of the same grid on the same device (a batch of
// many instances tunes each distinct grid once).

namespace {

using TuneMemoKey = std::tuple<int, int, int, int, int, unsigned long long>;  // device, d, n0, n1, n2, key
std::mutex g_tune_mutex;
std::map<TuneMemoKey, std::pair<PassGeom, PassGeom>> g_tune_memo;  // (best, default)
std::map<TuneMemoKey, std::pair<double, double>> g_tune_times;     // (best us, default us)

// Mean duration in microseconds of `reps` launches of one configuration with geometry g (one untimed
// launch first); +inf if the geometry cannot launch.
// A tuned geometry replaces the default only when it is faster by more than this fraction.
constexpr double kTuneMargin = 0.03;

double time_geometry(rfnse_ctx* c, const TuneRecord& r, const PassGeom& g, int reps, cudaEvent_t e0,
                     cudaEvent_t e1) {
  if (r.launch(g) != cudaSuccess) {
    cudaGetLastError();
    return std::numeric_limits<double>::infinity();
  }
  // the fastest of three trials of reps launches: one trial disturbed by other work on the GPU does
  // not decide the choice
  double best = std::numeric_limits<double>::infinity();
  for (int trial = 0; trial < 3; ++trial) {
    cudaEventRecord(e0, c->stream);
    for (int i = 0; i < reps; ++i)
      if (r.launch(g) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(c->stream);
        return std::numeric_limits<double>::infinity();
      }
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return std::numeric_limits<double>::infinity();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, 1e3 * ms / reps);
  }
  return best;
}

// Run, in recording mode, every line-pass configuration the context's solves launch: the Arnoldi
// step's preconditioner and product (with the first MGS dot product), the solution update, and the
// FP64 products of the right-hand side and the residual.  The operands are the context's own work
// vectors (zeroed; their contents do not change a pass's duration).
cudaError_t record_solver_passes(rfnse_ctx* c, std::vector<TuneRecord>* rec) {
  const long long N = c->N;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  chk(cudaMemsetAsync(c->D, 0, sizeof(double) * N, s));
  chk(cudaMemsetAsync(c->r, 0, sizeof(double2) * N, s));
  chk(cudaMemsetAsync(c->x, 0, sizeof(double2) * N, s));
  chk(cudaMemsetAsync(c->f, 0, sizeof(double2) * N, s));
  chk(cudaMemsetAsync(c->w, 0, sizeof(double2) * N, s));
  chk(prepare_D(c, c->D));
  if (e != cudaSuccess) return e;
  Dyn dot0;
  dot0.vbase = c->V;
  dot0.dot0 = true;
  c->tune_rec = rec;
  for (int half = 0; half < 2 && e == cudaSuccess; ++half) {
    if (c->p.precision == 1) {
      chk((run_precon<float, double2, float2, float2, float2, true, true>(
          c, c->r, &c->gs->inv_beta, c->V, c->Z32, 0, c->D, c->w, c->wp32, nullptr, kOne, kI, half, c->t1f, c->t2f,
          dot0)));
    } else {
      chk((run_precon<double, double2, double2, double2, double2, true, true>(
          c, c->r, &c->gs->inv_beta, c->V, c->zb, 0, c->D, c->w, c->w, nullptr, kOne, kI, half, c->t1, c->t2,
          dot0)));
      chk((run_precon<double, double2, double2, double2, double2, false, false>(
          c, c->r, nullptr, nullptr, c->x, 1, c->D, nullptr, nullptr, nullptr, kOne, kI, half, c->t1, c->t2)));
    }
    chk(run_matvec_fp64(c, c->x, c->D, c->r, c->f, kMinusOne, kMinusI, half, nullptr));
  }
  c->tune_rec = nullptr;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace

rfnse_status autotune(rfnse_ctx* c, int reps, int force, int* n_configs, int* n_changed, double* est_speedup) {
  NvtxRange range("rfnse autotune");
  int dev = 0;
  RFNSE_CUDA_TRY(c, cudaGetDevice(&dev));
  std::vector<TuneRecord> rec;
  c->tune.clear();
  RFNSE_CUDA_TRY(c, record_solver_passes(c, &rec));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RFNSE_CUDA_TRY(c, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    c->err = "autotune: event creation failed";
    return RFNSE_ECUDA;
  }
  int changed = 0;
  double t_best = 0.0, t_dflt = 0.0;
  rfnse_status st = RFNSE_OK;
  for (const TuneRecord& r : rec) {
    const TuneMemoKey mk{dev, c->d, c->n[0], c->n[1], c->n[2], r.key};
    PassGeom best = r.dflt;
    double tb = 0.0, td = 0.0;
    bool have = false;
    if (!force) {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      const auto it = g_tune_memo.find(mk);
      if (it != g_tune_memo.end()) {
        best = it->second.first;
        tb = g_tune_times[mk].first;
        td = g_tune_times[mk].second;
        have = true;
      }
    }
    if (!have) {
      td = time_geometry(c, r, r.dflt, reps, e0, e1);
      tb = td;
      for (const PassGeom& g : r.cands) {
        const double t = time_geometry(c, r, g, reps, e0, e1);
        if (t < tb) {
          tb = t;
          best = g;
        }
      }
      if (tb > (1.0 - kTuneMargin) * td) {  // within the timing noise of the default: keep the default
        best = r.dflt;
        tb = td;
      }
      if (!(td < std::numeric_limits<double>::infinity())) {
        st = RFNSE_ECUDA;
        c->err = "autotune: a pass failed with its default geometry";
        break;
      }
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tune_memo[mk] = {best, r.dflt};
      g_tune_times[mk] = {tb, td};
    }
    c->tune[r.key] = best;
    if (best.B != r.dflt.B || best.nt != r.dflt.nt || best.variant != r.dflt.variant) ++changed;
    t_best += tb;
    t_dflt += td;
  }
  // the cooperative Arnoldi kernel's grid: 1..4 blocks per SM (all co-resident), timed on column j = 1
  // of the context's own basis (two sweeps and a grid-wide barrier, then the norm sweep)
  const bool tune_mgs = st == RFNSE_OK && c->N > 4096 && c->p.restart >= 1;
  if (tune_mgs) {
    const TuneMemoKey mk{dev, -1, (int)(c->N >> 31), (int)(c->N & 0x7fffffff), 0, 0ull};
    int best = -1;
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      const auto it = g_tune_memo.find(mk);
      if (!force && it != g_tune_memo.end()) best = it->second.first.B;
    }
    if (best < 0) {
      const int bmax = coop_blocks_max(c->N);
      int sms = 152;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const SolveCfg cfg = make_cfg(c, c->p.precision == 1 ? 1 : 0);
      double tbest = std::numeric_limits<double>::infinity();
      // candidates: 1..4 blocks per SM of the grid-wide kernel; for grids of at most 2^21 points also
      // one cluster of 8 or 16 CTAs (negative counts)
      std::vector<int> cands;
      for (int k = 1; k <= 4; ++k) {
        const int blocks = std::min(bmax, sms * k);
        if (k > 1 && blocks == std::min(bmax, sms * (k - 1))) break;
        cands.push_back(blocks);
      }
      if (c->N <= (1LL << 21))
        for (int cs : {8, 16})
          if (mgs_cluster_fits(cs)) cands.push_back(-cs);
      // each candidate: the fastest of three trials of reps launches; the default launch stays unless a
      // candidate beats it by more than kTuneMargin (as for the passes)
      const int dflt = c->coop_blocks;
      double tdflt = std::numeric_limits<double>::infinity();
      for (const int blocks : cands) {
        auto one = [&]() {
          launch_set_column(c->gs, 1, c->stream);
          return launch_mgs_step(c->gs, c->V, c->N, c->w, c->N, c->coop_partials, c->bar, cfg, 0, 0, blocks,
                                 c->stream);
        };
        cudaError_t e = one();
        double tc = std::numeric_limits<double>::infinity();
        for (int trial = 0; trial < 3 && e == cudaSuccess; ++trial) {
          e = cudaEventRecord(e0, c->stream);
          for (int r = 0; r < reps && e == cudaSuccess; ++r) e = one();
          if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
          if (e == cudaSuccess) tc = std::min(tc, (double)ms);
        }
        if (e != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        if (blocks == dflt) tdflt = tc;
        if (tc < tbest) {
          tbest = tc;
          best = blocks;
        }
      }
      if (best != dflt && tbest > (1.0 - kTuneMargin) * tdflt) best = dflt;
      if (best > 0) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_memo[mk] = {PassGeom{best, 0, 0}, PassGeom{c->coop_blocks, 0, 0}};
      }
    }
    if (best > 0) {
      if (best != c->coop_blocks) ++changed;
      c->coop_blocks = best;
    }
    RFNSE_CUDA_TRY(c, cudaMemsetAsync(c->gs, 0, sizeof(GmresState), c->stream));
    RFNSE_CUDA_TRY(c, cudaMemsetAsync(c->bar, 0, sizeof(GridBarrier), c->stream));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RFNSE_OK) {
    c->tune.clear();
    return st;
  }
  // the cached solve graphs hold the old geometries: capture them again on the next solve
  for (int a = 0; a < 2; ++a)
    for (int h = 0; h < 2; ++h) {
      if (c->graph_exec[a][h]) cudaGraphExecDestroy(c->graph_exec[a][h]);
      if (c->graph[a][h]) cudaGraphDestroy(c->graph[a][h]);
      c->graph_exec[a][h] = nullptr;
      c->graph[a][h] = nullptr;
    }
  if (n_configs) *n_configs = (int)rec.size() + (tune_mgs ? 1 : 0);
  if (n_changed) *n_changed = changed;
  if (est_speedup) *est_speedup = (t_best > 0.0) ? t_dflt / t_best : 1.0;
  return RFNSE_OK;
}

}  // namespace rfnse
