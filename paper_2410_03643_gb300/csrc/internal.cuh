// Library-internal declarations: the context, the device-resident GMRES state and the kernels
// shared between translation units.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>
#include "../../include/rfnse.h"

namespace rfnse {

constexpr int kMaxM = 256;  // largest supported restart length
// Largest grid of a last matrix-product pass that hands its <v_0, w> partials to the Arnoldi kernel
// (every block of that kernel sums them; larger grids keep the kernel's own first sweep).
constexpr int kDot0MaxBlocks = 4096;
constexpr int kNormPartMax = 4096;  // largest grid whose squared-norm partials a norm kernel sums

// Number of kernels this library has launched in the process (all contexts).
extern std::atomic<long long> g_kernel_launches;
inline void count_launch(long long k = 1) { g_kernel_launches.fetch_add(k, std::memory_order_relaxed); }

// NVTX range for the span of a scope (time steps, solves, passes, the tuner), so that profilers can
// group or select the kernels by what launched them (e.g. ncu --nvtx --nvtx-include "rfnse step/").
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device and pinned-host allocations of contexts, batches and tapes go through these two (api.cu), so
// that rfnse_test_fail_allocations can make them fail without exhausting the GPU's memory.
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t host_alloc_pinned(void** p, size_t bytes);

// Checks of the problem description shared by rfnse_create and rfnse_apply_prec_static: d, grid,
// box, alpha, rho, dt, omega (api.cu).  Returns null when valid, else the reason.
const char* validate_problem(const rfnse_params* p);

// Device-resident Arnoldi / Givens state of one GMRES cycle.  H is stored by columns:
// H(i, j) = H[j * (kMaxM + 1) + i].
struct GmresState {
  // --- prefix read by the host (GmresPeek) ---
  double beta;      // norm of the residual that starts the cycle
  double relres;    // |g_{j+1}| / ref after the last Givens update
  int done;         // 0 running, 1 converged, 2 exact breakdown, 3 non-finite value
  int pad_;
  int it;           // Arnoldi steps of the current solve
  int outer;        // outer (restart / refinement) cycles of the current solve
  int err;          // 1: a bounded device-side wait gave up
  int j;            // next Arnoldi column of the cycle (= columns built so far)
  // --- device-only ---
  double inv_beta;  // 1 / beta
  double ref;       // reference norm of the relative residual test
  double tol;       // stop when |g_{j+1}| / ref < tol
  double inv_h;     // 1 / h_{j+1,j}
  double fnorm;     // ||f|| of the solve
  const double2* src;  // vector that starts the next Arnoldi column (r or w) ...
  double src_scale;    // ... and the factor that normalises it (1/beta or 1/h)
  int no_restart;   // 1 when the cycle ended converged or out of iterations (restart kernels skip)
  int upd;          // mixed form: 1 when this cycle's residual is formed from the Arnoldi basis
  double upd_err;   // ... and a bound on that residual's relative error (added to the stopping test)
  double H[(kMaxM + 1) * kMaxM];
  double cs[kMaxM], sn[kMaxM], g[kMaxM + 1], y[kMaxM];
  double q[kMaxM + 1];  // residual coefficients: r = sum_i q_i v_i (v_k = w / h_{k,k-1})
};

// Host-visible copy of the prefix of GmresState that the control loop reads.
struct GmresPeek {
  double beta, relres;
  int done, pad_;
  int it, outer, err, j;
};

// Settings of a solve that the device-side control reads.
struct SolveCfg {
  int m;            // restart length
  int max_it;       // Arnoldi steps per solve
  int max_outer;    // refinement cycles (mixed form)
  int mixed;        // 1: mixed form (inner tolerance from eta_min, FP64 outer residual)
  double tol;       // relative residual tolerance of the solve
  double eta_min;   // mixed form: smallest inner tolerance
};

// Geometry of a line-pass launch (passes.cuh): lines per block, threads per line, kernel variant
// (1 = the prefetching fixed-length FP32 kernel, 0 = k_line_pass).
struct PassGeom {
  int B, nt, variant;
};

// One pass configuration seen while rfnse_autotune records a solver's passes: its key, the geometry it
// gets without tuning, the geometries to try, and a function that launches it with a given geometry.
struct TuneRecord {
  unsigned long long key = 0;
  PassGeom dflt{};
  std::vector<PassGeom> cands;
  std::function<cudaError_t(const PassGeom&)> launch;
};

// Device tables of batched launches (the lock-step batch): a device buffer and its host image, filled
// while a graph is captured (the kernels only read them when the graph runs) and copied to the device
// once the capture has ended.
struct TableArena {
  char* dev = nullptr;     // device buffer of cap bytes
  size_t cap = 0;
  std::vector<char> host;  // host image; host.size() bytes in use
  // Reserve `bytes` (16-byte aligned), copy src into the host image, return the device address (null
  // when the buffer is full).
  void* put(const void* src, size_t bytes) {
    const size_t off = (host.size() + 15) & ~(size_t)15;
    if (off + bytes > cap) return nullptr;
    host.resize(off + bytes);
    if (bytes) std::memcpy(host.data() + off, src, bytes);
    return dev + off;
  }
};

struct ParamRecord;  // passes.cuh: a pass's parameters and its batched launcher (lock-step capture)

// Arrival counters of the cooperative kernels' grid-wide sums (coop.cuh); zero-initialised, and zero
// again when a launch ends (cleared by its last block).
struct GridBarrier {
  unsigned count;  // arrivals at the grid-wide sums of the current launch
  unsigned done;   // arrivals at the launch's last sum
};

// ---- device-side control (control.cu) -----------------------------------------------------------
int coop_blocks_for(long long N);  // blocks of the cooperative Arnoldi kernel (all co-resident)
int coop_blocks_max(long long N);  // the most it may use (up to four per SM, co-resident)
bool mgs_cluster_fits(int csize);  // one cluster of csize CTAs of the cluster variant is resident
void launch_set_column(GmresState* gs, int j, cudaStream_t s);  // state for timing column j (autotune)
// pre_part / pre_n: partials of h_0j = <v_0, w> written by the last product pass (pre_n = 0: none);
// blocks > 0: the cooperative grid-wide kernel on that many blocks; blocks < 0: one thread-block cluster
// of -blocks CTAs (hardware cluster barriers, distributed-shared-memory reductions)
cudaError_t launch_mgs_step(GmresState* gs, const double2* V, long long ldv, double2* w, long long N,
                            double* partials, GridBarrier* bar, const SolveCfg& cfg,
                            cudaGraphConditionalHandle h_inner, int set_cond, int blocks, cudaStream_t s,
                            const double* pre_part = nullptr, int pre_n = 0);
// pa/na, pb/nb: block partials of ||x||^2 left by x's producer (mode 0: pa; mode 2: pa when the
// residual came from the recurrence, pb when from the product); a count 0 means sweep x
void launch_norm_ctl(const double2* x, GmresState* gs, long long N, int blocks, double* partials, unsigned* counter,
                     GridBarrier* bar, const SolveCfg& cfg, int mode, cudaGraphConditionalHandle h_outer,
                     int set_cond, cudaStream_t s, const double* pa = nullptr, int na = 0,
                     const double* pb = nullptr, int nb = 0);
void launch_cycle_begin(GmresState* gs, const SolveCfg& cfg, cudaGraphConditionalHandle h_inner,
                        cudaGraphConditionalHandle h_outer, int set_cond, cudaStream_t s);
void launch_backsolve_dev(GmresState* gs, cudaStream_t s);
// Mixed form, end of a refinement cycle (graph form): back-substitution, x += Z y and the residual
// recurrence's decision and coefficients in one launch (control.cu k_cycle_end_mixed).
void launch_cycle_end_mixed(const float2* Z, long long ldz, GmresState* gs, double2* x, long long N, double tol,
                            cudaStream_t s);
// Mixed form, end of a refinement cycle of k Arnoldi steps (k < 0: gs->j).  Decides whether the new
// residual is formed from the Arnoldi basis (upd < 0: on the device, when the cycle's starting
// residual beta <= kUpdRatio * tol * ||f||; otherwise upd as given) and, if so, stores its
// coefficients q = Q^T g_k e_k (the Givens rotations undone on the last residual estimate).
constexpr double kUpdRatio = 1e5;
constexpr double kUpdErr = 4e-7;  // relative error of an FP32 product, times beta / ||f||: the bound
void launch_resid_coeffs(GmresState* gs, int k, int upd, double err, double tol, cudaStream_t s);
// r = sum_{i<k} q_i V_i + q_k inv_h w when gs->upd (else nothing); k < 0: gs->j
void launch_resid_update(const double2* V, long long ldv, const double2* w, const GmresState* gs, int k,
                         double2* r, long long N, cudaStream_t s, double* nrm_part = nullptr);
void launch_tu_from_residual_dev(const GmresState* gs, const double* D, const double2* f, const double2* x,
                                 const double2* r, double2* Tu, long long N, cudaStream_t s);
void launch_gather_peeks(GmresState* const* gs, GmresPeek* out, int count, cudaStream_t s);
void launch_combine_dev(const double2* V, long long ldv, const GmresState* gs, double2* out, long long N,
                        cudaStream_t s);
void launch_combine_f32_add_dev(const float2* Z, long long ldz, const GmresState* gs, double2* x, long long N,
                                cudaStream_t s);

inline int choose_reduce_blocks(long long N) {
  long long b = (N + 511) / 512;   // enough blocks to cover all 152 SMs; fixed for a given N
  if (b < 1) b = 1;
  if (b > 4 * 152) b = 4 * 152;
  return (int)b;
}

// ---- Krylov / pointwise kernels (krylov.cu) -----------------------------------------------------
// All reductions are deterministic: fixed grid, per-block partials, the last block to finish sums
// the partials in block order.
void launch_norm(const double2* x, GmresState* gs, long long N, int blocks, double* partials, unsigned* counter,
                 cudaStream_t s);
void launch_backsolve(GmresState* gs, int k, cudaStream_t s);
void launch_combine(const double2* V, long long ldv, const GmresState* gs, int k, double2* out, long long N,
                    cudaStream_t s);
void launch_combine_f32_add(const float2* Z, long long ldz, const GmresState* gs, int k, double2* x, long long N,
                            cudaStream_t s);
void launch_diag(const double2* u, const double2* u2, double* D, double rho_dt, long long N, cudaStream_t s);
void launch_neg_i(const double2* b, double2* f, long long N, cudaStream_t s);
void launch_zero(double2* x, long long N, cudaStream_t s);
// *flag = 1 if a and b differ in any bit of their N complex FP64 values, else 0
void launch_differs(const double2* a, const double2* b, long long N, int* flag, cudaStream_t s);
void launch_start_cycle(GmresState* gs, double ref, double tol, cudaStream_t s);
// Tu = scale (D x - i (f - x - r)) from the residual r = f - x - i(T - D)x
void launch_tu_from_residual(const double* D, const double2* f, const double2* x, const double2* r, double2* Tu,
                             double scale, long long N, cudaStream_t s);
// f = u - i (Tu - D u)
// D32 = D, dfac = 2w((w+1) + iD)/((w+1)^2 + D^2) in FP64 and FP32
void launch_prep_D(const double* D, float* D32, double2* dfac64, float2* dfac32, double omega, long long N,
                   cudaStream_t s);
// mixed form, steady step: D, f = u_prev - i (Tu_prev - D u_prev) and the prep_D tables in one sweep
void launch_step_prep(rfnse_ctx* c, const double2* uc, const double2* up, const double2* Tup, cudaStream_t s,
                      double* nrm_part = nullptr);
int step_prep_blocks(long long N);  // its grid (the number of partials it leaves)
int resid_update_blocks(long long N);

// Debug mode (rfnse_ctx::debug): after a line pass, wait for it and count the non-finite values among
// `count` complex values of storage `elem` bytes each (8: float2, 16: double2) at each of the outputs;
// the first pass with any is recorded in c->dbg_first with `what`.  Returns the launch or execution error.
cudaError_t debug_after_pass(rfnse_ctx* c, cudaStream_t s, const char* what, const void* const* outs,
                             const int* elems, int nout, long long count);

// ---- double-float Toeplitz passes (toep_df.cu) --------------------------------------------------
bool toeplitz_df_available(const rfnse_ctx* c);
// dfz_in / dfz_out: the double-float copy of z shared by the passes of a product (float4 per point; see
// PassParams), null when not used
cudaError_t run_toeplitz_df(rfnse_ctx* c, int axis, int half, bool first, const double2* z, const double* D,
                            const double2* add, double2* w, double2 a, double2 b, const int* skip,
                            double* nrm_part = nullptr, const void* dfz_in = nullptr, void* dfz_out = nullptr);
void launch_setup_df(int log2L, const double* c64h0, const double* c64h1, void* tw, void* c0, void* c1,
                     cudaStream_t s);

// ---- setup kernels (setup.cu) -------------------------------------------------------------------
void launch_setup_coefficients(double* c, int nmax, double alpha, cudaStream_t s);
void launch_setup_axis(const double* c, int n, int L, double* lam, double* circ, double2* tw64, float2* tw32,
                       cudaStream_t s);
// lamfac[g] = i dst_scale / (w + i sum_a mu_a lambda_a(k_a(g))) for every grid index g
// circ = 1: lamfac[g] = dst_scale / (w + i Lambda) (the circulant comparator in the DFT basis)
void launch_setup_lamfac(const double* lam0, const double* lam1, const double* lam2, int n0, int n1, int n2,
                         double mu0, double mu1, double mu2, double omega, double dst_scale, int circ,
                         double2* f64, float2* f32, long long N, cudaStream_t s);
// Strang-circulant comparator tables of one axis (setup.cu): eigenvalues, chirp, Bluestein spectrum
void launch_setup_circ(const double* c, int n, int L, double* lamC, double2* chirp64, float2* chirp32,
                       double2* bspec64, float2* bspec32, cudaStream_t s);
// scaled circulant spectrum circ * scale in FP64 and FP32
void launch_scale_circ(const double* circ, int L, double scale, double* c64, float* c32, cudaStream_t s);

}  // namespace rfnse

// The opaque context of the C ABI.
struct rfnse_ctx {
  rfnse_params p;
  cudaStream_t stream;
  int d;
  int n[3];
  long long stride[3];
  int L[3], log2L[3];
  long long N;
  double h[3], mu[3];
  // coefficients (device)
  double* c = nullptr;
  double* lam[3] = {nullptr, nullptr, nullptr};
  double* circ[3] = {nullptr, nullptr, nullptr};
  double2* tw64[3] = {nullptr, nullptr, nullptr};
  float2* tw32[3] = {nullptr, nullptr, nullptr};
  // time-stepping state (device)
  double2* u[3] = {nullptr, nullptr, nullptr};
  int iprev = 0, icur = 1, step = 0;
  double* D = nullptr;
  // work vectors (device)
  double2 *f = nullptr, *x = nullptr, *w = nullptr, *r = nullptr, *t1 = nullptr, *t2 = nullptr, *zb = nullptr;
  double2* V = nullptr;     // (m + 1) Krylov vectors
  float2* Z32 = nullptr;    // m preconditioned vectors of the mixed form
  float2 *t1f = nullptr, *t2f = nullptr;
  float2* wp32 = nullptr;   // FP32 partial matrix product between the Toeplitz passes (mixed form)
  // per-point factor tables in both precisions
  float* D32 = nullptr;                     // D of the current solve
  double2* dfac64 = nullptr;                // 2w((w+1) + iD)/((w+1)^2 + D^2) of the current solve
  float2* dfac32 = nullptr;
  double2* lamfac64[2] = {nullptr, nullptr};  // i dst_scale/(w + i Lambda(k)) per mode; [half]
  float2* lamfac32[2] = {nullptr, nullptr};
  double* circ64s[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};  // circ * mu_a hf / L
  float* circ32s[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  // Strang-circulant comparator (precond = 1): per axis the eigenvalues of Strang's circulant of T_0,
  // the chirp exp(i pi j^2/n) and the Bluestein filter spectrum (1/L folded in); per point
  // 1/(n_0 n_1 n_2 (w + i Lambda_C(k))) for [half]
  double* lamC[3] = {nullptr, nullptr, nullptr};
  double2* chirp64[3] = {nullptr, nullptr, nullptr};
  float2* chirp32[3] = {nullptr, nullptr, nullptr};
  double2* bspec64[3] = {nullptr, nullptr, nullptr};
  float2* bspec32[3] = {nullptr, nullptr, nullptr};
  double2* lamfacC64[2] = {nullptr, nullptr};
  float2* lamfacC32[2] = {nullptr, nullptr};
  // mixed form, double-float Toeplitz products of the residual (toep_df.cu): per axis the fixed-length
  // FFT's twiddles (complex double-float, 16 B each) and per [half][axis] the scaled circulant spectrum
  // (double-float, 8 B each); null when some axis has no fixed-length FFT
  void* twdf[3] = {nullptr, nullptr, nullptr};
  void* circdf[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  // mixed form: T u of each history vector, recovered from the final FP64 residual of the solve
  // that produced it (so the right-hand side two steps later needs no Toeplitz product)
  double2* Tu[3] = {nullptr, nullptr, nullptr};
  bool tu_valid[3] = {false, false, false};
  bool resid_current = false;               // c->r holds f - R x for the last solve's x
  bool tables_ready = false;                // the next solve's D tables are already built (k_step_prep)
  double* partials = nullptr;
  unsigned* counter = nullptr;
  int red_blocks = 1;
  rfnse::GmresState* gs = nullptr;
  rfnse::GmresPeek* peek = nullptr;  // pinned host
  // device-side control: cooperative Arnoldi kernel and one CUDA graph per (precision, half)
  rfnse::GridBarrier* bar = nullptr;
  double* coop_partials = nullptr;   // 2 * coop_blocks
  int coop_blocks = 1;               // < 0: one cluster of -coop_blocks CTAs (chosen by rfnse_autotune)
  double* dot_part = nullptr;        // kDot0MaxBlocks partials of <v_0, w> from the last product pass
  int dot0_blocks = 0;               // how many the last such launch wrote (0: none)
  // block partials of squared norms left by the kernel that produced the vector, so that the solve's
  // norm kernel only sums them: f (k_step_prep), r from the recurrence (k_resid_update), r from the
  // double-float product (its last pass); kNormPartMax each
  double* nrm_part = nullptr;        // 3 x kNormPartMax
  int nrm_df_blocks = 0;             // partials the last double-float product wrote (0: none)
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;   // private stream that captures the loop bodies
  cudaStream_t cap_stream2 = nullptr;  // private stream that captures a stand-alone solve graph
  cudaGraph_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaGraphExec_t graph_exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  // reverse pass (adjoint.cu): the taped forward run and its work vectors
  double2* keep_pred = nullptr;  // when set, the first time step copies its predictor here
  double2* tape = nullptr;       // checkpoints, segment states and gradient vectors
  size_t tape_vecs = 0;          // grid vectors allocated in tape
  double* adj_red = nullptr;     // per-block partial sums of the rho gradient, then the running sum
  int tape_steps = -1;           // steps of the taped run (-1: none)
  int tape_every = 0;            // checkpoint interval of the taped run
  // per-step statistics of the last solve
  int last_iters = 0, last_outer = 0;
  double last_relres = 0.0;
  // autotuned pass geometry (rfnse_autotune): per pass configuration the geometry that measured
  // fastest; empty until tuned.  tune_rec is set only while the tuner records the solver's passes.
  std::map<unsigned long long, rfnse::PassGeom> tune;
  std::vector<rfnse::TuneRecord>* tune_rec = nullptr;
  long long tuned_launches = 0;  // pass launches whose geometry came from `tune`
  // set only while a lock-step batch records this instance's pass sequence: the passes are recorded
  // (parameters and batched launcher) instead of launched
  std::vector<rfnse::ParamRecord>* param_rec = nullptr;
  // debug mode (environment RFNSE_DEBUG=1 at rfnse_create): host-driven loops, every line pass checked
  // after its launch (geometry covering the grid, launch and execution errors, non-finite outputs)
  bool debug = false;
  int* dbg_count = nullptr;        // device: non-finite values found by the last scan
  std::string dbg_first;           // the first pass whose output had a non-finite value ("" if none)
  int* cmp_flag = nullptr;         // device: result of the bitwise comparison in rfnse_set_state
  // kernel-class profiling (rfnse_profile): CUDA events around every launch of one pass kind
  int prof_kind = 0;
  std::vector<cudaEvent_t> prof_events;  // pairs (start, stop)
  size_t prof_used = 0;                  // events in use
  double prof_flops = 0.0, prof_bytes = 0.0;
  std::string err;
};

#define RFNSE_CUDA_TRY(ctx, expr)                                                              \
  do {                                                                                          \
    cudaError_t e__ = (expr);                                                                   \
    if (e__ != cudaSuccess) {                                                                   \
      (ctx)->err = std::string(#expr) + ": " + cudaGetErrorString(e__);                         \
      return RFNSE_ECUDA;                                                                       \
    }                                                                                           \
  } while (0)
