// Batched time stepping of many independent instances (different grids, alpha, rho, dt): every
// instance keeps its own context and stream; once all instances are past their first step, one time
// step of the whole batch is a single CUDA graph launch.  The graph holds, for every instance in its
// own branch, the pointwise set-up (D, right-hand side, sub-solve tables), the solve with its
// device-decided loops (capture_solve) writing u^{n+1} straight into the free history slot, and the
// update of the cached T u (mixed form); it ends by gathering every instance's statistics into pinned
// host memory.  The three history slots form a ring (u^{n-1}, u^n, u^{n+1} in slots v, v+1, v+2 mod 3),
// so there are three graphs, one per phase v, and a step moves no data.
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>
#include "internal.cuh"
#include "lockstep.cuh"
#include "passes.cuh"
#include "solve.cuh"

using namespace rfnse;

struct rfnse_batch {
  int count = 0;
  std::vector<rfnse_ctx*> ctx;
  std::vector<cudaStream_t> streams;  // one per instance (owned)
  cudaStream_t stream = nullptr;      // the caller's stream: the batch graph runs on it
  cudaStream_t cap = nullptr;         // private stream that captures the batch graph
  cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};  // one per ring phase
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  GmresState** d_gs = nullptr;        // device array of the instances' GMRES states
  GmresPeek* d_peeks = nullptr;
  GmresPeek* h_peeks = nullptr;       // pinned
  std::vector<cudaEvent_t> events;
  std::string err;
  // lock-step mode (lockstep.cuh): per step one graph whose every launch covers all instances
  bool lockstep = false;
  cudaStream_t cap2 = nullptr;          // captures the loop bodies of the lock-step graphs
  cudaGraph_t lgraph[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t lexec[3] = {nullptr, nullptr, nullptr};
  TableArena arena[3];                  // the batched launches' tables, one per ring phase
  LockFlags* flags = nullptr;           // device, one per instance
  GridBarrier* lbar = nullptr;          // barrier of the batched Arnoldi kernel
  unsigned* done_all = nullptr;         // arrival counter of the batched kernels
  unsigned long long* counts = nullptr;     // device: Arnoldi launches and cycles of the last step
  unsigned long long* h_counts = nullptr;   // pinned copy
  double* cpart = nullptr;              // partials of the batched Arnoldi kernel, 2 per block
  int maxb = 0;                         // blocks of the batched Arnoldi kernel
  long long arn_launches[3] = {0, 0, 0};  // batched pass launches per Arnoldi step, per phase graph
  long long res_launches[3] = {0, 0, 0};  // ... per residual product
};

namespace {

const double2 kOne = {1.0, 0.0};
const double2 kMinusOne = {-1.0, 0.0};
const double2 kMinusI = {0.0, -1.0};

void free_batch(rfnse_batch* b) {
  if (!b) return;
  for (int v = 0; v < 3; ++v) {
    if (b->exec[v]) cudaGraphExecDestroy(b->exec[v]);
    if (b->graph[v]) cudaGraphDestroy(b->graph[v]);
  }
  for (rfnse_ctx* c : b->ctx) rfnse_destroy(c);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int v = 0; v < 3; ++v) {
    if (b->lexec[v]) cudaGraphExecDestroy(b->lexec[v]);
    if (b->lgraph[v]) cudaGraphDestroy(b->lgraph[v]);
    cudaFree(b->arena[v].dev);
  }
  if (b->cap2) cudaStreamDestroy(b->cap2);
  cudaFree(b->flags);
  cudaFree(b->lbar);
  cudaFree(b->done_all);
  cudaFree(b->counts);
  if (b->h_counts) cudaFreeHost(b->h_counts);
  cudaFree(b->cpart);
  cudaFree(b->d_gs);
  cudaFree(b->d_peeks);
  if (b->h_peeks) cudaFreeHost(b->h_peeks);
  delete b;
}

// The ring phase of c's history: v when u^{n-1} is in slot v and u^n in slot v + 1 (mod 3), else -1.
int ring_phase(const rfnse_ctx* c) { return (c->icur == (c->iprev + 1) % 3) ? c->iprev : -1; }

// Put the history in ring phase v (u_prev in u[v], u_cur in u[v + 1 mod 3], each with its cached
// T u) so that the captured step of phase v can use fixed pointers.  Every copy goes into a slot that
// is free at that moment; nothing moves when c is already in phase v.
cudaError_t normalise_history(rfnse_ctx* c, int v) {
  int p = c->iprev, q = c->icur;
  const int tp = v, tq = (v + 1) % 3;
  if (p == tp && q == tq) return cudaSuccess;
  const size_t bytes = sizeof(double2) * (size_t)c->N;
  cudaError_t e = cudaSuccess;
  auto move = [&](int from, int to) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->u[to], c->u[from], bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && c->Tu[to])
      e = cudaMemcpyAsync(c->Tu[to], c->Tu[from], bytes, cudaMemcpyDeviceToDevice, c->stream);
    c->tu_valid[to] = c->tu_valid[from];
  };
  if (p != tp) {
    if (q == tp) {  // u_cur occupies u_prev's target: move it to the free slot first
      const int f = 3 - p - q;
      move(q, f);
      q = f;
    }
    move(p, tp);
    p = tp;
  }
  if (q != tq) move(q, tq);  // tq is the free slot now
  c->iprev = tp;
  c->icur = tq;
  c->tu_valid[(v + 2) % 3] = false;
  return e;
}

// Record one steady-state time step of instance c in ring phase v (u^{n-1} in slot v, u^n in slot
// v + 1, u^{n+1} into slot v + 2) on its stream, which is capturing into graph g.
cudaError_t capture_step(rfnse_ctx* c, cudaGraph_t g, int v) {
  const long long N = c->N;
  cudaStream_t s = c->stream;
  const int mixed = c->p.precision == 1;
  const int prev = v, cur = (v + 1) % 3, next = (v + 2) % 3;
  cudaError_t e;
  double* f_part = nullptr;
  int f_n = 0;
  if (mixed) {  // the set-up also leaves the partials of ||f||^2 for the solve's first norm
    f_part = c->nrm_part;
    f_n = step_prep_blocks(N);
    launch_step_prep(c, c->u[cur], c->u[prev], c->Tu[prev], s, f_part);
  } else {
    launch_diag(c->u[cur], nullptr, c->D, c->p.rho * c->p.dt, N, s);
    if ((e = run_matvec_fp64(c, c->u[prev], c->D, c->f, nullptr, kOne, kMinusI, 0, nullptr)) != cudaSuccess)
      return e;
    if ((e = prepare_D(c, c->D)) != cudaSuccess) return e;
  }
  double2* const x_own = c->x;
  c->x = c->u[next];  // the solve's kernels write the solution into the free slot
  e = capture_solve(c, mixed, 0, g, s, f_part, f_n);
  if (e == cudaSuccess && mixed) launch_tu_from_residual_dev(c->gs, c->D, c->f, c->x, c->r, c->Tu[next], N, s);
  c->x = x_own;
  return e;
}

cudaError_t build_batch_graph(rfnse_batch* b, int v) {
  const long long launches_before = g_kernel_launches.load();
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(b->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaEvent_t fork = b->events[0];
    e = cudaEventRecord(fork, b->cap);
    for (int i = 0; i < b->count && e == cudaSuccess; ++i) {
      rfnse_ctx* c = b->ctx[i];
      e = cudaStreamWaitEvent(c->stream, fork, 0);
      if (e == cudaSuccess) e = capture_step(c, g, v);
      if (e == cudaSuccess) e = cudaEventRecord(b->events[1 + i], c->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->events[1 + i], 0);
    }
    if (e == cudaSuccess) {
      launch_gather_peeks(b->d_gs, b->d_peeks, b->count, b->cap);
      e = cudaMemcpyAsync(b->h_peeks, b->d_peeks, sizeof(GmresPeek) * b->count, cudaMemcpyDeviceToHost, b->cap);
    }
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &out);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[v], g, 0);
  g_kernel_launches.store(launches_before);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    b->exec[v] = nullptr;
    cudaGetLastError();
    return e;
  }
  b->graph[v] = g;
  return cudaSuccess;
}

// Lock-step mode needs instances whose solves run the same kernels: the mixed form with the sine-transform
// preconditioner, the same dimension, double-float residual products (every axis n + 1 in 128..1024),
// at most 1024 instances and no more than the batched Arnoldi kernel's blocks.
bool lockstep_eligible(const rfnse_batch* b) {
  if (b->count < 1 || b->count > 1024) return false;
  const int d = b->ctx[0]->d;
  for (const rfnse_ctx* c : b->ctx)
    if (c->p.precision != 1 || c->p.precond != 0 || c->d != d || !c->Tu[0] || !toeplitz_df_available(c))
      return false;
  return b->count <= ls_mgs_max_blocks();
}

cudaError_t lockstep_alloc(rfnse_batch* b) {
  if (b->flags) return cudaSuccess;
  const int n = b->count;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  b->maxb = ls_mgs_max_blocks();
  chk(dev_alloc((void**)&b->flags, sizeof(LockFlags) * n));
  chk(dev_alloc((void**)&b->lbar, sizeof(GridBarrier)));
  chk(dev_alloc((void**)&b->done_all, sizeof(unsigned)));
  chk(dev_alloc((void**)&b->counts, 2 * sizeof(unsigned long long)));
  chk(host_alloc_pinned((void**)&b->h_counts, 2 * sizeof(unsigned long long)));
  chk(dev_alloc((void**)&b->cpart, 2 * sizeof(double) * (size_t)b->maxb));
  const size_t cap = 65536 + (size_t)n * 16384;  // LockInst + per pass launch a PassParams and an offset
  for (int v = 0; v < 3; ++v) {
    chk(dev_alloc((void**)&b->arena[v].dev, cap));
    b->arena[v].cap = cap;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemset(b->flags, 0, sizeof(LockFlags) * n);
  if (e == cudaSuccess) e = cudaMemset(b->lbar, 0, sizeof(GridBarrier));
  if (e == cudaSuccess) e = cudaMemset(b->done_all, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(b->counts, 0, 2 * sizeof(unsigned long long));
  return e;
}

// Record the lock-step graph of ring phase v: the set-up and solve start of all instances, the outer
// (refinement) loop whose body starts a cycle, runs the inner (Arnoldi) loop, and updates every
// instance's solution and residual, then the T u update and the statistics gather.  Each line pass of
// an Arnoldi step or residual product is one launch per FFT length over every instance's tiles.
cudaError_t build_lockstep_graph(rfnse_batch* b, int v) {
  const int n = b->count;
  cudaError_t e = lockstep_alloc(b);
  if (e != cudaSuccess) return e;
  TableArena& ar = b->arena[v];
  ar.host.clear();
  const int prev = v, cur = (v + 1) % 3, next = (v + 2) % 3;
  // the batched Arnoldi kernel's blocks, shared in proportion to the instances' sizes
  long long Ntot = 0;
  for (rfnse_ctx* c : b->ctx) Ntot += c->N;
  std::vector<int> ncb(n);
  int sum = 0;
  for (int i = 0; i < n; ++i) {
    const long long N = b->ctx[i]->N;
    long long want = (long long)((double)b->maxb * (double)N / (double)Ntot);
    const long long need = (N + 255) / 256;
    if (want > need) want = need;
    if (want < 1) want = 1;
    ncb[i] = (int)want;
    sum += ncb[i];
  }
  while (sum > b->maxb) {  // at most maxb blocks (each instance keeps one)
    int big = 0;
    for (int i = 1; i < n; ++i)
      if (ncb[i] > ncb[big]) big = i;
    if (ncb[big] <= 1) return cudaErrorInvalidConfiguration;
    --ncb[big];
    --sum;
  }
  std::vector<LockInst> li(n);
  long long blk = 0;
  int cb = 0;
  for (int i = 0; i < n; ++i) {
    rfnse_ctx* c = b->ctx[i];
    LockInst& I = li[i];
    I.gs = c->gs;
    I.fl = b->flags + i;
    I.cfg = solve_cfg(c, 1);
    I.N = c->N;
    I.u_prev = c->u[prev];
    I.u_cur = c->u[cur];
    I.Tu_prev = c->Tu[prev];
    I.x = c->u[next];
    I.Tu_next = c->Tu[next];
    I.f = c->f;
    I.r = c->r;
    I.w = c->w;
    I.V = c->V;
    I.Z32 = c->Z32;
    I.D = c->D;
    I.D32 = c->D32;
    I.dfac32 = c->dfac32;
    I.rho_dt = c->p.rho * c->p.dt;
    I.omega = c->p.omega;
    I.nrm_f = c->nrm_part;
    I.nrm_df = c->nrm_part + kNormPartMax;
    I.nrm_upd = c->nrm_part + 2 * kNormPartMax;
    I.nb_df = 0;
    I.dot_part = c->dot_part;
    I.dot_n = 0;
    I.blk0 = blk;
    I.nblk = lock_ew_blocks(c->N);
    blk += I.nblk;
    I.cb0 = cb;
    I.ncb = ncb[i];
    I.cpart = b->cpart + 2 * (size_t)cb;
    cb += ncb[i];
  }
  const long long blk_total = blk;
  const int cb_total = cb;
  // every instance's passes of one Arnoldi step and of one residual product, recorded, not launched
  std::vector<std::vector<ParamRecord>> arn(n), res(n);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    rfnse_ctx* c = b->ctx[i];
    double2* const x_own = c->x;
    c->x = li[i].x;
    c->param_rec = &arn[i];
    e = record_mixed_arnoldi_passes(c, &b->flags[i].iskip);
    c->param_rec = &res[i];
    if (e == cudaSuccess)
      e = run_matvec_fp64(c, c->x, c->D, c->r, c->f, kMinusOne, kMinusI, 0, &b->flags[i].dfskip, li[i].nrm_df);
    c->param_rec = nullptr;
    c->x = x_own;
  }
  if (e != cudaSuccess) return e;
  for (int i = 1; i < n; ++i) {
    if (arn[i].size() != arn[0].size() || res[i].size() != res[0].size()) return cudaErrorInvalidValue;
    for (size_t k = 0; k < arn[0].size(); ++k)
      if (arn[i][k].key != arn[0][k].key) return cudaErrorInvalidValue;
    for (size_t k = 0; k < res[0].size(); ++k)
      if (res[i][k].key != res[0][k].key) return cudaErrorInvalidValue;
  }
  LockInst* dli = static_cast<LockInst*>(ar.put(li.data(), sizeof(LockInst) * n));
  if (!dli) return cudaErrorMemoryAllocation;
  const size_t li_off = (size_t)((char*)dli - ar.dev);
  // one batched launch per FFT length at pass position k; after() sees each member's tile count
  long long launches = 0;
  // one launch per FFT length at pass position k, one after another (each fills the GPU: measured faster
  // than running a position's groups as parallel graph branches on the 64-instance workload)
  auto launch_position = [&](std::vector<std::vector<ParamRecord>>& recs, size_t k, cudaStream_t s, bool last_arn,
                             bool last_res) -> cudaError_t {
    std::map<int, std::vector<int>> groups;
    for (int i = 0; i < n; ++i) groups[recs[i][k].p.log2L].push_back(i);
    for (auto& kv : groups) {
      std::vector<PassParams> ps;
      for (int i : kv.second) ps.push_back(recs[i][k].p);
      std::vector<long long> grids;
      int dot0 = 0;
      const cudaError_t r = recs[kv.second[0]][k].group(ps, PassGeom{0, 0, 0}, ar, s, grids, &dot0);
      if (r != cudaSuccess) return r;
      ++launches;
      for (size_t m = 0; m < kv.second.size(); ++m) {
        LockInst& I = li[kv.second[m]];
        if (last_arn) I.dot_n = dot0 ? (int)grids[m] : 0;
        if (last_res) I.nb_df = ps[m].nrm_part ? (int)grids[m] : 0;
      }
    }
    return cudaSuccess;
  };
  const long long launches_before = g_kernel_launches.load();  // capture records, it does not launch
  cudaGraph_t g = nullptr;
  cudaStream_t cs = b->cap, bs = b->cap2;
  cudaGraphConditionalHandle ho = 0, hi = 0;
  cudaGraph_t obody = nullptr, ibody = nullptr;
  bool cs_open = false, bs_open = false;
  e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  cs_open = e == cudaSuccess;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&ho, g, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    launch_ls_step_prep(dli, n, blk_total, b->counts, cs);
    launch_ls_norm_start(dli, n, b->lbar, b->done_all, ho, cs);
    e = add_while_node(cs, ho, &obody);
  }
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hi, obody, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(bs, obody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  bs_open = e == cudaSuccess;
  if (e == cudaSuccess) {  // outer body: one refinement cycle of every active instance
    launch_ls_cycle_begin(dli, n, b->counts, hi, ho, bs);
    e = add_while_node(bs, hi, &ibody);
  }
  if (e == cudaSuccess) {
    launch_ls_backsolve(dli, n, bs);
    launch_ls_combine_add(dli, n, blk_total, bs);
    launch_ls_resid_coeffs(dli, n, bs);
    launches = 0;
    for (size_t k = 0; k < res[0].size() && e == cudaSuccess; ++k)
      e = launch_position(res, k, bs, false, k + 1 == res[0].size());
    b->res_launches[v] = launches;
  }
  if (e == cudaSuccess) {
    launch_ls_resid_update(dli, n, blk_total, bs);
    launch_ls_norm_resid(dli, n, b->done_all, ho, bs);
  }
  if (bs_open) {
    const cudaError_t e2 = cudaStreamEndCapture(bs, &obody);
    if (e == cudaSuccess) e = e2;
    bs_open = false;
  }
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(bs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  bs_open = e == cudaSuccess;
  if (e == cudaSuccess) {  // inner body: one Arnoldi step of every instance still iterating
    launches = 0;
    for (size_t k = 0; k < arn[0].size() && e == cudaSuccess; ++k)
      e = launch_position(arn, k, bs, k + 1 == arn[0].size(), false);
    b->arn_launches[v] = launches;
    if (e == cudaSuccess) e = launch_ls_mgs(dli, n, cb_total, b->lbar, b->done_all, b->counts, hi, bs);
  }
  if (bs_open) {
    const cudaError_t e2 = cudaStreamEndCapture(bs, &ibody);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) {
    launch_ls_tu(dli, n, blk_total, cs);
    launch_gather_peeks(b->d_gs, b->d_peeks, n, cs);
    e = cudaMemcpyAsync(b->h_peeks, b->d_peeks, sizeof(GmresPeek) * n, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->h_counts, b->counts, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, cs);
  }
  if (cs_open) {
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &out);
    if (e == cudaSuccess) e = e2;
  }
  g_kernel_launches.store(launches_before);
  if (e == cudaSuccess) {  // the tables with every instance's partial counts, then the graph
    std::memcpy(ar.host.data() + li_off, li.data(), sizeof(LockInst) * n);
    e = cudaMemcpy(ar.dev, ar.host.data(), ar.host.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->lexec[v], g, 0);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    b->lexec[v] = nullptr;
    cudaGetLastError();
    return e;
  }
  b->lgraph[v] = g;
  return cudaSuccess;
}

bool steady(const rfnse_ctx* c) { return c->step >= 1 && (c->p.precision == 0 || c->tu_valid[c->iprev]); }

// Kernels one captured solve executed, from its statistics (as counted for stand-alone solves).
long long solve_kernels(const rfnse_ctx* c, const GmresPeek& pk) {
  const int d = c->d;
  const int mixed = c->p.precision == 1;
  const long long step_k = (d == 1 ? 1 : 3 * d - 2) + 1;
  const long long cycle_k = mixed ? 1 + 1 + d + 1 + 1 : 1 + 1 + 1 + (d == 1 ? 1 : 2 * d - 1) + d + 1;
  const long long cycles = mixed ? pk.outer : (pk.it > 0 ? pk.outer + 1 : 0);
  return 2 + step_k * pk.it + cycle_k * cycles;
}

thread_local std::string g_batch_create_error;

constexpr int kLockstepMinCount = 8;  // batches of at least this many eligible instances start in lock-step

}  // namespace

extern "C" {

int rfnse_batch_create(const rfnse_params* params, int count, void* stream, rfnse_batch** out) {
  if (!out) return RFNSE_EINVAL;
  *out = nullptr;
  if (!params || count < 1) {
    g_batch_create_error = "need count >= 1 parameter sets";
    return RFNSE_EINVAL;
  }
  rfnse_batch* b = new (std::nothrow) rfnse_batch();
  if (!b) return RFNSE_ENOMEM;
  b->count = count;
  b->stream = (cudaStream_t)stream;
  b->ctx.assign(count, nullptr);
  b->streams.assign(count, nullptr);
  int st = RFNSE_OK;
  for (int i = 0; i < count && st == RFNSE_OK; ++i) {
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      st = RFNSE_ECUDA;
      break;
    }
    st = rfnse_create(&params[i], b->streams[i], &b->ctx[i]);
    if (st != RFNSE_OK) g_batch_create_error = "instance " + std::to_string(i) + ": " + rfnse_last_error(nullptr);
    if (st == RFNSE_OK && !b->ctx[i]->Tu[0] && params[i].precision == 1) st = RFNSE_ENOMEM;
  }
  if (st == RFNSE_OK) {
    b->events.assign(count + 1, nullptr);
    for (auto& e : b->events)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = RFNSE_ECUDA;
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) st = RFNSE_ECUDA;
    if (dev_alloc((void**)&b->d_gs, sizeof(GmresState*) * count) != cudaSuccess ||
        dev_alloc((void**)&b->d_peeks, sizeof(GmresPeek) * count) != cudaSuccess ||
        host_alloc_pinned((void**)&b->h_peeks, sizeof(GmresPeek) * count) != cudaSuccess)
      st = RFNSE_ENOMEM;
  }
  if (st == RFNSE_OK) {
    std::vector<GmresState*> h(count);
    for (int i = 0; i < count; ++i) h[i] = b->ctx[i]->gs;
    if (cudaMemcpy(b->d_gs, h.data(), sizeof(GmresState*) * count, cudaMemcpyHostToDevice) != cudaSuccess)
      st = RFNSE_ECUDA;
  }
  if (st != RFNSE_OK) {
    if (g_batch_create_error.empty()) g_batch_create_error = "batch set-up failed";
    free_batch(b);
    return st;
  }
  // lock-step pays off for many instances (64 uneven 2-D instances: 8.3e8 -> 9.1e8 DOF.steps/s); a few
  // large ones are faster as concurrent per-instance graphs (three 511^2: 8.9e8 against 7.1e8)
  b->lockstep = count >= kLockstepMinCount && lockstep_eligible(b);
  *out = b;
  return RFNSE_OK;
}

int rfnse_batch_set_lockstep(rfnse_batch* b, int on) {
  if (!b || (on != 0 && on != 1)) return RFNSE_EINVAL;
  if (on && !lockstep_eligible(b)) {
    b->err = "lock-step mode needs mixed-precision instances of one dimension with the sine-transform "
             "preconditioner and n + 1 in 128..1024 on every axis";
    return RFNSE_EINVAL;
  }
  b->lockstep = on != 0;
  return RFNSE_OK;
}

int rfnse_batch_lockstep(const rfnse_batch* b) { return (b && b->lockstep) ? 1 : 0; }

void rfnse_batch_destroy(rfnse_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_batch(b);
}

const char* rfnse_batch_last_error(const rfnse_batch* b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

rfnse_ctx* rfnse_batch_context(rfnse_batch* b, int i) {
  if (!b || i < 0 || i >= b->count) return nullptr;
  return b->ctx[i];
}

int rfnse_batch_autotune(rfnse_batch* b, int reps, int* n_configs, int* n_changed) {
  if (!b || reps < 1 || reps > 1000) return RFNSE_EINVAL;
  int total = 0, changed = 0;
  for (int i = 0; i < b->count; ++i) {
    int nc = 0, ch = 0;
    const int st = rfnse_autotune(b->ctx[i], reps, 0, &nc, &ch, nullptr);
    if (st != RFNSE_OK) {
      b->err = "instance " + std::to_string(i) + ": " + rfnse_last_error(b->ctx[i]);
      return st;
    }
    total += nc;
    changed += ch;
  }
  // the batch graphs hold the old geometries: capture them again on the next step
  for (int v = 0; v < 3; ++v) {
    if (b->exec[v]) cudaGraphExecDestroy(b->exec[v]);
    if (b->graph[v]) cudaGraphDestroy(b->graph[v]);
    b->exec[v] = nullptr;
    b->graph[v] = nullptr;
  }
  if (n_configs) *n_configs = total;
  if (n_changed) *n_changed = changed;
  return RFNSE_OK;
}

int rfnse_batch_run(rfnse_batch* b, int nsteps, int* iters, double* relres) {
  if (!b || nsteps < 0) return RFNSE_EINVAL;
  int worst = RFNSE_OK;
  for (int s = 0; s < nsteps; ++s) {
    NvtxRange range("rfnse step");
    bool all_steady = true;
    for (rfnse_ctx* c : b->ctx) all_steady = all_steady && steady(c);
    // a failing instance does not stop the others' step: every instance takes this step (or fails it),
    // then the first failure is reported
    int fail = RFNSE_OK;
    if (!all_steady) {  // first steps: every instance on its own (host-driven) until all are steady
      for (int i = 0; i < b->count; ++i) {
        int it = 0;
        double rr = 0.0;
        const int st = rfnse_run(b->ctx[i], 1, nullptr, &it, &rr, 1);
        if (st != RFNSE_OK && st != RFNSE_ENOCONV && fail == RFNSE_OK) {
          b->err = "instance " + std::to_string(i) + ": " + rfnse_last_error(b->ctx[i]);
          fail = st;
        }
        if (st == RFNSE_ENOCONV) worst = RFNSE_ENOCONV;
        if (iters) iters[(size_t)s * b->count + i] = it;
        if (relres) relres[(size_t)s * b->count + i] = rr;
      }
      if (fail != RFNSE_OK) return fail;
      continue;
    }
    // the ring phase of the first instance (or 0); the others are brought to it (no copies once
    // every instance has advanced through the batch)
    const int v = ring_phase(b->ctx[0]) >= 0 ? ring_phase(b->ctx[0]) : 0;
    for (rfnse_ctx* c : b->ctx) {
      if (normalise_history(c, v) != cudaSuccess) {
        b->err = "history normalisation failed";
        return RFNSE_ECUDA;
      }
    }
    for (rfnse_ctx* c : b->ctx) {
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        b->err = "stream synchronisation failed";
        return RFNSE_ECUDA;
      }
    }
    cudaGraphExec_t* exec = b->lockstep ? &b->lexec[v] : &b->exec[v];
    if (!*exec) {
      const cudaError_t e = b->lockstep ? build_lockstep_graph(b, v) : build_batch_graph(b, v);
      if (e != cudaSuccess) {
        b->err = std::string(b->lockstep ? "lock-step graph: " : "batch graph: ") + cudaGetErrorString(e);
        return RFNSE_ECUDA;
      }
    }
    cudaError_t e = cudaGraphLaunch(*exec, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
      b->err = std::string("batch step: ") + cudaGetErrorString(e);
      return RFNSE_ECUDA;
    }
    if (b->lockstep) {  // every kernel of the graph ran for all instances: count them from the loop counts
      const long long cycles = (long long)b->h_counts[1], steps = (long long)b->h_counts[0];
      count_launch(2 + cycles * (1 + 3 + b->res_launches[v] + 2) + steps * (b->arn_launches[v] + 1) + 2);
    } else {
      count_launch(1);  // the statistics gather
    }
    for (int i = 0; i < b->count; ++i) {
      rfnse_ctx* c = b->ctx[i];
      const GmresPeek& pk = b->h_peeks[i];
      // set-up (mixed: one kernel; FP64: D, the product passes, the sub-solve tables), the solve,
      // and (mixed) T u from the final residual
      if (!b->lockstep) count_launch(solve_kernels(c, pk) + (c->p.precision == 1 ? 2 : 2 + c->d));
      c->step += 1;
      c->iprev = (v + 1) % 3;
      c->icur = (v + 2) % 3;
      c->tu_valid[(v + 1) % 3] = c->tu_valid[(v + 2) % 3] = (c->p.precision == 1);
      c->tu_valid[v] = false;
      if (iters) iters[(size_t)s * b->count + i] = pk.it;
      if (relres) relres[(size_t)s * b->count + i] = pk.relres;
      if (pk.err && fail == RFNSE_OK) {
        b->err = "instance " + std::to_string(i) + ": a bounded device-side wait gave up";
        fail = RFNSE_ETIMEOUT;
      }
      if (pk.done == 3 && fail == RFNSE_OK) {
        b->err = "instance " + std::to_string(i) + ": non-finite value in the solve";
        fail = RFNSE_ENUMERIC;
      }
      const bool trivial = pk.beta == 0.0 && pk.it == 0;
      if (!trivial && pk.done != 1 && pk.done != 2) worst = RFNSE_ENOCONV;
    }
    if (fail != RFNSE_OK) return fail;
  }
  return worst;
}

}  // extern "C"
