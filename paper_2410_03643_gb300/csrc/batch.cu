// Batched time stepping of many independent instances (different grids, alpha, rho, dt): every
// instance keeps its own context and stream; once all instances are past their first step, one time
// step of the whole batch is a single CUDA graph launch.  The graph holds, for every instance in its
// own branch, the pointwise set-up (D, right-hand side, sub-solve tables), the solve with its
// device-decided loops (capture_solve) writing u^{n+1} straight into the free history slot, and the
// update of the cached T u (mixed form); it ends by gathering every instance's statistics into pinned
// host memory.  The three history slots form a ring (u^{n-1}, u^n, u^{n+1} in slots v, v+1, v+2 mod 3),
// so there are three graphs, one per phase v, and a step moves no data.
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include "internal.cuh"
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
};

namespace {

const double2 kOne = {1.0, 0.0};
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

bool steady(const rfnse_ctx* c) { return c->step >= 1 && (c->p.precision == 0 || c->tu_valid[c->iprev]); }

// Kernels one captured solve executed, from its statistics (as counted for stand-alone solves).
long long solve_kernels(const rfnse_ctx* c, const GmresPeek& pk) {
  const int d = c->d;
  const int mixed = c->p.precision == 1;
  const long long step_k = (d == 1 ? 1 : 3 * d - 2) + 1;
  const long long cycle_k = mixed ? 1 + 1 + 1 + 1 + d + 1 + 1 : 1 + 1 + 1 + (d == 1 ? 1 : 2 * d - 1) + d + 1;
  const long long cycles = mixed ? pk.outer : (pk.it > 0 ? pk.outer + 1 : 0);
  return 2 + step_k * pk.it + cycle_k * cycles;
}

thread_local std::string g_batch_create_error;

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
  *out = b;
  return RFNSE_OK;
}

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
    if (!b->exec[v]) {
      const cudaError_t e = build_batch_graph(b, v);
      if (e != cudaSuccess) {
        b->err = std::string("batch graph: ") + cudaGetErrorString(e);
        return RFNSE_ECUDA;
      }
    }
    cudaError_t e = cudaGraphLaunch(b->exec[v], b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    count_launch(1);  // the statistics gather
    if (e != cudaSuccess) {
      b->err = std::string("batch step: ") + cudaGetErrorString(e);
      return RFNSE_ECUDA;
    }
    for (int i = 0; i < b->count; ++i) {
      rfnse_ctx* c = b->ctx[i];
      const GmresPeek& pk = b->h_peeks[i];
      // set-up (mixed: one kernel; FP64: D, the product passes, the sub-solve tables), the solve,
      // and (mixed) T u from the final residual
      count_launch(solve_kernels(c, pk) + (c->p.precision == 1 ? 2 : 2 + c->d));
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
