// Lock-step time steps of a batch of independent instances (lockstep.cu, batch.cu).
//
// Every instance keeps its own solve (its own Krylov basis, Hessenberg matrix, Givens rotations,
// tolerance and convergence), but the instances advance through the solve together: each Arnoldi step
// of all instances that are still iterating is one launch per line pass over a work list of every
// instance's tiles and one cooperative launch of modified Gram-Schmidt over every instance's vectors;
// each refinement cycle's bookkeeping is one launch per kernel for all instances.  Instances that have
// finished their cycle (or their solve) skip their share of a launch.  The graph's loops run while any
// instance is still iterating.
#pragma once
#include "internal.cuh"

namespace rfnse {

// Per-instance loop state of a lock-step solve (device memory).
struct LockFlags {
  int act;      // 1 while the instance's solve needs another refinement cycle
  int iskip;    // 1 when the instance takes no further Arnoldi step in the current cycle
  int oskip;    // 1 when the instance's solve is finished (its cycle kernels skip it)
  int dfskip;   // 1 when the instance's residual product does not run this cycle
  unsigned arrive;  // arrivals of the instance's blocks at the end of the cooperative Arnoldi kernel
  int pad_[3];
};

// Per-instance description read by the batched kernels (device memory, one per instance).
struct LockInst {
  GmresState* gs;
  LockFlags* fl;
  SolveCfg cfg;
  long long N;
  const double2* u_prev;    // u^{n-1}
  const double2* u_cur;     // u^n
  const double2* Tu_prev;   // T u^{n-1} (cached by the previous step)
  double2* x;               // the solution, written into the free history slot (u^{n+1})
  double2* Tu_next;         // T u^{n+1}, recovered from the final residual
  double2 *f, *r, *w, *V;   // right-hand side, residual, Arnoldi vector, basis (N-strided)
  float2* Z32;              // preconditioned basis (FP32, N-strided)
  double* D;
  float* D32;
  float2* dfac32;
  double rho_dt, omega;
  double* nrm_f;            // partials of ||f||^2 (one per element-wise block)
  double* nrm_upd;          // partials of ||r||^2 from the residual recurrence (one per element-wise block)
  double* nrm_df;           // partials of ||r||^2 from the last double-float product pass
  int nb_df;                // their count (0: sweep r instead)
  const double* dot_part;   // partials of <v_0, w> from the last product pass of the Arnoldi step
  int dot_n;                // their count (0: the Arnoldi kernel sweeps itself)
  long long blk0, nblk;     // element-wise launches: this instance's blocks
  int cb0, ncb;             // cooperative launch: this instance's blocks
  double* cpart;            // cooperative partials, 2 * ncb
};

constexpr int kLockEwThreads = 256;

// Element-wise blocks of an instance of N points in a batched element-wise launch.
long long lock_ew_blocks(long long N);

// Launchers (one launch each for all n instances; `li` is the device table of LockInst).
// (also clears counts: [0] Arnoldi launches, [1] cycles of this step)
void launch_ls_step_prep(const LockInst* li, int n, long long blocks, unsigned long long* counts, cudaStream_t s);
void launch_ls_norm_start(const LockInst* li, int n, GridBarrier* bar, unsigned* done_all,
                          cudaGraphConditionalHandle h_outer, cudaStream_t s);
void launch_ls_cycle_begin(const LockInst* li, int n, unsigned long long* counts,
                           cudaGraphConditionalHandle h_inner, cudaGraphConditionalHandle h_outer, cudaStream_t s);
cudaError_t launch_ls_mgs(const LockInst* li, int n, int blocks, GridBarrier* bar, unsigned* done_all,
                          unsigned long long* counts, cudaGraphConditionalHandle h_inner, cudaStream_t s);
void launch_ls_backsolve(const LockInst* li, int n, cudaStream_t s);
void launch_ls_combine_add(const LockInst* li, int n, long long blocks, cudaStream_t s);
void launch_ls_resid_coeffs(const LockInst* li, int n, cudaStream_t s);
void launch_ls_resid_update(const LockInst* li, int n, long long blocks, cudaStream_t s);
void launch_ls_norm_resid(const LockInst* li, int n, unsigned* done_all, cudaGraphConditionalHandle h_outer,
                          cudaStream_t s);
void launch_ls_tu(const LockInst* li, int n, long long blocks, cudaStream_t s);
int ls_mgs_max_blocks();  // co-resident blocks of the cooperative kernel on this device

}  // namespace rfnse
