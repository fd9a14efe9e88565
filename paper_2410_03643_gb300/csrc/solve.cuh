// Host-side solver entry points shared by the C ABI (api.cu) and the drivers (solve.cu).
#pragma once
#include "internal.cuh"

namespace rfnse {

// nrm_part: when the double-float passes run, the last leaves block partials of ||w||^2 there
// (c->nrm_df_blocks of them; 0 when not)
cudaError_t run_matvec_fp64(rfnse_ctx* c, const double2* z, const double* D, double2* w, const double2* add,
                            double2 a, double2 b, int half, const int* skip, double* nrm_part = nullptr);
cudaError_t run_dst(rfnse_ctx* c, int axis, const double2* in, double2* out, int precision);
cudaError_t run_toeplitz(rfnse_ctx* c, int axis, const double2* in, double2* out, int half);
cudaError_t run_apply_prec(rfnse_ctx* c, const double2* v, double2* z, const double* D, int half, int precision);
cudaError_t run_apply_A(rfnse_ctx* c, const double2* u, double2* out, const double* D, int half);
rfnse_status solve_block(rfnse_ctx* c, const double* D, const double2* f, double2* x, int half, int* iters,
                         double* relres);
rfnse_status time_step(rfnse_ctx* c, int* iters, double* relres);
rfnse_status tban_solve(rfnse_ctx* c, const double* D, const double2* f, double2* x, int half, int* iters,
                        double* relres);
cudaError_t prepare_D(rfnse_ctx* c, const double* D);
// f_part / f_n: block partials of ||f||^2 left by f's producer in the same graph (f_n = 0: none)
// the settings of c's solves (mixed = 1: the mixed form)
SolveCfg solve_cfg(const rfnse_ctx* c, int mixed);
// a conditional WHILE node at the capture position of s, made the capture's dependency; its body graph
cudaError_t add_while_node(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body);
// lock-step batches: record (c->param_rec) the passes of one mixed-form Arnoldi step, skipped when *skip
cudaError_t record_mixed_arnoldi_passes(rfnse_ctx* c, const int* skip);
// rfnse_autotune: tune the geometry of every line-pass configuration of c's solves (reps timed launches
// per candidate; force = 1 ignores choices made for the same grid by other contexts)
rfnse_status autotune(rfnse_ctx* c, int reps, int force, int* n_configs, int* n_changed, double* est_speedup);
cudaError_t capture_solve(rfnse_ctx* c, int mixed, int half, cudaGraph_t g, cudaStream_t s,
                          const double* f_part = nullptr, int f_n = 0);

}  // namespace rfnse
