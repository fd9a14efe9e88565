// Host-side solver entry points shared by the C ABI (api.cu) and the drivers (solve.cu).
#pragma once
#include "internal.cuh"

namespace rfnse {

cudaError_t run_matvec_fp64(rfnse_ctx* c, const double2* z, const double* D, double2* w, const double2* add,
                            double2 a, double2 b, int half, const int* skip);
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
cudaError_t capture_solve(rfnse_ctx* c, int mixed, int half, cudaGraph_t g, cudaStream_t s);

}  // namespace rfnse
