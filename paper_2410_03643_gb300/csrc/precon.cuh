// The preconditioner sequence of line passes, shared by the solver drivers (solve.cu) and the
// comparator instantiations (comparators.cu).
#pragma once
#include <cmath>
#include <utility>
#include "internal.cuh"
#include "passes.cuh"

namespace rfnse {

static const double2 kOne = {1.0, 0.0};
static const double2 kI = {0.0, 1.0};
static const double2 kMinusOne = {-1.0, 0.0};
static const double2 kMinusI = {0.0, -1.0};

template <typename R> struct Tables;
template <> struct Tables<double> {
  static const void* tw(const rfnse_ctx* c, int a) { return c->tw64[a]; }
  static const void* circ(const rfnse_ctx* c, int h, int a) { return c->circ64s[h][a]; }
  static const void* lamfac(const rfnse_ctx* c, int h) {
    return c->p.precond == 1 ? (const void*)c->lamfacC64[h] : (const void*)c->lamfac64[h];
  }
  static const void* dfac(const rfnse_ctx* c) { return c->dfac64; }
  static const void* Dr(const rfnse_ctx* c, const double* D) { return D; }
  static const void* chirp(const rfnse_ctx* c, int a) { return c->chirp64[a]; }
  static const void* bspec(const rfnse_ctx* c, int a) { return c->bspec64[a]; }
};
template <> struct Tables<float> {
  static const void* tw(const rfnse_ctx* c, int a) { return c->tw32[a]; }
  static const void* circ(const rfnse_ctx* c, int h, int a) { return c->circ32s[h][a]; }
  static const void* lamfac(const rfnse_ctx* c, int h) {
    return c->p.precond == 1 ? (const void*)c->lamfacC32[h] : (const void*)c->lamfac32[h];
  }
  static const void* dfac(const rfnse_ctx* c) { return c->dfac32; }
  static const void* Dr(const rfnse_ctx* c, const double*) { return c->D32; }
  static const void* chirp(const rfnse_ctx* c, int a) { return c->chirp32[a]; }
  static const void* bspec(const rfnse_ctx* c, int a) { return c->bspec32[a]; }
};

template <typename R>
PassParams base_params(const rfnse_ctx* c, int axis, int half) {
  PassParams p{};
  p.n = c->n[axis];
  p.L = c->L[axis];
  p.log2L = c->log2L[axis];
  p.stride = c->stride[axis];
  p.nlines = c->N / c->n[axis];
  p.tw = Tables<R>::tw(c, axis);
  p.circ = Tables<R>::circ(c, half ? 1 : 0, axis);
  p.dst_scale = 1.0 / std::sqrt((double)p.L);
  p.chirp = Tables<R>::chirp(c, axis);
  p.bspec = Tables<R>::bspec(c, axis);
  p.ca = kOne;
  p.cb = kI;
  return p;
}

// Device-resolved operands of the Arnoldi step (see PassParams::gdyn) and a skip flag.
struct Dyn {
  const GmresState* gs = nullptr;
  double2* vbase = nullptr;
  void* zbase = nullptr;
  long long ldv = 0;
  const int* skip = nullptr;
  // the last product pass also leaves the block partials of <v_0, w> (v_0 = vbase) in c->dot_part
  // for the Arnoldi kernel, and their count in c->dot0_blocks (F_DOT0)
  bool dot0 = false;
};

// ---------------------------------------------------------------------------------------------
// z = F~^{-1} v (eq. 'taupre'), optionally followed by w = add + a z + b (T - D) z.
//   R     compute precision of the transforms
//   TIN   storage of v (double2 when INSC: v is scaled by *in_scale and copied to copy_v)
//   TMP   storage of the intermediate vectors t1, t2
//   TZ    storage of z
//   TW    storage of the partial products between Toeplitz passes (w itself when TW = double2)
// The caller has run prepare_D for D.  With dyn.gs set, the scaled input, its copy V[j] and (with
// dyn.zbase) the output Z[j] are resolved on the device.
//   PC    preconditioner: 0 the sine-transform F~ (Sec. 4), 1 the circulant comparator F_C (Sec. 5:
//         the same pass sequence with length-n DFTs in place of S), 2 none (z = v)
template <int PC, typename R, typename TIN, typename TMP, typename TZ, typename TW, bool INSC, bool MATVEC>
cudaError_t run_precon_pc(rfnse_ctx* c, const TIN* v, const double* in_scale, double2* copy_v, TZ* z, int z_add,
                          const double* D, double2* w, TW* wtmp, const double2* w_add, double2 a, double2 b,
                          int half, TMP* t1, TMP* t2, const Dyn& dyn) {
  cudaStream_t s = c->stream;
  cudaError_t e;
  constexpr int IS = INSC ? F_INSCALE : 0;
  constexpr int TX = MATVEC ? F_TOEP_X : 0;
  constexpr int CF = (PC == 1) ? F_CIRC : 0;
  const int h = half ? 1 : 0;
  auto with_dyn = [&](PassParams& p) {
    p.gdyn = dyn.gs;
    p.vbase = dyn.vbase;
    p.zbase = dyn.zbase;
    p.ldv = dyn.ldv;
    p.skip = dyn.skip;
  };
  const bool dot0 = MATVEC && dyn.dot0;
  if (MATVEC) c->dot0_blocks = 0;
  auto with_dot0 = [&](PassParams& p) {
    p.dot_v0 = dyn.vbase;
    p.dot_part = c->dot_part;
  };
  if constexpr (PC == 2) {  // no preconditioner: z = v, then the product along x
    PassParams p = base_params<R>(c, 0, h);
    p.in = v; p.in_scale = in_scale; p.copy_out = copy_v; p.out = z; p.z_add = z_add;
    p.Dr = Tables<R>::Dr(c, D); p.dfac = nullptr;
    p.acc_in = w_add; p.ca = a; p.cb = b;
    with_dyn(p);
    if (c->d == 1) {
      p.acc_out = w;
      if (dot0) {
        with_dot0(p);
        return launch_pass<R, TIN, TZ, double2, double2, IS | F_DSCALE | TX | (MATVEC ? F_DOT0 : 0)>(c, p, s);
      }
      return launch_pass<R, TIN, TZ, double2, double2, IS | F_DSCALE | TX>(c, p, s);
    }
    p.acc_out = wtmp;
    if ((e = launch_pass<R, TIN, TZ, double2, TW, IS | F_DSCALE | TX>(c, p, s)) != cudaSuccess) return e;
  } else {
    if (c->d == 1) {
      PassParams p = base_params<R>(c, 0, h);
      p.in = v; p.in_scale = in_scale; p.copy_out = copy_v; p.out = z; p.z_add = z_add;
      p.Dr = Tables<R>::Dr(c, D); p.dfac = Tables<R>::dfac(c); p.lamfac = Tables<R>::lamfac(c, h);
      p.acc_in = w_add; p.acc_out = w; p.ca = a; p.cb = b;
      with_dyn(p);
      if (dot0) {
        with_dot0(p);
        return launch_pass<R, TIN, TZ, double2, double2,
                           IS | F_DST | CF | F_LAM | F_DSCALE | TX | (MATVEC ? F_DOT0 : 0)>(c, p, s);
      }
      return launch_pass<R, TIN, TZ, double2, double2, IS | F_DST | CF | F_LAM | F_DSCALE | TX>(c, p, s);
    }
    {  // first axis: forward DST (and the Arnoldi normalisation)
      PassParams p = base_params<R>(c, 0, h);
      p.in = v; p.in_scale = in_scale; p.copy_out = copy_v; p.out = t1;
      with_dyn(p);
      p.zbase = nullptr;
      if ((e = launch_pass<R, TIN, TMP, double2, double2, IS | F_DST | CF>(c, p, s)) != cudaSuccess) return e;
    }
    TMP* cur = t1;
    TMP* nxt = t2;
    for (int a2 = 1; a2 < c->d - 1; ++a2) {  // middle axes (d = 3): forward DST
      PassParams p = base_params<R>(c, a2, h);
      p.in = cur; p.out = nxt; p.skip = dyn.skip;
      if ((e = launch_pass<R, TMP, TMP, double2, double2, F_DST | CF>(c, p, s)) != cudaSuccess) return e;
      std::swap(cur, nxt);
    }
    {  // last axis: DST, multiply by i s/(w + i Lambda), DST
      PassParams p = base_params<R>(c, c->d - 1, h);
      p.in = cur; p.out = nxt; p.lamfac = Tables<R>::lamfac(c, h); p.skip = dyn.skip;
      if ((e = launch_pass<R, TMP, TMP, double2, double2, F_DST | CF | F_LAM>(c, p, s)) != cudaSuccess) return e;
      std::swap(cur, nxt);
    }
    for (int a2 = c->d - 2; a2 >= 1; --a2) {  // middle axes: inverse DST (S is involutory)
      PassParams p = base_params<R>(c, a2, h);
      p.in = cur; p.out = nxt; p.skip = dyn.skip; p.inv_dft = 1;
      if ((e = launch_pass<R, TMP, TMP, double2, double2, F_DST | CF>(c, p, s)) != cudaSuccess) return e;
      std::swap(cur, nxt);
    }
    {  // first axis: inverse DST, (wI + D)^{-1} sub-solve, optional Toeplitz along x
      PassParams p = base_params<R>(c, 0, h);
      p.in = cur; p.out = z; p.z_add = z_add;
      p.Dr = Tables<R>::Dr(c, D); p.dfac = Tables<R>::dfac(c);
      p.acc_in = w_add; p.acc_out = wtmp; p.ca = a; p.cb = b; p.inv_dft = 1;
      with_dyn(p);
      if ((e = launch_pass<R, TMP, TZ, double2, TW, F_DST | CF | F_DSCALE | TX>(c, p, s)) != cudaSuccess) return e;
    }
  }
  if (MATVEC) {
    for (int a2 = 1; a2 < c->d; ++a2) {
      PassParams p = base_params<R>(c, a2, h);
      p.in = z; p.acc_in = wtmp; p.cb = b;
      with_dyn(p);
      p.in_dyn_z = (dyn.gs && dyn.zbase) ? 1 : 0;
      if (a2 == c->d - 1) {
        p.acc_out = w;
        if (dot0) {
          with_dot0(p);
          e = launch_pass<R, TZ, TZ, TW, double2, F_TOEP_ACC | F_DOT0>(c, p, s);
        } else {
          e = launch_pass<R, TZ, TZ, TW, double2, F_TOEP_ACC>(c, p, s);
        }
      } else {
        p.acc_out = wtmp;
        e = launch_pass<R, TZ, TZ, TW, TW, F_TOEP_ACC>(c, p, s);
      }
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}


// The instantiations the drivers use, for PC = 1 and 2 compiled in comparators.cu (so that the
// comparator kernels build in parallel with the rest): X(PC, R, TIN, TMP, TZ, TW, INSC, MATVEC)
#define RFNSE_PRECON_VARIANTS(X, PC)                                  \
  X(PC, float, double2, float2, double2, float2, false, false)       \
  X(PC, double, double2, double2, double2, double2, false, false)    \
  X(PC, double, double2, double2, double2, double2, true, true)      \
  X(PC, float, double2, float2, float2, float2, true, true)

#define RFNSE_PRECON_SIG(PC, R, TIN, TMP, TZ, TW, INSC, MATVEC)                                        \
  template cudaError_t run_precon_pc<PC, R, TIN, TMP, TZ, TW, INSC, MATVEC>(                          \
      rfnse_ctx*, const TIN*, const double*, double2*, TZ*, int, const double*, double2*, TW*,         \
      const double2*, double2, double2, int, TMP*, TMP*, const Dyn&);
#define RFNSE_PRECON_EXTERN(PC, R, TIN, TMP, TZ, TW, INSC, MATVEC) extern RFNSE_PRECON_SIG(PC, R, TIN, TMP, TZ, TW, INSC, MATVEC)

}  // namespace rfnse
