// Toeplitz products of the mixed form's outer residual in double-float arithmetic (dfloat.cuh):
// w = add + a z + b (mu_a T_0 z - D z) along the first axis and w += b mu_a T_0 z along the others
// (paper Sec. 2, eq. 'equ2'; the product by circulant embedding as in the FP64 passes), with the two
// length-L FFTs of the embedding in double-float on the FP32 pipes and the pointwise epilogue in FP64.
// The FFT is the fixed-length Stockham FFT of fft_fixed.cuh (radix kFixedLogRDF) instantiated for
// complex double-float; its twiddles and the scaled circulant spectrum are double-float tables built at set-up.
// Only for FFT lengths that have a fixed-length FFT (fixed_fft_length); the caller falls back to the
// FP64 passes otherwise.
#include <cmath>
#include "internal.cuh"
#include "dfloat.cuh"
#include "fft_fixed.cuh"
#include "passes.cuh"

namespace rfnse {

// c v for a coefficient given by code (0: 0, 1: +1, 2: -1, 3: +i, 4: -i) or, for code -1, in full
__device__ __forceinline__ double2 coef_mul(int code, double2 c, double2 v) {
  switch (code) {
    case 0: return make_double2(0.0, 0.0);
    case 1: return v;
    case 2: return make_double2(-v.x, -v.y);
    case 3: return make_double2(-v.y, v.x);
    case 4: return make_double2(v.y, -v.x);
    default: return cmul(c, v);
  }
}

static int coef_code(double2 c) {
  if (c.x == 0.0 && c.y == 0.0) return 0;
  if (c.x == 1.0 && c.y == 0.0) return 1;
  if (c.x == -1.0 && c.y == 0.0) return 2;
  if (c.x == 0.0 && c.y == 1.0) return 3;
  if (c.x == 0.0 && c.y == -1.0) return 4;
  return -1;
}

template <int LOG2L, bool FIRST>
__device__ __forceinline__ void toeplitz_df_body(const PassParams& p, const long long tile) {
  using V = cdf;
  if (p.skip && *p.skip) return;  // uniform
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int L = 1 << LOG2L;
  constexpr int Nh = L >> 1;  // the grids have n + 1 = L / 2 points per axis
  const int B = p.B;
  const int Lp = fft_line_stride(L);
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const bool xax = (p.stride == 1);
  const V zero = cdf{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};

  long long line0 = 0, hi = 0, lo0 = 0;
  if (xax) {
    line0 = tile * B;
  } else {
    hi = tile / p.tiles_inner;
    lo0 = (tile - hi * p.tiles_inner) * B;
  }
  // the tiling of k_line_pass (TileWalk): x lines contiguous, strided tiles of B lines adjacent in x
  auto at = [&](int l, int i) -> V& { return buf[(size_t)l * Lp + fft_pad(i)]; };

  // load z into positions 1..n of the embedding, zero the rest.  In a product along several axes the
  // first pass splits z into double-float and leaves the split copy for the others (FP64 work saved)
  const double2* in = reinterpret_cast<const double2*>(p.in);
  const float4* zdf_in = reinterpret_cast<const float4*>(p.dfz_in);
  float4* zdf_out = reinterpret_cast<float4*>(p.dfz_out);
  for (TileWalk it(p, xax, tid, nthr, line0, hi, lo0); it.more(); it.next()) {
    const int l = it.l, pos = it.pos;
    const bool valid = it.valid;
    const long long g = it.g;
    cdf v = zero;
    if (valid) {
      if (zdf_in) {
        v = cdf_ld(zdf_in[g]);
      } else {
        v = cdf_from(in[g]);
        if (zdf_out) zdf_out[g] = cdf_st(v);
      }
    }
    at(l, 1 + pos) = v;
  }
  for (int e = tid; e < B * Nh; e += nthr) {  // positions 0 and n+1 .. L-1 (n + 1 = L/2)
    const int l = e / Nh, k = e - l * Nh;
    at(l, k == 0 ? 0 : Nh + k) = zero;
  }
  for (int l = tid; l < B; l += nthr) at(l, Nh) = zero;
  __syncthreads();

  const V* tw = reinterpret_cast<const V*>(p.tw);
  fft_lines_fixed<LOG2L, kFixedLogRDF, false, true, false>(buf, Lp, B, tw);   // zero upper half in
  const dfl* circ = reinterpret_cast<const dfl*>(p.circ);
  for (int e = tid; e < B * L; e += nthr) {
    const int l = e >> LOG2L, k = e & (L - 1);
    at(l, k) = cscale(at(l, k), circ[k]);
  }
  __syncthreads();
  fft_lines_fixed<LOG2L, kFixedLogRDF, true, false, true>(buf, Lp, B, tw);    // lower half out

  // epilogue in FP64: FIRST acc = add + a z + b (t - D z); otherwise acc = acc + b t.  The block
  // partials of ||result||^2 only where asked for (the last pass of a product): two FP64 FMAs per point
  // less elsewhere (GB300's FP64 pipe issues 1/64 of the FP32 rate, and it bounds these passes)
  const double2* accin = reinterpret_cast<const double2*>(p.acc_in);
  double2* accout = reinterpret_cast<double2*>(p.acc_out);
  const double* D = reinterpret_cast<const double*>(p.Dr);
  const bool want_nrm = p.nrm_part != nullptr;
  double nacc = 0.0;
  for (TileWalk it(p, xax, tid, nthr, line0, hi, lo0); it.more(); it.next()) {
    const int l = it.l, pos = it.pos;
    const bool valid = it.valid;
    const long long g = it.g;
    if (!valid) continue;
    double2 t = cdf_to(at(l, 1 + pos));
    double2 acc = accin ? accin[g] : make_double2(0.0, 0.0);
    if (FIRST) {
      const double2 z = in[g];
      const double Dj = D ? D[g] : 0.0;
      t.x -= Dj * z.x;
      t.y -= Dj * z.y;
      acc = cadd(acc, coef_mul(p.ca_code, p.ca, z));
    }
    const double2 out = cadd(acc, coef_mul(p.cb_code, p.cb, t));
    accout[g] = out;
    if (want_nrm) {
      nacc = fma(out.x, out.x, nacc);
      nacc = fma(out.y, out.y, nacc);
    }
  }
  if (want_nrm) block_sum_store(nacc, p.nrm_part + tile);  // share of ||result||^2 (uniform)
}

template <int LOG2L, bool FIRST>
__global__ void __launch_bounds__(kPassMaxThreads) k_toeplitz_df(const PassParams p) {
  toeplitz_df_body<LOG2L, FIRST>(p, blockIdx.x);
}

// batched over several instances' tiles (lock-step batch), as k_line_pass_wl
template <int LOG2L, bool FIRST>
__global__ void __launch_bounds__(kPassMaxThreads) k_toeplitz_df_wl(const PassWork w) {
  __shared__ PassParams ps;
  __shared__ long long tile;
  pass_work_item(w, ps, tile);
  toeplitz_df_body<LOG2L, FIRST>(ps, tile);
}

template <int LOG2L>
static cudaError_t launch_df(rfnse_ctx* c, const PassParams& p, bool first, size_t smem, unsigned grid, int threads,
                             cudaStream_t s) {
  auto kern = first ? k_toeplitz_df<LOG2L, true> : k_toeplitz_df<LOG2L, false>;
  static const cudaError_t attr =
      [] {
        cudaError_t e1 = cudaFuncSetAttribute(k_toeplitz_df<LOG2L, true>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaError_t e2 = cudaFuncSetAttribute(k_toeplitz_df<LOG2L, false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return e1 != cudaSuccess ? e1 : e2;
      }();
  if (attr != cudaSuccess) return attr;
  kern<<<grid, threads, smem, s>>>(p);
  count_launch();
  return cudaGetLastError();
}

template <int LOG2L>
static cudaError_t launch_df_wl(const PassWork& w, bool first, size_t smem, unsigned grid, int threads,
                                cudaStream_t s) {
  auto kern = first ? k_toeplitz_df_wl<LOG2L, true> : k_toeplitz_df_wl<LOG2L, false>;
  static const cudaError_t attr =
      [] {
        cudaError_t e1 = cudaFuncSetAttribute(k_toeplitz_df_wl<LOG2L, true>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaError_t e2 = cudaFuncSetAttribute(k_toeplitz_df_wl<LOG2L, false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return e1 != cudaSuccess ? e1 : e2;
      }();
  if (attr != cudaSuccess) return attr;
  {
    NvtxRange range("rfnse pass group");
    kern<<<grid, threads, smem, s>>>(w);
  }
  count_launch();
  return cudaGetLastError();
}

// Tile geometry of a double-float pass for nlines lines with `avail` lines adjacent (x: all).
static void df_geometry(PassParams& p, long long avail, long long nlines) {
  const bool xax = (p.stride == 1);
  pass_geometry_fixed(p.L, xax, avail, nlines, p.nt, p.B, kFixedLogRDF);
  p.log2B = 0;
  while ((1 << p.log2B) < p.B) ++p.log2B;
}

// Batched double-float pass over a group of instances with the same FFT length on this axis (the
// lock-step batch's residual products).  A member whose grid is too large for its norm partials gets
// nrm_part = null (grids[i] still reports its tile count).
static cudaError_t launch_df_group(std::vector<PassParams>& ps, bool first, TableArena& ar, cudaStream_t s,
                                   std::vector<long long>& grids) {
  if (ps.empty()) return cudaSuccess;
  const bool xax = (ps[0].stride == 1);
  long long avail = xax ? 0 : (1LL << 62), lines = 0;
  for (const PassParams& p : ps) {
    lines += p.nlines;
    if (xax) avail += p.nlines;
    else if (p.stride < avail) avail = p.stride;
  }
  PassParams g = ps[0];
  df_geometry(g, avail, lines);
  if (g.B * g.nt > kPassMaxThreads || g.B * g.nt < 1) return cudaErrorInvalidConfiguration;
  std::vector<long long> start(ps.size() + 1, 0);
  grids.assign(ps.size(), 0);
  for (size_t i = 0; i < ps.size(); ++i) {
    PassParams& p = ps[i];
    if (p.L != g.L || p.L != 2 * (p.n + 1)) return cudaErrorInvalidValue;  // the kernel takes n = L/2 - 1
    p.B = g.B;
    p.nt = g.nt;
    p.log2B = g.log2B;
    long long grid;
    if (p.stride == 1) {
      grid = (p.nlines + p.B - 1) / p.B;
      p.tiles_inner = 1;
    } else {
      p.tiles_inner = (p.stride + p.B - 1) / p.B;
      grid = p.tiles_inner * (p.nlines / p.stride);
    }
    if (p.nrm_part && grid > kNormPartMax) p.nrm_part = nullptr;
    grids[i] = grid;
    start[i + 1] = start[i] + grid;
  }
  if (start.back() <= 0) return cudaSuccess;
  const void* dp = ar.put(ps.data(), sizeof(PassParams) * ps.size());
  const void* ds = ar.put(start.data(), sizeof(long long) * start.size());
  if (!dp || !ds) return cudaErrorMemoryAllocation;
  const PassWork w{static_cast<const PassParams*>(dp), static_cast<const long long*>(ds), (int)ps.size()};
  const size_t smem = (size_t)g.B * fft_line_stride(g.L) * sizeof(cdf);
  const unsigned grid = (unsigned)start.back();
  switch (g.log2L) {
    case 8: return launch_df_wl<8>(w, first, smem, grid, g.B * g.nt, s);
    case 9: return launch_df_wl<9>(w, first, smem, grid, g.B * g.nt, s);
    case 10: return launch_df_wl<10>(w, first, smem, grid, g.B * g.nt, s);
    case 11: return launch_df_wl<11>(w, first, smem, grid, g.B * g.nt, s);
    default: return cudaErrorInvalidValue;
  }
}

bool toeplitz_df_available(const rfnse_ctx* c) {
  if (!c->twdf[0]) return false;
  for (int a = 0; a < c->d; ++a)
    if (!fixed_fft_length(c->log2L[a])) return false;
  return true;
}

// One Toeplitz pass along `axis` in double-float: first = the x-pass with diagonal and coupling.
cudaError_t run_toeplitz_df(rfnse_ctx* c, int axis, int half, bool first, const double2* z, const double* D,
                            const double2* add, double2* w, double2 a, double2 b, const int* skip,
                            double* nrm_part, const void* dfz_in, void* dfz_out) {
  PassParams p{};
  p.dfz_in = dfz_in;
  p.dfz_out = dfz_out;
  p.n = c->n[axis];
  p.L = c->L[axis];
  p.log2L = c->log2L[axis];
  if (p.L != 2 * (p.n + 1)) return cudaErrorInvalidValue;  // the kernel takes n = L/2 - 1
  p.stride = c->stride[axis];
  p.nlines = c->N / c->n[axis];
  p.tw = c->twdf[axis];
  p.circ = c->circdf[half ? 1 : 0][axis];
  p.in = z;
  p.Dr = D;
  p.acc_in = add;
  p.acc_out = w;
  p.ca = a;
  p.cb = b;
  p.ca_code = coef_code(a);
  p.cb_code = coef_code(b);
  p.skip = skip;
  const bool xax = (p.stride == 1);
  if (c->param_rec) {  // a lock-step batch records the pass instead of launching it
    ParamRecord r;
    r.key = (first ? F_TOEP_X : F_TOEP_ACC) | RFNSE_K_DF | ((unsigned long long)axis << 13);
    p.nrm_part = nrm_part;
    r.p = p;
    r.df = true;
    r.group = [first](std::vector<PassParams>& ps, const PassGeom&, TableArena& ar, cudaStream_t st,
                      std::vector<long long>& grids, int*) { return launch_df_group(ps, first, ar, st, grids); };
    c->param_rec->push_back(std::move(r));
    return cudaSuccess;
  }
  df_geometry(p, xax ? p.nlines : p.stride, p.nlines);
  long long grid;
  if (xax) {
    grid = (p.nlines + p.B - 1) / p.B;
    p.tiles_inner = 1;
  } else {
    p.tiles_inner = (p.stride + p.B - 1) / p.B;
    grid = p.tiles_inner * (p.nlines / p.stride);
  }
  if (grid <= 0) return cudaSuccess;
  if (p.B * p.nt > kPassMaxThreads || p.B * p.nt < 1) return cudaErrorInvalidConfiguration;
  if (nrm_part) {  // partials of ||w||^2 for the norm kernel, if it can sum this many
    p.nrm_part = grid <= kNormPartMax ? nrm_part : nullptr;
    c->nrm_df_blocks = grid <= kNormPartMax ? (int)grid : 0;
  }
  const size_t smem = (size_t)p.B * fft_line_stride(p.L) * sizeof(cdf);
  // kernel-class profiling (rfnse_profile): kind = Toeplitz flag | RFNSE_K_DF
  const int kind = (first ? F_TOEP_X : F_TOEP_ACC) | RFNSE_K_DF;
  const bool prof = c->prof_kind != 0 && c->prof_kind == kind;
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
  cudaError_t e;
  switch (p.log2L) {
    case 8: e = launch_df<8>(c, p, first, smem, (unsigned)grid, p.B * p.nt, c->stream); break;
    case 9: e = launch_df<9>(c, p, first, smem, (unsigned)grid, p.B * p.nt, c->stream); break;
    case 10: e = launch_df<10>(c, p, first, smem, (unsigned)grid, p.B * p.nt, c->stream); break;
    case 11: e = launch_df<11>(c, p, first, smem, (unsigned)grid, p.B * p.nt, c->stream); break;
    default: return cudaErrorInvalidValue;
  }
  cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
  if (e == cudaSuccess && c->debug && cudaStreamIsCapturing(c->stream, &cap_st) == cudaSuccess &&
      cap_st == cudaStreamCaptureStatusNone) {  // debug mode: the result (or its double-float running sum)
    const void* outs[1] = {w};
    const int elems[1] = {16};
    e = debug_after_pass(c, c->stream, first ? "double-float Toeplitz pass (first axis)" : "double-float Toeplitz pass",
                         outs, elems, 1, c->N);
  }
  if (prof) {
    cudaEventRecord(e1, c->stream);
    const double lines = (double)p.nlines, N = lines * p.n;
    c->prof_flops += lines * 2.0 * 5.0 * p.L * p.log2L;  // two FFTs of length L per line
    // z (or its double-float copy) in, the result out, the additive vector or running sum in, D in; the
    // first pass of a product along several axes also stores z split
    c->prof_bytes += N * (16.0 + 16.0 + (add ? 16.0 : 0.0) + ((first && D) ? 8.0 : 0.0) + (dfz_out ? 16.0 : 0.0));
  }
  return e;
}

// Set-up: the fixed-length FFT's twiddle table in double-float (from FP64 sin/cos of exact binary
// fractions) and the scaled circulant spectra split into double-float.
__global__ void k_df_tables(int log2L, const double* __restrict__ c64h0, const double* __restrict__ c64h1,
                            cdf* __restrict__ tw, dfl* __restrict__ c0, dfl* __restrict__ c1) {
  const int L = 1 << log2L;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  int R, ns, r, kk;
  fixed_twiddle_entry(log2L, kFixedLogRDF, k, R, ns, r, kk);
  double sn = 0.0, cs = 1.0;
  if (R > 1) sincospi(2.0 * (double)(r * kk) / (double)(R * ns), &sn, &cs);
  tw[k] = cvec<dfl>::make(dfl(cs), dfl(-sn));
  c0[k] = dfl(c64h0[k]);
  c1[k] = dfl(c64h1[k]);
}

void launch_setup_df(int log2L, const double* c64h0, const double* c64h1, void* tw, void* c0, void* c1,
                     cudaStream_t s) {
  const int L = 1 << log2L;
  count_launch();
  k_df_tables<<<(L + 127) / 128, 128, 0, s>>>(log2L, c64h0, c64h1, reinterpret_cast<cdf*>(tw),
                                              reinterpret_cast<dfl*>(c0), reinterpret_cast<dfl*>(c1));
}

}  // namespace rfnse
