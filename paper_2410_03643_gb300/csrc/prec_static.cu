// rfnse_apply_prec_static: the preconditioner apply of rfnse_apply_prec (FP64) without any device
// allocation.  Some callers cannot call cudaMalloc: plug-ins whose host application owns the whole
// device-memory budget, real-time loops that must not allocate once they are running, and programs
// whose memory comes from an allocator other than CUDA's.  They still pass their own inputs and
// outputs; everything else this call needs (the coefficient, eigenvalue, twiddle and factor tables
// and the intermediate grid vectors between the line passes) lives in one file-scope device array.
//
// The array is a static __device__ object: every GPU that loads this library holds it (about 17 MB)
// until the process exits.  All calls on a device share it, and it keeps whatever the last call
// wrote; this entry point overwrites every part it reads, so nothing has to start at zero.  Two
// calls whose work overlaps on the GPU (different streams, or different host threads) race on the
// array and give wrong results: serialise them.
#include <cmath>
#include "internal.cuh"
#include "solve.cuh"

namespace {

constexpr long long kStaticMaxN = 1LL << 18;   // largest grid: N = n0*n1*n2 <= 262144 complex values
constexpr int kStaticMaxL = 4096;              // FFT length 2(n+1) for n + 1 <= 2048

// Layout of the array, in double2 units:
//   [t1: kStaticMaxN][t2: kStaticMaxN][dfac64: kStaticMaxN][lamfac64: kStaticMaxN]
//   [c: 1024 (2048 doubles)]
//   per axis a < 3: [lam: 1024 (2048 doubles)][circ: 2048 (4096 doubles)][tw64: 4096][tw32: 2048 (4096 float2)]
// The FP32 companions the set-up kernels also write (lamfac32, D32, dfac32) are not read by this FP64
// path; they are pointed at t1 and t2, which the first passes overwrite.
constexpr long long kTableElems = 1024 + 3LL * (1024 + 2048 + 4096 + 2048);
constexpr long long kStaticElems = 4 * kStaticMaxN + kTableElems;

static __device__ __align__(256) double2 g_prec_scratch[kStaticElems];

// Device address of g_prec_scratch on the current device.  Host code may not use the symbol itself
// (it is a host-side stand-in); cudaGetSymbolAddress gives the real address.  It is looked up on every
// call rather than cached, so the address stays right after the primary context has been reset and the
// module reloaded elsewhere in the process.
cudaError_t scratch_address(double2** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_prec_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double2*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" int rfnse_apply_prec_static(const rfnse_params* p, const void* v, void* z, const double* D, int half,
                                       void* stream) {
  using namespace rfnse;
  if (!p || !v || !z || !D || v == z) return RFNSE_EINVAL;
  if (validate_problem(p)) return RFNSE_EINVAL;  // the checks of rfnse_create on d, grid, box, alpha, rho, dt, omega
  long long N = 1;
  for (int a = 0; a < p->d; ++a) N *= p->n[a];
  if (N > kStaticMaxN) return RFNSE_EINVAL;  // larger grids need rfnse_create / rfnse_apply_prec
  // A CUDA error already pending in this thread belongs to the caller: leave it for the caller's own
  // check and do nothing, so that every error seen below is one this call caused.
  if (cudaPeekAtLastError() != cudaSuccess) return RFNSE_ECUDA;

  double2* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return RFNSE_ECUDA;

  // A context on the stack whose arrays all point into the static scratch: no allocation.
  rfnse_ctx c;
  c.p = *p;
  c.p.precision = 0;
  c.p.precond = 0;  // the sine-transform preconditioner F~ only
  c.stream = (cudaStream_t)stream;
  c.d = p->d;
  c.N = 1;
  int nmax = 0;
  for (int a = 0; a < 3; ++a) {
    c.n[a] = (a < c.d) ? p->n[a] : 1;
    c.stride[a] = c.N;
    c.N *= c.n[a];
    c.L[a] = (a < c.d) ? 2 * (c.n[a] + 1) : 0;
    c.log2L[a] = 0;
    while (a < c.d && (1 << c.log2L[a]) < c.L[a]) ++c.log2L[a];
    c.h[a] = (a < c.d) ? (p->hi[a] - p->lo[a]) / (c.n[a] + 1) : 0.0;
    c.mu[a] = (a < c.d) ? p->dt / std::pow(c.h[a], p->alpha) : 0.0;
    if (a < c.d && c.n[a] > nmax) nmax = c.n[a];
  }
  c.t1 = base;
  c.t2 = base + kStaticMaxN;
  c.dfac64 = base + 2 * kStaticMaxN;
  const int hidx = half ? 1 : 0;
  c.lamfac64[hidx] = base + 3 * kStaticMaxN;
  c.lamfac32[hidx] = reinterpret_cast<float2*>(c.t1);
  c.dfac32 = reinterpret_cast<float2*>(c.t2);                       // 8 N bytes
  c.D32 = reinterpret_cast<float*>(c.t2) + 2 * kStaticMaxN;          // 4 N bytes after dfac32
  double2* tab = base + 4 * kStaticMaxN;
  c.c = reinterpret_cast<double*>(tab);
  tab += 1024;
  for (int a = 0; a < 3; ++a) {
    double* lam = reinterpret_cast<double*>(tab);
    double* circ = reinterpret_cast<double*>(tab + 1024);
    double2* tw64 = tab + 1024 + 2048;
    float2* tw32 = reinterpret_cast<float2*>(tab + 1024 + 2048 + kStaticMaxL);
    tab += 1024 + 2048 + kStaticMaxL + 2048;
    if (a < c.d) {
      c.lam[a] = lam;
      c.circ[a] = circ;
      c.tw64[a] = tw64;
      c.tw32[a] = tw32;
    }
  }

  // Tables first (they are rewritten on every call), then the same passes as rfnse_apply_prec.
  launch_setup_coefficients(c.c, nmax, p->alpha, c.stream);
  for (int a = 0; a < c.d; ++a)
    launch_setup_axis(c.c, c.n[a], c.L[a], c.lam[a], c.circ[a], c.tw64[a], c.tw32[a], c.stream);
  const double hf = half ? 0.5 : 1.0;
  launch_setup_lamfac(c.lam[0], c.lam[1], c.lam[2], c.n[0], c.n[1], c.n[2], hf * c.mu[0], hf * c.mu[1],
                      hf * c.mu[2], p->omega, 1.0 / std::sqrt((double)c.L[c.d - 1]), 0, c.lamfac64[hidx],
                      c.lamfac32[hidx], c.N, c.stream);
  if (cudaGetLastError() != cudaSuccess) return RFNSE_ECUDA;  // a set-up launch of this call failed
  if (run_apply_prec(&c, (const double2*)v, (double2*)z, D, half ? 1 : 0, 0) != cudaSuccess) return RFNSE_ECUDA;
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) return RFNSE_ECUDA;
  return RFNSE_OK;
}
