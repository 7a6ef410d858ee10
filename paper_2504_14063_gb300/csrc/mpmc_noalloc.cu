// mpmc_rhs_noalloc: the right-hand-side evaluation of mpmc_rhs for callers
// that cannot allocate device memory -- code that runs where cudaMalloc is
// forbidden or unsafe (inside another framework's memory pool or arena that
// owns the whole device, in a real-time or embedded host loop that must not
// block on the allocator, or before any allocator exists).  All scratch
// (primitive cache, face fluxes, reduction scalars) lives in one file-scope
// device array of fixed size, held by every GPU that loads the library until
// the process exits.  The kernels are the library's FP64 kernels.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/mpmc.h"
#include "mpmc_device.cuh"
#include "mpmc_params.h"
#include "mpmc_ops.h"

namespace mpmc {
// defined with the context entry points (time-step scalars)
__global__ void k_dt(const KParams P, unsigned long long* red, double* scal, double dt_fixed, double gamma_fixed,
                     double* dt_hist, int* counter);

namespace {

constexpr size_t kScratchBytes = (size_t)MPMC_NOALLOC_SCRATCH_BYTES;
constexpr size_t kHeader = 4096;  // scalars, flags, inflow state

// The shared scratch.  In host code `g_scratch` only names a host-side
// stand-in; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_addr[kMaxDevices] = {nullptr};

// device address of g_scratch on the current device, looked up once per
// device and cached: it is not valid after cudaDeviceReset of that device
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPMC_CUDA_ERROR;
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MPMC_CUDA_ERROR;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MPMC_OK;
}

struct Inflow {
  double w[32];
};

__global__ void k_put(Inflow in, double* dst, int n) {
  const int i = threadIdx.x;
  if (i < n) dst[i] = in.w[i];
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Kernel parameters as mpmc_create sets them up (FP64, WENO5-Z only)
int params(const mpmc_grid* g, const mpmc_eos* eos, const mpmc_model* m, KParams& P) {
  if (m && (m->precision != MPMC_FP64 || m->recon != MPMC_RECON_WENO5Z)) return MPMC_INVALID_ARG;
  const int rc = build_params(g, eos, m, P);
  // no characteristic boundaries: their ghost buffers are not laid out here
  return rc ? rc : (P.nslots ? MPMC_INVALID_ARG : MPMC_OK);
}

}  // namespace
}  // namespace mpmc

using namespace mpmc;

extern "C" int mpmc_rhs_noalloc(const mpmc_grid* grid, const mpmc_eos* eos, const mpmc_model* model, void* stream,
                                const double* U, double* dUdt, const mpmc_stage* st, size_t* scratch_bytes) {
  KParams P;
  int rc = params(grid, eos, model, P);
  if (rc) return rc;
  // scratch layout: header | primitive cache | face fluxes of each direction
  long long nface[3] = {0, 0, 0};
  size_t need = kHeader + round256((size_t)P.nW * (size_t)P.wstride * sizeof(double));
  size_t foff[3] = {0, 0, 0};
  for (int d = 0; d < P.dim; ++d) {
    nface[d] = 1;
    for (int e = 0; e < 3; ++e) nface[d] *= (long long)(P.n[e] + (e == d));
    foff[d] = need;
    need += round256((size_t)P.nv * (size_t)nface[d] * sizeof(double));
  }
  if (scratch_bytes) *scratch_bytes = need;
  if (need > kScratchBytes) return MPMC_INVALID_ARG;
  if (!U || !dUdt) return MPMC_INVALID_ARG;
  // an error left pending by earlier work of the caller is reported as it
  // is and not cleared: the final check below then only sees this call's
  if (cudaPeekAtLastError() != cudaSuccess) return MPMC_CUDA_ERROR;
  const Ops ops = P.dim == 1 ? ops_fp64_d1(P.ns) : (P.dim == 2 ? ops_fp64_d2(P.ns) : ops_fp64_d3(P.ns));
  if (!ops.face) return MPMC_INVALID_ARG;
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  double* scal = reinterpret_cast<double*>(b + 0);                     // 8 doubles
  unsigned long long* red = reinterpret_cast<unsigned long long*>(b + 256);  // 4 words
  int* status = reinterpret_cast<int*>(b + 512);
  int* counter = reinterpret_cast<int*>(b + 768);
  double* Uin = reinterpret_cast<double*>(b + 1024);                  // 32 doubles
  P.gn = Uin;   // the inflow state serves U^n and the stage state alike
  double* prim_in = reinterpret_cast<double*>(b + 2048);              // 32 doubles
  double* Wc = reinterpret_cast<double*>(b + kHeader);
  double* F[3] = {nullptr, nullptr, nullptr};
  for (int d = 0; d < P.dim; ++d) F[d] = reinterpret_cast<double*>(b + foff[d]);

  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear what starts at zero
  if (cudaMemsetAsync(b, 0, kHeader, s) != cudaSuccess) {
    cudaGetLastError();
    return MPMC_CUDA_ERROR;
  }
  if (P.has_inflow) {
    Inflow in;
    memset(&in, 0, sizeof(in));
    for (int v = 0; v < P.ns + P.dim + 2; ++v) in.w[v] = grid->inflow[v];
    k_put<<<1, 32, 0, s>>>(in, prim_in, 32);
    ops.init(P, s, prim_in, Uin, 1);
  }
  const double* Un = st && st->U_n ? st->U_n : U;
  const double rk0 = st ? st->rk0 : 1.0, rk1 = st ? st->rk1 : 0.0, rk2 = st ? st->rk2 : 1.0;
  const double dt = st ? st->dt : 0.0, G = st ? st->Gamma : -1.0;
  ops.prim(P, s, Un, Uin, Wc, red, status);
  k_dt<<<1, 1, 0, s>>>(P, red, scal, dt, G, nullptr, counter);
  if (Un != U) ops.prim(P, s, U, Uin, Wc, nullptr, status);
  for (int d = 0; d < P.dim; ++d)
    ops.face(P, s, d, Wc, Un, U, Uin, scal, rk0, rk1, rk2, F[d], nullptr, nullptr);
  ops.update(P, s, Un, U, F, scal, rk0, rk1, rk2, nullptr, dUdt, status);
  if (cudaGetLastError() != cudaSuccess) return MPMC_CUDA_ERROR;
  return MPMC_OK;
}
