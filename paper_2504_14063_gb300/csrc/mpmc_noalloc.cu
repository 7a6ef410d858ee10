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

// device address of g_scratch on the current device (looked up once per device)
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

// Kernel parameters from the public structs: the same fields and cache
// layout that mpmc_create sets up.
int params(const mpmc_grid* g, const mpmc_eos* eos, const mpmc_model* m, KParams& P) {
  if (!g || !eos || !m) return MPMC_INVALID_ARG;
  if (g->dim < 1 || g->dim > 3 || eos->n_species < 1 || eos->n_species > MPMC_MAXS || !(g->dx > 0.0))
    return MPMC_INVALID_ARG;
  if (m->precision != MPMC_FP64) return MPMC_INVALID_ARG;
  for (int d = 0; d < 3; ++d) {
    if (d < g->dim && g->n[d] < 3) return MPMC_INVALID_ARG;
    if (d >= g->dim && g->n[d] != 1) return MPMC_INVALID_ARG;
    if (d < g->dim && (g->bc_lo[d] < 0 || g->bc_lo[d] > 3 || g->bc_hi[d] < 0 || g->bc_hi[d] > 3))
      return MPMC_INVALID_ARG;
    if (d < g->dim && ((g->bc_lo[d] == MPMC_BC_PERIODIC) != (g->bc_hi[d] == MPMC_BC_PERIODIC)))
      return MPMC_INVALID_ARG;
  }
  memset(&P, 0, sizeof(P));
  const int ns = eos->n_species, D = g->dim;
  P.dim = D;
  P.ns = ns;
  P.nv = ns + D + 1;
  for (int d = 0; d < 3; ++d) {
    P.n[d] = g->n[d];
    P.bc_lo[d] = d < D ? g->bc_lo[d] : 0;
    P.bc_hi[d] = d < D ? g->bc_hi[d] : 0;
    if (d < D && (P.bc_lo[d] == MPMC_BC_INFLOW || P.bc_hi[d] == MPMC_BC_INFLOW)) P.has_inflow = 1;
  }
  P.ncell = (long long)g->n[0] * g->n[1] * g->n[2];
  P.dx = g->dx;
  P.inv_dx = 1.0 / g->dx;
  bool has0 = false, has1 = false;
  for (int k = 0; k < ns; ++k) {
    P.phase[k] = eos->phase[k] ? 1 : 0;
    (P.phase[k] ? has1 : has0) = true;
    P.cv[k] = eos->cv[k];
    P.gam[k] = eos->gamma[k];
    P.q[k] = eos->q[k];
    P.b[k] = eos->b[k];
    P.pinf[k] = eos->pinf[k];
    P.W[k] = eos->W[k];
    P.mu[k] = eos->mu[k];
    P.Sc[k] = eos->Sc[k];
    P.Rk[k] = (eos->gamma[k] - 1.0) * eos->cv[k];
    if (eos->b[k] != 0.0) P.has_b = 1;
    if (eos->q[k] != 0.0) P.has_q = 1;
    P.cp[k] = eos->gamma[k] * eos->cv[k];
  }
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < ns; ++j) {
      const double Wij = P.W[i] / P.W[j];
      const double t = 1.0 + std::sqrt(P.mu[i] / P.mu[j]) * std::pow(P.W[j] / P.W[i], 0.25);
      P.wilke[i][j] = Wij * (t * t / (std::sqrt(8.0) * std::sqrt(1.0 + Wij)));
    }
  P.two_phase = has0 && has1;
  P.weno_eps = m->weno_eps;
  P.cdi = m->cdi ? 1 : 0;
  P.diffusion = m->diffusion ? 1 : 0;
  P.pos_limiter = m->pos_limiter ? 1 : 0;
  P.cdi_eps = m->cdi_eps > 0.0 ? m->cdi_eps : g->dx;
  P.cdi_gamma = m->cdi_gamma;
  P.phi_min = m->phi_min;
  P.psi_delta = m->psi_delta;
  P.cfl = m->cfl;
  P.mu_liquid = m->mu_liquid;
  P.sharp0 = 4.0 * m->phi_min * (1.0 - m->phi_min);
  int f = 0;
  P.wT = f++;
  P.wP = f++;
  P.wRho = f++;
  P.wA = f++;
  P.wY = f;
  f += ns;
  P.wU = f;
  f += D;
  if (P.cdi) {
    P.wPhi0 = f++;
    P.wPsi = f++;
    P.wYrho = f;
    f += ns;
    P.wHrho = f;
    f += 2;
  }
  if (P.diffusion) {
    P.wXr = f;
    f += ns;
    P.wB = f;
    f += ns;
  }
  P.nW = f;
  P.wstride = P.ncell + 1;
  return MPMC_OK;
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
  double* prim_in = reinterpret_cast<double*>(b + 2048);              // 32 doubles
  double* Wc = reinterpret_cast<double*>(b + kHeader);
  double* F[3] = {nullptr, nullptr, nullptr};
  for (int d = 0; d < P.dim; ++d) F[d] = reinterpret_cast<double*>(b + foff[d]);

  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear what starts at zero
  cudaMemsetAsync(b, 0, kHeader, s);
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
