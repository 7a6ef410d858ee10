// Internal launch table of the MPMC kernels: one entry per (species count,
// dimension) instantiation.  Not part of the public C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpmc {

struct KParams;

struct Ops {
  void (*init)(const KParams&, cudaStream_t, const double* prim, double* U, long long n);
  void (*prim)(const KParams&, cudaStream_t, const double* U, const double* Uin, double* Wc,
               unsigned long long* red, int* status);
  void (*face)(const KParams&, cudaStream_t, int d, const double* Wc, const double* Un, const double* Uk,
               const double* Uin, const double* scal, double rk0, double rk1, double rk2, double* F,
               uint32_t* flags, unsigned long long* stats);
  void (*update)(const KParams&, cudaStream_t, const double* Un, const double* Uk, double* const* F,
                 const double* scal, double rk0, double rk1, double rk2, double* Uout, double* dUdt, int* status);
};

// per-dimension tables, defined in mpmc_kernels_d{1,2,3}.cu (FP64) and
// mpmc_mixed_d{1,2,3}.cu (mixed precision; init is the FP64 one)
Ops ops_fp64_d1(int ns);
Ops ops_fp64_d2(int ns);
Ops ops_fp64_d3(int ns);
Ops ops_mixed_d1(int ns);
Ops ops_mixed_d2(int ns);
Ops ops_mixed_d3(int ns);

}  // namespace mpmc
