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
  // ghost states of the characteristic boundaries of U into its ghost buffer
  // G (FP64 on both paths; nothing to do without such boundaries)
  void (*ghost)(const KParams&, cudaStream_t, const double* U, double* G);
};

// discrete adjoint (FP64): per-face contributions of one direction into a
// slot buffer, their per-cell gather, the per-cell primitive-recovery VJP
// fused with the reverse RK combination, and the VJP of the initialisation
struct AdjOps {
  int (*slots)(const KParams&);
  void (*face)(const KParams&, cudaStream_t, int d, const double* Wc, const double* Uk, const double* Uin,
               const double* scal, const uint32_t* tape, const double* lamL, double coef, int mul_dt, double* C);
  // the viscous stress and conduction flux of the same faces, reversed (adds
  // to the slots the face pass wrote)
  void (*face_visc)(const KParams&, cudaStream_t, int d, const double* Wc, const double* scal,
                    const uint32_t* tape, const double* lamL, double coef, int mul_dt, double* C);
  void (*gather)(const KParams&, cudaStream_t, int d, const double* C, int first, double* gW, double* gU);
  // Wc (nullable): U's primitive cache, whose T and P the reverse takes
  // instead of solving the p-T equilibrium again
  void (*cell)(const KParams&, cudaStream_t, const double* U, const double* Wc, const double* gW, const double* gU,
               double* out, double a, const double* x, double b, const double* y, double cz, const double* z);
  void (*init)(const KParams&, cudaStream_t, const double* prim, const double* lamU, double* lprim, long long n);
};

using FaceFn = decltype(Ops::face);
// FP64 face passes with Sec. 4.1's other ENO-type interpolations, for
// (dimension, species count), null if none: defined in
// mpmc_recon_{weno5js,teno5,teno6}.cu
FaceFn face_fp64_weno5js(int dim, int ns);
FaceFn face_fp64_teno5(int dim, int ns);
FaceFn face_fp64_teno6(int dim, int ns);
// the same for mixed-precision contexts: mpmc_mixed_recon_{weno5js,teno5,teno6}.cu
FaceFn face_mixed_weno5js(int dim, int ns);
FaceFn face_mixed_teno5(int dim, int ns);
FaceFn face_mixed_teno6(int dim, int ns);

using AdjFaceFn = decltype(AdjOps::face);
// adjoint face passes with Sec. 4.1's other interpolations:
// mpmc_adjoint_recon_{weno5js,teno5,teno6}.cu
AdjFaceFn adj_face_weno5js(int dim, int ns);
AdjFaceFn adj_face_teno5(int dim, int ns);
AdjFaceFn adj_face_teno6(int dim, int ns);

// per-dimension tables, defined in mpmc_kernels_d{1,2,3}.cu (FP64) and
// mpmc_mixed_d{1,2,3}.cu (mixed precision; init is the FP64 one)
Ops ops_fp64_d1(int ns);
Ops ops_fp64_d2(int ns);
Ops ops_fp64_d3(int ns);
Ops ops_mixed_d1(int ns);
Ops ops_mixed_d2(int ns);
Ops ops_mixed_d3(int ns);
// defined in mpmc_adjoint_d{1,2,3}.cu
AdjOps adj_ops_d1(int ns);
AdjOps adj_ops_d2(int ns);
AdjOps adj_ops_d3(int ns);

}  // namespace mpmc
