// Divergence of the face fluxes (Eq. DiscreteGoverningEquations) and the
// SSP-RK combination (Eq. SSPRK3) of one cell, from FP64 face fluxes
// F_d[v][face]; shared by the FP64 and mixed-precision update kernels (the
// mixed face kernel stores its FP32 fluxes widened to FP64, exactly, so that
// every flux enters its two cells with the same FP64 value and the sum over
// cells telescopes to FP64 rounding).
#pragma once
#include "mpmc_device.cuh"

namespace mpmc {

template <int NS, int D>
__device__ __forceinline__ void update_cell(const KParams& P, const long long c, const double* __restrict__ Un,
                                            const double* __restrict__ Uk, const double* __restrict__ F0,
                                            const double* __restrict__ F1, const double* __restrict__ F2,
                                            const double* __restrict__ scal, const double rk0, const double rk1,
                                            const double rk2, double* __restrict__ Uout, double* __restrict__ dUdt,
                                            int* __restrict__ status) {
  constexpr int NV = NS + D + 1;
  const int n0 = P.n[0], n1 = P.n[1];
  int ijk[3];
  unflatten(c, n0, n1, ijk);
  const int i = ijk[0], j = ijk[1], k = ijk[2];
  const double* Fd[3] = {F0, F1, F2};
  long long fm[3], fp[3], nf[3];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int f0 = n0 + (d == 0), f1 = n1 + (d == 1), f2 = P.n[2] + (d == 2);
    nf[d] = (long long)f0 * f1 * f2;
    fm[d] = ((long long)k * f1 + j) * f0 + i;
    fp[d] = fm[d] + (d == 0 ? 1 : (d == 1 ? f0 : (long long)f0 * f1));
  }
  const double dt = scal[0];
  // U = rk0 U^n + rk1 U^(k) + rk2 dt L, L = sum_d (F_{-1/2} - F_{+1/2}) / dx:
  // the flux differences are summed first and scaled once (the FP64 pipe
  // binds this kernel on GB300); a zero coefficient skips its state's load
  const double sdx = (rk2 * dt) * P.inv_dx;
  // the coefficient tests, once per thread as integers (FP64 comparisons
  // issue on the FP64 pipe, and would otherwise be repeated per variable)
  const int keep = dt == 0.0, use_k = rk1 != 0.0, use_n = rk0 != 0.0;
  double Uo[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double fs = Fd[0][(long long)v * nf[0] + fm[0]] - Fd[0][(long long)v * nf[0] + fp[0]];
#pragma unroll
    for (int d = 1; d < D; ++d) fs += Fd[d][(long long)v * nf[d] + fm[d]] - Fd[d][(long long)v * nf[d] + fp[d]];
    if (dUdt) dUdt[(long long)v * P.ncell + c] = fs * P.inv_dx;
    // a zero-length step (a run past its end time) leaves the state as it is
    if (keep) {
      Uo[v] = Uk[(long long)v * P.ncell + c];
    } else {
      double t = sdx * fs;
      if (use_k) t = fma(rk1, Uk[(long long)v * P.ncell + c], t);
      if (use_n) t = fma(rk0, Un[(long long)v * P.ncell + c], t);
      Uo[v] = t;
    }
  }
  if (Uout) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Uout[(long long)v * P.ncell + c] = Uo[v];
    if (!admissible<NS, D>(P, Uo)) atomicMax(status, (int)ST_INADMISSIBLE);
  }
}

}  // namespace mpmc
