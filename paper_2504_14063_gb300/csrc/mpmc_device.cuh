// Device building blocks of the MPMC right-hand side (arXiv 2504.14063):
// kernel parameters, boundary index mapping, NASG mixture EOS, WENO5-Z,
// HLLC, admissibility.  Everything here is FP64; the mixed-precision path
// adds its own FP32 pieces in mpmc_mixed.cuh.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mpmc_narrow.h"

namespace mpmc {

constexpr int MAXS = 4;
// round-off allowance on partial densities in every admissibility test
constexpr double YTOL = 1e-14;
// threshold below which a phase (or species) counts as absent
constexpr double ABSENT = 1e-300;
// |grad psi| below which the interface normal of the regularization is zero
constexpr double GTOL = 1e-8;
// per species: |sum Y - 1| up to which the Y limiter does not renormalize
constexpr double YSUM_TOL = 1e-15;

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_ZEROGRAD = 2, BC_INFLOW = 3, BC_CHAR = 4 };
enum { ST_OK = 0, ST_INADMISSIBLE = 3, ST_EOS_NO_CONVERGE = 4 };
enum : uint32_t {
  F_THETA_T_L = 1u << 0, F_THETA_T_R = 1u << 1, F_THETA_P_L = 1u << 2, F_THETA_P_R = 1u << 3,
  F_HLLC_FALLBACK = 1u << 4, F_CDI_DROPPED = 1u << 5, F_YLIM_L = 1u << 6, F_YLIM_R = 1u << 7,
  F_DIFF_DROPPED = 1u << 8
};

// Everything a kernel needs, passed by value (lives in the constant bank).
struct KParams {
  int dim, ns, nv;
  int n[3];
  long long ncell;
  double dx, inv_dx;
  int bc_lo[3], bc_hi[3];
  int phase[MAXS];
  double cv[MAXS], gam[MAXS], q[MAXS], b[MAXS], pinf[MAXS], W[MAXS], mu[MAXS], Sc[MAXS];
  double Rk[MAXS], cp[MAXS];
  double wilke[MAXS][MAXS];  // (W_i / W_j) Phi_ij of Wilke's rule (gas species)
  double weno_eps;
  int cdi, diffusion, pos_limiter, two_phase, has_inflow;
  int recon;  // MPMC_RECON_* (the face kernels take it as a template parameter)
  int viscous;  // viscous stress and heat conduction
  double prandtl, lambda_liquid;
  int has_b, has_q;  // some species has a nonzero NASG covolume b / reference energy q
  double cdi_eps, cdi_gamma, phi_min, psi_delta, cfl, mu_liquid, sharp0;
  // primitive cache: field f of cell c at Wc[f * wstride + c]; slot ncell
  // holds the inflow state, slots ncell + 1 .. ncell + nslots the ghost
  // states of the characteristic boundaries (one per boundary cell: the low
  // x side first, then the high one, each ordered like the cells of an
  // x-plane)
  int wT, wP, wRho, wA, wY, wU, wPhi0, wPsi, wYrho, wHrho, wXr, wB, wMu, wLam, nW;
  long long wstride;
  // conserved states of those slots: ghost buffers [nv][gstride], column 0
  // the inflow (far-field) state, column 1 + s slot s.  Kernels get the
  // buffer of U^(k) as an argument; gn is the one of U^n.
  int nslots, char_lo, char_hi;  // char_*: the x side is characteristic
  long long gstride, nextra;     // nextra: cache slots beyond ncell (0, or 1 + nslots)
  const double* gn;
  // mixed precision only: FP32 copy of U^n ([nv][wstride]) written by the
  // primitive pass that computes the step's dt and Gamma; FP32 copies of
  // U^(k) live in the FP32 cache at fields nW .. nW + nv - 1
  float* unf;
  // FP32 roundings of the constants above, made once on the host: the
  // mixed-precision kernels read these instead of converting per thread (a
  // double -> float conversion issues on the FP64 pipe)
  struct Consts32 {
    float cv[MAXS], gam[MAXS], q[MAXS], b[MAXS], pinf[MAXS], Rk[MAXS], cp[MAXS];
    float W[MAXS], mu[MAXS], Sc[MAXS], wilke[MAXS][MAXS];
    float inv_dx, cdi_eps, sharp0, mu_liquid, prandtl, lambda_liquid;
  } f32;
};

// fills P.f32 from the FP64 fields (host)
inline void round_consts32(KParams& P) {
  for (int k = 0; k < MAXS; ++k) {
    P.f32.cv[k] = (float)P.cv[k];
    P.f32.gam[k] = (float)P.gam[k];
    P.f32.q[k] = (float)P.q[k];
    P.f32.b[k] = (float)P.b[k];
    P.f32.pinf[k] = (float)P.pinf[k];
    P.f32.Rk[k] = (float)P.Rk[k];
    P.f32.cp[k] = (float)P.cp[k];
    P.f32.W[k] = (float)P.W[k];
    P.f32.mu[k] = (float)P.mu[k];
    P.f32.Sc[k] = (float)P.Sc[k];
    for (int j = 0; j < MAXS; ++j) P.f32.wilke[k][j] = (float)P.wilke[k][j];
  }
  P.f32.inv_dx = (float)P.inv_dx;
  P.f32.cdi_eps = (float)P.cdi_eps;
  P.f32.sharp0 = (float)P.sharp0;
  P.f32.mu_liquid = (float)P.mu_liquid;
  P.f32.prandtl = (float)P.prandtl;
  P.f32.lambda_liquid = (float)P.lambda_liquid;
}

// (x, y, z) of the linear index l of an n0 x n1 x n2 box, in 32-bit unsigned
// arithmetic, cheaper than 64-bit division (mpmc_create admits no grid with
// 2^31 - 1 cells or faces)
__device__ __forceinline__ void unflatten(long long l, int n0, int n1, int* x) {
  const unsigned u = (unsigned)l, a = (unsigned)n0, b = (unsigned)n1;
  const unsigned r = u / a;
  const unsigned z = r / b;
  x[0] = (int)(u - r * a);
  x[1] = (int)(r - z * b);
  x[2] = (int)z;
}

// ---------------------------------------------------------------------------
// boundary ghosts by index mapping.  Directions are resolved in order x, y,
// z: periodic and zero-gradient remap the coordinate, a wall mirrors it and
// negates that velocity component, an inflow face replaces the cell by the
// inflow state (later walls still mirror it).
struct CRef {
  int idx;         // cell index, or ncell for the inflow state (the host keeps
                   // every cell, slot and face index below 2^31 - 1)
  unsigned flip;   // bit d: negate u_d / m_d
};

// MASK bit d: coordinate d may lie outside the grid (the others are known to
// be inside, so their tests and the slot arithmetic they would need are
// compiled out at the call sites that know it)
// CHR = false: the caller's context has no characteristic boundary (the
// adjoint refuses them), so their slot arithmetic is compiled out as well
template <unsigned MASK, bool CHR = true>
__device__ __forceinline__ CRef map_cell_m(const KParams& P, int i, int j, int k) {
  int c[3] = {i, j, k};
  unsigned flip = 0u;
  bool inflow = false;
  int chr = 0;  // a characteristic x boundary: 1 low side, 2 high side
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (((MASK >> d) & 1u) && d < P.dim) {
      const int n = P.n[d];
      if (c[d] < 0 || c[d] >= n) {
        const bool lo = c[d] < 0;
        const int bc = lo ? P.bc_lo[d] : P.bc_hi[d];
        const int l = lo ? -1 - c[d] : c[d] - n;
        if (bc == BC_PERIODIC) {
          c[d] = lo ? c[d] + n : c[d] - n;
        } else if (bc == BC_WALL) {
          c[d] = lo ? l : n - 1 - l;
          flip ^= 1u << d;
        } else if (bc == BC_ZEROGRAD) {
          c[d] = lo ? 0 : n - 1;
        } else if (CHR && d == 0 && bc == BC_CHAR) {
          // the ghost slot of the boundary cell of this row (x only): the
          // other directions still map the row's coordinates (and walls
          // mirror the ghost's velocity)
          chr = lo ? 1 : 2;
          c[d] = 0;
        } else {
          inflow = true;
          flip = 0u;
        }
      }
    }
  }
  CRef r;
  r.flip = flip;
  // a row's cells, or its characteristic slot after the inflow slot
  const int nc = (int)P.ncell;
  const int row = c[2] * P.n[1] + c[1];
  const int slot = nc + 1 + (chr == 2 && P.char_lo ? P.n[1] * P.n[2] : 0) + row;
  r.idx = inflow ? nc : ((CHR && (MASK & 1u) && chr) ? slot : row * P.n[0] + c[0]);
  return r;
}

__device__ __forceinline__ CRef map_cell(const KParams& P, int i, int j, int k) {
  return map_cell_m<7u>(P, i, j, k);
}

// a neighbour whose coordinates DIR and t (a tangential direction) may lie
// outside the grid
template <int DIR, bool CHR = true>
__device__ __forceinline__ CRef map_cell_dt(const KParams& P, int t, int i, int j, int k) {
  if (t == 0) return map_cell_m<(1u << DIR) | 1u, CHR>(P, i, j, k);
  if (t == 1) return map_cell_m<(1u << DIR) | 2u, CHR>(P, i, j, k);
  return map_cell_m<(1u << DIR) | 4u, CHR>(P, i, j, k);
}

__device__ __forceinline__ double sgn_flip(unsigned flip, int d) { return (flip >> d) & 1u ? -1.0 : 1.0; }

// conserved vector of a mapped cell (U has ncell entries per component; the
// inflow state and the characteristic ghosts come from U's ghost buffer G)
template <int NS, int D>
__device__ __forceinline__ void load_U(const KParams& P, const double* __restrict__ U,
                                       const double* __restrict__ G, CRef r, double* out) {
  constexpr int NV = NS + D + 1;
  if (r.idx >= P.ncell) {
    const long long col = r.idx - P.ncell;
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = G[(long long)v * P.gstride + col];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = U[(long long)v * P.ncell + r.idx];
  }
#pragma unroll
  for (int d = 0; d < D; ++d) out[NS + d] *= sgn_flip(r.flip, d);
}

__device__ __forceinline__ double wget(const KParams& P, const double* __restrict__ Wc, int f, CRef r) {
  return Wc[(long long)f * P.wstride + r.idx];
}

// ---------------------------------------------------------------------------
// NASG EOS per species (Eq. NASG_EOS)
__device__ __forceinline__ double v_k(const KParams& P, int k, double p, double T) {
  return P.Rk[k] * T / (p + P.pinf[k]) + P.b[k];
}
__device__ __forceinline__ double e_k(const KParams& P, int k, double p, double T) {
  return P.cv[k] * T * (p + P.gam[k] * P.pinf[k]) / (p + P.pinf[k]) + P.q[k];
}
__device__ __forceinline__ double h_k(const KParams& P, int k, double p, double T) {
  return P.cp[k] * T + P.b[k] * p + P.q[k];
}

// common-pressure residual of NASG_T1 = NASG_T2 and its first two
// derivatives, f(x) = sum_k w_k / (x + Pinf_k) - Cv with w_k = Y_k R_k
// (E' - Pinf_k) precomputed for the species present (mag: the sum of the
// magnitudes of its terms, the scale of its rounding).  The ideal-gas
// species share one reciprocal 1/x.
template <int NS>
__device__ __forceinline__ void pt_residual(const KParams& P, const double* Y, const double* w, double Cv, double x,
                                            double& f, double& df, double& d2f, double& mag) {
  f = -Cv;
  df = 0.0;
  d2f = 0.0;
  mag = Cv;
  double rg = 0.0;
  bool have_rg = false;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (nonzero(Y[k])) {
      double r;
      if (!nonzero(P.pinf[k])) {
        if (!have_rg) {
          rg = 1.0 / x;
          have_rg = true;
        }
        r = rg;
      } else {
        r = 1.0 / (x + P.pinf[k]);
      }
      const double t = w[k] * r;
      f += t;
      df -= t * r;
      d2f += 2.0 * t * r * r;
      mag += fabs(t);
    }
  }
}

// Non-contracting arithmetic for the inversion U -> (P, T).  The pressure of
// a stiff liquid (P << Pinf) is the small difference of terms ~ gamma Pinf,
// so it inherits the rounding of every operation before it; evaluating in
// a fixed order without fused multiply-adds makes it reproducible.
// EX = false: ordinary (contractible) arithmetic, for the uses that need no
// bit-for-bit reproduction (face-average scalars, the mixed path)
template <bool EX = true>
__device__ __forceinline__ double mul_(double a, double b) { return EX ? __dmul_rn(a, b) : a * b; }
template <bool EX = true>
__device__ __forceinline__ double add_(double a, double b) { return EX ? __dadd_rn(a, b) : a + b; }
template <bool EX = true>
__device__ __forceinline__ double sub_(double a, double b) { return EX ? __dsub_rn(a, b) : a - b; }

// mixture decode of a conserved vector: rho, Y, |u|^2, specific e, v
template <int NS, int D, bool EX = true>
__device__ __forceinline__ void decode(const double* U, double& rho, double* Y, double* u, double& e, double& v) {
  rho = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) rho = add_<EX>(rho, U[k]);
  if (EX) {
#pragma unroll
    for (int k = 0; k < NS; ++k) Y[k] = U[k] / rho;
    double ke = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      u[d] = d < D ? U[NS + d] / rho : 0.0;
      ke = add_(ke, mul_(u[d], u[d]));
    }
    e = sub_(U[NS + D] / rho, mul_(0.5, ke));
    v = 1.0 / rho;
  } else {
    const double ir = 1.0 / rho;
#pragma unroll
    for (int k = 0; k < NS; ++k) Y[k] = U[k] * ir;
    double ke = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      u[d] = d < D ? U[NS + d] * ir : 0.0;
      ke += u[d] * u[d];
    }
    e = U[NS + D] * ir - 0.5 * ke;
    v = ir;
  }
}

// the same residual solved in FP32 (its coefficients rounded once, on the
// integer pipes, the constants from KParams.f32) by safeguarded Halley steps
// from x0: a start for the FP64 iteration that costs little on the FP32 pipe.
// Its root is within FP32 rounding of the residual's terms (for a stiff
// liquid, P to ~eps32 Pinf), from which one or two FP64 steps reach the
// FP64 root.
template <int NS>
__device__ __forceinline__ double pt_start_f32(const KParams& P, const double* Y, const double* w, double Cv,
                                               double lo, double x0) {
  float wf[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) wf[k] = nonzero(Y[k]) ? narrow(w[k]) : 0.f;
  const float cvf = narrow(Cv), lof = narrow(lo);
  float x = narrow(x0), a = lof, b = INFINITY;
  for (int it = 0; it < 40; ++it) {
    float f = -cvf, df = 0.f, d2f = 0.f, mag = cvf, rg = 0.f;
    bool have_rg = false;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (nonzero(Y[k])) {
        float r;
        if (P.f32.pinf[k] == 0.f) {
          if (!have_rg) {
            rg = __frcp_rn(x);
            have_rg = true;
          }
          r = rg;
        } else {
          r = __frcp_rn(x + P.f32.pinf[k]);
        }
        const float t = wf[k] * r;
        f += t;
        df -= t * r;
        d2f += 2.f * t * r * r;
        mag += fabsf(t);
      }
    }
    if (f > 0.f) a = x;
    else b = x;
    if (fabsf(f) <= 16.f * 1.1920929e-7f * mag) break;
    const float hd = 2.f * df * df - f * d2f;
    float xn = hd > 0.f ? x - 2.f * f * df / hd : x - f / df;
    if (!(xn > a && xn < b)) xn = b == INFINITY ? x + fmaxf(x - lof, 1.f) : 0.5f * (a + b);
    const bool done = fabsf(xn - x) <= 2.4e-7f * fabsf(xn);
    x = xn;
    if (done || !(b > a)) break;
  }
  return (double)x;
}

// p-T equilibrium from mass fractions, specific internal energy and volume
// (Eqs. NASG_T1, NASG_T2, NASG_P).  One stiffened component (or several
// sharing Pinf): the quadratic of NASG_P, larger root in cancellation-free
// form, linear root without gas.  Several distinct Pinf: safeguarded Halley
// steps on the common-pressure residual from the caller's guess or, without
// one, from an FP32 solve started at the quadratic with a Y-weighted Pinf,
// at most 100 iterations.
// F32OUT: the caller keeps P and T only in FP32 (the mixed path's cache).
// The FP64 iteration then stops after a Halley step smaller than 1e-6 of the
// distance to the nearest pole of the residual (x - lo): the terms are
// analytic within that distance, so the step leaves an error of order
// 1e-18 (x - lo), far below FP32 rounding of P.  T follows in FP32 (its
// ratios (P + gamma Pinf) / (P + Pinf) are well conditioned).  The
// contracted FP64 solve (EX = false) stops the same way at 1e-7.
template <int NS, bool EX = true, bool F32OUT = false>
__device__ int pt_equilibrium(const KParams& P, const double* Y, double e, double v, double& p, double& T,
                              double rho = 0.0, double guess = -1e300) {
  double Cv = 0.0, q = 0.0, b = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    Cv = add_<EX>(Cv, mul_<EX>(Y[k], P.cv[k]));
    q = add_<EX>(q, mul_<EX>(Y[k], P.q[k]));
    b = add_<EX>(b, mul_<EX>(Y[k], P.b[k]));
  }
  const double em = sub_<EX>(e, q), vm = sub_<EX>(v, b);
  int st = ST_OK;
  if (!positive(em) || !positive(vm)) st = ST_INADMISSIBLE;
  // (the contracted form takes E' = (e - q) rho, one division fewer, when no
  // species has a covolume and the caller passes rho = 1/v)
  const double Ep = (!EX && !P.has_b && positive(rho)) ? em * rho : em / vm;
  double pl = -1.0, pmin = 1e300, Rg = 0.0, Rl = 0.0, wpl = 0.0;
  bool multi = false, gas = false;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (positive(Y[k])) {
      pmin = fmin(pmin, P.pinf[k]);
      if (positive(P.pinf[k])) {
        if (pl < 0.0) pl = P.pinf[k];
        else if (P.pinf[k] != pl) multi = true;
        Rl = add_<EX>(Rl, mul_<EX>(Y[k], P.Rk[k]));
        wpl += Y[k] * P.Rk[k] * P.pinf[k];
      } else {
        gas = true;
        Rg = add_<EX>(Rg, mul_<EX>(Y[k], P.Rk[k]));
      }
    }
  }
  if (!multi) {
    if (pl < 0.0) {
      p = mul_<EX>(Ep, Rg) / Cv;
    } else if (!gas) {
      p = sub_<EX>(sub_<EX>(mul_<EX>(Ep, Rl), mul_<EX>(pl, Cv)), mul_<EX>(pl, Rl)) / Cv;
    } else {
      const double a1 = Cv;
      const double a2 = sub_<EX>(sub_<EX>(mul_<EX>(Ep, add_<EX>(Rg, Rl)), mul_<EX>(pl, Cv)), mul_<EX>(pl, Rl));
      const double a3 = mul_<EX>(mul_<EX>(Ep, pl), Rg);
      const double sq = sqrt(add_<EX>(mul_<EX>(a2, a2), mul_<EX>(mul_<EX>(4.0, a1), a3)));
      p = a2 >= 0.0 ? add_<EX>(a2, sq) / mul_<EX>(2.0, a1) : mul_<EX>(2.0, a3) / sub_<EX>(sq, a2);
    }
  } else {
    // Halley steps on the residual from the caller's guess (a nearby
    // pressure) or the quadratic with the liquids merged into one, kept
    // inside the bracket (a, bb) of the root on (lo, inf); the upper end is
    // found only if a step leaves the bracket while it is still open
    const double lo = -pmin;
    double w[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) w[k] = nonzero(Y[k]) ? Y[k] * P.Rk[k] * (Ep - P.pinf[k]) : 0.0;
    double a = lo, bb = INFINITY;
    double x;
    if (guess > lo && guess < 1e300) {
      x = guess;
    } else {
      const double pe = wpl / Rl;
      const double a2 = Ep * (Rg + Rl) - pe * Cv - pe * Rl, a3 = Ep * pe * Rg;
      x = gas ? (a2 >= 0.0 ? (a2 + sqrt(a2 * a2 + 4.0 * Cv * a3)) / (2.0 * Cv)
                           : 2.0 * a3 / (sqrt(a2 * a2 + 4.0 * Cv * a3) - a2))
              : (Ep * Rl - pe * Cv - pe * Rl) / Cv;
      if (!(x > a)) x = lo + fmax(fabs(lo), 1.0);
      const double xs = pt_start_f32<NS>(P, Y, w, Cv, lo, x);
      if (xs > a && xs < 1e300) x = xs;
    }
    double f, df, d2f, mag;
    bool conv = false;
    if (F32OUT) {
      // FP32 output: one Newton step from the FP32 root suffices (its error,
      // dxn^2 / (x - lo) <= 1e-12 (x - lo), is below FP32 rounding of P);
      // the reciprocals 1/(x + Pinf_k) from an FP32 seed and one Newton
      // refinement (relative error ~1e-14).  A larger step, or a seed that
      // is not a normal number, falls through to the iteration below.
      double fn = -Cv, dfn = 0.0;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        if (nonzero(Y[k])) {
          const double y = x + P.pinf[k];
          double r = (double)__frcp_rn((float)y);
          r = r * (2.0 - y * r);
          const double t = w[k] * r;
          fn += t;
          dfn -= t * r;
        }
      }
      const double xn = x - fn / dfn;
      if (xn > lo && fabs(xn - x) <= 1e-6 * (x - lo)) {
        x = xn;
        conv = true;
      }
    }
    for (int it = 0; it < 100 && !conv; ++it) {
      pt_residual<NS>(P, Y, w, Cv, x, f, df, d2f, mag);
      if (positive(f)) a = x;
      else bb = x;
      // the residual is a difference of terms of size mag: once it is at its
      // own rounding level, x is the root as far as the data determine it
      // (a stiff liquid with trace gas: the iterate would wander in that band)
      if (fabs(f) <= 16.0 * 2.220446049250313e-16 * mag) { conv = true; break; }
      const double hd = 2.0 * df * df - f * d2f;
      double xn = positive(hd) ? x - 2.0 * f * df / hd : x - f / df;
      if (!(xn > a && xn < bb)) {
        if (bb == INFINITY) {
          xn = x + fmax(x - lo, 1.0);       // root above every point tried so far
        } else {
          const double da = a - lo, db = bb - lo;
          xn = (da > 0.0 && db > 16.0 * da) ? lo + sqrt(da * db) : 0.5 * (a + bb);
        }
      }
      const double dxn = fabs(xn - x);
      x = xn;
      // the contracted solve (face averages, the mixed cell inversion) takes
      // a Halley step below 1e-7 (FP32 output: 1e-6) of the distance to the
      // nearest pole as final: the error it leaves is of order dxn^3 /
      // (x - lo)^2, 1e-21 (FP32 output: 1e-18) of x - lo
      if (!EX && dxn <= (F32OUT ? 1e-6 : 1e-7) * (x - lo)) { conv = true; break; }
      if (dxn <= 4.5e-16 * fabs(x) || !(bb > a)) {
        pt_residual<NS>(P, Y, w, Cv, x, f, df, d2f, mag);
        x = x - f / df;   // one more Newton step at full accuracy
        conv = true;
        break;
      }
    }
    if (!conv && st == ST_OK) st = ST_EOS_NO_CONVERGE;
    p = x;
    if (F32OUT) {
      const float pf = narrow(p);
      float den = 0.f;
#pragma unroll
      for (int k = 0; k < NS; ++k)
        if (nonzero(Y[k])) {
          const float r = P.f32.pinf[k] == 0.f
                              ? 1.f
                              : __fdividef(pf + P.f32.gam[k] * P.f32.pinf[k], pf + P.f32.pinf[k]);
          den += narrow(Y[k]) * P.f32.cv[k] * r;
        }
      T = (double)__fdividef(narrow(em), den);
      return st;
    }
  }
  if (!EX && !multi && positive(pl)) {
    // every stiffened species present shares P + pl: T = em (P + pl) /
    // (sum_gas Y cv (P + pl) + sum_liquid Y cv (P + gamma pl)), one division
    // (a species with another Pinf can only be a trace below zero, which
    // did not set pl: it keeps its own ratio)
    const double pp = p + pl;
    double g = 0.0, l = 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k)
      if (nonzero(Y[k])) {
        if (!nonzero(P.pinf[k]))
          g += Y[k] * P.cv[k];
        else if (P.pinf[k] == pl)
          l += Y[k] * P.cv[k] * (p + P.gam[k] * pl);
        else
          g += Y[k] * P.cv[k] * (p + P.gam[k] * P.pinf[k]) / (p + P.pinf[k]);
      }
    T = em * pp / (g * pp + l);
    return st;
  }
  double den = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k)
    if (nonzero(Y[k])) {
      if (!EX && !nonzero(P.pinf[k]))
        den += Y[k] * P.cv[k];   // (P + gamma Pinf) / (P + Pinf) = 1
      else
        den = add_<EX>(den, mul_<EX>(mul_<EX>(Y[k], P.cv[k]), add_<EX>(p, mul_<EX>(P.gam[k], P.pinf[k]))) /
                                add_<EX>(p, P.pinf[k]));
    }
  T = em / den;
  return st;
}

// forward EOS at (P, T, Y): density (Amagat), specific internal energy and
// the sound speed of Eq. SpeedOfSound with the NASG alpha, beta
template <int NS>
__device__ __forceinline__ void eos_forward(const KParams& P, const double* Y, double p, double T, double& rho,
                                            double& e, double& a, double& alpha, double& beta) {
  double v = 0.0, cp = 0.0, sa = 0.0, sb = 0.0, rg = 0.0;
  bool have_rg = false;
  e = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (nonzero(Y[k])) {
      // ideal-gas species share 1/(P + 0) = 1/P (the same value bit for bit)
      double r;
      if (!nonzero(P.pinf[k])) {
        if (!have_rg) {
          rg = 1.0 / p;
          have_rg = true;
        }
        r = rg;
      } else {
        r = 1.0 / (p + P.pinf[k]);
      }
      const double RT = P.Rk[k] * T;
      v += Y[k] * (RT * r + P.b[k]);
      e += Y[k] * (P.cv[k] * T * (p + P.gam[k] * P.pinf[k]) * r + P.q[k]);
      cp += Y[k] * P.cp[k];
      sa += Y[k] * P.Rk[k] * r;
      sb += Y[k] * RT * r * r;
    }
  }
  rho = 1.0 / v;
  alpha = rho * sa;
  beta = rho * sb;
  // sqrt(cp / den) as cp rsqrt(cp den): one reciprocal square root in place
  // of a division and a square root (cp > 0; den <= 0 gives NaN or inf alike)
  a = cp * rsqrt(cp * (rho * beta * cp - alpha * alpha * T));
}

// the sound speed, alpha and beta of eos_forward at a state whose density
// rho is already known (the face average: its (P, T) come from inverting
// that density, so v(P, T, Y) = 1/rho up to rounding)
template <int NS>
__device__ __forceinline__ void eos_char(const KParams& P, const double* Y, double p, double T, double rho,
                                         double& a, double& alpha, double& beta) {
  double cp = 0.0, sa = 0.0, sb = 0.0, rg = 0.0;
  bool have_rg = false;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (nonzero(Y[k])) {
      double r;
      if (!nonzero(P.pinf[k])) {
        if (!have_rg) {
          rg = 1.0 / p;
          have_rg = true;
        }
        r = rg;
      } else {
        r = 1.0 / (p + P.pinf[k]);
      }
      cp += Y[k] * P.cp[k];
      sa += Y[k] * P.Rk[k] * r;
      sb += Y[k] * P.Rk[k] * T * r * r;
    }
  }
  alpha = rho * sa;
  beta = rho * sb;
  // sqrt(cp / den) as cp rsqrt(cp den): one reciprocal square root in place
  // of a division and a square root (cp > 0; den <= 0 gives NaN or inf alike)
  a = cp * rsqrt(cp * (rho * beta * cp - alpha * alpha * T));
}

// ---------------------------------------------------------------------------
// WENO5-Z (Borges et al. 2008), exponent 1: value at the right face of v2.
// Same weights, fewer FP64 instructions: the candidates are carried as
// 6 q_0, 36 q_1, 18 q_2 (the 1/6 of the stencils and the ideal weights
// d = (1, 6, 3)/10 folded into their coefficients), and alpha_k = d_k (1 +
// tau/(b_k+eps)) over the common denominator prod_j (b_j+eps) reads
// (c_k + tau) prod_{j!=k} c_j; the quotient is scaled back by the 6 in the
// denominator.
__device__ __forceinline__ void weno5z_nd(double v0, double v1, double v2, double v3, double v4, double eps,
                                          double& num, double& den) {
  const double q0 = 2.0 * v0 - 7.0 * v1 + 11.0 * v2;
  const double q1 = -6.0 * v1 + 30.0 * v2 + 12.0 * v3;
  const double q2 = 6.0 * v2 + 15.0 * v3 - 3.0 * v4;
  double t = v0 - 2.0 * v1 + v2, s = v0 - 4.0 * v1 + 3.0 * v2;
  const double b0 = (13.0 / 12.0) * t * t + 0.25 * s * s;
  t = v1 - 2.0 * v2 + v3;
  s = v1 - v3;
  const double b1 = (13.0 / 12.0) * t * t + 0.25 * s * s;
  t = v2 - 2.0 * v3 + v4;
  s = 3.0 * v2 - 4.0 * v3 + v4;
  const double b2 = (13.0 / 12.0) * t * t + 0.25 * s * s;
  const double tau = fabs(b0 - b2);
  const double c0 = b0 + eps, c1 = b1 + eps, c2 = b2 + eps;
  const double a0 = (c0 + tau) * (c1 * c2);
  const double a1 = (c1 + tau) * (c0 * c2);
  const double a2 = (c2 + tau) * (c0 * c1);
  num = a0 * q0 + a1 * q1 + a2 * q2;
  den = 6.0 * a0 + 36.0 * a1 + 18.0 * a2;
}

__device__ __forceinline__ double weno5z(double v0, double v1, double v2, double v3, double v4, double eps) {
  double num, den;
  weno5z_nd(v0, v1, v2, v3, v4, eps, num, den);
  return num / den;
}

// ---------------------------------------------------------------------------
// The other ENO-type interpolations that Sec. 4.1 runs beside WENO5-Z:
// WENO5-JS (Jiang & Shu 1996) and TENO5 / TENO6 (Fu, Hu & Adams 2016), as
// those works define them (the paper cites them).  Value at the right face of
// cell i from the cells i-2..i+3 (v5 is read by TENO6 alone).  Readings:
// WENO5-JS eps = 1e-6, exponent 2; TENO C = 1, q = 6, eps = 1e-40,
// CT = 1e-5 (TENO5) / 1e-7 (TENO6).
enum { RC_WENO5Z = 0, RC_WENO5JS = 1, RC_TENO5 = 2, RC_TENO6 = 3 };

// the three-cell candidates (left i-2..i, central i-1..i+1, right i..i+2)
// and their Jiang-Shu indicators
struct Eno3 {
  double ql, qc, qr, bl, bc, br;
};

__device__ __forceinline__ Eno3 eno3(double v0, double v1, double v2, double v3, double v4) {
  Eno3 e;
  e.ql = (2.0 * v0 - 7.0 * v1 + 11.0 * v2) * (1.0 / 6.0);
  e.qc = (-v1 + 5.0 * v2 + 2.0 * v3) * (1.0 / 6.0);
  e.qr = (2.0 * v2 + 5.0 * v3 - v4) * (1.0 / 6.0);
  double t = v0 - 2.0 * v1 + v2, s = v0 - 4.0 * v1 + 3.0 * v2;
  e.bl = (13.0 / 12.0) * t * t + 0.25 * s * s;
  t = v1 - 2.0 * v2 + v3;
  s = v1 - v3;
  e.bc = (13.0 / 12.0) * t * t + 0.25 * s * s;
  t = v2 - 2.0 * v3 + v4;
  s = 3.0 * v2 - 4.0 * v3 + v4;
  e.br = (13.0 / 12.0) * t * t + 0.25 * s * s;
  return e;
}

// eno3 of both sides of a face: L of w[0..4], R of w[5..1].  The sides share
// two candidates (the central one of each is the right one of the other)
// and the second differences w1 - 2 w2 + w3, w2 - 2 w3 + w4.
__device__ __forceinline__ void eno3_lr(const double* w, Eno3& L, Eno3& R) {
  const double qa = (-w[1] + 5.0 * w[2] + 2.0 * w[3]) * (1.0 / 6.0);
  const double qb = (2.0 * w[2] + 5.0 * w[3] - w[4]) * (1.0 / 6.0);
  const double t123 = w[1] - 2.0 * w[2] + w[3], t234 = w[2] - 2.0 * w[3] + w[4];
  const double e123 = (13.0 / 12.0) * t123 * t123, e234 = (13.0 / 12.0) * t234 * t234;
  L.ql = (2.0 * w[0] - 7.0 * w[1] + 11.0 * w[2]) * (1.0 / 6.0);
  L.qc = qa;
  L.qr = qb;
  double t = w[0] - 2.0 * w[1] + w[2], s = w[0] - 4.0 * w[1] + 3.0 * w[2];
  L.bl = (13.0 / 12.0) * t * t + 0.25 * s * s;
  s = w[1] - w[3];
  L.bc = e123 + 0.25 * s * s;
  s = 3.0 * w[2] - 4.0 * w[3] + w[4];
  L.br = e234 + 0.25 * s * s;
  R.ql = (2.0 * w[5] - 7.0 * w[4] + 11.0 * w[3]) * (1.0 / 6.0);
  R.qc = qb;
  R.qr = qa;
  t = w[5] - 2.0 * w[4] + w[3];
  s = w[5] - 4.0 * w[4] + 3.0 * w[3];
  R.bl = (13.0 / 12.0) * t * t + 0.25 * s * s;
  s = w[4] - w[2];
  R.bc = e234 + 0.25 * s * s;
  s = 3.0 * w[3] - 4.0 * w[2] + w[1];
  R.br = e123 + 0.25 * s * s;
}

__device__ __forceinline__ double weno5js_e(const Eno3& e) {
  constexpr double eps = 1e-6;
  const double il = 1.0 / (eps + e.bl), ic = 1.0 / (eps + e.bc), ir = 1.0 / (eps + e.br);
  const double al = 0.1 * il * il, ac = 0.6 * ic * ic, ar = 0.3 * ir * ir;
  return (al * e.ql + ac * e.qc + ar * e.qr) / (al + ac + ar);
}

__device__ __forceinline__ double weno5js(double v0, double v1, double v2, double v3, double v4) {
  return weno5js_e(eno3(v0, v1, v2, v3, v4));
}

// TENO selection: r_k = C + tau / (beta_k + eps); chi_k = r_k^q / sum r^q,
// formed from r_k / max r (r_k^6 overflows beside a large jump); candidates
// with chi_k < CT are cut off (bit k of the result clear)
template <int K>
__device__ __forceinline__ unsigned teno_kept(const double* b, double tau, double CT) {
  // 1 / (beta_k + eps) from one reciprocal of their product (each factor lies
  // in [1e-40, ~1e20], the product of four within range), then r_k
  double cfac[K], pre[K], suf[K];
#pragma unroll
  for (int k = 0; k < K; ++k) cfac[k] = b[k] + 1e-40;
  pre[0] = 1.0;
#pragma unroll
  for (int k = 1; k < K; ++k) pre[k] = pre[k - 1] * cfac[k - 1];
  suf[K - 1] = 1.0;
#pragma unroll
  for (int k = K - 2; k >= 0; --k) suf[k] = suf[k + 1] * cfac[k + 1];
  const double iprod = 1.0 / (pre[K - 1] * cfac[K - 1]);
  double r[K], rmax = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    r[k] = 1.0 + tau * (iprod * pre[k] * suf[k]);
    rmax = fmax(rmax, r[k]);
  }
  // scale by the power of two 2^-floor(log2 rmax) (exact; r_k^6 would
  // overflow beside a large jump): chi_k is unchanged by a common factor
  const int ex = min((__double2hiint(rmax) >> 20) & 0x7ff, 2045);  // rmax >= 1, finite
  const double scale = __hiloint2double((2046 - ex) << 20, 0);
  double g[K], gs = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double x = r[k] * scale, x2 = x * x;
    g[k] = x2 * x2 * x2;
    gs += g[k];
  }
  unsigned kept = 0u;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (!(g[k] < CT * gs)) kept |= 1u << k;
  return kept;
}

// the kept candidates with their optimal weights renormalized
template <int K>
__device__ __forceinline__ double teno_combine(const double* q, const double* dk, unsigned kept) {
  double num = 0.0, den = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (kept & (1u << k)) {
      num += dk[k] * q[k];
      den += dk[k];
    }
  return num / den;
}

// TENO5: optimal weights (3/5, 1/10, 3/10) for (central, left, right),
// tau5 = |beta_left - beta_right|
__device__ constexpr double TENO5_D[3] = {0.6, 0.1, 0.3};
__device__ constexpr double TENO6_D[4] = {0.45, 0.05, 0.3, 0.2};

__device__ __forceinline__ unsigned teno5_kept(const Eno3& e) {
  const double b[3] = {e.bc, e.bl, e.br};
  return teno_kept<3>(b, fabs(e.bl - e.br), 1e-5);
}

__device__ __forceinline__ double teno5_e(const Eno3& e) {
  const double q[3] = {e.qc, e.ql, e.qr};
  return teno_combine<3>(q, TENO5_D, teno5_kept(e));
}

__device__ __forceinline__ double teno5(double v0, double v1, double v2, double v3, double v4) {
  return teno5_e(eno3(v0, v1, v2, v3, v4));
}

// TENO6: adds the four-cell candidate i..i+3; optimal weights
// (9/20, 1/20, 3/10, 1/5) reproduce the six-cell interpolation;
// tau6 = |beta6 - (beta_left + beta_right + 4 beta_central) / 6|.  The four-
// and six-cell Jiang-Shu indicators are written as positive multiples of
// squared zero-sum combinations (exact rational coefficients), evaluated on
// deviations from cell i.
__device__ __forceinline__ unsigned teno6_kept(const Eno3& e, double v0, double v1, double v2, double v3, double v4,
                                               double v5) {
  const double e0 = v0 - v2, e1 = v1 - v2, e3 = v3 - v2, e4 = v4 - v2, e5 = v5 - v2;
  const double s = 18.0 * e3 - 9.0 * e4 + 2.0 * e5, t = -5.0 * e3 + 4.0 * e4 - e5, u = 3.0 * e3 - 3.0 * e4 + e5;
  const double b4 = (1.0 / 36.0) * s * s + (13.0 / 12.0) * t * t + (781.0 / 720.0) * u * u;
  const double c1 = 3.0 * e0 - 30.0 * e1 + 60.0 * e3 - 15.0 * e4 + 2.0 * e5;
  const double c2 = -11.0 * e0 + 174.0 * e1 + 174.0 * e3 - 11.0 * e4;
  const double c3 = -16315.0 * e0 - 16831.0 * e1 - 230474.0 * e3 + 115237.0 * e4 - 16487.0 * e5;
  const double c4 = e0 - 4.0 * e1 - 4.0 * e3 + e4;
  const double c5 = -e0 + 5.0 * e1 + 10.0 * e3 - 5.0 * e4 + e5;
  const double b6 = (1.0 / 3600.0) * c1 * c1 + (1.0 / 15600.0) * c2 * c2 + (1.0 / 3967729920.0) * c3 * c3 +
                    (1421461.0 / 1310400.0) * c4 * c4 + (21520059541.0 / 19838649600.0) * c5 * c5;
  const double b[4] = {e.bc, e.bl, e.br, b4};
  return teno_kept<4>(b, fabs(b6 - (e.bl + e.br + 4.0 * e.bc) * (1.0 / 6.0)), 1e-7);
}

__device__ __forceinline__ double teno6_e(const Eno3& e, double v0, double v1, double v2, double v3, double v4,
                                         double v5) {
  const double q[4] = {e.qc, e.ql, e.qr, (3.0 * v2 + 13.0 * v3 - 5.0 * v4 + v5) * (1.0 / 12.0)};
  return teno_combine<4>(q, TENO6_D, teno6_kept(e, v0, v1, v2, v3, v4, v5));
}

__device__ __forceinline__ double teno6(double v0, double v1, double v2, double v3, double v4, double v5) {
  return teno6_e(eno3(v0, v1, v2, v3, v4), v0, v1, v2, v3, v4, v5);
}

// the interpolation of kind RC on the stencil v0..v5 (left side: cells
// i-2..i+3; right side: the same cells mirrored)
template <int RC>
__device__ __forceinline__ double recon(double v0, double v1, double v2, double v3, double v4, double v5,
                                        double eps) {
  if constexpr (RC == RC_WENO5JS) return weno5js(v0, v1, v2, v3, v4);
  else if constexpr (RC == RC_TENO5) return teno5(v0, v1, v2, v3, v4);
  else if constexpr (RC == RC_TENO6) return teno6(v0, v1, v2, v3, v4, v5);
  else return weno5z(v0, v1, v2, v3, v4, eps);
}

// both face values of one field from the cells y[0..5] = i-2..i+3 around
// the face i+1/2: L from the left (recon of y[0..5]), R from the right (of
// y[5..0]).  WENO5-Z shares the two sides' common candidates and second
// differences (weno5z_lr_nd) and forms the two quotients with one reciprocal,
// num_L d_R / (d_L d_R) and num_R d_L / (d_L d_R), while d_L d_R is a
// normal number whose reciprocal is normal too (exponent field 2..2044,
// tested on the integer pipe), else with two divisions.
// WENO5-Z weights of one side over the common denominator: a_k = (c_k +
// tau) prod_{j!=k} c_j, c_k = b_k + eps (as weno5z_nd)
__device__ __forceinline__ void weno5z_alpha(double b0, double b1, double b2, double eps, double& a0, double& a1,
                                             double& a2) {
  const double tau = fabs(b0 - b2);
  const double c0 = b0 + eps, c1 = b1 + eps, c2 = b2 + eps;
  a0 = (c0 + tau) * (c1 * c2);
  a1 = (c1 + tau) * (c0 * c2);
  a2 = (c2 + tau) * (c0 * c1);
}

// numerators and denominators of both sides of a face (weno5z_nd of
// w[0..4] and of w[5..1]).  The two sides share two candidate stencils:
// 6 q_1 of the left side (cells w1..w3) is 6 q_2 of the right one, and
// 6 q_2 of the left (w2..w4) is 6 q_1 of the right; and two second
// differences (w1 - 2 w2 + w3, w2 - 2 w3 + w4) with their (13/12) t^2 terms.
__device__ __forceinline__ void weno5z_lr_nd(const double* w, double eps, double& nL, double& dL, double& nR,
                                             double& dR) {
  const double t123 = w[1] - 2.0 * w[2] + w[3], t234 = w[2] - 2.0 * w[3] + w[4];
  const double e123 = (13.0 / 12.0) * t123 * t123, e234 = (13.0 / 12.0) * t234 * t234;
  const double A = -w[1] + 5.0 * w[2] + 2.0 * w[3];
  const double B = 2.0 * w[2] + 5.0 * w[3] - w[4];
  {
    const double t = w[0] - 2.0 * w[1] + w[2], s = w[0] - 4.0 * w[1] + 3.0 * w[2];
    const double b0 = (13.0 / 12.0) * t * t + 0.25 * s * s;
    const double s1 = w[1] - w[3], s2 = 3.0 * w[2] - 4.0 * w[3] + w[4];
    const double b1 = e123 + 0.25 * s1 * s1, b2 = e234 + 0.25 * s2 * s2;
    double a0, a1, a2;
    weno5z_alpha(b0, b1, b2, eps, a0, a1, a2);
    const double Q0 = 2.0 * w[0] - 7.0 * w[1] + 11.0 * w[2];
    nL = a0 * Q0 + a1 * (6.0 * A) + a2 * (3.0 * B);
    dL = 6.0 * a0 + 36.0 * a1 + 18.0 * a2;
  }
  {
    const double t = w[5] - 2.0 * w[4] + w[3], s = w[5] - 4.0 * w[4] + 3.0 * w[3];
    const double b0 = (13.0 / 12.0) * t * t + 0.25 * s * s;
    const double s1 = w[4] - w[2], s2 = 3.0 * w[3] - 4.0 * w[2] + w[1];
    const double b1 = e234 + 0.25 * s1 * s1, b2 = e123 + 0.25 * s2 * s2;
    double a0, a1, a2;
    weno5z_alpha(b0, b1, b2, eps, a0, a1, a2);
    const double Q0 = 2.0 * w[5] - 7.0 * w[4] + 11.0 * w[3];
    nR = a0 * Q0 + a1 * (6.0 * B) + a2 * (3.0 * A);
    dR = 6.0 * a0 + 36.0 * a1 + 18.0 * a2;
  }
}

template <int RC>
__device__ __forceinline__ void recon_lr(const double* y, double eps, double& L, double& R) {
  if constexpr (RC == RC_WENO5Z) {
    double nL, dL, nR, dR;
    weno5z_lr_nd(y, eps, nL, dL, nR, dR);
    const double dd = dL * dR;
    const unsigned ex = ((unsigned)__double2hiint(dd) >> 20) & 0x7ffu;
    if (ex - 2u <= 2042u) {
      const double r = 1.0 / dd;
      L = nL * (dR * r);
      R = nR * (dL * r);
    } else {
      L = nL / dL;
      R = nR / dR;
    }
  } else {
    // the other interpolations share the sides' three-cell terms too
    Eno3 eL, eR;
    eno3_lr(y, eL, eR);
    if constexpr (RC == RC_WENO5JS) {
      L = weno5js_e(eL);
      R = weno5js_e(eR);
    } else if constexpr (RC == RC_TENO5) {
      L = teno5_e(eL);
      R = teno5_e(eR);
    } else {
      L = teno6_e(eL, y[0], y[1], y[2], y[3], y[4], y[5]);
      R = teno6_e(eR, y[5], y[4], y[3], y[2], y[1], y[0]);
    }
  }
}

// ---------------------------------------------------------------------------
// HLLC (Appendix B)
template <int NS>
struct State {
  double rho, rhoY[NS], u[3], m[3], p, E, a;
};

// F(S) + s (U*_S - U_S): the HLLC flux on the side S of the contact the
// face lies on (s = min(0, s_L) for the left side, max(0, s_R) for the right,
// sS its wave speed, dS = sS - u_S)
template <int NS, int D>
__device__ __forceinline__ void hllc_side(int d, const State<NS>& S, double s, double sS, double dS, double ss,
                                          double* F) {
  const double f = dS / (sS - ss);
#pragma unroll
  for (int k = 0; k < NS; ++k) F[k] = S.rhoY[k] * S.u[d] + s * (f * S.rhoY[k] - S.rhoY[k]);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const double Fs = S.rho * S.u[d] * S.u[j] + (j == d ? S.p : 0.0);
    const double Us = f * S.rho * (j == d ? ss : S.u[j]);
    F[NS + j] = Fs + s * (Us - S.m[j]);
  }
  const double Fs = S.u[d] * (S.E + S.p);
  const double Us = f * (S.E + (ss - S.u[d]) * (S.rho * ss + S.p / dS));
  F[NS + D] = Fs + s * (Us - S.E);
}

template <int NS, int D>
__device__ __forceinline__ void hllc(int d, const State<NS>& L, const State<NS>& R, double* F) {
  const double ub = 0.5 * (L.u[d] + R.u[d]), ab = 0.5 * (L.a + R.a);
  const double sL = fmin(ub - ab, L.u[d] - L.a);
  const double sR = fmax(ub + ab, R.u[d] + R.a);
  const double sm = fmin(0.0, sL), sp = fmax(0.0, sR);
  const double dL = sL - L.u[d], dR = sR - R.u[d];
  const double ss = (R.p - L.p + L.rho * L.u[d] * dL - R.rho * R.u[d] * dR) / (L.rho * dL - R.rho * dR);
  // only the side of the contact the face lies on is evaluated; sign(0) = 0
  // takes both with weight 1/2
  if (positive(ss)) {
    hllc_side<NS, D>(d, L, sm, sL, dL, ss, F);
  } else if (negative(ss)) {
    hllc_side<NS, D>(d, R, sp, sR, dR, ss, F);
  } else {
    constexpr int NV = NS + D + 1;
    double FL[NV], FR[NV];
    hllc_side<NS, D>(d, L, sm, sL, dL, ss, FL);
    hllc_side<NS, D>(d, R, sp, sR, dR, ss, FR);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = 0.5 * FL[v] + 0.5 * FR[v];
  }
}

// face-side state from reconstructed (Y, u, P, T) (steps 4-5 of Sec. 3.1.3)
template <int NS>
__device__ __forceinline__ void state_from_primitive(const KParams& P, const double* Y, const double* u, double p,
                                                     double T, State<NS>& s) {
  double e, al, be;
  eos_forward<NS>(P, Y, p, T, s.rho, e, s.a, al, be);
  double ke = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    s.u[d] = u[d];
    s.m[d] = s.rho * u[d];
    ke += u[d] * u[d];
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) s.rhoY[k] = s.rho * Y[k];
  s.p = p;
  s.E = s.rho * (e + 0.5 * ke);
}

// Eqs. PositivityReqs1/2 on a conserved vector, division free:
// rhoY_k >= -YTOL rho, rho > 0, 1 - sum rhoY_k b_k > 0,
// rho E - |m|^2/2 - rho sum rhoY_k q_k > 0
template <int NS, int D>
__device__ __forceinline__ bool admissible_bq(const double* b, const double* q, bool has_b, bool has_q,
                                              const double* U) {
  double rho = 0.0, sb = 0.0, sq = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    rho += U[k];
    if (has_b) sb += U[k] * b[k];
    if (has_q) sq += U[k] * q[k];
  }
  // (without covolumes or reference energies the b and q terms are zero:
  // they are skipped, not evaluated as 1 - 0 and x - 0)
  bool ok = positive(rho) && (!has_b || positive(1.0 - sb));
#pragma unroll
  for (int k = 0; k < NS; ++k) ok = ok && (U[k] >= -YTOL * rho);
  double mm = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) mm += U[NS + d] * U[NS + d];
  const double ei = rho * U[NS + D] - 0.5 * mm;
  return ok && positive(has_q ? ei - rho * sq : ei);
}

template <int NS, int D>
__device__ __forceinline__ bool admissible(const KParams& P, const double* U) {
  return admissible_bq<NS, D>(P.b, P.q, P.has_b, P.has_q, U);
}

// mass-fraction limiter of Sec. 3.3.1 on one face side (Yc: cell values)
template <int NS>
__device__ __forceinline__ bool y_limiter(double* Y, const double* Yc) {
  bool active = false;
#pragma unroll
  for (int k = 0; k < NS; ++k)
    if (negative(Y[k])) {
      Y[k] = 0.0;
      active = true;
    }
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) sum += Y[k];
  // a sum that is one to rounding is left alone: the correction would be
  // below the data's resolution and split by a ratio of rounding errors
  if (fabs(sum - 1.0) > NS * YSUM_TOL) {
    const bool over = sum > 1.0;
    double dd[NS], Sig = 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      dd[k] = (over ? fmin(Y[k], Yc[k]) : fmax(Y[k], Yc[k])) - Y[k];
      Sig += dd[k];
    }
    if (nonzero(Sig)) {
      const double f = (1.0 - sum) / Sig;
#pragma unroll
      for (int k = 0; k < NS; ++k) Y[k] += f * dd[k];
      active = true;
    }
  }
  return active;
}

}  // namespace mpmc
