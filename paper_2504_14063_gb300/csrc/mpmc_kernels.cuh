// FP64 kernels of the MPMC stage (arXiv 2504.14063), templated on the
// species count NS and the dimension D, and their launchers.
//   k_init   : primitive fields -> U (Eq. NASG_EOS, Amagat mixing)
//   k_prim   : U -> primitive cache (Sec. 2.2-2.3, Eq. SpeedOfSound, the CDI
//              and diffusion ingredients) + CFL / Gamma block maxima
//   k_face   : one face of direction d: Godunov approach of Sec. 3.1.3 with
//              limiters (Sec. 3.3), HLLC (App. B), CDI (Sec. 3.2), diffusion
//   k_update : divergence (Eq. DiscreteGoverningEquations) + SSP-RK
//              combination (Eq. SSPRK3)
#pragma once
#include "mpmc_device.cuh"
#include "mpmc_ops.h"
#include "mpmc_update.cuh"

namespace mpmc {

constexpr int FACE_THREADS = 128;
constexpr int CELL_THREADS = 256;

// ---------------------------------------------------------------------------
template <int NS, int D>
__global__ void __launch_bounds__(CELL_THREADS) k_init(const KParams P, const double* __restrict__ prim,
                                                       double* __restrict__ U, long long n) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double p = prim[(long long)(NS + D) * n + c];
  const double T = prim[(long long)(NS + D + 1) * n + c];
  double rho = 0.0, e = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double a = prim[(long long)k * n + c];
    double ry = 0.0;
    if (a != 0.0) {
      ry = a / v_k(P, k, p, T);
      e += ry * e_k(P, k, p, T);
    }
    U[(long long)k * n + c] = ry;
    rho += ry;
  }
  double ke = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double u = prim[(long long)(NS + d) * n + c];
    U[(long long)(NS + d) * n + c] = rho * u;
    ke += rho * u * u;
  }
  U[(long long)(NS + D) * n + c] = e + 0.5 * ke;
}

// ---------------------------------------------------------------------------
// ghost states of the characteristic x boundaries (the non-reflecting inflow
// / outflow conditions Sec. 3.5 cites, in their locally one-dimensional
// inviscid form): at each boundary cell, the characteristic decomposition of
// Appendix A at that cell's state -- the acoustic invariants P +- rho a u_x
// (speeds u_x +- a) and, with speed u_x, T - X P, the mass fractions and the
// tangential velocity.  A field leaving the domain (speed along the outward
// normal > 0, >= 0 for u_x) keeps the cell's value, an entering one takes
// the far-field state's (G column 0, the inflow state).  A ghost that is not
// admissible (T <= 0, or P + Pinf_k <= 0 for a species present) is the
// boundary cell itself.  G: U's ghost buffer; slot s is written to column 1 + s.
template <int NS, int D>
__global__ void __launch_bounds__(CELL_THREADS)
    k_char_ghost(const KParams P, const double* __restrict__ U, double* __restrict__ G) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.nslots) return;
  constexpr int NV = NS + D + 1;
  const long long plane = (long long)P.n[1] * P.n[2];
  const int side = (P.char_lo && s < plane) ? 0 : 1;
  const long long row = s - (side == 1 && P.char_lo ? plane : 0);
  const long long cb = row * P.n[0] + (side == 0 ? 0 : P.n[0] - 1);
  double Ub[NV], Ut[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    Ub[v] = U[(long long)v * P.ncell + cb];
    Ut[v] = G[(long long)v * P.gstride];
  }
  double rho, Y[NS], u[3], e, vol, p, T;
  decode<NS, D>(Ub, rho, Y, u, e, vol);
  pt_equilibrium<NS>(P, Y, e, vol, p, T);
  double r2, e2, a, al, be;
  eos_forward<NS>(P, Y, p, T, r2, e2, a, al, be);
  const double X = (rho * a * a * be - 1.0) / (al * a * a * rho), c = a * rho;
  double rt, Yt[NS], ut[3], et, vt, pt, Tt;
  decode<NS, D>(Ut, rt, Yt, ut, et, vt);
  pt_equilibrium<NS>(P, Yt, et, vt, pt, Tt);
  const double out = side == 0 ? -1.0 : 1.0;
  const double un = u[0];
  const bool out_p = out * (un + a) > 0.0, out_m = out * (un - a) > 0.0, out_0 = out * un >= 0.0;
  const double wp = out_p ? p + c * un : pt + c * ut[0];
  const double wm = out_m ? p - c * un : pt - c * ut[0];
  const double Pg = 0.5 * (wp + wm);
  const double Tg = (out_0 ? T - X * p : Tt - X * pt) + X * Pg;
  double Yg[NS], ug[3];
#pragma unroll
  for (int k = 0; k < NS; ++k) Yg[k] = out_0 ? Y[k] : Yt[k];
#pragma unroll
  for (int t = 0; t < 3; ++t) ug[t] = out_0 ? u[t] : ut[t];
  ug[0] = (wp - wm) / (2.0 * c);
  bool ok = Tg > 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k)
    if (positive(Yg[k]) && !positive(Pg + P.pinf[k])) ok = false;
  double Ug[NV];
  if (ok) {
    State<NS> st;
    state_from_primitive<NS>(P, Yg, ug, Pg, Tg, st);
#pragma unroll
    for (int k = 0; k < NS; ++k) Ug[k] = st.rhoY[k];
#pragma unroll
    for (int d = 0; d < D; ++d) Ug[NS + d] = st.m[d];
    Ug[NS + D] = st.E;
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) Ug[v] = Ub[v];
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) G[(long long)v * P.gstride + 1 + s] = Ug[v];
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Block maxima of two non-negative values -> atomicMax on their bit patterns
// (IEEE order of non-negative doubles equals the order of their bits).
__device__ __forceinline__ void block_max2(double a, double b, unsigned long long* red) {
  __shared__ double sa[32], sb[32];
  a = warp_max(a);
  b = warp_max(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sa[wid] = a;
    sb[wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    a = warp_max(a);
    b = warp_max(b);
    if (lane == 0) {
      atomicMax(red + 0, (unsigned long long)__double_as_longlong(a));
      atomicMax(red + 1, (unsigned long long)__double_as_longlong(b));
    }
  }
}

template <int NS, int D>
__global__ void __launch_bounds__(CELL_THREADS)
    k_prim(const KParams P, const double* __restrict__ U, const double* __restrict__ Uin, double* __restrict__ Wc,
           unsigned long long* __restrict__ red, int* __restrict__ status) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double smax = 0.0, gmax = 0.0;
  if (c < P.ncell + P.nextra) {
    constexpr int NV = NS + D + 1;
    double Uc[NV];
    if (c >= P.ncell) {
      // the inflow state or a characteristic ghost, from U's ghost buffer
#pragma unroll
      for (int v = 0; v < NV; ++v) Uc[v] = Uin[(long long)v * P.gstride + (c - P.ncell)];
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) Uc[v] = U[(long long)v * P.ncell + c];
    }
    const long long ws = P.wstride;
    double rho, Y[NS], u[3], e, irho;
    decode<NS, D>(Uc, rho, Y, u, e, irho);
    int st = positive(rho) ? ST_OK : ST_INADMISSIBLE;
#pragma unroll
    for (int k = 0; k < NS; ++k)
      if (Uc[k] < -YTOL * rho) st = ST_INADMISSIBLE;
    double p, T;
    const int st2 = pt_equilibrium<NS>(P, Y, e, irho, p, T);
    if (st == ST_OK) st = st2;
    double r2, e2, a, al, be;
    eos_forward<NS>(P, Y, p, T, r2, e2, a, al, be);
    Wc[P.wT * ws + c] = T;
    Wc[P.wP * ws + c] = p;
    Wc[P.wRho * ws + c] = rho;
    Wc[P.wA * ws + c] = a;
#pragma unroll
    for (int k = 0; k < NS; ++k) Wc[(P.wY + k) * ws + c] = Y[k];
#pragma unroll
    for (int d = 0; d < D; ++d) Wc[(P.wU + d) * ws + c] = u[d];

    double mu = 0.0, lam = 0.0;
    if (P.cdi || P.diffusion || P.viscous) {
      double phi[2], Yp[2];
#pragma unroll
      for (int ph = 0; ph < 2; ++ph) {
        double f = 0.0, hr = 0.0, yp = 0.0;
#pragma unroll
        for (int k = 0; k < NS; ++k)
          if (P.phase[k] == ph) {
            yp += Y[k];
            if (nonzero(Uc[k])) {
              // the oracle's operation order without contraction
              const double vk = add_(mul_(P.Rk[k], T) / add_(p, P.pinf[k]), P.b[k]);
              const double hk = add_(add_(mul_(P.cp[k], T), mul_(P.b[k], p)), P.q[k]);
              f = add_(f, mul_(Uc[k], vk));
              hr = add_(hr, mul_(Uc[k], hk));
            }
          }
        phi[ph] = f;
        Yp[ph] = yp;
        if (P.cdi) {
          const bool present = yp >= ABSENT;
          Wc[(P.wHrho + ph) * ws + c] = present ? hr / f : 0.0;
#pragma unroll
          for (int k = 0; k < NS; ++k)
            if (P.phase[k] == ph) Wc[(P.wYrho + k) * ws + c] = present ? Uc[k] / f : 0.0;
        }
      }
      if (P.cdi) {
        Wc[P.wPhi0 * ws + c] = phi[0];
        Wc[P.wPsi * ws + c] = P.cdi_eps * log((phi[0] + P.psi_delta) / (phi[1] + P.psi_delta));
      }
      // phase viscosities: liquid constant, gas by Wilke's rule
      double mup[2] = {P.mu_liquid, 0.0};
      if (P.diffusion || P.viscous) {
        double num = 0.0;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          if (P.phase[i] != 1) continue;
          double den = 0.0;
#pragma unroll
          for (int j = 0; j < NS; ++j)
            if (P.phase[j] == 1) den += Y[j] * P.wilke[i][j];
          if (positive(den)) num += Y[i] * P.mu[i] / den;
        }
        mup[1] = Yp[1] >= ABSENT ? num : 0.0;
        mu = phi[0] * mup[0] + phi[1] * mup[1];
      }
      if (P.viscous) {
        // heat conductivity: liquid constant, gas (mu_g / Pr) sum (Y^c/Y_g) Cp^c
        double cpY = 0.0;
#pragma unroll
        for (int k = 0; k < NS; ++k)
          if (P.phase[k] == 1) cpY += Y[k] * P.cp[k];
        const double lam_g = Yp[1] >= ABSENT ? mup[1] / P.prandtl * (cpY / Yp[1]) : 0.0;
        lam = phi[0] * P.lambda_liquid + phi[1] * lam_g;
        Wc[P.wMu * ws + c] = mu;
        Wc[P.wLam * ws + c] = lam;
      }
      if (P.diffusion) {
#pragma unroll
        for (int ph = 0; ph < 2; ++ph) {
          double sY = 0.0;
#pragma unroll
          for (int j = 0; j < NS; ++j)
            if (P.phase[j] == ph) sY += Y[j] / P.W[j];
          const bool present = Yp[ph] >= ABSENT && sY >= ABSENT;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            if (P.phase[k] != ph) continue;
            double xr = 0.0, B = 0.0;
            if (present) {
              xr = (Y[k] / P.W[k]) / sY;
              const double WcWp = P.W[k] * sY / Yp[ph];
              const double rho_p = rho * Yp[ph] / phi[ph];
              B = WcWp * (mup[ph] / (rho_p * P.Sc[k]));
            }
            Wc[(P.wXr + k) * ws + c] = xr;
            Wc[(P.wB + k) * ws + c] = B;
          }
        }
      }
    }
    if (st != ST_OK) atomicMax(status, st);
    if (c < P.ncell) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const double ud = fabs(u[d]);
        smax = fmax(smax, (ud + a) * P.inv_dx);
        gmax = fmax(gmax, ud);
      }
      if (P.diffusion || P.viscous) smax = fmax(smax, 4.0 * mu / rho * (P.inv_dx * P.inv_dx));
      if (P.viscous) {
        // conduction limit with the thermal diffusivity lambda / (rho cv)
        double cv = 0.0;
#pragma unroll
        for (int k = 0; k < NS; ++k) cv += Y[k] * P.cv[k];
        smax = fmax(smax, 4.0 * lam / (rho * cv) * (P.inv_dx * P.inv_dx));
      }
    }
  }
  if (red) block_max2(smax, gmax, red);
}


// ---------------------------------------------------------------------------
// DIR: the face direction, a template parameter so that every array indexed
// by it is indexed by a constant (registers, not the stack).  RC: the
// ENO-type interpolation (RC_WENO5Z, the method's, or one of Sec. 4.1's others)
template <int NS, int D, int DIR, int RC>
__global__ void __launch_bounds__(FACE_THREADS)
    k_face(const KParams P, const double* __restrict__ Wc, const double* __restrict__ Un,
           const double* __restrict__ Uk, const double* __restrict__ Uin, const double* __restrict__ scal,
           const double rk0, const double rk1, const double rk2, double* __restrict__ F,
           uint32_t* __restrict__ flags, unsigned long long* __restrict__ stats) {
  constexpr int NV = NS + D + 1;
  constexpr int d = DIR;
  const int f0 = P.n[0] + (d == 0), f1 = P.n[1] + (d == 1), f2 = P.n[2] + (d == 2);
  const long long nf = (long long)f0 * f1 * f2;
  const long long fid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (fid >= nf) return;
  int fc[3];
  unflatten(fid, f0, f1, fc);
  int ci[3] = {fc[0], fc[1], fc[2]};
  ci[d] -= 1;  // the cell on the low side of the face
  const double dt = scal[0], Gamma = scal[1];
  const long long ws = P.wstride;

  CRef cr[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    int cc[3] = {ci[0], ci[1], ci[2]};
    cc[d] += j - 2;
    cr[j] = map_cell_m<1u << d>(P, cc[0], cc[1], cc[2]);
  }
  const CRef ri = cr[2], rj = cr[3];
  uint32_t fl = 0u;

  // step 1: averaged conserved state on the face, its EOS, the scalars of
  // the characteristic matrices (Appendix A)
  double X, c, ic;
  {
    double Ui[NV], Uj[NV];
    load_U<NS, D>(P, Uk, Uin, ri, Ui);
    load_U<NS, D>(P, Uk, Uin, rj, Uj);
#pragma unroll
    for (int v = 0; v < NV; ++v) Ui[v] = 0.5 * (Ui[v] + Uj[v]);
    // these scalars only shape the projection: ordinary (contracted) arithmetic
    double rho, Y[NS], uu[3], e, vol;
    decode<NS, D, false>(Ui, rho, Y, uu, e, vol);
    double p, T, a, al, be;
    // the Newton start of several stiffened liquids: the mean of the two
    // cells' pressures, close to the averaged state's
    pt_equilibrium<NS, false>(P, Y, e, vol, p, T, rho,
                              0.5 * (wget(P, Wc, P.wP, ri) + wget(P, Wc, P.wP, rj)));
    eos_char<NS>(P, Y, p, T, rho, a, al, be);
    X = (rho * a * a * be - 1.0) / (al * a * a * rho);
    c = a * rho;
    ic = 1.0 / c;
  }

  // steps 2-3: project, interpolate both sides (WENO5-Z unless RC says
  // otherwise), back to physical space
  double YL[NS], YR[NS], uL[3] = {0.0, 0.0, 0.0}, uR[3] = {0.0, 0.0, 0.0}, PL, PR, TL, TR;
  const double eps = P.weno_eps;
  {
    double w1[6], w5[6], w6[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const double T = wget(P, Wc, P.wT, cr[j]);
      const double p = wget(P, Wc, P.wP, cr[j]);
      const double un = wget(P, Wc, P.wU + d, cr[j]) * sgn_flip(cr[j].flip, d);
      w1[j] = T - X * p;
      w5[j] = (0.5 * c) * un + 0.5 * p;
      w6[j] = (-0.5 * c) * un + 0.5 * p;
    }
    double w1L, w1R, w5L, w5R, w6L, w6R;
    recon_lr<RC>(w1, eps, w1L, w1R);
    recon_lr<RC>(w5, eps, w5L, w5R);
    recon_lr<RC>(w6, eps, w6L, w6R);
    TL = w1L + X * w5L + X * w6L;
    TR = w1R + X * w5R + X * w6R;
    uL[d] = ic * w5L + (-ic) * w6L;
    uR[d] = ic * w5R + (-ic) * w6R;
    PL = w5L + w6L;
    PR = w5R + w6R;
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    double y[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) y[j] = wget(P, Wc, P.wY + k, cr[j]);
    recon_lr<RC>(y, eps, YL[k], YR[k]);
  }
#pragma unroll
  for (int t = 0; t < D; ++t) {
    if (t == d) continue;
    double y[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) y[j] = wget(P, Wc, P.wU + t, cr[j]) * sgn_flip(cr[j].flip, t);
    recon_lr<RC>(y, eps, uL[t], uR[t]);
  }

  // cell values of the two face neighbours
  double Yi[NS], Yj[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    Yi[k] = wget(P, Wc, P.wY + k, ri);
    Yj[k] = wget(P, Wc, P.wY + k, rj);
  }
  const double Ti = wget(P, Wc, P.wT, ri), Tj = wget(P, Wc, P.wT, rj);
  const double Pi = wget(P, Wc, P.wP, ri), Pj = wget(P, Wc, P.wP, rj);

  // interpolation limiters (Sec. 3.3.1)
  if (P.pos_limiter) {
    if (y_limiter<NS>(YL, Yi)) fl |= F_YLIM_L;
    if (y_limiter<NS>(YR, Yj)) fl |= F_YLIM_R;
    if (!positive(TL)) { TL = Ti; fl |= F_THETA_T_L; }
    if (!positive(TR)) { TR = Tj; fl |= F_THETA_T_R; }
    bool okL = true, okR = true;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (positive(YL[k]) && !positive(PL + P.pinf[k])) okL = false;
      if (positive(YR[k]) && !positive(PR + P.pinf[k])) okR = false;
    }
    if (!okL) { PL = Pi; fl |= F_THETA_P_L; }
    if (!okR) { PR = Pj; fl |= F_THETA_P_R; }
  }

  // steps 4-6: face EOS, conserved face states, HLLC
  double Fx[NV];
  {
    State<NS> sL, sR;
    state_from_primitive<NS>(P, YL, uL, PL, TL, sL);
    state_from_primitive<NS>(P, YR, uR, PR, TR, sR);
    hllc<NS, D>(d, sL, sR, Fx);
  }

  // flux limiter (Sec. 3.3.2): pseudo-updates of both cells
  // Bi, Bj: the RK combination rk0 U^n + rk1 U^(k) of both cells, formed
  // once for the (up to three) pseudo-update tests of this face
  double Bi[NV], Bj[NV], Uki[NV], Ukj[NV];
  const double lam = 2.0 * D * rk2 * dt * P.inv_dx;
  if (P.pos_limiter || P.cdi) {
    load_U<NS, D>(P, Uk, Uin, ri, Uki);
    load_U<NS, D>(P, Uk, Uin, rj, Ukj);
    load_U<NS, D>(P, Un, P.gn, ri, Bi);
    load_U<NS, D>(P, Un, P.gn, rj, Bj);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Bi[v] = rk0 * Bi[v] + rk1 * Uki[v];
      Bj[v] = rk0 * Bj[v] + rk1 * Ukj[v];
    }
  }
  auto passes = [&](const double* Ft) {
    double Ti_[NV], Tj_[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Ti_[v] = Bi[v] - lam * Ft[v];
      Tj_[v] = Bj[v] + lam * Ft[v];
    }
    return admissible<NS, D>(P, Ti_) && admissible<NS, D>(P, Tj_);
  };
  if (P.pos_limiter && !passes(Fx)) {
    State<NS> si, sj;
    si.rho = wget(P, Wc, P.wRho, ri);
    sj.rho = wget(P, Wc, P.wRho, rj);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      si.rhoY[k] = Uki[k];
      sj.rhoY[k] = Ukj[k];
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      si.u[t] = t < D ? wget(P, Wc, P.wU + t, ri) * sgn_flip(ri.flip, t) : 0.0;
      sj.u[t] = t < D ? wget(P, Wc, P.wU + t, rj) * sgn_flip(rj.flip, t) : 0.0;
      si.m[t] = t < D ? Uki[NS + t] : 0.0;
      sj.m[t] = t < D ? Ukj[NS + t] : 0.0;
    }
    si.p = Pi;
    sj.p = Pj;
    si.E = Uki[NS + D];
    sj.E = Ukj[NS + D];
    si.a = wget(P, Wc, P.wA, ri);
    sj.a = wget(P, Wc, P.wA, rj);
    hllc<NS, D>(d, si, sj, Fx);
    fl |= F_HLLC_FALLBACK;
  }

  // interface regularization (Sec. 3.2), KEEP split form, with its limiter
  if (P.cdi && P.two_phase) {
    bool pres_i[2] = {false, false}, pres_j[2] = {false, false};
    {
      // (branches on the phase rather than ypi[P.phase[k]]: an array indexed
      // at run time would live on the stack)
      double ypi[2] = {0.0, 0.0}, ypj[2] = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        if (P.phase[k]) {
          ypi[1] += Yi[k];
          ypj[1] += Yj[k];
        } else {
          ypi[0] += Yi[k];
          ypj[0] += Yj[k];
        }
      }
#pragma unroll
      for (int ph = 0; ph < 2; ++ph) {
        pres_i[ph] = ypi[ph] >= ABSENT;
        pres_j[ph] = ypj[ph] >= ABSENT;
      }
    }
    if ((pres_i[0] || pres_j[0]) && (pres_i[1] || pres_j[1])) {
      const double ceps = P.cdi_eps;
      const double psi_i = wget(P, Wc, P.wPsi, ri), psi_j = wget(P, Wc, P.wPsi, rj);
      const double dphi = (wget(P, Wc, P.wPhi0, rj) - wget(P, Wc, P.wPhi0, ri)) * P.inv_dx;
      double g[3] = {0.0, 0.0, 0.0};
      g[d] = (psi_j - psi_i) * P.inv_dx;
#pragma unroll
      for (int t = 0; t < D; ++t) {
        if (t == d) continue;
        int a0[3] = {ci[0], ci[1], ci[2]}, a1[3] = {ci[0], ci[1], ci[2]};
        int b0[3] = {ci[0], ci[1], ci[2]}, b1[3] = {ci[0], ci[1], ci[2]};
        a0[t] += 1;
        a1[t] -= 1;
        b0[t] += 1;
        b1[t] -= 1;
        b0[d] += 1;
        b1[d] += 1;
        const double pip = wget(P, Wc, P.wPsi, map_cell_dt<d>(P, t, a0[0], a0[1], a0[2]));
        const double pim = wget(P, Wc, P.wPsi, map_cell_dt<d>(P, t, a1[0], a1[1], a1[2]));
        const double pjp = wget(P, Wc, P.wPsi, map_cell_dt<d>(P, t, b0[0], b0[1], b0[2]));
        const double pjm = wget(P, Wc, P.wPsi, map_cell_dt<d>(P, t, b1[0], b1[1], b1[2]));
        g[t] = 0.5 * ((pip - pim) * (0.5 * P.inv_dx) + (pjp - pjm) * (0.5 * P.inv_dx));
      }
      const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      const double nd = gn >= GTOL ? g[d] / gn : 0.0;
      // 1 - tanh^2 as 1 / cosh^2 (no cancellation near the phi_min floor)
      const double ch = cosh((0.5 * (psi_i + psi_j)) / (2.0 * ceps));
      const double sech2 = 1.0 / (ch * ch);
      const double ahat0 = Gamma * (ceps * dphi - 0.25 * (sech2 - P.sharp0) * nd);
      double Fdi[NV], Rtot = 0.0, hR = 0.0;
#pragma unroll
      for (int ph = 0; ph < 2; ++ph) {
        const double ahat = ph == 0 ? ahat0 : -ahat0;
        const bool pi = pres_i[ph], pj = pres_j[ph];
        auto keep = [&](double a, double b) { return pi && pj ? 0.5 * (a + b) : (pi ? a : (pj ? b : 0.0)); };
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          if (P.phase[k] != ph) continue;
          const double R = -keep(wget(P, Wc, P.wYrho + k, ri), wget(P, Wc, P.wYrho + k, rj)) * ahat;
          Fdi[k] = R;
          Rtot += R;
        }
        hR -= keep(wget(P, Wc, P.wHrho + ph, ri), wget(P, Wc, P.wHrho + ph, rj)) * ahat;
      }
      double kb = 0.0;
#pragma unroll
      for (int t = 0; t < D; ++t) {
        const double ui = wget(P, Wc, P.wU + t, ri) * sgn_flip(ri.flip, t);
        const double uj = wget(P, Wc, P.wU + t, rj) * sgn_flip(rj.flip, t);
        kb += ui * uj;
        Fdi[NS + t] = 0.5 * (ui + uj) * Rtot;
      }
      Fdi[NS + D] = 0.5 * kb * Rtot + hR;
      double Ft[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Ft[v] = Fx[v] + Fdi[v];
      if (P.pos_limiter && !passes(Ft)) {
        fl |= F_CDI_DROPPED;
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) Fx[v] = Ft[v];
      }
    }
  }

  // diffusive flux F_nu: species diffusion (Eq. SpeciesMassDiffusion),
  // viscous stress and heat conduction.  It passes the same flux limiter as
  // the regularization flux: added to the admissible flux when both
  // pseudo-updates stay admissible, else not added at this face.
  double Fnu[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Fnu[v] = 0.0;
  if (P.diffusion) {
    const double rb = 0.5 * (wget(P, Wc, P.wRho, ri) + wget(P, Wc, P.wRho, rj));
    double Jh = 0.0;
#pragma unroll
    for (int ph = 0; ph < 2; ++ph) {
      double Yp = 0.0, S = 0.0, Bf[NS], G[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        Bf[k] = 0.0;
        G[k] = 0.0;
        if (P.phase[k] != ph) continue;
        Yp += 0.5 * (Yi[k] + Yj[k]);
        Bf[k] = 0.5 * (wget(P, Wc, P.wB + k, ri) + wget(P, Wc, P.wB + k, rj));
        G[k] = (wget(P, Wc, P.wXr + k, rj) - wget(P, Wc, P.wXr + k, ri)) * P.inv_dx;
        S += Bf[k] * G[k];
      }
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        if (P.phase[k] != ph) continue;
        const double J = -rb * (Yp * Bf[k] * G[k] - 0.5 * (Yi[k] + Yj[k]) * S);
        Fnu[k] = J;
        Jh += J * (0.5 * (h_k(P, k, Pi, Ti) + h_k(P, k, Pj, Tj)));
      }
    }
    Fnu[NS + D] = Jh;
  }

  // viscous stress and heat conduction (Eq. DiffusionTerms), second-order
  // central: face averages of the two cells, normal derivative
  // (q_j - q_i)/dx, a tangential one the mean of the two cells' central
  // differences; the energy row carries -u.tau + q
  if (P.viscous) {
    double gu[3][3];  // gu[i][j] = d u_i / d x_j on the face
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) gu[i][j] = 0.0;
    double ui[3] = {0.0, 0.0, 0.0}, uj[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < D; ++i) {
      ui[i] = wget(P, Wc, P.wU + i, ri) * sgn_flip(ri.flip, i);
      uj[i] = wget(P, Wc, P.wU + i, rj) * sgn_flip(rj.flip, i);
      gu[i][d] = (uj[i] - ui[i]) * P.inv_dx;
    }
#pragma unroll
    for (int t = 0; t < D; ++t) {
      if (t == d) continue;
      int a0[3] = {ci[0], ci[1], ci[2]}, a1[3] = {ci[0], ci[1], ci[2]};
      a0[t] += 1;
      a1[t] -= 1;
      int b0[3] = {a0[0], a0[1], a0[2]}, b1[3] = {a1[0], a1[1], a1[2]};
      b0[d] += 1;
      b1[d] += 1;
      const CRef ip = map_cell_dt<d>(P, t, a0[0], a0[1], a0[2]), im = map_cell_dt<d>(P, t, a1[0], a1[1], a1[2]);
      const CRef jp = map_cell_dt<d>(P, t, b0[0], b0[1], b0[2]), jm = map_cell_dt<d>(P, t, b1[0], b1[1], b1[2]);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const double dip = wget(P, Wc, P.wU + i, ip) * sgn_flip(ip.flip, i) -
                           wget(P, Wc, P.wU + i, im) * sgn_flip(im.flip, i);
        const double djp = wget(P, Wc, P.wU + i, jp) * sgn_flip(jp.flip, i) -
                           wget(P, Wc, P.wU + i, jm) * sgn_flip(jm.flip, i);
        gu[i][t] = 0.25 * P.inv_dx * (dip + djp);
      }
    }
    double div = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) div += gu[k][k];
    const double mub = 0.5 * (wget(P, Wc, P.wMu, ri) + wget(P, Wc, P.wMu, rj));
    const double lamb = 0.5 * (wget(P, Wc, P.wLam, ri) + wget(P, Wc, P.wLam, rj));
    double work = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double tau = mub * (gu[i][d] + gu[d][i] - (i == d ? (2.0 / 3.0) * div : 0.0));
      Fnu[NS + i] = -tau;
      work += 0.5 * (ui[i] + uj[i]) * tau;
    }
    Fnu[NS + D] -= work + lamb * (Tj - Ti) * P.inv_dx;
  }
  if (P.diffusion || P.viscous) {
    double Ft[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Ft[v] = Fx[v] + Fnu[v];
    if (P.pos_limiter && !passes(Ft)) {
      fl |= F_DIFF_DROPPED;
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) Fx[v] = Ft[v];
    }
  }

#pragma unroll
  for (int v = 0; v < NV; ++v) F[(long long)v * nf + fid] = Fx[v];
  if (flags) flags[fid] = fl;
  if (stats && fl) {
    if (fl & F_HLLC_FALLBACK) atomicAdd(stats + 1, 1ull);
    if (fl & F_CDI_DROPPED) atomicAdd(stats + 2, 1ull);
    if (fl & (F_THETA_P_L | F_THETA_P_R)) atomicAdd(stats + 3, 1ull);
    if (fl & (F_THETA_T_L | F_THETA_T_R)) atomicAdd(stats + 4, 1ull);
    if (fl & (F_YLIM_L | F_YLIM_R)) atomicAdd(stats + 5, 1ull);
    if (fl & F_DIFF_DROPPED) atomicAdd(stats + 6, 1ull);
  }
}

// ---------------------------------------------------------------------------
template <int NS, int D>
__global__ void __launch_bounds__(CELL_THREADS)
    k_update(const KParams P, const double* __restrict__ Un, const double* __restrict__ Uk,
             const double* __restrict__ F0, const double* __restrict__ F1, const double* __restrict__ F2,
             const double* __restrict__ scal, const double rk0, const double rk1, const double rk2,
             double* __restrict__ Uout, double* __restrict__ dUdt, int* __restrict__ status) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.ncell) return;
  update_cell<NS, D>(P, c, Un, Uk, F0, F1, F2, scal, rk0, rk1, rk2, Uout, dUdt, status);
}

// ---------------------------------------------------------------------------
inline unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// the FP64 face pass of one direction with interpolation RC
template <int NS, int D, int RC>
struct FaceImpl {
  static void face(const KParams& P, cudaStream_t s, int d, const double* Wc, const double* Un, const double* Uk,
                   const double* Uin, const double* scal, double rk0, double rk1, double rk2, double* F,
                   uint32_t* flags, unsigned long long* stats) {
    long long nf = 1;
    for (int e = 0; e < 3; ++e) nf *= (long long)(P.n[e] + (e == d));
    const unsigned nb = nblocks(nf, FACE_THREADS);
    if (d == 0)
      k_face<NS, D, 0, RC><<<nb, FACE_THREADS, 0, s>>>(P, Wc, Un, Uk, Uin, scal, rk0, rk1, rk2, F, flags, stats);
    else if (d == 1)
      k_face<NS, D, (D > 1 ? 1 : 0), RC><<<nb, FACE_THREADS, 0, s>>>(P, Wc, Un, Uk, Uin, scal, rk0, rk1, rk2, F,
                                                                     flags, stats);
    else
      k_face<NS, D, (D > 2 ? 2 : 0), RC><<<nb, FACE_THREADS, 0, s>>>(P, Wc, Un, Uk, Uin, scal, rk0, rk1, rk2, F,
                                                                     flags, stats);
  }
};

// the face pass of interpolation RC for (dimension, species count), or null
template <int RC>
FaceFn face_fp64(int dim, int ns) {
  switch (dim * 8 + ns) {
    case 9: return &FaceImpl<1, 1, RC>::face;
    case 10: return &FaceImpl<2, 1, RC>::face;
    case 11: return &FaceImpl<3, 1, RC>::face;
    case 12: return &FaceImpl<4, 1, RC>::face;
    case 17: return &FaceImpl<1, 2, RC>::face;
    case 18: return &FaceImpl<2, 2, RC>::face;
    case 19: return &FaceImpl<3, 2, RC>::face;
    case 20: return &FaceImpl<4, 2, RC>::face;
    case 25: return &FaceImpl<1, 3, RC>::face;
    case 26: return &FaceImpl<2, 3, RC>::face;
    case 27: return &FaceImpl<3, 3, RC>::face;
    case 28: return &FaceImpl<4, 3, RC>::face;
    default: return nullptr;
  }
}

template <int NS, int D>
struct Impl {
  static void init(const KParams& P, cudaStream_t s, const double* prim, double* U, long long n) {
    if (n > 0) k_init<NS, D><<<nblocks(n, CELL_THREADS), CELL_THREADS, 0, s>>>(P, prim, U, n);
  }
  static void prim(const KParams& P, cudaStream_t s, const double* U, const double* Uin, double* Wc,
                   unsigned long long* red, int* status) {
    k_prim<NS, D><<<nblocks(P.ncell + P.nextra, CELL_THREADS), CELL_THREADS, 0, s>>>(P, U, Uin, Wc, red,
                                                                                            status);
  }
  static void face(const KParams& P, cudaStream_t s, int d, const double* Wc, const double* Un, const double* Uk,
                   const double* Uin, const double* scal, double rk0, double rk1, double rk2, double* F,
                   uint32_t* flags, unsigned long long* stats) {
    FaceImpl<NS, D, RC_WENO5Z>::face(P, s, d, Wc, Un, Uk, Uin, scal, rk0, rk1, rk2, F, flags, stats);
  }
  static void update(const KParams& P, cudaStream_t s, const double* Un, const double* Uk, double* const* F,
                     const double* scal, double rk0, double rk1, double rk2, double* Uout, double* dUdt,
                     int* status) {
    k_update<NS, D><<<nblocks(P.ncell, CELL_THREADS), CELL_THREADS, 0, s>>>(
        P, Un, Uk, F[0], D > 1 ? F[1] : F[0], D > 2 ? F[2] : F[0], scal, rk0, rk1, rk2, Uout, dUdt, status);
  }
  static void ghost(const KParams& P, cudaStream_t s, const double* U, double* G) {
    if (P.nslots > 0) k_char_ghost<NS, D><<<nblocks(P.nslots, CELL_THREADS), CELL_THREADS, 0, s>>>(P, U, G);
  }
  static Ops ops() {
    Ops o;
    o.init = &init;
    o.prim = &prim;
    o.face = &face;
    o.update = &update;
    o.ghost = &ghost;
    return o;
  }
};

}  // namespace mpmc
