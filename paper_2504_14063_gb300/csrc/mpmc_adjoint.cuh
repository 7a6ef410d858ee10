// Discrete adjoint of the FP64 stage (reverse of k_prim / k_face / k_update)
// with the discrete decisions of the forward pass (interpolation limiters,
// first-order fallback, dropped regularization flux) replayed from the tape;
// dt and Gamma are frozen.  Each block of the face pipeline is recomputed
// forward and swept in reverse by hand.  The p-T equilibrium is reversed
// through the implicit-function theorem of its two defining equations
// (NASG_T1 and NASG_T2), which holds for the closed form and for the Newton
// solve alike.
#pragma once
#include "mpmc_device.cuh"

namespace mpmc {
namespace adj {

// ---------------------------------------------------------------------------
// relative stencil variation below which the weights are noise: the
// derivative there is taken with the ideal weights (the value is each
// candidate to rounding, and the weights' own derivative grows like 1/eps)
constexpr double WENO_FLAT = 1e-10;

// WENO5-Z (the forward kernel's form: candidates carried as 6 q_0, 36 q_1,
// 18 q_2, weights over one common denominator): its value and gradient
// g[j] = d(out)/d(v_j) in one pass
__device__ __forceinline__ double weno_val_grad(double v0, double v1, double v2, double v3, double v4, double eps,
                                                double* g) {
  const double Q0 = 2.0 * v0 - 7.0 * v1 + 11.0 * v2;
  const double Q1 = -6.0 * v1 + 30.0 * v2 + 12.0 * v3;
  const double Q2 = 6.0 * v2 + 15.0 * v3 - 3.0 * v4;
  const double t0 = v0 - 2.0 * v1 + v2, s0 = v0 - 4.0 * v1 + 3.0 * v2;
  const double t1 = v1 - 2.0 * v2 + v3, s1 = v1 - v3;
  const double t2 = v2 - 2.0 * v3 + v4, s2 = 3.0 * v2 - 4.0 * v3 + v4;
  const double b0 = (13.0 / 12.0) * t0 * t0 + 0.25 * s0 * s0;
  const double b1 = (13.0 / 12.0) * t1 * t1 + 0.25 * s1 * s1;
  const double b2 = (13.0 / 12.0) * t2 * t2 + 0.25 * s2 * s2;
  const double tau = fabs(b0 - b2);
  const double c0 = b0 + eps, c1 = b1 + eps, c2 = b2 + eps;
  const double p12 = c1 * c2, p02 = c0 * c2, p01 = c0 * c1;
  const double A0 = (c0 + tau) * p12, A1 = (c1 + tau) * p02, A2 = (c2 + tau) * p01;
  // out = sum_k A_k Q_k / S, S = 6 A0 + 36 A1 + 18 A2 (the ideal weights
  // 1/10, 6/10, 3/10 and the candidates' 1/6 folded in)
  const double iS = 1.0 / (6.0 * A0 + 36.0 * A1 + 18.0 * A2);
  const double out = (A0 * Q0 + A1 * Q1 + A2 * Q2) * iS;
  double M = fmax(fmax(fabs(v0), fabs(v1)), fmax(fmax(fabs(v2), fabs(v3)), fabs(v4)));
  const double tol = (WENO_FLAT * M) * (WENO_FLAT * M);
  if (b0 <= tol && b1 <= tol && b2 <= tol) {
    // ideal weights 1/10, 6/10, 3/10 on the three candidates
    g[0] = 1.0 / 30.0;
    g[1] = -13.0 / 60.0;
    g[2] = 47.0 / 60.0;
    g[3] = 9.0 / 20.0;
    g[4] = -1.0 / 20.0;
    return out;
  }
  // dA_k -> (Q_k - w_k out)/S with w = (6, 36, 18); dQ_k -> A_k/S
  const double lA0 = (Q0 - 6.0 * out) * iS, lA1 = (Q1 - 36.0 * out) * iS, lA2 = (Q2 - 18.0 * out) * iS;
  const double lQ0 = A0 * iS, lQ1 = A1 * iS, lQ2 = A2 * iS;
  // A0 = (c0 + tau) c1 c2 and cyclically
  const double lc0 = lA0 * p12 + lA1 * (c1 + tau) * c2 + lA2 * (c2 + tau) * c1;
  const double lc1 = lA1 * p02 + lA0 * (c0 + tau) * c2 + lA2 * (c2 + tau) * c0;
  const double lc2 = lA2 * p01 + lA0 * (c0 + tau) * c1 + lA1 * (c1 + tau) * c0;
  const double ltau = lA0 * p12 + lA1 * p02 + lA2 * p01;
  const double sg = (b0 - b2) >= 0.0 ? 1.0 : -1.0;
  const double lb0 = lc0 + sg * ltau, lb1 = lc1, lb2 = lc2 - sg * ltau;
  const double lt0 = lb0 * (13.0 / 6.0) * t0, ls0 = lb0 * 0.5 * s0;
  const double lt1 = lb1 * (13.0 / 6.0) * t1, ls1 = lb1 * 0.5 * s1;
  const double lt2 = lb2 * (13.0 / 6.0) * t2, ls2 = lb2 * 0.5 * s2;
  g[0] = lt0 + ls0 + 2.0 * lQ0;
  g[1] = -2.0 * lt0 - 4.0 * ls0 + lt1 + ls1 - 7.0 * lQ0 - 6.0 * lQ1;
  g[2] = lt0 + 3.0 * ls0 - 2.0 * lt1 + lt2 + 3.0 * ls2 + 11.0 * lQ0 + 30.0 * lQ1 + 6.0 * lQ2;
  g[3] = lt1 - ls1 - 2.0 * lt2 - 4.0 * ls2 + 12.0 * lQ1 + 15.0 * lQ2;
  g[4] = lt2 + ls2 - 3.0 * lQ2;
  return out;
}

// gradient of the three-cell candidates and indicators: given the adjoints
// lq[k] of the candidate values and lb[k] of the indicators (k = left,
// central, right), adds d/dv0..v4 to g
__device__ __forceinline__ void eno3_rev(double v0, double v1, double v2, double v3, double v4, const double* lq,
                                         const double* lb, double* g) {
  const double t0 = v0 - 2.0 * v1 + v2, s0 = v0 - 4.0 * v1 + 3.0 * v2;
  const double t1 = v1 - 2.0 * v2 + v3, s1 = v1 - v3;
  const double t2 = v2 - 2.0 * v3 + v4, s2 = 3.0 * v2 - 4.0 * v3 + v4;
  const double lt0 = lb[0] * (13.0 / 6.0) * t0, ls0 = lb[0] * 0.5 * s0;
  const double lt1 = lb[1] * (13.0 / 6.0) * t1, ls1 = lb[1] * 0.5 * s1;
  const double lt2 = lb[2] * (13.0 / 6.0) * t2, ls2 = lb[2] * 0.5 * s2;
  g[0] += lt0 + ls0 + lq[0] * (2.0 / 6.0);
  g[1] += -2.0 * lt0 - 4.0 * ls0 + lt1 + ls1 - lq[0] * (7.0 / 6.0) - lq[1] * (1.0 / 6.0);
  g[2] += lt0 + 3.0 * ls0 - 2.0 * lt1 + lt2 + 3.0 * ls2 + lq[0] * (11.0 / 6.0) + lq[1] * (5.0 / 6.0) +
          lq[2] * (2.0 / 6.0);
  g[3] += lt1 - ls1 - 2.0 * lt2 - 4.0 * ls2 + lq[1] * (2.0 / 6.0) + lq[2] * (5.0 / 6.0);
  g[4] += lt2 + ls2 - lq[2] * (1.0 / 6.0);
}

// WENO5-JS (alpha_k = d_k / (eps + beta_k)^2, eps = 1e-6): value and
// gradient w.r.t. v0..v4 (g[5] = 0)
__device__ __forceinline__ double weno5js_val_grad(double v0, double v1, double v2, double v3, double v4, double* g) {
  const Eno3 e = eno3(v0, v1, v2, v3, v4);
  constexpr double eps = 1e-6;
  const double il = 1.0 / (eps + e.bl), ic = 1.0 / (eps + e.bc), ir = 1.0 / (eps + e.br);
  const double A[3] = {0.1 * il * il, 0.6 * ic * ic, 0.3 * ir * ir};
  const double q[3] = {e.ql, e.qc, e.qr}, ib[3] = {il, ic, ir};
  const double S = A[0] + A[1] + A[2];
  const double out = (A[0] * q[0] + A[1] * q[1] + A[2] * q[2]) / S;
  // out = sum A_k q_k / S: dA_k -> (q_k - out) / S; dq_k -> A_k / S;
  // dA_k / dbeta_k = -2 A_k / (eps + beta_k)
  double lq[3], lb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lq[k] = A[k] / S;
    lb[k] = (q[k] - out) / S * (-2.0 * A[k] * ib[k]);
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) g[j] = 0.0;
  eno3_rev(v0, v1, v2, v3, v4, lq, lb, g);
  return out;
}

// TENO5 / TENO6: with the kept candidates fixed by the forward values (the
// replayed decision) the value is linear in v; its gradient is the kept
// candidates' coefficients with their renormalized optimal weights
template <int RC>
__device__ __forceinline__ double teno_val_grad(double v0, double v1, double v2, double v3, double v4, double v5,
                                                double* g) {
  const Eno3 e = eno3(v0, v1, v2, v3, v4);
  constexpr int K = RC == RC_TENO6 ? 4 : 3;
  // candidate coefficients on v0..v5: central, left, right, right four-cell
  const double cf[4][6] = {{0.0, -1.0 / 6.0, 5.0 / 6.0, 2.0 / 6.0, 0.0, 0.0},
                           {2.0 / 6.0, -7.0 / 6.0, 11.0 / 6.0, 0.0, 0.0, 0.0},
                           {0.0, 0.0, 2.0 / 6.0, 5.0 / 6.0, -1.0 / 6.0, 0.0},
                           {0.0, 0.0, 3.0 / 12.0, 13.0 / 12.0, -5.0 / 12.0, 1.0 / 12.0}};
  unsigned kept;
  double q[4] = {e.qc, e.ql, e.qr, 0.0};
  const double* dk;
  if constexpr (RC == RC_TENO6) {
    kept = teno6_kept(e, v0, v1, v2, v3, v4, v5);
    q[3] = (3.0 * v2 + 13.0 * v3 - 5.0 * v4 + v5) * (1.0 / 12.0);
    dk = TENO6_D;
  } else {
    kept = teno5_kept(e);
    dk = TENO5_D;
  }
  const double out = teno_combine<K>(q, dk, kept);
  // on a stencil flat to rounding the selection is rounding noise: the
  // derivative is the linear scheme's (every candidate kept), as the
  // oracle's tangent takes it
  {
    double M = fmax(fmax(fabs(v0), fabs(v1)), fmax(fmax(fabs(v2), fabs(v3)), fabs(v4)));
    if constexpr (RC == RC_TENO6) M = fmax(M, fabs(v5));
    const double tol = (WENO_FLAT * M) * (WENO_FLAT * M);
    bool flat = e.bl <= tol && e.bc <= tol && e.br <= tol;
    if constexpr (RC == RC_TENO6) {
      const double e3 = v3 - v2, e4 = v4 - v2, e5 = v5 - v2;
      const double s = 18.0 * e3 - 9.0 * e4 + 2.0 * e5, t = -5.0 * e3 + 4.0 * e4 - e5, u = 3.0 * e3 - 3.0 * e4 + e5;
      const double b4 = (1.0 / 36.0) * s * s + (13.0 / 12.0) * t * t + (781.0 / 720.0) * u * u;
      flat = flat && b4 <= tol;
    }
    if (flat) kept = (1u << K) - 1u;
  }
  double den = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (kept & (1u << k)) den += dk[k];
#pragma unroll
  for (int j = 0; j < 6; ++j) g[j] = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (kept & (1u << k)) {
      const double w = dk[k] / den;
#pragma unroll
      for (int j = 0; j < 6; ++j) g[j] += w * cf[k][j];
    }
  return out;
}

// value and gradient w.r.t. the six stencil values of the interpolation RC
// (left side: cells i-2..i+3; right side: the same cells mirrored)
template <int RC>
__device__ __forceinline__ double recon_val_grad(double v0, double v1, double v2, double v3, double v4, double v5,
                                                 double eps, double* g) {
  if constexpr (RC == RC_WENO5JS) {
    return weno5js_val_grad(v0, v1, v2, v3, v4, g);
  } else if constexpr (RC == RC_TENO5 || RC == RC_TENO6) {
    return teno_val_grad<RC>(v0, v1, v2, v3, v4, v5, g);
  } else {
    const double out = weno_val_grad(v0, v1, v2, v3, v4, eps, g);
    g[5] = 0.0;
    return out;
  }
}

// ---------------------------------------------------------------------------
// Thermodynamic sums at (P, T, Y) shared by the forward EOS, the sound speed
// and their reverse.
template <int NS>
struct Thermo {
  double Y[NS], p, T;
  double r[NS];          // 1 / (P + Pinf_k)
  double v, e, cp, sa, sb, rho, al, be, den, a;
};

template <int NS>
__device__ __forceinline__ void thermo_fwd(const KParams& P, Thermo<NS>& t) {
  t.v = 0.0; t.e = 0.0; t.cp = 0.0; t.sa = 0.0; t.sb = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    t.r[k] = 1.0 / (t.p + P.pinf[k]);
    if (nonzero(t.Y[k])) {
      const double RT = P.Rk[k] * t.T;
      t.v += t.Y[k] * (RT * t.r[k] + P.b[k]);
      t.e += t.Y[k] * (P.cv[k] * t.T * (t.p + P.gam[k] * P.pinf[k]) * t.r[k] + P.q[k]);
      t.cp += t.Y[k] * P.cp[k];
      t.sa += t.Y[k] * P.Rk[k] * t.r[k];
      t.sb += t.Y[k] * RT * t.r[k] * t.r[k];
    }
  }
  t.rho = 1.0 / t.v;
  t.al = t.rho * t.sa;
  t.be = t.rho * t.sb;
  t.den = t.rho * t.be * t.cp - t.al * t.al * t.T;
  t.a = sqrt(t.cp / t.den);
}

// reverse of thermo_fwd: adjoints of (rho, e, a, alpha, beta) -> (Y, P, T)
template <int NS>
__device__ __forceinline__ void thermo_rev(const KParams& P, const Thermo<NS>& t, double lrho, double le, double la,
                                           double lal, double lbe, double* lY, double& lp, double& lT) {
  // a = sqrt(cp / den)
  double lcp = 0.0, lden = 0.0;
  if (nonzero(la)) {
    const double g = la * 0.5 / t.a, iden = 1.0 / t.den;
    lcp += g * iden;
    lden -= g * t.cp * iden * iden;
  }
  // den = rho be cp - al^2 T
  lrho += lden * t.be * t.cp;
  lbe += lden * t.rho * t.cp;
  lcp += lden * t.rho * t.be;
  lal -= lden * 2.0 * t.al * t.T;
  lT -= lden * t.al * t.al;
  // al = rho sa, be = rho sb
  lrho += lal * t.sa + lbe * t.sb;
  const double lsa = lal * t.rho, lsb = lbe * t.rho;
  // rho = 1 / v
  const double lv = -lrho * t.rho * t.rho;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (!nonzero(t.Y[k])) continue;
    const double r = t.r[k], RT = P.Rk[k] * t.T, pg = t.p + P.gam[k] * P.pinf[k];
    const double vk = RT * r + P.b[k];
    const double ek = P.cv[k] * t.T * pg * r + P.q[k];
    lY[k] += lv * vk + le * ek + lcp * P.cp[k] + lsa * P.Rk[k] * r + lsb * RT * r * r;
    const double y = t.Y[k];
    // d/dT
    lT += lv * y * P.Rk[k] * r + le * y * P.cv[k] * pg * r + lsb * y * P.Rk[k] * r * r;
    // d/dP: through pg in ek and through r everywhere
    lp += le * y * P.cv[k] * t.T * r;
    const double lr = lv * y * RT + le * y * P.cv[k] * t.T * pg + lsa * y * P.Rk[k] + lsb * y * RT * 2.0 * r;
    lp -= lr * r * r;
  }
}

// Reverse of the p-T equilibrium (Y, e, v) -> (P, T) by the implicit-function
// theorem of   G1 = T A(P,Y) - (v - b) = 0,   G2 = T B(P,Y) - (e - q) = 0,
// A = sum Y_k R_k / (P + Pinf_k)  (NASG_T2),  B = sum Y_k cv_k (P + g Pinf)/(P + Pinf)  (NASG_T1).
template <int NS>
__device__ __forceinline__ void pt_rev(const KParams& P, const double* Y, double p, double T, const double* r,
                                       double lp, double lT, double* lY, double& le, double& lv) {
  // r[k] = 1 / (P + Pinf_k)
  double A = 0.0, B = 0.0, AP = 0.0, BP = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (!nonzero(Y[k])) continue;
    A += Y[k] * P.Rk[k] * r[k];
    AP -= Y[k] * P.Rk[k] * r[k] * r[k];
    const double g = (p + P.gam[k] * P.pinf[k]) * r[k];
    B += Y[k] * P.cv[k] * g;
    // d/dP of (P + g Pinf)/(P + Pinf) = (Pinf - g Pinf) r^2
    BP += Y[k] * P.cv[k] * (P.pinf[k] - P.gam[k] * P.pinf[k]) * r[k] * r[k];
  }
  // J = [[T AP, A], [T BP, B]] (rows G1, G2; columns P, T); solve J^T mu = (lp, lT)
  const double j11 = T * AP, j12 = A, j21 = T * BP, j22 = B;
  const double idet = 1.0 / (j11 * j22 - j12 * j21);
  // J^T = [[j11, j21], [j12, j22]]
  const double mu1 = (lp * j22 - lT * j21) * idet;
  const double mu2 = (j11 * lT - j12 * lp) * idet;
  // lambda_x = -mu^T dG/dx
  lv += mu1;   // dG1/dv = -1
  le += mu2;   // dG2/de = -1
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (!nonzero(Y[k])) continue;
    const double dG1 = T * P.Rk[k] * r[k] + P.b[k];
    const double dG2 = T * P.cv[k] * (p + P.gam[k] * P.pinf[k]) * r[k] + P.q[k];
    lY[k] -= mu1 * dG1 + mu2 * dG2;
  }
}

// reverse of decode: U -> (rho, Y, u, e, v); adds into lU
template <int NS, int D>
__device__ __forceinline__ void decode_rev(const double* U, double rho, const double* Y, const double* u, double lrho,
                                           const double* lY, const double* lu, double le, double lv, double* lU) {
  // e = E/rho - |u|^2/2, v = 1/rho, u = m/rho, Y = U/rho, rho = sum U_k
  const double ir = 1.0 / rho;
  double lu2[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) lu2[t] = (t < D ? lu[t] : 0.0) - le * u[t];
  lU[NS + D] += le * ir;
  lrho -= (le * U[NS + D] + lv) * ir * ir;
#pragma unroll
  for (int t = 0; t < D; ++t) {
    lU[NS + t] += lu2[t] * ir;
    lrho -= lu2[t] * u[t] * ir;
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    lU[k] += lY[k] * ir;
    lrho -= lY[k] * Y[k] * ir;
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) lU[k] += lrho;
}

// ---------------------------------------------------------------------------
// HLLC (Appendix B), forward with intermediates, and reverse
template <int NS>
struct St {
  double rho, rhoY[NS], u[3], m[3], p, E, a;
};

template <int NS>
struct StAdj {
  double rho, rhoY[NS], u[3], m[3], p, E, a;
  __device__ __forceinline__ void zero() {
    rho = 0.0; p = 0.0; E = 0.0; a = 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k) rhoY[k] = 0.0;
#pragma unroll
    for (int t = 0; t < 3; ++t) { u[t] = 0.0; m[t] = 0.0; }
  }
};

template <int NS, int D>
__device__ __forceinline__ void hllc_rev(int d, const St<NS>& L, const St<NS>& R, const double* lF, StAdj<NS>& gL,
                                         StAdj<NS>& gR) {
  const double ub = 0.5 * (L.u[d] + R.u[d]), ab = 0.5 * (L.a + R.a);
  const bool bl = (ub - ab) <= (L.u[d] - L.a);   // fmin(ub - ab, uL - aL) picks ub - ab
  const double sL = bl ? ub - ab : L.u[d] - L.a;
  const bool br = (ub + ab) >= (R.u[d] + R.a);
  const double sR = br ? ub + ab : R.u[d] + R.a;
  const double sm = fmin(0.0, sL), sp = fmax(0.0, sR);
  const double dL = sL - L.u[d], dR = sR - R.u[d];
  const double num = R.p - L.p + L.rho * L.u[d] * dL - R.rho * R.u[d] * dR;
  const double den = L.rho * dL - R.rho * dR;
  const double ss = num / den;
  const double wl = positive(ss) ? 1.0 : (ss < 0.0 ? 0.0 : 0.5);
  const double wr = 1.0 - wl;
  const double eL = sL - ss, eR = sR - ss;
  const double fL = dL / eL, fR = dR / eR;
  double lsm = 0.0, lsp = 0.0, lfL = 0.0, lfR = 0.0, lss = 0.0, ldL = 0.0, ldR = 0.0;
  // species
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double a = wl * lF[k], b = wr * lF[k];
    gL.rhoY[k] += a * (L.u[d] + sm * (fL - 1.0));
    gL.u[d] += a * L.rhoY[k];
    lsm += a * (fL * L.rhoY[k] - L.rhoY[k]);
    lfL += a * sm * L.rhoY[k];
    gR.rhoY[k] += b * (R.u[d] + sp * (fR - 1.0));
    gR.u[d] += b * R.rhoY[k];
    lsp += b * (fR * R.rhoY[k] - R.rhoY[k]);
    lfR += b * sp * R.rhoY[k];
  }
  // momentum
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const double a = wl * lF[NS + j], b = wr * lF[NS + j];
    // FL = rhoL uLd uLj + (j==d) PL ; UsL = fL rhoL (j==d ? ss : uLj)
    const double vjL = j == d ? ss : L.u[j], vjR = j == d ? ss : R.u[j];
    const double UsL = fL * L.rho * vjL, UsR = fR * R.rho * vjR;
    gL.rho += a * (L.u[d] * L.u[j] + sm * fL * vjL);
    gL.u[d] += a * L.rho * L.u[j];
    gL.u[j] += a * L.rho * L.u[d];
    if (j == d) gL.p += a;
    lsm += a * (UsL - L.m[j]);
    lfL += a * sm * L.rho * vjL;
    if (j == d) lss += a * sm * fL * L.rho;
    else gL.u[j] += a * sm * fL * L.rho;
    gL.m[j] -= a * sm;
    gR.rho += b * (R.u[d] * R.u[j] + sp * fR * vjR);
    gR.u[d] += b * R.rho * R.u[j];
    gR.u[j] += b * R.rho * R.u[d];
    if (j == d) gR.p += b;
    lsp += b * (UsR - R.m[j]);
    lfR += b * sp * R.rho * vjR;
    if (j == d) lss += b * sp * fR * R.rho;
    else gR.u[j] += b * sp * fR * R.rho;
    gR.m[j] -= b * sp;
  }
  // energy: F = u (E + P) + s (f (E + (ss - u)(rho ss + P/dK)) - E)
  {
    const double a = wl * lF[NS + D], b = wr * lF[NS + D];
    const double idL = 1.0 / dL, idR = 1.0 / dR;
    const double kL = L.rho * ss + L.p * idL, kR = R.rho * ss + R.p * idR;
    const double inL = L.E + (ss - L.u[d]) * kL, inR = R.E + (ss - R.u[d]) * kR;
    gL.u[d] += a * (L.E + L.p);
    gL.E += a * (L.u[d] + sm * (fL - 1.0));
    gL.p += a * L.u[d];
    lsm += a * (fL * inL - L.E);
    lfL += a * sm * inL;
    {
      const double g = a * sm * fL;   // adjoint of inL
      lss += g * kL;
      gL.u[d] -= g * kL;
      const double gk = g * (ss - L.u[d]);
      gL.rho += gk * ss;
      lss += gk * L.rho;
      gL.p += gk * idL;
      ldL -= gk * L.p * idL * idL;
    }
    gR.u[d] += b * (R.E + R.p);
    gR.E += b * (R.u[d] + sp * (fR - 1.0));
    gR.p += b * R.u[d];
    lsp += b * (fR * inR - R.E);
    lfR += b * sp * inR;
    {
      const double g = b * sp * fR;
      lss += g * kR;
      gR.u[d] -= g * kR;
      const double gk = g * (ss - R.u[d]);
      gR.rho += gk * ss;
      lss += gk * R.rho;
      gR.p += gk * idR;
      ldR -= gk * R.p * idR * idR;
    }
  }
  // fK = dK / (sK - ss)
  double lsL = 0.0, lsR = 0.0;
  const double ieL = 1.0 / eL, ieR = 1.0 / eR, iden = 1.0 / den;
  ldL += lfL * ieL;
  lsL -= lfL * fL * ieL;
  lss += lfL * fL * ieL;
  ldR += lfR * ieR;
  lsR -= lfR * fR * ieR;
  lss += lfR * fR * ieR;
  // ss = num / den
  const double lnum = lss * iden, lden = -lss * ss * iden;
  gR.p += lnum;
  gL.p -= lnum;
  gL.rho += lnum * L.u[d] * dL + lden * dL;
  gL.u[d] += lnum * L.rho * dL;
  ldL += lnum * L.rho * L.u[d] + lden * L.rho;
  gR.rho -= lnum * R.u[d] * dR + lden * dR;
  gR.u[d] -= lnum * R.rho * dR;
  ldR -= lnum * R.rho * R.u[d] + lden * R.rho;
  // dK = sK - uK
  lsL += ldL;
  gL.u[d] -= ldL;
  lsR += ldR;
  gR.u[d] -= ldR;
  if (sL < 0.0) lsL += lsm;
  if (positive(sR)) lsR += lsp;
  double lub = 0.0, lab = 0.0;
  if (bl) { lub += lsL; lab -= lsL; } else { gL.u[d] += lsL; gL.a -= lsL; }
  if (br) { lub += lsR; lab += lsR; } else { gR.u[d] += lsR; gR.a += lsR; }
  gL.u[d] += 0.5 * lub;
  gR.u[d] += 0.5 * lub;
  gL.a += 0.5 * lab;
  gR.a += 0.5 * lab;
}

// face-side state from (Y, u, P, T) and its reverse (adjoint of the state ->
// adjoints of Y, u, P, T)
template <int NS>
__device__ __forceinline__ void face_state(const KParams& P, Thermo<NS>& t, const double* u, St<NS>& s) {
  thermo_fwd<NS>(P, t);
  double ke = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    s.u[d] = u[d];
    s.m[d] = t.rho * u[d];
    ke += u[d] * u[d];
  }
  s.rho = t.rho;
#pragma unroll
  for (int k = 0; k < NS; ++k) s.rhoY[k] = t.rho * t.Y[k];
  s.p = t.p;
  s.E = t.rho * (t.e + 0.5 * ke);
  s.a = t.a;
}

template <int NS>
__device__ __forceinline__ void face_state_rev(const KParams& P, const Thermo<NS>& t, const St<NS>& s,
                                               const StAdj<NS>& g, double* lY, double* lu, double& lp, double& lT) {
  double ke = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) ke += s.u[d] * s.u[d];
  double lrho = g.rho + g.E * (t.e + 0.5 * ke);
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    lrho += g.rhoY[k] * t.Y[k];
    lY[k] += g.rhoY[k] * t.rho;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lrho += g.m[d] * s.u[d];
    lu[d] += g.u[d] + g.m[d] * t.rho + g.E * t.rho * s.u[d];
  }
  lp += g.p;
  thermo_rev<NS>(P, t, lrho, g.E * t.rho, g.a, 0.0, 0.0, lY, lp, lT);
}

}  // namespace adj
}  // namespace mpmc
