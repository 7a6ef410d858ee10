/*
 * CPU oracle for the four-equation MPMC finite-volume right-hand side
 * (arXiv 2504.14063).  TEST INFRASTRUCTURE ONLY: the product path never
 * loads it.  See mpmc_oracle.h for layouts.
 *
 * Written plainly in the paper's order, in FP64:
 *   conserved -> primitive  : Sec. 2.2-2.3, Eqs. NASG_EOS, NASG_T1, NASG_T2,
 *                             NASG_P; sound speed Eq. SpeedOfSound
 *   face states             : Sec. 3.1.3 (Godunov approach) with the
 *                             characteristic matrices of Appendix A and the
 *                             WENO5-Z interpolation (Borges et al. 2008, the
 *                             scheme the paper uses by default, Sec. 4)
 *   interpolation limiters  : Sec. 3.3.1
 *   HLLC                    : Appendix B
 *   flux limiter            : Sec. 3.3.2
 *   interface regularization: Sec. 3.2, Eqs. InterfaceRegularization,
 *                             psi_transformation, MPMC_ACDI and the KEEP
 *                             split form SkewSymmetricSplitting_Regularization*
 *   species diffusion       : Eq. SpeciesMassDiffusion (third form), D_p^c
 *                             of Sec. 2.2.3, Wilke viscosity of Sec. 2.2.2
 *   time integration        : Eq. SSPRK3 and the CFL condition of Sec. 3.4
 *
 * Readings of passages that are silent, garbled or ambiguous are marked
 * "reading:" where they are used.  Every numeric routine is a template over
 * the scalar type R so that a forward-mode dual number can be substituted.
 */
#include "mpmc_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle_scalar.hpp"

namespace orc {

constexpr int MAXS = ORC_MAXS;
constexpr int MAXV = MAXS + 4;   // conserved variables
constexpr int MAXC = MAXS + 4;   // characteristic variables
constexpr double YTOL = 1e-14;   // round-off allowance on partial densities
constexpr double GTOL = 1e-8;    // |grad psi| below which the interface normal is zero
constexpr double YSUM_TOL = 1e-15;  // per species: |sum Y - 1| treated as rounding
constexpr double WENO_FLAT = 1e-10; // relative stencil variation treated as noise (derivative only)

using std::vector;

/* ------------------------------------------------------------------------ */
/* species constants                                                         */
/* ------------------------------------------------------------------------ */
inline double Rgas(const orc_params& p, int k) { return (p.gamma[k] - 1.0) * p.cv[k]; }
inline double Cp(const orc_params& p, int k) { return p.gamma[k] * p.cv[k]; }

/* Eq. NASG_EOS: specific volume, internal energy and enthalpy of species k */
template <class R> R v_k(const orc_params& p, int k, const R& P, const R& T) {
  return Rgas(p, k) * T / (P + p.pinf[k]) + p.b[k];
}
template <class R> R e_k(const orc_params& p, int k, const R& P, const R& T) {
  return p.cv[k] * T * (P + p.gamma[k] * p.pinf[k]) / (P + p.pinf[k]) + p.q[k];
}
template <class R> R h_k(const orc_params& p, int k, const R& P, const R& T) {
  return Cp(p, k) * T + p.b[k] * P + p.q[k];
}

/* ------------------------------------------------------------------------ */
/* p-T equilibrium: Eqs. NASG_T1, NASG_T2, NASG_P                            */
/* ------------------------------------------------------------------------ */
/* Residual of the common-pressure condition obtained by equating NASG_T1 and
 * NASG_T2 (reading for several stiffened components, where the paper only
 * names an iterative procedure):
 *     f(P) = sum_k Y_k R_k (E' - Pinf_k) / (P + Pinf_k) - C_v,
 *     E' = (e - q) / (v - b).
 * For one stiffened component this is the quadratic of Eq. NASG_P. */
template <class R>
R pt_residual(const orc_params& p, const R* Y, const R& Ep, const R& Cv, const R& P) {
  R f = -Cv;
  for (int k = 0; k < p.ns; ++k)
    if (val(Y[k]) != 0.0) f = f + Y[k] * Rgas(p, k) * (Ep - p.pinf[k]) / (P + p.pinf[k]);
  return f;
}

template <class R>
int pt_equilibrium(const orc_params& p, const R* Y, const R& e, const R& v, R& P, R& T) {
  R Cv(0.0), q(0.0), b(0.0);
  for (int k = 0; k < p.ns; ++k) {
    Cv = Cv + Y[k] * p.cv[k];
    q = q + Y[k] * p.q[k];
    b = b + Y[k] * p.b[k];
  }
  R em = e - q, vm = v - b;
  int st = ORC_OK;
  if (!(val(em) > 0.0) || !(val(vm) > 0.0)) st = ORC_INADMISSIBLE; /* Eq. PositivityReqs1 */
  R Ep = em / vm;
  /* distinct stiffening pressures among the species present */
  double pl = -1.0, pmin = 1e300;
  bool multi = false, gas = false;
  for (int k = 0; k < p.ns; ++k) {
    if (!(val(Y[k]) > 0.0)) continue;
    pmin = std::min(pmin, p.pinf[k]);
    if (p.pinf[k] > 0.0) {
      if (pl < 0.0) pl = p.pinf[k];
      else if (p.pinf[k] != pl) multi = true;
    } else {
      gas = true;
    }
  }
  if (!multi && !p.eos_iterative) {
    R Rg(0.0), Rl(0.0);
    for (int k = 0; k < p.ns; ++k) {
      if (!(val(Y[k]) > 0.0)) continue;
      if (p.pinf[k] > 0.0) Rl = Rl + Y[k] * Rgas(p, k);
      else Rg = Rg + Y[k] * Rgas(p, k);
    }
    if (pl < 0.0) {
      /* no stiffened component: a3 = 0 and P = a2 / a1 */
      P = Ep * Rg / Cv;
    } else if (!gas) {
      /* reading: without gas a3 = 0 and the root is the linear one, a2/a1,
       * which may be negative (tension is admissible, Sec. 3.3) */
      P = (Ep * Rl - pl * Cv - pl * Rl) / Cv;
    } else {
      /* Eq. NASG_P, a1 = C_v, a2, a3 as printed; the larger root, written
       * without cancellation when a2 < 0 */
      R a1 = Cv;
      R a2 = Ep * (Rg + Rl) - pl * Cv - pl * Rl;
      R a3 = Ep * pl * Rg;
      R sq = sqrt(a2 * a2 + 4.0 * a1 * a3);
      if (val(a2) >= 0.0) P = (a2 + sq) / (2.0 * a1);
      else P = 2.0 * a3 / (sq - a2);
    }
  } else {
    /* bisection to the last ulp on (-min Pinf, inf) */
    const double lo0 = -pmin;
    double lo = lo0;
    double hi = std::max(std::fabs(val(Ep)), 1.0) + std::fabs(lo0);
    double Epv = val(Ep), Cvv = val(Cv);
    double Yv[MAXS];
    for (int k = 0; k < p.ns; ++k) Yv[k] = val(Y[k]);
    int it = 0;
    while (pt_residual<double>(p, Yv, Epv, Cvv, hi) >= 0.0 && it < 2100) { hi *= 2.0; ++it; }
    if (it >= 2100) st = ORC_EOS_NO_CONVERGE;
    for (it = 0; it < 2200; ++it) {
      double mid = lo + 0.5 * (hi - lo);
      if (!(mid > lo) || !(mid < hi)) break;
      if (pt_residual<double>(p, Yv, Epv, Cvv, mid) > 0.0) lo = mid;
      else hi = mid;
    }
    double P0;
    if (lo == lo0) P0 = hi;
    else P0 = std::fabs(pt_residual<double>(p, Yv, Epv, Cvv, lo)) <
                      std::fabs(pt_residual<double>(p, Yv, Epv, Cvv, hi))
                  ? lo
                  : hi;
    P = R(P0);
    if (is_dual<R>::value) {
      /* derivative of the root by the implicit-function theorem: one Newton
       * step taken in R arithmetic from the converged value */
      R f = pt_residual<R>(p, Y, Ep, Cv, P);
      R dfdP(0.0);
      for (int k = 0; k < p.ns; ++k)
        if (Yv[k] != 0.0) {
          double den = P0 + p.pinf[k];
          dfdP = dfdP - Y[k] * Rgas(p, k) * (Ep - p.pinf[k]) / (den * den);
        }
      P = P - f / R(val(dfdP));
    }
  }
  /* Eq. NASG_T1 (reading: T1 is used; species absent from the cell skipped) */
  R den(0.0);
  for (int k = 0; k < p.ns; ++k)
    if (val(Y[k]) != 0.0)
      den = den + Y[k] * p.cv[k] * (P + p.gamma[k] * p.pinf[k]) / (P + p.pinf[k]);
  T = em / den;
  return st;
}

/* forward EOS at (P, T, Y): density (Amagat), internal energy, and the
 * sound speed of Eq. SpeedOfSound with alpha, beta of the NASG EOS */
template <class R>
void eos_forward(const orc_params& p, const R* Y, const R& P, const R& T, R& rho, R& e, R& a,
                 R& alpha, R& beta, R& cp) {
  R v(0.0);
  e = R(0.0);
  cp = R(0.0);
  R sa(0.0), sb(0.0);
  for (int k = 0; k < p.ns; ++k) {
    if (val(Y[k]) == 0.0) continue;
    v = v + Y[k] * v_k(p, k, P, T);
    e = e + Y[k] * e_k(p, k, P, T);
    cp = cp + Y[k] * Cp(p, k);
    R pp = P + p.pinf[k];
    sa = sa + Y[k] * Rgas(p, k) / pp;
    sb = sb + Y[k] * Rgas(p, k) * T / (pp * pp);
  }
  rho = 1.0 / v;
  alpha = rho * sa;
  beta = rho * sb;
  R a2 = cp / (rho * beta * cp - alpha * alpha * T);
  a = sqrt(a2);
}

/* ------------------------------------------------------------------------ */
/* per-cell state                                                            */
/* ------------------------------------------------------------------------ */
template <class R>
struct Cell {
  /* conserved */
  R rhoY[MAXS], m[3], E;
  /* primitive and thermodynamic */
  R rho, Y[MAXS], u[3], e, P, T, a;
  /* interface regularization: phase volume fraction, psi, (Y^c/Y_p) rho_p, h_p rho_p */
  R phi[2], psi, yrho[MAXS], hrho[2];
  bool present[2];
  /* diffusion: X^c/X_p, W^c D^c_p / W_p, h^c; mixture viscosity and heat
   * conductivity */
  R xr[MAXS], B[MAXS], h[MAXS], mu, lam;
  int status;
};

struct Geom {
  int dim, n[3], g[3], N[3];
  size_t npad, ncell;
  explicit Geom(const orc_params& p) {
    dim = p.dim;
    for (int d = 0; d < 3; ++d) {
      n[d] = d < dim ? p.n[d] : 1;
      g[d] = d < dim ? 3 : 0;
      N[d] = n[d] + 2 * g[d];
    }
    npad = (size_t)N[0] * N[1] * N[2];
    ncell = (size_t)n[0] * n[1] * n[2];
  }
  size_t pad(int i, int j, int k) const {
    return ((size_t)(k + g[2]) * N[1] + (size_t)(j + g[1])) * N[0] + (size_t)(i + g[0]);
  }
  size_t cell(int i, int j, int k) const { return ((size_t)k * n[1] + j) * n[0] + i; }
  long stride(int d) const { return d == 0 ? 1 : (d == 1 ? (long)N[0] : (long)N[0] * N[1]); }
  /* faces of direction d: n[d]+1 along d */
  size_t nface(int d) const {
    size_t s = 1;
    for (int e = 0; e < 3; ++e) s *= (size_t)(n[e] + (e == d ? 1 : 0));
    return s;
  }
  size_t face(int d, int i, int j, int k) const { /* i, j, k: face-local indices */
    int f0 = n[0] + (d == 0), f1 = n[1] + (d == 1);
    return ((size_t)k * f1 + j) * f0 + i;
  }
};

/* mixture quantities of one cell from its conserved vector (Sec. 2.2, 2.3,
 * Appendix E mixing identities) */
template <class R>
void cell_from_conserved(const orc_params& p, int D, const R* U, Cell<R>& c) {
  const int ns = p.ns;
  c.status = ORC_OK;
  c.rho = R(0.0);
  for (int k = 0; k < ns; ++k) {
    c.rhoY[k] = U[k];
    c.rho = c.rho + U[k];
  }
  /* Eq. PositivityReqs2 (reading: partial densities >= -YTOL rho) */
  for (int k = 0; k < ns; ++k)
    if (val(U[k]) < -YTOL * val(c.rho)) c.status = ORC_INADMISSIBLE;
  for (int d = 0; d < 3; ++d) c.m[d] = R(0.0);
  for (int d = 0; d < D; ++d) c.m[d] = U[ns + d];
  c.E = U[ns + D];
  if (!(val(c.rho) > 0.0)) c.status = ORC_INADMISSIBLE;
  for (int k = 0; k < ns; ++k) c.Y[k] = c.rhoY[k] / c.rho;
  R ke(0.0);
  for (int d = 0; d < 3; ++d) {
    c.u[d] = c.m[d] / c.rho;
    ke = ke + c.u[d] * c.u[d];
  }
  /* reading: e is the specific internal energy, E = rho e + rho |u|^2 / 2 */
  c.e = c.E / c.rho - 0.5 * ke;
  R v = 1.0 / c.rho;
  int st = pt_equilibrium(p, c.Y, c.e, v, c.P, c.T);
  if (st != ORC_OK && c.status == ORC_OK) c.status = st;
  R rho2, e2, alpha, beta, cp;
  eos_forward(p, c.Y, c.P, c.T, rho2, e2, c.a, alpha, beta, cp);

  /* phase volume fractions, psi transform, KEEP face quantities */
  for (int ph = 0; ph < 2; ++ph) {
    R phi(0.0), Yp(0.0), hr(0.0);
    for (int k = 0; k < ns; ++k)
      if (p.phase[k] == ph) {
        Yp = Yp + c.Y[k];
        if (val(c.rhoY[k]) != 0.0) {
          phi = phi + c.rhoY[k] * v_k(p, k, c.P, c.T);
          hr = hr + c.rhoY[k] * h_k(p, k, c.P, c.T);
        }
      }
    c.phi[ph] = phi;
    /* reading: ratios over an absent phase are zero */
    bool present = val(Yp) >= 1e-300;
    c.present[ph] = present;
    c.hrho[ph] = present ? hr / phi : R(0.0);
    for (int k = 0; k < ns; ++k)
      if (p.phase[k] == ph) c.yrho[k] = present ? c.rhoY[k] / phi : R(0.0);
  }

  /* Eq. psi_transformation for phase 0.  reading: 1 - phi_0 is written as
   * phi_1 (equal by the mixing identities of Appendix E), which keeps full
   * precision where either fraction is tiny */
  c.psi = p.cdi_eps * log((c.phi[0] + p.psi_delta) / (c.phi[1] + p.psi_delta));

  /* phase viscosities: constant in the liquid, Wilke's rule in the gas
   * (reading: the standard rule written in mass fractions) */
  R mu_p[2];
  mu_p[0] = R(p.mu_liquid);
  {
    R num(0.0), Yg(0.0);
    R den_i[MAXS];
    for (int i = 0; i < ns; ++i) {
      den_i[i] = R(0.0);
      if (p.phase[i] != 1) continue;
      Yg = Yg + c.Y[i];
      for (int j = 0; j < ns; ++j) {
        if (p.phase[j] != 1) continue;
        double Wij = p.W[i] / p.W[j];
        double t = 1.0 + std::sqrt(p.mu[i] / p.mu[j]) * std::pow(p.W[j] / p.W[i], 0.25);
        double Phi = t * t / (std::sqrt(8.0) * std::sqrt(1.0 + Wij));
        den_i[i] = den_i[i] + c.Y[j] * Wij * Phi;
      }
    }
    for (int i = 0; i < ns; ++i)
      if (p.phase[i] == 1 && val(den_i[i]) > 0.0) num = num + c.Y[i] * p.mu[i] / den_i[i];
    mu_p[1] = val(Yg) >= 1e-300 ? num : R(0.0);
  }
  /* mixture viscosity mu = sum_p phi_p mu_p (Sec. 2.2.2) */
  c.mu = c.phi[0] * mu_p[0] + c.phi[1] * mu_p[1];
  /* mixture heat conductivity lambda = sum_p phi_p lambda_p: constant in the
   * liquid, lambda_g = (mu_g / Pr) sum_{c in gas} (Y^c / Y_g) Cp^c (Sec. 2.2.2) */
  {
    R Yg(0.0), cpY(0.0);
    for (int k = 0; k < ns; ++k)
      if (p.phase[k] == 1) {
        Yg = Yg + c.Y[k];
        cpY = cpY + c.Y[k] * Cp(p, k);
      }
    R lam_g = val(Yg) >= 1e-300 ? mu_p[1] / p.prandtl * (cpY / Yg) : R(0.0);
    c.lam = c.phi[0] * p.lambda_liquid + c.phi[1] * lam_g;
  }

  /* species diffusion ingredients (Eq. SpeciesMassDiffusion, third form):
   *   X^c/X_p = (Y^c/W^c) / sum_{j in p} Y^j/W^j,
   *   W^c/W_p = W^c sum_{j in p} (Y^j/Y_p)/W^j,
   *   D^c_p  = mu_p / (rho_p Sc^c_p),  rho_p = rho Y_p / phi_p  */
  for (int ph = 0; ph < 2; ++ph) {
    R sY(0.0), Yp(0.0);
    for (int j = 0; j < ns; ++j)
      if (p.phase[j] == ph) {
        sY = sY + c.Y[j] / p.W[j];
        Yp = Yp + c.Y[j];
      }
    bool present = val(Yp) >= 1e-300 && val(sY) >= 1e-300;
    for (int k = 0; k < ns; ++k) {
      if (p.phase[k] != ph) continue;
      if (!present) {
        c.xr[k] = R(0.0);
        c.B[k] = R(0.0);
        continue;
      }
      c.xr[k] = (c.Y[k] / p.W[k]) / sY;
      R WcWp = p.W[k] * sY / Yp;
      R rho_p = c.rho * Yp / c.phi[ph];
      R Dk = mu_p[ph] / (rho_p * p.Sc[k]);
      c.B[k] = WcWp * Dk;
    }
  }
  for (int k = 0; k < ns; ++k) c.h[k] = h_k(p, k, c.P, c.T);
}

/* ------------------------------------------------------------------------ */
/* WENO5-Z (Borges et al. 2008): value at the right face of the middle cell  */
/* of the five-cell stencil v0..v4                                            */
/* ------------------------------------------------------------------------ */
template <class R>
R weno5z(const R& v0, const R& v1, const R& v2, const R& v3, const R& v4, double eps) {
  R q0 = (2.0 * v0 - 7.0 * v1 + 11.0 * v2) / 6.0;
  R q1 = (-v1 + 5.0 * v2 + 2.0 * v3) / 6.0;
  R q2 = (2.0 * v2 + 5.0 * v3 - v4) / 6.0;
  R t;
  t = v0 - 2.0 * v1 + v2;
  R s0 = v0 - 4.0 * v1 + 3.0 * v2;
  R b0 = (13.0 / 12.0) * t * t + 0.25 * s0 * s0;
  t = v1 - 2.0 * v2 + v3;
  R s1 = v1 - v3;
  R b1 = (13.0 / 12.0) * t * t + 0.25 * s1 * s1;
  t = v2 - 2.0 * v3 + v4;
  R s2 = 3.0 * v2 - 4.0 * v3 + v4;
  R b2 = (13.0 / 12.0) * t * t + 0.25 * s2 * s2;
  R tau5 = fabs(b0 - b2);
  /* reading: exponent q = 1 */
  R a0 = 0.1 * (1.0 + tau5 / (b0 + eps));
  R a1 = 0.6 * (1.0 + tau5 / (b1 + eps));
  R a2 = 0.3 * (1.0 + tau5 / (b2 + eps));
  R out = (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
  if (is_dual<R>::value) {
    /* reading (derivative only): on a stencil flat to rounding (every
     * smoothness indicator below (WENO_FLAT max|v|)^2) the weights are
     * ratios of rounding errors whose derivative grows like 1/eps, while
     * the value is each candidate to rounding; the tangent there is taken
     * with the ideal weights (the linear fifth-order scheme). */
    double M = 0.0;
    const double vv[5] = {val(v0), val(v1), val(v2), val(v3), val(v4)};
    for (int j = 0; j < 5; ++j) M = std::max(M, std::fabs(vv[j]));
    const double tol = (WENO_FLAT * M) * (WENO_FLAT * M);
    if (val(b0) <= tol && val(b1) <= tol && val(b2) <= tol) {
      R lin = 0.1 * q0 + 0.6 * q1 + 0.3 * q2;
      return with_value(lin, val(out));
    }
  }
  return out;
}

/* ------------------------------------------------------------------------ */
/* The other ENO-type interpolations the paper runs beside WENO5-Z (Sec. 4.1 */
/* gas-liquid Riemann problem, Table DropAdvectionIECResults, Shu-Osher and  */
/* 2D Riemann problems): WENO5-JS (Jiang & Shu 1996), TENO5 and TENO6 (Fu,   */
/* Hu & Adams 2016).  The paper cites them without restating them; these    */
/* follow the cited definitions.  v[0..5] are the cells i-2..i+3 of a value */
/* at the right face of cell i (TENO6 alone reads v[5]).                    */
/* ------------------------------------------------------------------------ */

/* Candidate polynomial of the stencil of n cells starting at offset o
 * (cell i is [0,1], cell c is [c, c+1]) from its cell averages, taken as
 * deviations from cell i (a constant changes neither the smoothness
 * indicator nor the deviation of the value): a_k of p(x) = sum a_k x^k solve
 * sum_k a_k int_c^{c+1} x^k dx = v_c - v_i.  The moment matrix depends on
 * (o, n) alone; its inverse is formed once, by Gauss-Jordan elimination
 * with partial pivoting, for every stencil inside i-2..i+3. */
struct MomentInverses {
  double inv[3][7][6][6];  /* [o + 2][n][row][col] */
  MomentInverses() {
    for (int o = -2; o <= 0; ++o)
      for (int n = 1; n <= 6; ++n) {
        if (o + n - 1 > 3) continue;
        double A[6][12];
        for (int r = 0; r < n; ++r) {
          const double c = o + r;
          for (int k = 0; k < n; ++k) A[r][k] = (std::pow(c + 1.0, k + 1) - std::pow(c, k + 1)) / (k + 1);
          for (int k = 0; k < n; ++k) A[r][n + k] = r == k ? 1.0 : 0.0;
        }
        for (int col = 0; col < n; ++col) {
          int piv = col;
          for (int r = col + 1; r < n; ++r)
            if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
          for (int k = 0; k < 2 * n; ++k) std::swap(A[piv][k], A[col][k]);
          const double pv = A[col][col];
          for (int k = 0; k < 2 * n; ++k) A[col][k] /= pv;
          for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = A[r][col];
            for (int k = 0; k < 2 * n; ++k) A[r][k] -= f * A[col][k];
          }
        }
        for (int r = 0; r < n; ++r)
          for (int k = 0; k < n; ++k) inv[o + 2][n][r][k] = A[r][n + k];
      }
  }
};

template <class R>
void candidate_poly(const R* v, int o, int n, R* a) {
  static const MomentInverses M;
  const double(*Ai)[6] = M.inv[o + 2][n];
  for (int k = 0; k < n; ++k) {
    R s(0.0);
    for (int r = 0; r < n; ++r) s = s + Ai[k][r] * (v[2 + o + r] - v[2]);
    a[k] = s;
  }
}

/* Jiang-Shu smoothness indicator of a candidate polynomial on cell i:
 * sum_{l=1}^{n-1} int_0^1 (d^l p / dx^l)^2 dx (unit cell width) */
template <class R>
R jiang_shu_beta(const R* a, int n) {
  R beta(0.0);
  for (int l = 1; l < n; ++l) {
    R c[6];
    int m = 0;
    for (int k = l; k < n; ++k) {
      double f = 1.0;
      for (int j = 0; j < l; ++j) f *= (k - j);
      c[m++] = f * a[k];  /* coefficient of x^(k-l) */
    }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) beta = beta + c[i] * c[j] / (double)(i + j + 1);
  }
  return beta;
}

/* value at x = 1 (the right face of cell i) */
template <class R>
R poly_at_one(const R& vi, const R* a, int n) {
  R s = vi;
  for (int k = 0; k < n; ++k) s = s + a[k];
  return s;
}

/* WENO5-JS: the WENO5 candidates and indicators, alpha_k = d_k / (eps + beta_k)^2
 * (reading: eps = 1e-6 and exponent 2, the values of Jiang & Shu) */
template <class R>
R weno5js(const R* v) {
  const double eps = 1e-6;
  R q0 = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
  R q1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
  R q2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
  R t = v[0] - 2.0 * v[1] + v[2], s = v[0] - 4.0 * v[1] + 3.0 * v[2];
  R b0 = (13.0 / 12.0) * t * t + 0.25 * s * s;
  t = v[1] - 2.0 * v[2] + v[3];
  s = v[1] - v[3];
  R b1 = (13.0 / 12.0) * t * t + 0.25 * s * s;
  t = v[2] - 2.0 * v[3] + v[4];
  s = 3.0 * v[2] - 4.0 * v[3] + v[4];
  R b2 = (13.0 / 12.0) * t * t + 0.25 * s * s;
  R a0 = 0.1 / ((eps + b0) * (eps + b0));
  R a1 = 0.6 / ((eps + b1) * (eps + b1));
  R a2 = 0.3 / ((eps + b2) * (eps + b2));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/* TENO selection: gamma_k = (C + tau / (beta_k + eps))^q with C = 1, q = 6,
 * eps = 1e-40; chi_k = gamma_k / sum gamma; a candidate is kept when
 * chi_k >= CT; the kept candidates combine with their optimal weights
 * renormalized.  (Reading: chi_k is formed from (r_k / max r)^6, the same
 * ratio, because r_k^6 overflows FP64 when a stencil is exactly flat beside
 * a jump.) */
template <class R>
R teno_select(int K, const R* q, const R* beta, const double* d, const R& tau, double CT) {
  const double eps = 1e-40;
  R r[4];
  double rmax = 0.0;
  for (int k = 0; k < K; ++k) {
    r[k] = 1.0 + tau / (beta[k] + eps);
    rmax = std::max(rmax, val(r[k]));
  }
  double g[4], gs = 0.0;
  for (int k = 0; k < K; ++k) {
    const double x = val(r[k]) / rmax;
    const double x2 = x * x;
    g[k] = x2 * x2 * x2;
    gs += g[k];
  }
  R num(0.0);
  double den = 0.0;
  for (int k = 0; k < K; ++k)
    if (!(g[k] < CT * gs)) {
      num = num + d[k] * q[k];
      den += d[k];
    }
  return num / den;
}

/* reading (derivative only, as for WENO5-Z): on a stencil flat to rounding
 * (every indicator below (WENO_FLAT max|v|)^2) the candidates TENO keeps are
 * chosen by rounding noise while every candidate is the value to rounding;
 * the tangent there is that of the linear scheme (all candidates kept) */
template <class R>
R teno_flat_tangent(const R* v, int nv, int K, const R* q, const R* beta, const double* d, const R& out) {
  if (!is_dual<R>::value) return out;
  double M = 0.0;
  for (int j = 0; j < nv; ++j) M = std::max(M, std::fabs(val(v[j])));
  const double tol = (WENO_FLAT * M) * (WENO_FLAT * M);
  for (int k = 0; k < K; ++k)
    if (val(beta[k]) > tol) return out;
  R lin(0.0);
  for (int k = 0; k < K; ++k) lin = lin + d[k] * q[k];
  return with_value(lin, val(out));
}

/* TENO5: candidates central (i-1..i+1), left (i-2..i), right (i..i+2) with
 * optimal weights (3/5, 1/10, 3/10); tau5 = |beta_left - beta_right|;
 * reading: CT = 1e-5 */
template <class R>
R teno5(const R* v) {
  const R ql = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
  const R qc = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
  const R qr = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
  R t = v[0] - 2.0 * v[1] + v[2], s = v[0] - 4.0 * v[1] + 3.0 * v[2];
  const R bl = (13.0 / 12.0) * t * t + 0.25 * s * s;
  t = v[1] - 2.0 * v[2] + v[3];
  s = v[1] - v[3];
  const R bc = (13.0 / 12.0) * t * t + 0.25 * s * s;
  t = v[2] - 2.0 * v[3] + v[4];
  s = 3.0 * v[2] - 4.0 * v[3] + v[4];
  const R br = (13.0 / 12.0) * t * t + 0.25 * s * s;
  const R q[3] = {qc, ql, qr}, beta[3] = {bc, bl, br};
  const double d[3] = {0.6, 0.1, 0.3};
  const R out = teno_select(3, q, beta, d, fabs(bl - br), 1e-5);
  return teno_flat_tangent(v, 5, 3, q, beta, d, out);
}

/* TENO6: TENO5's three candidates plus the four-cell right candidate
 * (i..i+3), optimal weights (9/20, 1/20, 3/10, 1/5) reproducing the six-cell
 * interpolation; tau6 = |beta6 - (beta_left + beta_right + 4 beta_central) / 6|
 * with beta6 the indicator of the six-cell polynomial (the combination that
 * vanishes to O(dx^6) on smooth data); reading: CT = 1e-7.  The new
 * candidate and both new indicators come from the definitions above. */
template <class R>
R teno6(const R* v) {
  R a4[6], a6[6];
  candidate_poly(v, 0, 4, a4);
  candidate_poly(v, -2, 6, a6);
  const R ql = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
  const R qc = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
  const R qr = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
  const R q4 = poly_at_one(v[2], a4, 4);
  R t = v[0] - 2.0 * v[1] + v[2], s = v[0] - 4.0 * v[1] + 3.0 * v[2];
  const R bl = (13.0 / 12.0) * t * t + 0.25 * s * s;
  t = v[1] - 2.0 * v[2] + v[3];
  s = v[1] - v[3];
  const R bc = (13.0 / 12.0) * t * t + 0.25 * s * s;
  t = v[2] - 2.0 * v[3] + v[4];
  s = 3.0 * v[2] - 4.0 * v[3] + v[4];
  const R br = (13.0 / 12.0) * t * t + 0.25 * s * s;
  const R b4 = jiang_shu_beta(a4, 4);
  const R b6 = jiang_shu_beta(a6, 6);
  const R q[4] = {qc, ql, qr, q4}, beta[4] = {bc, bl, br, b4};
  const double d[4] = {0.45, 0.05, 0.3, 0.2};
  const R out = teno_select(4, q, beta, d, fabs(b6 - (bl + br + 4.0 * bc) / 6.0), 1e-7);
  return teno_flat_tangent(v, 6, 4, q, beta, d, out);
}

/* the interpolation the model selects (ORC_RECON_*) */
template <class R>
R reconstruct(int kind, const R* v, double eps) {
  switch (kind) {
    case 1: return weno5js(v);
    case 2: return teno5(v);
    case 3: return teno6(v);
    default: return weno5z(v[0], v[1], v[2], v[3], v[4], eps);
  }
}

/* ------------------------------------------------------------------------ */
/* characteristic matrices, Appendix A                                       */
/* ------------------------------------------------------------------------ */
/* Ordering.  W  = [T, Y_0..Y_{ns-2}, u_0..u_{D-1}, P]                        */
/*            W~ = [w1, Y_0..Y_{ns-2}, tangential velocities, w5, w6]         */
/* (reading: the species left out of the projection is the last one)        */
template <class R>
void char_matrices(int ns, int D, int d, const R& X, const R& rhoa, R* Sinv, R* S) {
  const int nc = ns + D + 1;
  for (int i = 0; i < nc * nc; ++i) {
    Sinv[i] = R(0.0);
    S[i] = R(0.0);
  }
  const int iT = 0, iY0 = 1, iu0 = ns, iP = ns + D;
  const int i5 = nc - 2, i6 = nc - 1;
  /* S^{-1}: w1 = T - X P */
  Sinv[0 * nc + iT] = R(1.0);
  Sinv[0 * nc + iP] = -X;
  /* mass fractions: identity */
  for (int k = 0; k < ns - 1; ++k) Sinv[(iY0 + k) * nc + iY0 + k] = R(1.0);
  /* tangential velocities */
  int row = ns;
  for (int t = 0; t < D; ++t) {
    if (t == d) continue;
    Sinv[row * nc + iu0 + t] = R(1.0);
    ++row;
  }
  /* acoustic pair */
  Sinv[i5 * nc + iu0 + d] = 0.5 * rhoa;
  Sinv[i5 * nc + iP] = R(0.5);
  Sinv[i6 * nc + iu0 + d] = -0.5 * rhoa;
  Sinv[i6 * nc + iP] = R(0.5);

  /* S */
  S[iT * nc + 0] = R(1.0);
  S[iT * nc + i5] = X;
  S[iT * nc + i6] = X;
  for (int k = 0; k < ns - 1; ++k) S[(iY0 + k) * nc + iY0 + k] = R(1.0);
  row = ns;
  for (int t = 0; t < D; ++t) {
    if (t == d) continue;
    S[(iu0 + t) * nc + row] = R(1.0);
    ++row;
  }
  S[(iu0 + d) * nc + i5] = 1.0 / rhoa;
  S[(iu0 + d) * nc + i6] = -1.0 / rhoa;
  S[iP * nc + i5] = R(1.0);
  S[iP * nc + i6] = R(1.0);
}

/* scalars of the characteristic matrices at a conserved state */
template <class R>
int char_scalars(const orc_params& p, int D, const R* U, R& rho, R& a, R& alpha, R& beta, R& X,
                 R& rhoa) {
  Cell<R> c;
  cell_from_conserved(p, D, U, c);
  R rho2, e2, cp;
  eos_forward(p, c.Y, c.P, c.T, rho2, e2, a, alpha, beta, cp);
  rho = c.rho;
  /* X = (rho a^2 beta - 1) / (alpha a^2 rho), Appendix A */
  X = (rho * a * a * beta - 1.0) / (alpha * a * a * rho);
  rhoa = a * rho;
  return c.status;
}

/* ------------------------------------------------------------------------ */
/* HLLC, Appendix B                                                          */
/* ------------------------------------------------------------------------ */
template <class R>
struct State {
  R rho, rhoY[MAXS], u[3], m[3], P, E, a;
};

template <class R>
void physical_flux(int ns, int D, int d, const State<R>& s, R* F) {
  for (int k = 0; k < ns; ++k) F[k] = s.rhoY[k] * s.u[d];
  /* reading: the mass row of H is rho Y w */
  for (int j = 0; j < D; ++j) F[ns + j] = s.rho * s.u[d] * s.u[j] + (j == d ? s.P : R(0.0));
  F[ns + D] = s.u[d] * (s.E + s.P);
}

template <class R>
void conserved_of(int ns, int D, const State<R>& s, R* U) {
  for (int k = 0; k < ns; ++k) U[k] = s.rhoY[k];
  for (int j = 0; j < D; ++j) U[ns + j] = s.m[j];
  U[ns + D] = s.E;
}

template <class R>
void star_state(int ns, int D, int d, const State<R>& s, const R& sK, const R& ss, R* Us) {
  R fac = (sK - s.u[d]) / (sK - ss);
  for (int k = 0; k < ns; ++k) Us[k] = fac * s.rhoY[k];
  for (int j = 0; j < D; ++j) Us[ns + j] = fac * s.rho * (j == d ? ss : s.u[j]);
  Us[ns + D] = fac * (s.E + (ss - s.u[d]) * (s.rho * ss + s.P / (sK - s.u[d])));
}

template <class R>
void hllc(int ns, int D, int d, const State<R>& L, const State<R>& Rr, R* F) {
  const int nv = ns + D + 1;
  /* reading: the averages in the wave-speed estimates are arithmetic
   * averages of the two face states */
  R ub = 0.5 * (L.u[d] + Rr.u[d]);
  R ab = 0.5 * (L.a + Rr.a);
  R sL = rmin(ub - ab, L.u[d] - L.a);
  R sR = rmax(ub + ab, Rr.u[d] + Rr.a);
  R sm = rmin(R(0.0), sL);
  R sp = rmax(R(0.0), sR);
  R ss = (Rr.P - L.P + L.rho * L.u[d] * (sL - L.u[d]) - Rr.rho * Rr.u[d] * (sR - Rr.u[d])) /
         (L.rho * (sL - L.u[d]) - Rr.rho * (sR - Rr.u[d]));
  R FL[MAXV], FR[MAXV], UL[MAXV], UR[MAXV], UsL[MAXV], UsR[MAXV];
  physical_flux(ns, D, d, L, FL);
  physical_flux(ns, D, d, Rr, FR);
  conserved_of(ns, D, L, UL);
  conserved_of(ns, D, Rr, UR);
  star_state(ns, D, d, L, sL, ss, UsL);
  star_state(ns, D, d, Rr, sR, ss, UsR);
  /* reading: sign(0) = 0 */
  double sg = val(ss) > 0.0 ? 1.0 : (val(ss) < 0.0 ? -1.0 : 0.0);
  for (int v = 0; v < nv; ++v)
    F[v] = 0.5 * (1.0 + sg) * (FL[v] + sm * (UsL[v] - UL[v])) +
           0.5 * (1.0 - sg) * (FR[v] + sp * (UsR[v] - UR[v]));
}

/* State of a reconstructed face side from (Y, u, P, T): steps 4-5 of the
 * Godunov approach (Sec. 3.1.3) */
template <class R>
void state_from_primitive(const orc_params& p, int D, const R* Y, const R* u, const R& P, const R& T,
                          State<R>& s) {
  R e, alpha, beta, cp;
  eos_forward(p, Y, P, T, s.rho, e, s.a, alpha, beta, cp);
  R ke(0.0);
  for (int d = 0; d < 3; ++d) {
    s.u[d] = u[d];
    s.m[d] = s.rho * u[d];
    ke = ke + u[d] * u[d];
  }
  for (int k = 0; k < p.ns; ++k) s.rhoY[k] = s.rho * Y[k];
  s.P = P;
  s.E = s.rho * (e + 0.5 * ke);
  (void)D;
}

template <class R>
void state_from_cell(int ns, const Cell<R>& c, State<R>& s) {
  s.rho = c.rho;
  for (int k = 0; k < ns; ++k) s.rhoY[k] = c.rhoY[k];
  for (int d = 0; d < 3; ++d) {
    s.u[d] = c.u[d];
    s.m[d] = c.m[d];
  }
  s.P = c.P;
  s.E = c.E;
  s.a = c.a;
}

/* admissible conserved state: Eqs. PositivityReqs1, PositivityReqs2 checked
 * on U alone (Sec. 3.3.2).  reading: partial densities >= -YTOL rho, so that
 * a rounding-level negative left by the final RK combination does not fail
 * every later pseudo-update of its cell */
template <class R>
bool admissible(const orc_params& p, int D, const R* U) {
  const int ns = p.ns;
  R rho(0.0), sb(0.0), sq(0.0);
  for (int k = 0; k < ns; ++k) {
    rho = rho + U[k];
    sb = sb + U[k] * p.b[k];
    sq = sq + U[k] * p.q[k];
  }
  if (!(val(rho) > 0.0)) return false;
  for (int k = 0; k < ns; ++k)
    if (!(val(U[k]) >= -YTOL * val(rho))) return false;
  /* rho (v - b) = 1 - sum rhoY_k b_k */
  if (!(val(1.0 - sb) > 0.0)) return false;
  /* rho (e - q) = E - |m|^2 / (2 rho) - sum rhoY_k q_k */
  R mm(0.0);
  for (int d = 0; d < D; ++d) mm = mm + U[ns + d] * U[ns + d];
  R rem = U[ns + D] - 0.5 * mm / rho - sq;
  return val(rem) > 0.0;
}

/* ------------------------------------------------------------------------ */
/* solver                                                                   */
/* ------------------------------------------------------------------------ */
template <class R>
struct Solver {
  const orc_params& p;
  Geom G;
  int ns, D, nv, nc;
  vector<R> Unp, Ukp;       /* padded conserved arrays [nv][npad] */
  vector<Cell<R>> cells;    /* padded */
  R Uin[MAXV];              /* conserved inflow state */

  explicit Solver(const orc_params& pp) : p(pp), G(pp) {
    ns = p.ns;
    D = p.dim;
    nv = ns + D + 1;
    nc = ns + D + 1;
    Unp.assign((size_t)nv * G.npad, R(0.0));
    Ukp.assign((size_t)nv * G.npad, R(0.0));
    cells.resize(G.npad);
    conserved_from_primitive(p.inflow, Uin);
  }

  /* init: rhoY_k = alpha_k / v_k(P, T), m = rho u, E = sum rhoY_k e_k + rho|u|^2/2 */
  template <class Wt>
  void conserved_from_primitive(const Wt* w, R* U) const {
    R P(w[ns + D]), T(w[ns + D + 1]);
    R rho(0.0), e(0.0);
    for (int k = 0; k < ns; ++k) {
      R a(w[k]);
      U[k] = val(a) != 0.0 ? a / v_k(p, k, P, T) : R(0.0);
      rho = rho + U[k];
      if (val(a) != 0.0) e = e + U[k] * e_k(p, k, P, T);
    }
    R ke(0.0);
    for (int d = 0; d < D; ++d) {
      U[ns + d] = rho * w[ns + d];
      ke = ke + rho * w[ns + d] * w[ns + d];
    }
    U[ns + D] = e + 0.5 * ke;
  }

  void load(const R* U, vector<R>& Up) const {
    for (int v = 0; v < nv; ++v)
      for (int k = 0; k < G.n[2]; ++k)
        for (int j = 0; j < G.n[1]; ++j)
          for (int i = 0; i < G.n[0]; ++i)
            Up[(size_t)v * G.npad + G.pad(i, j, k)] = U[(size_t)v * G.ncell + G.cell(i, j, k)];
  }

  /* ghost state of a characteristic boundary (Sec. 3.5: the non-reflecting
   * inflow / outflow conditions of Thompson and of Poinsot & Lele).  The paper
   * gives no formulation; reading: their locally one-dimensional inviscid
   * form, realized through the ghost state with the characteristic
   * decomposition of Appendix A at the boundary cell: the acoustic
   * invariants P +- rho a u_n (speeds u_n +- a) and, with speed u_n, the
   * entropy variable T - X P, the mass fractions and the tangential
   * velocity.  A field that leaves the domain (its speed along the outward
   * normal > 0; >= 0 for speed u_n) keeps the boundary cell's value, one
   * that enters takes the far-field state's (the inflow state), so that no
   * wave is reflected by the boundary in the linear limit and the incoming
   * waves carry the far field in.  A ghost that is not admissible (T <= 0,
   * or P + Pinf_k <= 0 for a species present) is replaced by the boundary
   * cell.  side 0: low boundary of direction d, 1: high. */
  void char_ghost(int d, int side, const R* Ub, R* Ug) const {
    Cell<R> cb, ct;
    cell_from_conserved(p, D, Ub, cb);
    cell_from_conserved(p, D, Uin, ct);
    R rho, a, al, be, X, c;
    char_scalars(p, D, Ub, rho, a, al, be, X, c);
    const double out = side == 0 ? -1.0 : 1.0;
    const R un = cb.u[d];
    const bool out_p = val(out * (un + a)) > 0.0;
    const bool out_m = val(out * (un - a)) > 0.0;
    const bool out_0 = val(out * un) >= 0.0;
    const R wp = out_p ? cb.P + c * un : ct.P + c * ct.u[d];
    const R wm = out_m ? cb.P - c * un : ct.P - c * ct.u[d];
    const R Pg = 0.5 * (wp + wm);
    const R w1 = out_0 ? cb.T - X * cb.P : ct.T - X * ct.P;
    const R Tg = w1 + X * Pg;
    R Yg[MAXS], ug[3];
    for (int k = 0; k < ns; ++k) Yg[k] = out_0 ? cb.Y[k] : ct.Y[k];
    for (int t = 0; t < 3; ++t) ug[t] = out_0 ? cb.u[t] : ct.u[t];
    ug[d] = (wp - wm) / (2.0 * c);
    bool ok = val(Tg) > 0.0;
    for (int k = 0; k < ns; ++k)
      if (val(Yg[k]) > 0.0 && !(val(Pg + p.pinf[k]) > 0.0)) ok = false;
    if (!ok) {
      for (int v = 0; v < nv; ++v) Ug[v] = Ub[v];
      return;
    }
    State<R> s;
    state_from_primitive(p, D, Yg, ug, Pg, Tg, s);
    conserved_of(ns, D, s, Ug);
  }

  /* ghost layers, one direction after the other (x, y, z) over the full
   * padded extent of the other directions */
  void fill_ghosts(vector<R>& Up) const {
    for (int d = 0; d < D; ++d) {
      const int n = G.n[d], g = G.g[d];
      for (int side = 0; side < 2; ++side) {
        int bc = side == 0 ? p.bc_lo[d] : p.bc_hi[d];
        for (int l = 0; l < g; ++l) {
          int gi = side == 0 ? -1 - l : n + l; /* ghost index along d */
          int src;
          switch (bc) {
            case ORC_BC_PERIODIC: src = side == 0 ? n - 1 - l : l; break;
            case ORC_BC_WALL: src = side == 0 ? l : n - 1 - l; break;
            case ORC_BC_ZEROGRAD: src = side == 0 ? 0 : n - 1; break;
            default: src = -100; break;
          }
          int lo[3], hi[3];
          for (int e = 0; e < 3; ++e) {
            lo[e] = -G.g[e];
            hi[e] = G.n[e] + G.g[e];
          }
          lo[d] = 0;
          hi[d] = 1;
          for (int k = lo[2]; k < hi[2]; ++k)
            for (int j = lo[1]; j < hi[1]; ++j)
              for (int i = lo[0]; i < hi[0]; ++i) {
                int ig[3] = {i, j, k}, is[3] = {i, j, k};
                ig[d] = gi;
                is[d] = src;
                size_t dst = G.pad(ig[0], ig[1], ig[2]);
                if (bc == ORC_BC_INFLOW) {
                  for (int v = 0; v < nv; ++v) Up[(size_t)v * G.npad + dst] = Uin[v];
                } else if (bc == ORC_BC_CHAR) {
                  /* every ghost layer takes the ghost state of the boundary
                   * cell of its row (rows outside the other directions'
                   * ranges are overwritten when those directions are filled) */
                  is[d] = side == 0 ? 0 : n - 1;
                  R Ub[MAXV], Ug[MAXV];
                  cell_U(Up, G.pad(is[0], is[1], is[2]), Ub);
                  char_ghost(d, side, Ub, Ug);
                  for (int v = 0; v < nv; ++v) Up[(size_t)v * G.npad + dst] = Ug[v];
                } else {
                  size_t s = G.pad(is[0], is[1], is[2]);
                  for (int v = 0; v < nv; ++v) Up[(size_t)v * G.npad + dst] = Up[(size_t)v * G.npad + s];
                  if (bc == ORC_BC_WALL) Up[(size_t)(ns + d) * G.npad + dst] = -Up[(size_t)(ns + d) * G.npad + dst];
                }
              }
        }
      }
    }
  }

  void cell_U(const vector<R>& Up, size_t c, R* U) const {
    for (int v = 0; v < nv; ++v) U[v] = Up[(size_t)v * G.npad + c];
  }

  int compute_cells(const vector<R>& Up) {
    int st = ORC_OK;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)G.npad; ++c) {
      R U[MAXV];
      for (int v = 0; v < nv; ++v) U[v] = Up[(size_t)v * G.npad + c];
      cell_from_conserved(p, D, U, cells[c]);
    }
    /* status over interior cells */
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) st = std::max(st, cells[G.pad(i, j, k)].status);
    return st;
  }

  /* the Y limiter of Sec. 3.3.1 on one face side; Yc = cell values.
   * reading of the garbled step formulas: Sigma = sum_k (min(Y_k, Yc_k) - Y_k)
   * and eps_k = ((1 - sum Y) / Sigma) (min(Y_k, Yc_k) - Y_k) when sum Y > 1,
   * the same with max when sum Y < 1; first Y_k <- max(Y_k, 0). */
  bool y_limiter(R* Y, const R* Yc) const {
    bool active = false;
    for (int k = 0; k < ns; ++k)
      if (val(Y[k]) < 0.0) {
        Y[k] = R(0.0);
        active = true;
      }
    R sum(0.0);
    for (int k = 0; k < ns; ++k) sum = sum + Y[k];
    /* reading: no renormalization when sum Y is one to rounding
     * (|sum Y - 1| <= ns YSUM_TOL).  The correction would then be below the
     * resolution of the data, distributed by a ratio of rounding errors
     * (Sigma itself is rounding-level where the reconstruction equals the
     * cell values), which makes the limiter discontinuous to round-off. */
    if (std::fabs(val(sum) - 1.0) <= ns * YSUM_TOL) return active;
    if (val(sum) > 1.0) {
      R d[MAXS], Sig(0.0);
      for (int k = 0; k < ns; ++k) {
        d[k] = rmin(Y[k], Yc[k]) - Y[k];
        Sig = Sig + d[k];
      }
      if (val(Sig) != 0.0) {
        R f = (1.0 - sum) / Sig;
        for (int k = 0; k < ns; ++k) Y[k] = Y[k] + f * d[k];
        active = true;
      }
    } else if (val(sum) < 1.0) {
      R d[MAXS], Sig(0.0);
      for (int k = 0; k < ns; ++k) {
        d[k] = rmax(Y[k], Yc[k]) - Y[k];
        Sig = Sig + d[k];
      }
      if (val(Sig) != 0.0) {
        R f = (1.0 - sum) / Sig;
        for (int k = 0; k < ns; ++k) Y[k] = Y[k] + f * d[k];
        active = true;
      }
    }
    return active;
  }

  /* reading of the P, T admissibility of Sec. 3.3.1: T > 0 and
   * P + Pinf_k > 0 for every species present on that side */
  bool p_admissible(const R* Y, const R& P) const {
    for (int k = 0; k < ns; ++k)
      if (val(Y[k]) > 0.0 && !(val(P + p.pinf[k]) > 0.0)) return false;
    return true;
  }

  /* face states of the face between padded cells c0 and c1 = c0 +
   * stride(d) (Sec. 3.1.3 steps 1-3 and the interpolation limiters of
   * Sec. 3.3.1): mass fractions, velocity, pressure and temperature of each
   * side.  Returns the interpolation-limiter flag bits. */
  uint32_t face_states(int d, size_t c0, R* YL, R* YR, R* uL, R* uR, R& PL, R& PR, R& TL,
                       R& TR) const {
    const long st = G.stride(d);
    uint32_t flags = 0;
    const Cell<R>* cc[6];
    for (int j = 0; j < 6; ++j) cc[j] = &cells[(size_t)((long)c0 + (j - 2) * st)];
    const Cell<R>& ci = *cc[2];
    const Cell<R>& cj = *cc[3];
    const size_t c1 = (size_t)((long)c0 + st);

    if (p.recon_basis == 0) {
      /* step 1: averaged state on the face, its EOS and the matrices */
      R Ui[MAXV], Uj[MAXV], Ub[MAXV];
      cell_U(Ukp, c0, Ui);
      cell_U(Ukp, c1, Uj);
      for (int v = 0; v < nv; ++v) Ub[v] = 0.5 * (Ui[v] + Uj[v]);
      R rb, ab, alb, beb, X, rhoa;
      char_scalars(p, D, Ub, rb, ab, alb, beb, X, rhoa);
      R Sinv[MAXC * MAXC], S[MAXC * MAXC];
      char_matrices(ns, D, d, X, rhoa, Sinv, S);
      /* project W_j = [T, Y_0..Y_{ns-2}, u, P] of the six stencil cells */
      R Wt[6][MAXC];
      for (int j = 0; j < 6; ++j) {
        R W[MAXC];
        W[0] = cc[j]->T;
        for (int k = 0; k < ns - 1; ++k) W[1 + k] = cc[j]->Y[k];
        for (int t = 0; t < D; ++t) W[ns + t] = cc[j]->u[t];
        W[ns + D] = cc[j]->P;
        for (int r = 0; r < nc; ++r) {
          R s(0.0);
          for (int q = 0; q < nc; ++q) s = s + Sinv[r * nc + q] * W[q];
          Wt[j][r] = s;
        }
      }
      /* step 2: ENO-type interpolation (WENO5-Z unless the model selects
       * another) of each characteristic variable, both sides */
      R WtL[MAXC], WtR[MAXC];
      for (int r = 0; r < nc; ++r) {
        const R sl[6] = {Wt[0][r], Wt[1][r], Wt[2][r], Wt[3][r], Wt[4][r], Wt[5][r]};
        const R sr[6] = {Wt[5][r], Wt[4][r], Wt[3][r], Wt[2][r], Wt[1][r], Wt[0][r]};
        WtL[r] = reconstruct(p.recon, sl, p.weno_eps);
        WtR[r] = reconstruct(p.recon, sr, p.weno_eps);
      }
      /* step 3: back to physical space */
      R WL[MAXC], WR[MAXC];
      for (int r = 0; r < nc; ++r) {
        R sl(0.0), sr(0.0);
        for (int q = 0; q < nc; ++q) {
          sl = sl + S[r * nc + q] * WtL[q];
          sr = sr + S[r * nc + q] * WtR[q];
        }
        WL[r] = sl;
        WR[r] = sr;
      }
      TL = WL[0];
      TR = WR[0];
      for (int k = 0; k < ns - 1; ++k) {
        YL[k] = WL[1 + k];
        YR[k] = WR[1 + k];
      }
      for (int t = 0; t < 3; ++t) {
        uL[t] = t < D ? WL[ns + t] : R(0.0);
        uR[t] = t < D ? WR[ns + t] : R(0.0);
      }
      PL = WL[ns + D];
      PR = WR[ns + D];
      /* the species left out of the projection, interpolated on its own */
      const int kl = ns - 1;
      {
        const R sl[6] = {cc[0]->Y[kl], cc[1]->Y[kl], cc[2]->Y[kl], cc[3]->Y[kl], cc[4]->Y[kl], cc[5]->Y[kl]};
        const R sr[6] = {cc[5]->Y[kl], cc[4]->Y[kl], cc[3]->Y[kl], cc[2]->Y[kl], cc[1]->Y[kl], cc[0]->Y[kl]};
        YL[kl] = reconstruct(p.recon, sl, p.weno_eps);
        YR[kl] = reconstruct(p.recon, sr, p.weno_eps);
      }
    } else {
      /* negative control: component-wise [rhoY, u, P] without projection;
       * T on the face then follows from rho, P, Y through NASG_T2 */
      R rYL[MAXS], rYR[MAXS];
      auto both = [&](const R* s6, R& l, R& r) {
        const R sr[6] = {s6[5], s6[4], s6[3], s6[2], s6[1], s6[0]};
        l = reconstruct(p.recon, s6, p.weno_eps);
        r = reconstruct(p.recon, sr, p.weno_eps);
      };
      for (int k = 0; k < ns; ++k) {
        const R s6[6] = {cc[0]->rhoY[k], cc[1]->rhoY[k], cc[2]->rhoY[k], cc[3]->rhoY[k], cc[4]->rhoY[k], cc[5]->rhoY[k]};
        both(s6, rYL[k], rYR[k]);
      }
      for (int t = 0; t < 3; ++t) {
        if (t < D) {
          const R s6[6] = {cc[0]->u[t], cc[1]->u[t], cc[2]->u[t], cc[3]->u[t], cc[4]->u[t], cc[5]->u[t]};
          both(s6, uL[t], uR[t]);
        } else {
          uL[t] = R(0.0);
          uR[t] = R(0.0);
        }
      }
      {
        const R s6[6] = {cc[0]->P, cc[1]->P, cc[2]->P, cc[3]->P, cc[4]->P, cc[5]->P};
        both(s6, PL, PR);
      }
      R rl(0.0), rr(0.0);
      for (int k = 0; k < ns; ++k) {
        rl = rl + rYL[k];
        rr = rr + rYR[k];
      }
      for (int k = 0; k < ns; ++k) {
        YL[k] = rYL[k] / rl;
        YR[k] = rYR[k] / rr;
      }
      R bl(0.0), br(0.0), sl(0.0), sr(0.0);
      for (int k = 0; k < ns; ++k) {
        bl = bl + YL[k] * p.b[k];
        br = br + YR[k] * p.b[k];
        sl = sl + YL[k] * Rgas(p, k) / (PL + p.pinf[k]);
        sr = sr + YR[k] * Rgas(p, k) / (PR + p.pinf[k]);
      }
      TL = (1.0 / rl - bl) / sl;
      TR = (1.0 / rr - br) / sr;
    }

    /* interpolation limiters (Sec. 3.3.1) */
    if (p.pos_limiter) {
      if (p.recon_basis == 0) {
        if (y_limiter(YL, ci.Y)) flags |= ORC_F_YLIM_L;
        if (y_limiter(YR, cj.Y)) flags |= ORC_F_YLIM_R;
      }
      if (!(val(TL) > 0.0)) { TL = ci.T; flags |= ORC_F_THETA_T_L; }
      if (!(val(TR) > 0.0)) { TR = cj.T; flags |= ORC_F_THETA_T_R; }
      if (!p_admissible(YL, PL)) { PL = ci.P; flags |= ORC_F_THETA_P_L; }
      if (!p_admissible(YR, PR)) { PR = cj.P; flags |= ORC_F_THETA_P_R; }
    }
    return flags;
  }

  /* numerical flux through the face between padded cells c0 and c1 = c0 +
   * stride(d).  Un/Uk: padded U^n and U^(k).  Returns flag bits. */
  uint32_t face_flux(int d, size_t c0, double rk0, double rk1, double rk2, double dt,
                     const R& Gamma, R* F) const {
    const long st = G.stride(d);
    const Cell<R>& ci = cells[c0];
    const Cell<R>& cj = cells[(size_t)((long)c0 + st)];
    const size_t c1 = (size_t)((long)c0 + st);
    R YL[MAXS], YR[MAXS], uL[3], uR[3], PL, PR, TL, TR;
    uint32_t flags = face_states(d, c0, YL, YR, uL, uR, PL, PR, TL, TR);

    /* steps 4-6: face density from the EOS, conserved face states, HLLC */
    State<R> sLf, sRf;
    state_from_primitive(p, D, YL, uL, PL, TL, sLf);
    state_from_primitive(p, D, YR, uR, PR, TR, sRf);
    hllc(ns, D, d, sLf, sRf, F);

    /* flux limiter (Sec. 3.3.2).  reading: pseudo-update factor
     * 2 D RK2 dt / dx, minus on cell i, plus on cell i+1 */
    R Uni[MAXV], Unj[MAXV], Uki[MAXV], Ukj[MAXV];
    cell_U(Unp, c0, Uni);
    cell_U(Unp, c1, Unj);
    cell_U(Ukp, c0, Uki);
    cell_U(Ukp, c1, Ukj);
    const double lam = 2.0 * D * rk2 * dt / p.dx;
    auto passes = [&](const R* Ft) {
      R Ti[MAXV], Tj[MAXV];
      for (int v = 0; v < nv; ++v) {
        Ti[v] = rk0 * Uni[v] + rk1 * Uki[v] - lam * Ft[v];
        Tj[v] = rk0 * Unj[v] + rk1 * Ukj[v] + lam * Ft[v];
      }
      return admissible(p, D, Ti) && admissible(p, D, Tj);
    };
    if (p.pos_limiter && !passes(F)) {
      State<R> si, sj;
      state_from_cell(ns, ci, si);
      state_from_cell(ns, cj, sj);
      hllc(ns, D, d, si, sj, F);
      flags |= ORC_F_HLLC_FALLBACK;
    }

    /* interface regularization (Sec. 3.2), KEEP split form */
    bool two_phase = false, has0 = false, has1 = false;
    for (int k = 0; k < ns; ++k) (p.phase[k] == 0 ? has0 : has1) = true;
    two_phase = has0 && has1;
    /* reading: no regularization through a face where a phase is absent
     * from both cells (psi is flat to round-off there and its normalized
     * gradient would be noise) */
    const bool both_phases = (ci.present[0] || cj.present[0]) && (ci.present[1] || cj.present[1]);
    if (p.cdi && two_phase && both_phases) {
      R Fdi[MAXV];
      for (int v = 0; v < nv; ++v) Fdi[v] = R(0.0);
      const double eps = p.cdi_eps;
      const double sharp0 = 4.0 * p.phi_min * (1.0 - p.phi_min);
      R Rtot(0.0), hR(0.0);
      /* regularization velocity of phase 0.  reading: for two phases the
       * second phase takes the negative (phi_1 = 1 - phi_0, psi_1 = -psi_0,
       * n_1 = -n_0 in the continuous model); evaluating both phases
       * separately lets round-off in a saturated phase fraction produce a net
       * volume flux, which breaks the interface equilibrium */
      R dphi = (cj.phi[0] - ci.phi[0]) / p.dx;
      /* reading: normal of grad psi on the face; tangential components are
       * the average of the two cells' central differences */
      R g[3];
      for (int t = 0; t < 3; ++t) g[t] = R(0.0);
      g[d] = (cj.psi - ci.psi) / p.dx;
      for (int t = 0; t < D; ++t) {
        if (t == d) continue;
        const long sT = G.stride(t);
        const Cell<R>& ip = cells[(size_t)((long)c0 + sT)];
        const Cell<R>& im = cells[(size_t)((long)c0 - sT)];
        const Cell<R>& jp = cells[(size_t)((long)c1 + sT)];
        const Cell<R>& jm = cells[(size_t)((long)c1 - sT)];
        g[t] = 0.5 * ((ip.psi - im.psi) / (2.0 * p.dx) + (jp.psi - jm.psi) / (2.0 * p.dx));
      }
      R gn(0.0);
      for (int t = 0; t < 3; ++t) gn = gn + g[t] * g[t];
      gn = sqrt(gn);
      /* reading: the normal is taken as zero where |grad psi| is below
       * GTOL (psi near a signed distance has |grad psi| ~ 1; a flat far
       * field gives round-off, whose normalized direction is noise) */
      R nd = val(gn) >= GTOL ? g[d] / gn : R(0.0);
      R psib = 0.5 * (ci.psi + cj.psi);
      /* 1 - tanh^2(x) written as 1 / cosh^2(x): the same quantity without the
       * cancellation that 1 - tanh^2 suffers where the phase fraction is
       * near the phi_min floor and the bracket below nearly vanishes */
      R ch = cosh(psib / (2.0 * eps));
      R sech2 = 1.0 / (ch * ch);
      /* Eq. SkewSymmetricSplitting_Regularization_Expanded */
      R ahat0 = Gamma * (eps * dphi - 0.25 * (sech2 - sharp0) * nd);
      for (int ph = 0; ph < 2; ++ph) {
        R ahat = ph == 0 ? ahat0 : -ahat0;
        /* KEEP face interpolation of a phase quantity.  reading: where the
         * phase is absent from one cell its intensive quantities are
         * undefined and the face takes the other side's value (no flux of
         * a phase absent on both sides) */
        const bool pi = ci.present[ph], pj = cj.present[ph];
        auto keep = [&](const R& a, const R& b) {
          return pi && pj ? 0.5 * (a + b) : (pi ? a : (pj ? b : R(0.0)));
        };
        for (int k = 0; k < ns; ++k) {
          if (p.phase[k] != ph) continue;
          R Rk = -keep(ci.yrho[k], cj.yrho[k]) * ahat;
          Fdi[k] = Rk;
          Rtot = Rtot + Rk;
        }
        hR = hR - keep(ci.hrho[ph], cj.hrho[ph]) * ahat;
      }
      R kb(0.0);
      for (int t = 0; t < 3; ++t) kb = kb + ci.u[t] * cj.u[t];
      kb = 0.5 * kb;
      for (int t = 0; t < D; ++t) Fdi[ns + t] = 0.5 * (ci.u[t] + cj.u[t]) * Rtot;
      Fdi[ns + D] = kb * Rtot + hR;
      R Ft[MAXV];
      for (int v = 0; v < nv; ++v) Ft[v] = F[v] + Fdi[v];
      if (p.pos_limiter && !passes(Ft)) {
        flags |= ORC_F_CDI_DROPPED;
      } else {
        for (int v = 0; v < nv; ++v) F[v] = Ft[v];
      }
    }

    /* diffusive flux F_nu: species diffusion (energy carries sum_c J^c h^c;
     * reading: without the extra Y^c/Y_p factor), viscous stress and heat
     * conduction.  Reading: it passes the same flux limiter as the
     * regularization flux (Sec. 3.3.2, last paragraph) -- added to the
     * admissible flux when the pseudo-update stays admissible, else not
     * added at this face -- so that the next state is admissible with
     * every flux in */
    R Fnu[MAXV];
    for (int v = 0; v < nv; ++v) Fnu[v] = R(0.0);
    if (p.diffusion) {
      R rb = 0.5 * (ci.rho + cj.rho);
      R Jh(0.0);
      for (int ph = 0; ph < 2; ++ph) {
        R Yp(0.0), Ssum(0.0);
        R Bf[MAXS], Gf[MAXS];
        for (int k = 0; k < ns; ++k) {
          if (p.phase[k] != ph) continue;
          Yp = Yp + 0.5 * (ci.Y[k] + cj.Y[k]);
          Bf[k] = 0.5 * (ci.B[k] + cj.B[k]);
          Gf[k] = (cj.xr[k] - ci.xr[k]) / p.dx;
          Ssum = Ssum + Bf[k] * Gf[k];
        }
        for (int k = 0; k < ns; ++k) {
          if (p.phase[k] != ph) continue;
          R Yk = 0.5 * (ci.Y[k] + cj.Y[k]);
          R J = -rb * (Yp * Bf[k] * Gf[k] - Yk * Ssum);
          Fnu[k] = J;
          Jh = Jh + J * 0.5 * (ci.h[k] + cj.h[k]);
        }
      }
      Fnu[ns + D] = Jh;
    }

    /* viscous stress and heat conduction (Eq. DiffusionTerms and the stress
     * tensor and heat flux of Sec. 2.1), second-order central: face values
     * are the averages of the two cells; the normal derivative is
     * (q_{i+1} - q_i)/dx, a tangential one the average of the two cells'
     * central differences.  Reading: the energy row carries the physical
     * -u.tau + q (the printed row has the opposite sign to the printed
     * momentum rows -tau); q's enthalpy part is the diffusion block above. */
    if (p.viscous) {
      R gu[3][3];  /* gu[i][j] = d u_i / d x_j on the face */
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) gu[i][j] = R(0.0);
      for (int i = 0; i < D; ++i) gu[i][d] = (cj.u[i] - ci.u[i]) / p.dx;
      for (int t = 0; t < D; ++t) {
        if (t == d) continue;
        const long sT = G.stride(t);
        const Cell<R>& ip = cells[(size_t)((long)c0 + sT)];
        const Cell<R>& im = cells[(size_t)((long)c0 - sT)];
        const Cell<R>& jp = cells[(size_t)((long)c1 + sT)];
        const Cell<R>& jm = cells[(size_t)((long)c1 - sT)];
        for (int i = 0; i < D; ++i)
          gu[i][t] = 0.5 * ((ip.u[i] - im.u[i]) / (2.0 * p.dx) + (jp.u[i] - jm.u[i]) / (2.0 * p.dx));
      }
      R div(0.0);
      for (int k = 0; k < D; ++k) div = div + gu[k][k];
      const R mub = 0.5 * (ci.mu + cj.mu), lamb = 0.5 * (ci.lam + cj.lam);
      R work(0.0);
      for (int i = 0; i < D; ++i) {
        R tau = mub * (gu[i][d] + gu[d][i] - (i == d ? (2.0 / 3.0) * div : R(0.0)));
        Fnu[ns + i] = -tau;
        work = work + 0.5 * (ci.u[i] + cj.u[i]) * tau;
      }
      Fnu[ns + D] = Fnu[ns + D] - work - lamb * (cj.T - ci.T) / p.dx;
    }
    if (p.diffusion || p.viscous) {
      R Ft[MAXV];
      for (int v = 0; v < nv; ++v) Ft[v] = F[v] + Fnu[v];
      if (p.pos_limiter && !passes(Ft)) {
        flags |= ORC_F_DIFF_DROPPED;
      } else {
        for (int v = 0; v < nv; ++v) F[v] = Ft[v];
      }
    }
    return flags;
  }

  /* all face fluxes of direction d into Fd [nv][nface(d)] */
  void sweep(int d, double rk0, double rk1, double rk2, double dt, const R& Gamma, vector<R>& Fd,
             uint32_t* flags) const {
    const int f0 = G.n[0] + (d == 0), f1 = G.n[1] + (d == 1), f2 = G.n[2] + (d == 2);
    const size_t nf = G.nface(d);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < f2; ++k)
      for (int j = 0; j < f1; ++j)
        for (int i = 0; i < f0; ++i) {
          /* face index -> the cell on its low side (may be a ghost) */
          int ic[3] = {i, j, k};
          ic[d] -= 1;
          size_t c0 = G.pad(ic[0], ic[1], ic[2]);
          R F[MAXV];
          uint32_t fl = face_flux(d, c0, rk0, rk1, rk2, dt, Gamma, F);
          size_t fi = G.face(d, i, j, k);
          for (int v = 0; v < nv; ++v) Fd[(size_t)v * nf + fi] = F[v];
          if (flags) flags[fi] = fl;
        }
  }

  /* Eq. DiscreteGoverningEquations: L = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx */
  int evaluate(const R* Un, const R* Uk, double rk0, double rk1, double rk2, double dt,
               const R& Gamma, vector<vector<R>>& F, uint32_t* flags) {
    load(Un, Unp);
    load(Uk, Ukp);
    fill_ghosts(Unp);
    fill_ghosts(Ukp);
    int st = compute_cells(Ukp);
    F.assign(D, vector<R>());
    size_t foff = 0;
    for (int d = 0; d < D; ++d) {
      F[d].assign((size_t)nv * G.nface(d), R(0.0));
      sweep(d, rk0, rk1, rk2, dt, Gamma, F[d], flags ? flags + foff : nullptr);
      foff += G.nface(d);
    }
    return st;
  }

  int stage(const R* Un, const R* Uk, double rk0, double rk1, double rk2, double dt,
            const R& Gamma, R* Uout, R* dUdt, uint32_t* flags) {
    vector<vector<R>> F;
    int st = evaluate(Un, Uk, rk0, rk1, rk2, dt, Gamma, F, flags);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) {
          size_t c = G.cell(i, j, k);
          for (int v = 0; v < nv; ++v) {
            R L(0.0);
            for (int d = 0; d < D; ++d) {
              int ic[3] = {i, j, k};
              size_t fm = G.face(d, ic[0], ic[1], ic[2]);
              ic[d] += 1;
              size_t fp = G.face(d, ic[0], ic[1], ic[2]);
              size_t nf = G.nface(d);
              L = L - (F[d][(size_t)v * nf + fp] - F[d][(size_t)v * nf + fm]) / p.dx;
            }
            if (dUdt) dUdt[(size_t)v * G.ncell + c] = L;
            if (Uout)
              Uout[(size_t)v * G.ncell + c] =
                  rk0 * Un[(size_t)v * G.ncell + c] + rk1 * Uk[(size_t)v * G.ncell + c] + rk2 * dt * L;
          }
        }
    if (Uout) {
      for (size_t c = 0; c < G.ncell; ++c) {
        R U[MAXV];
        for (int v = 0; v < nv; ++v) U[v] = Uout[(size_t)v * G.ncell + c];
        if (!admissible(p, D, U)) {
          st = std::max(st, (int)ORC_INADMISSIBLE);
          break;
        }
      }
    }
    return st;
  }

  /* CFL condition of Sec. 3.4 (reading: (|u_d| + a)/dx per direction and
   * 4 mu / rho / dx^2 when diffusion is on) and Gamma = max |u_d| (Sec. 3.2) */
  int dt_gamma(const R* U, double& dt, double& Gamma) {
    load(U, Ukp);
    double smax = 0.0, gmax = 0.0;
    int st = ORC_OK;
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i) {
          R Uc[MAXV];
          cell_U(Ukp, G.pad(i, j, k), Uc);
          Cell<R> c;
          cell_from_conserved(p, D, Uc, c);
          st = std::max(st, c.status);
          for (int d = 0; d < D; ++d) {
            double ud = std::fabs(val(c.u[d]));
            smax = std::max(smax, (ud + val(c.a)) / p.dx);
            gmax = std::max(gmax, ud);
          }
          if (p.diffusion || p.viscous) smax = std::max(smax, 4.0 * val(c.mu) / val(c.rho) / (p.dx * p.dx));
          if (p.viscous) {
            /* reading: the conduction limit with the thermal diffusivity
             * lambda / (rho cv) */
            double cv = 0.0;
            for (int k = 0; k < ns; ++k) cv += val(c.Y[k]) * p.cv[k];
            smax = std::max(smax, 4.0 * val(c.lam) / (val(c.rho) * cv) / (p.dx * p.dx));
          }
        }
    dt = p.cfl / smax;
    Gamma = p.cdi_gamma > 0.0 ? p.cdi_gamma : gmax;
    return st;
  }
};

}  // namespace orc

/* ------------------------------------------------------------------------ */
/* C API                                                                    */
/* ------------------------------------------------------------------------ */
using namespace orc;

static int check(const orc_params* p) {
  if (!p || p->dim < 1 || p->dim > 3 || p->ns < 1 || p->ns > ORC_MAXS || !(p->dx > 0)) return ORC_INVALID;
  for (int d = 0; d < p->dim; ++d) {
    if (p->n[d] < 1) return ORC_INVALID;
    /* characteristic boundaries along x only (their ghost rows are then
     * never corners of two such boundaries) */
    if (d > 0 && (p->bc_lo[d] == ORC_BC_CHAR || p->bc_hi[d] == ORC_BC_CHAR)) return ORC_INVALID;
  }
#ifdef _OPENMP
  if (p->nthreads > 0) omp_set_num_threads(p->nthreads);
#endif
  return ORC_OK;
}

extern "C" {

int orc_nvars(const orc_params* p) { return p->ns + p->dim + 1; }

int orc_init_state(const orc_params* p, const double* prim, double* U) {
  if (check(p)) return ORC_INVALID;
  Solver<double> s(*p);
  const int ns = p->ns, D = p->dim, nv = ns + D + 1, nw = ns + D + 2;
  for (size_t c = 0; c < s.G.ncell; ++c) {
    double w[MAXV + 1], Uc[MAXV];
    for (int v = 0; v < nw; ++v) w[v] = prim[(size_t)v * s.G.ncell + c];
    s.conserved_from_primitive(w, Uc);
    for (int v = 0; v < nv; ++v) U[(size_t)v * s.G.ncell + c] = Uc[v];
  }
  return ORC_OK;
}

int orc_primitives(const orc_params* p, const double* U, double* out) {
  if (check(p)) return ORC_INVALID;
  Solver<double> s(*p);
  const int nv = s.nv;
  int st = ORC_OK;
  for (size_t c = 0; c < s.G.ncell; ++c) {
    double Uc[MAXV];
    for (int v = 0; v < nv; ++v) Uc[v] = U[(size_t)v * s.G.ncell + c];
    Cell<double> cl;
    cell_from_conserved(*p, p->dim, Uc, cl);
    st = std::max(st, cl.status);
    double o[8] = {cl.P, cl.T, cl.a, cl.rho, cl.phi[0], cl.phi[1], cl.psi, -cl.psi};
    for (int v = 0; v < 8; ++v) out[(size_t)v * s.G.ncell + c] = o[v];
  }
  return st;
}

int orc_dt_gamma(const orc_params* p, const double* U, double* dt, double* Gamma) {
  if (check(p)) return ORC_INVALID;
  Solver<double> s(*p);
  return s.dt_gamma(U, *dt, *Gamma);
}

int orc_stage(const orc_params* p, const double* U_n, const double* U_k, double rk0, double rk1,
              double rk2, double dt, double Gamma, double* U_out, double* dUdt, uint32_t* flags) {
  if (check(p)) return ORC_INVALID;
  Solver<double> s(*p);
  return s.stage(U_n, U_k, rk0, rk1, rk2, dt, Gamma, U_out, dUdt, flags);
}

int orc_face_fluxes(const orc_params* p, const double* U_n, const double* U_k, double rk0,
                    double rk1, double rk2, double dt, double Gamma, double* F) {
  if (check(p)) return ORC_INVALID;
  Solver<double> s(*p);
  std::vector<std::vector<double>> Fd;
  int st = s.evaluate(U_n, U_k, rk0, rk1, rk2, dt, Gamma, Fd, nullptr);
  size_t off = 0;
  for (int d = 0; d < p->dim; ++d) {
    std::memcpy(F + off, Fd[d].data(), Fd[d].size() * sizeof(double));
    off += Fd[d].size();
  }
  return st;
}

/* Eq. SSPRK3 */
int orc_rk_step(const orc_params* p, double* U, double dt, double* dt_used) {
  if (check(p)) return ORC_INVALID;
  Solver<double> s(*p);
  const size_t n = (size_t)s.nv * s.G.ncell;
  double Gamma = 0.0, dtc = 0.0;
  int st = s.dt_gamma(U, dtc, Gamma);
  if (dt <= 0.0) dt = dtc;
  std::vector<double> Un(U, U + n), U1(n), U2(n);
  st = std::max(st, s.stage(Un.data(), Un.data(), 1.0, 0.0, 1.0, dt, Gamma, U1.data(), nullptr, nullptr));
  st = std::max(st, s.stage(Un.data(), U1.data(), 0.75, 0.25, 0.25, dt, Gamma, U2.data(), nullptr, nullptr));
  st = std::max(st, s.stage(Un.data(), U2.data(), 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, dt, Gamma, U, nullptr, nullptr));
  if (dt_used) *dt_used = dt;
  return st;
}

int orc_run(const orc_params* p, double* U, int nsteps, double t_end, double* t_out, int* steps_out) {
  if (check(p)) return ORC_INVALID;
  double t = 0.0;
  int st = ORC_OK, it = 0;
  for (; it < nsteps; ++it) {
    double dtc, G;
    {
      Solver<double> s(*p);
      st = std::max(st, s.dt_gamma(U, dtc, G));
    }
    double dt = dtc;
    if (t_end > 0.0) {
      if (t >= t_end) break;
      if (t + dt > t_end) dt = t_end - t;
    }
    double used;
    st = std::max(st, orc_rk_step(p, U, dt, &used));
    t += used;
    if (st >= ORC_INADMISSIBLE) { ++it; break; }
  }
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = it;
  return st;
}

int orc_eos_pt(const orc_params* p, const double* Y, double e, double v, double* P, double* T) {
  return pt_equilibrium<double>(*p, Y, e, v, *P, *T);
}

int orc_eos_forward(const orc_params* p, const double* Y, double P, double T, double* out) {
  double rho, e, a, al, be, cp;
  eos_forward<double>(*p, Y, P, T, rho, e, a, al, be, cp);
  out[0] = rho; out[1] = e; out[2] = a; out[3] = al; out[4] = be; out[5] = cp;
  return ORC_OK;
}

double orc_weno5z(const double* v, double eps) { return weno5z<double>(v[0], v[1], v[2], v[3], v[4], eps); }

double orc_reconstruct(int kind, const double* v6, double eps) { return reconstruct<double>(kind, v6, eps); }

void orc_candidate(const double* v6, int offset, int n, double* value, double* beta) {
  double a[6];
  candidate_poly<double>(v6, offset, n, a);
  *value = poly_at_one<double>(v6[2], a, n);
  *beta = jiang_shu_beta<double>(a, n);
}

int orc_y_limiter(const orc_params* p, double* Y, const double* Yc) {
  if (check(p)) return -1;
  Solver<double> s(*p);
  return s.y_limiter(Y, Yc) ? 1 : 0;
}

int orc_face_states(const orc_params* p, const double* U, int d, int i, int j, int k, double* WL,
                    double* WR, uint32_t* flags) {
  if (check(p) || d < 0 || d >= p->dim) return ORC_INVALID;
  Solver<double> s(*p);
  int ic[3] = {i, j, k};
  for (int e = 0; e < 3; ++e)
    if (ic[e] < 0 || ic[e] >= s.G.n[e] + (e == d)) return ORC_INVALID;
  s.load(U, s.Ukp);
  s.fill_ghosts(s.Ukp);
  int st = s.compute_cells(s.Ukp);
  ic[d] -= 1; /* the cell on the face's low side */
  const size_t c0 = s.G.pad(ic[0], ic[1], ic[2]);
  double YL[MAXS], YR[MAXS], uL[3], uR[3], PL, PR, TL, TR;
  uint32_t fl = s.face_states(d, c0, YL, YR, uL, uR, PL, PR, TL, TR);
  const int ns = p->ns;
  for (int q = 0; q < ns; ++q) {
    WL[q] = YL[q];
    WR[q] = YR[q];
  }
  for (int t = 0; t < 3; ++t) {
    WL[ns + t] = uL[t];
    WR[ns + t] = uR[t];
  }
  WL[ns + 3] = PL;
  WR[ns + 3] = PR;
  WL[ns + 4] = TL;
  WR[ns + 4] = TR;
  if (flags) *flags = fl;
  return st;
}

int orc_char_matrices(const orc_params* p, int d, const double* Ubar, double* Sinv, double* S, double* scal) {
  double rho, a, al, be, X, rhoa;
  int st = char_scalars<double>(*p, p->dim, Ubar, rho, a, al, be, X, rhoa);
  char_matrices<double>(p->ns, p->dim, d, X, rhoa, Sinv, S);
  scal[0] = rho; scal[1] = a; scal[2] = al; scal[3] = be; scal[4] = X; scal[5] = rhoa;
  return st;
}

static void point_state(const orc_params* p, const double* W, State<double>& s) {
  const int ns = p->ns;
  double Y[ORC_MAXS], u[3] = {W[ns], W[ns + 1], W[ns + 2]};
  for (int k = 0; k < ns; ++k) Y[k] = W[k];
  state_from_primitive<double>(*p, p->dim, Y, u, W[ns + 3], W[ns + 4], s);
}

int orc_hllc_prim(const orc_params* p, int d, const double* WL, const double* WR, double* F) {
  State<double> L, R;
  point_state(p, WL, L);
  point_state(p, WR, R);
  hllc<double>(p->ns, p->dim, d, L, R, F);
  return ORC_OK;
}

int orc_physical_flux(const orc_params* p, int d, const double* W, double* F) {
  State<double> s;
  point_state(p, W, s);
  physical_flux<double>(p->ns, p->dim, d, s, F);
  return ORC_OK;
}

int orc_cons_from_point(const orc_params* p, const double* W, double* U) {
  State<double> s;
  point_state(p, W, s);
  conserved_of<double>(p->ns, p->dim, s, U);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Forward-mode tangents: the same routines evaluated in Dual<1> arithmetic,  */
/* i.e. exact directional derivatives of the oracle's own discrete map (with  */
/* its branches taken on values).  dt and Gamma are inputs and carry no       */
/* tangent.  The CPU reference for the discrete adjoint.                      */
/* ------------------------------------------------------------------------ */
typedef Dual<1> D1;

static std::vector<D1> dual_of(const double* v, const double* dv, size_t n) {
  std::vector<D1> out(n);
  for (size_t i = 0; i < n; ++i) {
    out[i].v = v[i];
    out[i].d[0] = dv ? dv[i] : 0.0;
  }
  return out;
}

static void split(const std::vector<D1>& x, double* v, double* dv) {
  for (size_t i = 0; i < x.size(); ++i) {
    if (v) v[i] = x[i].v;
    if (dv) dv[i] = x[i].d[0];
  }
}

int orc_stage_jvp(const orc_params* p, const double* U_n, const double* U_k, const double* dU_k, double rk0,
                  double rk1, double rk2, double dt, double Gamma, double* dUdt, double* d_dUdt) {
  if (check(p)) return ORC_INVALID;
  Solver<D1> s(*p);
  const size_t n = (size_t)s.nv * s.G.ncell;
  std::vector<D1> Un = dual_of(U_n, nullptr, n), Uk = dual_of(U_k, dU_k, n), L(n);
  int st = s.stage(Un.data(), Uk.data(), rk0, rk1, rk2, dt, D1(Gamma), nullptr, L.data(), nullptr);
  split(L, dUdt, d_dUdt);
  return st;
}

int orc_rk_step_jvp(const orc_params* p, const double* U, const double* dU, double dt, double Gamma,
                    double* U_out, double* dU_out) {
  if (check(p) || !(dt > 0.0) || !(Gamma >= 0.0)) return ORC_INVALID;
  Solver<D1> s(*p);
  const size_t n = (size_t)s.nv * s.G.ncell;
  std::vector<D1> Un = dual_of(U, dU, n), U1(n), U2(n), U3(n);
  const D1 G(Gamma);
  int st = s.stage(Un.data(), Un.data(), 1.0, 0.0, 1.0, dt, G, U1.data(), nullptr, nullptr);
  st = std::max(st, s.stage(Un.data(), U1.data(), 0.75, 0.25, 0.25, dt, G, U2.data(), nullptr, nullptr));
  st = std::max(st, s.stage(Un.data(), U2.data(), 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, dt, G, U3.data(), nullptr,
                            nullptr));
  split(U3, U_out, dU_out);
  return st;
}

int orc_primitives_jvp(const orc_params* p, const double* U, const double* dU, double* out, double* dout) {
  if (check(p)) return ORC_INVALID;
  Solver<D1> s(*p);
  const int nv = s.nv;
  int st = ORC_OK;
  for (size_t c = 0; c < s.G.ncell; ++c) {
    D1 Uc[MAXV];
    for (int v = 0; v < nv; ++v) {
      Uc[v].v = U[(size_t)v * s.G.ncell + c];
      Uc[v].d[0] = dU[(size_t)v * s.G.ncell + c];
    }
    Cell<D1> cl;
    cell_from_conserved(*p, p->dim, Uc, cl);
    st = std::max(st, cl.status);
    D1 o[8] = {cl.P, cl.T, cl.a, cl.rho, cl.phi[0], cl.phi[1], cl.psi, -cl.psi};
    for (int v = 0; v < 8; ++v) {
      out[(size_t)v * s.G.ncell + c] = o[v].v;
      dout[(size_t)v * s.G.ncell + c] = o[v].d[0];
    }
  }
  return st;
}

double orc_weno5z_jvp(const double* v5, const double* dv5, double eps, double* dout) {
  D1 v[5];
  for (int j = 0; j < 5; ++j) {
    v[j].v = v5[j];
    v[j].d[0] = dv5[j];
  }
  D1 r = weno5z(v[0], v[1], v[2], v[3], v[4], eps);
  *dout = r.d[0];
  return r.v;
}

int orc_init_state_jvp(const orc_params* p, const double* prim, const double* dprim, double* U, double* dU) {
  if (check(p)) return ORC_INVALID;
  Solver<D1> s(*p);
  const int ns = p->ns, D = p->dim, nv = ns + D + 1, nw = ns + D + 2;
  for (size_t c = 0; c < s.G.ncell; ++c) {
    D1 w[MAXV + 1], Uc[MAXV];
    for (int v = 0; v < nw; ++v) {
      w[v].v = prim[(size_t)v * s.G.ncell + c];
      w[v].d[0] = dprim[(size_t)v * s.G.ncell + c];
    }
    s.conserved_from_primitive(w, Uc);
    for (int v = 0; v < nv; ++v) {
      U[(size_t)v * s.G.ncell + c] = Uc[v].v;
      dU[(size_t)v * s.G.ncell + c] = Uc[v].d[0];
    }
  }
  return ORC_OK;
}

}  /* extern "C" */
