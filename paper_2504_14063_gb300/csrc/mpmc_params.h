// Kernel parameters (KParams) from the public descriptions of include/mpmc.h:
// grid and boundaries, NASG species constants (Sec. 2.2), model switches,
// the primitive-cache layout, and the FP32 roundings the mixed path reads.
// Shared by mpmc_create and mpmc_rhs_noalloc (host code).
#pragma once
#include <cmath>
#include <cstring>

#include "../../include/mpmc.h"
#include "mpmc_device.cuh"

namespace mpmc {

// MPMC_OK, or MPMC_INVALID_ARG for an ill-formed description (dimension,
// species count, cell counts, boundary codes, one-sided periodicity, dx,
// unknown precision).  P is fully written on success.
inline int build_params(const mpmc_grid* g, const mpmc_eos* eos, const mpmc_model* m, KParams& P) {
  if (!g || !eos || !m) return MPMC_INVALID_ARG;
  if (g->dim < 1 || g->dim > 3 || eos->n_species < 1 || eos->n_species > MPMC_MAXS || !(g->dx > 0.0))
    return MPMC_INVALID_ARG;
  if (m->precision != MPMC_FP64 && m->precision != MPMC_MIXED) return MPMC_INVALID_ARG;
  if (m->recon < MPMC_RECON_WENO5Z || m->recon > MPMC_RECON_TENO6) return MPMC_INVALID_ARG;
  if (m->viscous && (!(m->prandtl > 0.0) || !(m->lambda_liquid >= 0.0))) return MPMC_INVALID_ARG;
  for (int d = 0; d < 3; ++d) {
    if (d < g->dim && g->n[d] < 3) return MPMC_INVALID_ARG;
    if (d >= g->dim && g->n[d] != 1) return MPMC_INVALID_ARG;
    if (d < g->dim && (g->bc_lo[d] < 0 || g->bc_lo[d] > 4 || g->bc_hi[d] < 0 || g->bc_hi[d] > 4))
      return MPMC_INVALID_ARG;
    // characteristic boundaries along x only
    if (d > 0 && d < g->dim && (g->bc_lo[d] == MPMC_BC_CHAR || g->bc_hi[d] == MPMC_BC_CHAR))
      return MPMC_INVALID_ARG;
    if (d < g->dim && ((g->bc_lo[d] == MPMC_BC_PERIODIC) != (g->bc_hi[d] == MPMC_BC_PERIODIC)))
      return MPMC_INVALID_ARG;
  }
  // cells (plus the inflow slot and the characteristic ghost slots) and the
  // faces of each direction are indexed in 32 bits on the device
  {
    long long lim = (long long)g->n[0] * g->n[1] * g->n[2] + 1 + 2LL * g->n[1] * g->n[2];
    for (int d = 0; d < g->dim; ++d) {
      long long nf = 1;
      for (int e = 0; e < 3; ++e) nf *= (long long)g->n[e] + (e == d);
      if (nf > lim) lim = nf;
    }
    if (lim >= 2147483647LL) return MPMC_INVALID_ARG;
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
  // characteristic x boundaries: one ghost slot per boundary cell; their far
  // field is the inflow state
  P.char_lo = g->bc_lo[0] == MPMC_BC_CHAR ? 1 : 0;
  P.char_hi = g->bc_hi[0] == MPMC_BC_CHAR ? 1 : 0;
  P.nslots = (P.char_lo + P.char_hi) * g->n[1] * g->n[2];
  if (P.nslots) P.has_inflow = 1;
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
    P.cp[k] = eos->gamma[k] * eos->cv[k];
    if (eos->b[k] != 0.0) P.has_b = 1;
    if (eos->q[k] != 0.0) P.has_q = 1;
  }
  // Wilke's mixing rule (Sec. 2.4) in mass fractions: (W_i/W_j) Phi_ij
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < ns; ++j) {
      const double Wij = P.W[i] / P.W[j];
      const double t = 1.0 + std::sqrt(P.mu[i] / P.mu[j]) * std::pow(P.W[j] / P.W[i], 0.25);
      const double Phi = t * t / (std::sqrt(8.0) * std::sqrt(1.0 + Wij));
      P.wilke[i][j] = Wij * Phi;
    }
  P.two_phase = has0 && has1;
  P.weno_eps = m->weno_eps;
  P.cdi = m->cdi ? 1 : 0;
  P.diffusion = m->diffusion ? 1 : 0;
  P.pos_limiter = m->pos_limiter ? 1 : 0;
  P.recon = m->recon;
  P.viscous = m->viscous ? 1 : 0;
  P.prandtl = m->prandtl;
  P.lambda_liquid = m->lambda_liquid;
  P.cdi_eps = m->cdi_eps > 0.0 ? m->cdi_eps : g->dx;
  P.cdi_gamma = m->cdi_gamma;
  P.phi_min = m->phi_min;
  P.psi_delta = m->psi_delta;
  P.cfl = m->cfl;
  P.mu_liquid = m->mu_liquid;
  P.sharp0 = 4.0 * m->phi_min * (1.0 - m->phi_min);
  // primitive cache layout: field f of cell c at Wc[f * wstride + c]
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
  if (P.viscous) {
    P.wMu = f++;
    P.wLam = f++;
  }
  P.nW = f;
  P.wstride = P.ncell + 1 + P.nslots;
  P.gstride = 1 + P.nslots;
  P.nextra = P.has_inflow ? 1 + P.nslots : 0;
  round_consts32(P);
  return MPMC_OK;
}

}  // namespace mpmc
