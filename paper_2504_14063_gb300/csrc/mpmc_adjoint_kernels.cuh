// Kernels of the discrete adjoint (FP64), atomic-free and deterministic:
//   k_face_adj : per face of direction d, nu = c (lambda_{i+1} - lambda_i)/dx
//                and (dF/d inputs)^T nu, stored per face and per stencil
//                slot (plain stores, no accumulation)
//   k_gather   : per cell, the slots of every face whose stencil reaches the
//                cell (through the boundary mapping's preimages), summed in a
//                fixed order into the cell's cache adjoint gW and U adjoint
//   k_cell_adj : per cell, lambda_U = (dW/dU)^T gW + gU plus a linear
//                combination of stage adjoints (the reverse of Eq. SSPRK3)
//   k_init_vjp : reverse of the primitive -> conserved initialisation
// The forward decisions (theta_T, theta_P, first-order fallback, dropped
// regularization flux) come from the tape of the forward stage.
#pragma once
#include "mpmc_adjoint.cuh"
#include "mpmc_kernels.cuh"

namespace mpmc {
namespace adj {

constexpr int VJP_THREADS = 128;

// Slot layout of one face's contributions (field q of slot s at
// C[q_index * nf + face]):
//   line slots j = 0..5 (cells i-2..i+3 along d), NL fields each:
//     T, P, u_d, Y_0..Y_{NS-1}, the tangential u_t in increasing t
//   neighbour slots s = 0 (cell i), 1 (cell i+1), NB fields each:
//     rho, a, [CDI: (Y^c/Y_p)rho_p x NS, h_p rho_p x 2, phi_0, psi],
//     [diffusion: X^c/X_p x NS, W^c D^c_p/W_p x NS], U x NV
//   CDI: psi of the four tangential neighbours per tangential direction
//     (i + e_t, i - e_t, i + e_d + e_t, i + e_d - e_t)
//   viscous: mu, lambda in the neighbour slots, and the D velocity
//     components of the same four tangential neighbours per tangential
//     direction
// Values are adjoints of the quantities as the face sees them (wall-mirrored
// velocity components with their sign); the gather applies the mirror sign.
template <int NS, int D>
struct Lay {
  static constexpr int NV = NS + D + 1;
  static constexpr int NL = 2 + NS + D;
  int nb, qYr, qHr, qPhi, qPsi, qXr, qB, qMu, qLam, qU, psi0, vel0, total;
  __host__ __device__ Lay(int cdi, int diff, int visc = 0) {
    int q = 2;
    qYr = qHr = qPhi = qPsi = qXr = qB = qMu = qLam = -1;
    if (cdi) {
      qYr = q; q += NS;
      qHr = q; q += 2;
      qPhi = q++;
      qPsi = q++;
    }
    if (diff) {
      qXr = q; q += NS;
      qB = q; q += NS;
    }
    if (visc) {
      qMu = q++;
      qLam = q++;
    }
    qU = q;
    q += NV;
    nb = q;
    psi0 = 6 * NL + 2 * nb;
    vel0 = psi0 + (cdi ? 4 * (D - 1) : 0);
    total = vel0 + (visc ? 4 * (D - 1) * D : 0);
  }
  // velocity component i of tangential neighbour q (0..3) of tangential
  // direction number tt
  __host__ __device__ int vel(int tt, int q, int i) const { return vel0 + (tt * 4 + q) * D + i; }
  __host__ __device__ int line(int j, int q) const { return j * NL + q; }
  __host__ __device__ int nbq(int s, int q) const { return 6 * NL + s * nb + q; }
};

// mass-fraction limiter (Sec. 3.3.1) with its intermediates, and its reverse
template <int NS>
struct YLim {
  double Yin[NS], Yc[NS], Y1[NS], m[NS], f, Sig, sum;
  bool corrected, over, pick[NS];
};

template <int NS>
__device__ __forceinline__ void ylim_fwd(YLim<NS>& s, double* Y) {
  double sum = 0.0;
  for (int k = 0; k < NS; ++k) {
    s.Yin[k] = Y[k];
    s.Y1[k] = Y[k] < 0.0 ? 0.0 : Y[k];
    sum += s.Y1[k];
  }
  s.sum = sum;
  s.corrected = false;
  if (fabs(sum - 1.0) > NS * YSUM_TOL) {
    s.over = sum > 1.0;
    double Sig = 0.0;
    for (int k = 0; k < NS; ++k) {
      const double mm = s.over ? fmin(s.Y1[k], s.Yc[k]) : fmax(s.Y1[k], s.Yc[k]);
      s.pick[k] = s.over ? (s.Y1[k] <= s.Yc[k]) : (s.Y1[k] >= s.Yc[k]);
      s.m[k] = mm - s.Y1[k];
      Sig += s.m[k];
    }
    s.Sig = Sig;
    if (nonzero(Sig)) {
      s.f = (1.0 - sum) / Sig;
      s.corrected = true;
    }
  }
  for (int k = 0; k < NS; ++k) Y[k] = s.corrected ? s.Y1[k] + s.f * s.m[k] : s.Y1[k];
}

template <int NS>
__device__ __forceinline__ void ylim_rev(const YLim<NS>& s, const double* lout, double* lY, double* lYc) {
  double l1[NS];
  for (int k = 0; k < NS; ++k) l1[k] = lout[k];
  if (s.corrected) {
    double lf = 0.0;
    for (int k = 0; k < NS; ++k) lf += lout[k] * s.m[k];
    const double lsum = -lf / s.Sig;
    const double lSig = -lf * s.f / s.Sig;
    for (int k = 0; k < NS; ++k) {
      const double lm = lout[k] * s.f + lSig;
      l1[k] += lsum - lm;
      if (s.pick[k]) l1[k] += lm;
      else lYc[k] += lm;
    }
  }
  for (int k = 0; k < NS; ++k) lY[k] += s.Yin[k] < 0.0 ? 0.0 : l1[k];
}

// Face-average scalars of the characteristic matrices (Appendix A):
// X = (rho a^2 beta - 1) / (alpha a^2 rho) and c = rho a at the arithmetic
// average of the two cells' conserved states, with what the reverse needs.
template <int NS, int D>
struct FaceAvg {
  double Ub[NS + D + 1], rb, Yb[NS], ub[3], eb, vb, pb, Tb, XN, XD, X, c;
  Thermo<NS> tb;
};

template <int NS, int D>
__device__ __forceinline__ void face_avg_fwd(const KParams& P, const double* Uk, const double* Uin, CRef ri, CRef rj,
                                             FaceAvg<NS, D>& f, double p_guess) {
  constexpr int NV = NS + D + 1;
  double Ui[NV], Uj[NV];
  load_U<NS, D>(P, Uk, Uin, ri, Ui);
  load_U<NS, D>(P, Uk, Uin, rj, Uj);
#pragma unroll
  for (int v = 0; v < NV; ++v) f.Ub[v] = 0.5 * (Ui[v] + Uj[v]);
  decode<NS, D, false>(f.Ub, f.rb, f.Yb, f.ub, f.eb, f.vb);
  pt_equilibrium<NS, false>(P, f.Yb, f.eb, f.vb, f.pb, f.Tb, f.rb, p_guess);
#pragma unroll
  for (int k = 0; k < NS; ++k) f.tb.Y[k] = f.Yb[k];
  f.tb.p = f.pb;
  f.tb.T = f.Tb;
  thermo_fwd<NS>(P, f.tb);
  const double a2 = f.tb.a * f.tb.a;
  f.XN = f.rb * a2 * f.tb.be - 1.0;
  f.XD = f.tb.al * a2 * f.rb;
  f.X = f.XN / f.XD;
  f.c = f.tb.a * f.rb;
}

// adjoints of X and c -> adjoint of the averaged conserved state Ub
template <int NS, int D>
__device__ __forceinline__ void face_avg_rev(const KParams& P, const FaceAvg<NS, D>& f, double lX, double lc,
                                             double* lUb) {
  const double a = f.tb.a, a2 = a * a;
  double lrho = lc * a, la = lc * f.rb;
  const double lXN = lX / f.XD, lXD = -lX * f.X / f.XD;
  lrho += lXN * a2 * f.tb.be + lXD * f.tb.al * a2;
  la += (lXN * f.rb * f.tb.be + lXD * f.tb.al * f.rb) * 2.0 * a;
  const double lbe = lXN * f.rb * a2, lal = lXD * a2 * f.rb;
  double lYb[NS], lpb = 0.0, lTb = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) lYb[k] = 0.0;
  thermo_rev<NS>(P, f.tb, 0.0, 0.0, la, lal, lbe, lYb, lpb, lTb);
  double leb = 0.0, lvb = 0.0;
  pt_rev<NS>(P, f.Yb, f.pb, f.Tb, f.tb.r, lpb, lTb, lYb, leb, lvb);
  const double lub[3] = {0.0, 0.0, 0.0};
  decode_rev<NS, D>(f.Ub, f.rb, f.Yb, f.ub, lrho, lYb, lub, leb, lvb, lUb);
}

// DIR: the face direction, a template parameter so that every array indexed
// by it is indexed by a constant.  RC: the interpolation (RC_WENO5Z or one of
// Sec. 4.1's others)
template <int NS, int D, int DIR, int RC>
__global__ void __launch_bounds__(VJP_THREADS)
    k_face_adj(const KParams P, const double* __restrict__ Wc, const double* __restrict__ Uk,
               const double* __restrict__ Uin, const double* __restrict__ scal, const uint32_t* __restrict__ tape,
               const double* __restrict__ lamL, const double coef, const int mul_dt, double* __restrict__ C) {
  constexpr int NV = NS + D + 1;
  constexpr int d = DIR;
  const int f0 = P.n[0] + (d == 0), f1 = P.n[1] + (d == 1), f2 = P.n[2] + (d == 2);
  const long long nf = (long long)f0 * f1 * f2;
  const long long fid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (fid >= nf) return;
  const Lay<NS, D> L(P.cdi, P.diffusion, P.viscous);
  auto put = [&](int q, double v) { C[(long long)q * nf + fid] = v; };
  int fc[3];
  unflatten(fid, f0, f1, fc);
  int ci[3] = {fc[0], fc[1], fc[2]};
  ci[d] -= 1;
  const double Gamma = scal[1];
  const double eps = P.weno_eps;
  // d(stage output)/dF = coef (dt) (lambda_{i+1} - lambda_i) / dx
  const double sc = (mul_dt ? coef * scal[0] : coef) * P.inv_dx;

  CRef cr[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    int cc[3] = {ci[0], ci[1], ci[2]};
    cc[d] += j - 2;
    cr[j] = map_cell_m<1u << d, false>(P, cc[0], cc[1], cc[2]);
  }
  const CRef ri = cr[2], rj = cr[3];
  // adjoint of this face's flux: F enters L_i with -1/dx and L_{i+1} with +1/dx
  const bool real_i = ci[d] >= 0, real_j = ci[d] + 1 <= P.n[d] - 1;
  double nu[NV];
  bool any = false;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double a = real_j ? lamL[(long long)v * P.ncell + rj.idx] : 0.0;
    const double b = real_i ? lamL[(long long)v * P.ncell + ri.idx] : 0.0;
    nu[v] = (a - b) * sc;
    any = any || nonzero(nu[v]);
  }
  if (!any) {
    for (int q = 0; q < L.total; ++q) put(q, 0.0);
    return;
  }
  const uint32_t fl = tape[fid];
  // six-cell stencil of a cache field (velocity components with the wall sign)
  auto stencil = [&](int f, int t, double* y) {
#pragma unroll
    for (int j = 0; j < 6; ++j) y[j] = wget(P, Wc, f, cr[j]) * (t >= 0 ? sgn_flip(cr[j].flip, t) : 1.0);
  };

  // ================= forward recomputation (values only) =================
  FaceAvg<NS, D> fa;
  // the forward face kernel's start for the averaged state's pressure
  face_avg_fwd<NS, D>(P, Uk, Uin, ri, rj, fa, 0.5 * (wget(P, Wc, P.wP, ri) + wget(P, Wc, P.wP, rj)));
  const double X = fa.X, c = fa.c, ic = 1.0 / c;
  // reconstruction values with their gradients w.r.t. the stencil values
  double TL, TR, PL, PR, uL[3] = {0.0, 0.0, 0.0}, uR[3] = {0.0, 0.0, 0.0};
  // gradients over the six stencil cells (the last entry zero for the
  // five-cell interpolations); the right side's gradient index runs mirrored
  double g1L[6], g1R[6], g5L[6], g5R[6], g6L[6], g6R[6], w5L, w5R, w6L, w6R;
  double gYL[NS][6], gYR[NS][6], gtL[2][6], gtR[2][6];
  {
    double w1[6], w5[6], w6[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const double Tj_ = wget(P, Wc, P.wT, cr[j]), Pj_ = wget(P, Wc, P.wP, cr[j]);
      const double un = wget(P, Wc, P.wU + d, cr[j]) * sgn_flip(cr[j].flip, d);
      w1[j] = Tj_ - X * Pj_;
      w5[j] = (0.5 * c) * un + 0.5 * Pj_;
      w6[j] = (-0.5 * c) * un + 0.5 * Pj_;
    }
    const double w1L = recon_val_grad<RC>(w1[0], w1[1], w1[2], w1[3], w1[4], w1[5], eps, g1L);
    const double w1R = recon_val_grad<RC>(w1[5], w1[4], w1[3], w1[2], w1[1], w1[0], eps, g1R);
    w5L = recon_val_grad<RC>(w5[0], w5[1], w5[2], w5[3], w5[4], w5[5], eps, g5L);
    w5R = recon_val_grad<RC>(w5[5], w5[4], w5[3], w5[2], w5[1], w5[0], eps, g5R);
    w6L = recon_val_grad<RC>(w6[0], w6[1], w6[2], w6[3], w6[4], w6[5], eps, g6L);
    w6R = recon_val_grad<RC>(w6[5], w6[4], w6[3], w6[2], w6[1], w6[0], eps, g6R);
    TL = w1L + X * w5L + X * w6L;
    TR = w1R + X * w5R + X * w6R;
    uL[d] = ic * w5L + (-ic) * w6L;
    uR[d] = ic * w5R + (-ic) * w6R;
    PL = w5L + w6L;
    PR = w5R + w6R;
  }
  double YLp[NS], YRp[NS];   // before the Y limiter
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    double y[6];
    stencil(P.wY + k, -1, y);
    YLp[k] = recon_val_grad<RC>(y[0], y[1], y[2], y[3], y[4], y[5], eps, gYL[k]);
    YRp[k] = recon_val_grad<RC>(y[5], y[4], y[3], y[2], y[1], y[0], eps, gYR[k]);
  }
  {
    int tt = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      if (t == d) continue;
      double y[6];
      stencil(P.wU + t, t, y);
      uL[t] = recon_val_grad<RC>(y[0], y[1], y[2], y[3], y[4], y[5], eps, gtL[tt]);
      uR[t] = recon_val_grad<RC>(y[5], y[4], y[3], y[2], y[1], y[0], eps, gtR[tt]);
      ++tt;
    }
  }
  double Yi[NS], Yj[NS], YL[NS], YR[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    Yi[k] = wget(P, Wc, P.wY + k, ri);
    Yj[k] = wget(P, Wc, P.wY + k, rj);
    YL[k] = YLp[k];
    YR[k] = YRp[k];
  }
  const double Ti = wget(P, Wc, P.wT, ri), Tj = wget(P, Wc, P.wT, rj);
  const double Pi = wget(P, Wc, P.wP, ri), Pj = wget(P, Wc, P.wP, rj);
  if (P.pos_limiter) {
    YLim<NS> yl, yr;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      yl.Yc[k] = Yi[k];
      yr.Yc[k] = Yj[k];
    }
    ylim_fwd<NS>(yl, YL);
    ylim_fwd<NS>(yr, YR);
    if (fl & F_THETA_T_L) TL = Ti;
    if (fl & F_THETA_T_R) TR = Tj;
    if (fl & F_THETA_P_L) PL = Pi;
    if (fl & F_THETA_P_R) PR = Pj;
  }
  const bool fallback = (fl & F_HLLC_FALLBACK) != 0;

  // ================= reverse sweep =================
  // adjoints gathered on the two neighbour cells (slots 2 and 3) before the
  // reconstruction's reverse; index 0 = cell i, 1 = cell i+1
  double aT[2] = {0.0, 0.0}, aP[2] = {0.0, 0.0}, aY[2][NS], aU3[2][3], aRho[2] = {0.0, 0.0}, aA[2] = {0.0, 0.0};
  double aU[2][NV];
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
#pragma unroll
    for (int k = 0; k < NS; ++k) aY[s2][k] = 0.0;
#pragma unroll
    for (int t = 0; t < 3; ++t) aU3[s2][t] = 0.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) aU[s2][v] = 0.0;
  }

  // ---- species diffusion (Eq. SpeciesMassDiffusion), stores its cache slots
  // (zeros where the forward pass dropped the diffusive flux)
  if (P.diffusion) {
    const bool dropped = (fl & F_DIFF_DROPPED) != 0;
    const double rbar = 0.5 * (wget(P, Wc, P.wRho, ri) + wget(P, Wc, P.wRho, rj));
    double lrb = 0.0;
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
      double lYp = 0.0, lS = 0.0, lBf[NS], lG[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        lBf[k] = 0.0;
        lG[k] = 0.0;
        if (P.phase[k] != ph) continue;
        const double Ybk = 0.5 * (Yi[k] + Yj[k]);
        const double J = -rbar * (Yp * Bf[k] * G[k] - Ybk * S);
        const double hi = h_k(P, k, Pi, Ti), hj = h_k(P, k, Pj, Tj);
        const double lJ = dropped ? 0.0 : nu[k] + nu[NS + D] * 0.5 * (hi + hj);
        const double lh = dropped ? 0.0 : nu[NS + D] * J * 0.5;
        aT[0] += lh * P.cp[k];
        aP[0] += lh * P.b[k];
        aT[1] += lh * P.cp[k];
        aP[1] += lh * P.b[k];
        lrb -= lJ * (Yp * Bf[k] * G[k] - Ybk * S);
        lYp -= rbar * lJ * Bf[k] * G[k];
        lBf[k] -= rbar * lJ * Yp * G[k];
        lG[k] -= rbar * lJ * Yp * Bf[k];
        const double lYb = rbar * lJ * S;
        aY[0][k] += 0.5 * lYb;
        aY[1][k] += 0.5 * lYb;
        lS += rbar * lJ * Ybk;
      }
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        if (P.phase[k] != ph) continue;
        lBf[k] += lS * G[k];
        lG[k] += lS * Bf[k];
        aY[0][k] += 0.5 * lYp;
        aY[1][k] += 0.5 * lYp;
        put(L.nbq(0, L.qB + k), 0.5 * lBf[k]);
        put(L.nbq(1, L.qB + k), 0.5 * lBf[k]);
        put(L.nbq(1, L.qXr + k), lG[k] * P.inv_dx);
        put(L.nbq(0, L.qXr + k), -lG[k] * P.inv_dx);
      }
    }
    aRho[0] += 0.5 * lrb;
    aRho[1] += 0.5 * lrb;
  }

  // ---- interface regularization (if the forward added it), stores its slots
  if (P.cdi) {
    double cYr[2][NS], cHr[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, cPhi[2] = {0.0, 0.0}, cPsi[2] = {0.0, 0.0};
    double cPsiT[2][4];
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
#pragma unroll
      for (int k = 0; k < NS; ++k) cYr[s2][k] = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) cPsiT[s2][q] = 0.0;
    }
    bool pres_i[2], pres_j[2];
    {
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
    if (P.two_phase && !(fl & F_CDI_DROPPED) && (pres_i[0] || pres_j[0]) && (pres_i[1] || pres_j[1])) {
      const double ceps = P.cdi_eps;
      const double psi_i = wget(P, Wc, P.wPsi, ri), psi_j = wget(P, Wc, P.wPsi, rj);
      const double dphi = (wget(P, Wc, P.wPhi0, rj) - wget(P, Wc, P.wPhi0, ri)) * P.inv_dx;
      double g[3] = {0.0, 0.0, 0.0};
      g[d] = (psi_j - psi_i) * P.inv_dx;
#pragma unroll
      for (int t = 0; t < D; ++t) {
        if (t == d) continue;
        int a0[3] = {ci[0], ci[1], ci[2]}, a1[3] = {ci[0], ci[1], ci[2]};
        a0[t] += 1;
        a1[t] -= 1;
        int b0[3] = {a0[0], a0[1], a0[2]}, b1[3] = {a1[0], a1[1], a1[2]};
        b0[d] += 1;
        b1[d] += 1;
        g[t] = 0.5 * ((wget(P, Wc, P.wPsi, map_cell_dt<d, false>(P, t, a0[0], a0[1], a0[2])) -
                       wget(P, Wc, P.wPsi, map_cell_dt<d, false>(P, t, a1[0], a1[1], a1[2]))) * (0.5 * P.inv_dx) +
                      (wget(P, Wc, P.wPsi, map_cell_dt<d, false>(P, t, b0[0], b0[1], b0[2])) -
                       wget(P, Wc, P.wPsi, map_cell_dt<d, false>(P, t, b1[0], b1[1], b1[2]))) * (0.5 * P.inv_dx));
      }
      const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      const bool nact = gn >= GTOL;
      const double nd = nact ? g[d] / gn : 0.0;
      const double xarg = (0.5 * (psi_i + psi_j)) / (2.0 * ceps);
      const double ch = cosh(xarg);
      const double sech2 = 1.0 / (ch * ch);
      const double ahat0 = Gamma * (ceps * dphi - 0.25 * (sech2 - P.sharp0) * nd);
      double Rtot = 0.0, kb = 0.0;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const bool pi = P.phase[k] ? pres_i[1] : pres_i[0], pj = P.phase[k] ? pres_j[1] : pres_j[0];
        const double yi = wget(P, Wc, P.wYrho + k, ri), yj = wget(P, Wc, P.wYrho + k, rj);
        const double kp = pi && pj ? 0.5 * (yi + yj) : (pi ? yi : (pj ? yj : 0.0));
        Rtot += -kp * (P.phase[k] == 0 ? ahat0 : -ahat0);
      }
      double ui[3] = {0.0, 0.0, 0.0}, uj[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int t = 0; t < D; ++t) {
        ui[t] = wget(P, Wc, P.wU + t, ri) * sgn_flip(ri.flip, t);
        uj[t] = wget(P, Wc, P.wU + t, rj) * sgn_flip(rj.flip, t);
        kb += ui[t] * uj[t];
      }
      double lRtot = nu[NS + D] * 0.5 * kb;
      const double lkb = nu[NS + D] * 0.5 * Rtot;
#pragma unroll
      for (int t = 0; t < D; ++t) {
        lRtot += nu[NS + t] * 0.5 * (ui[t] + uj[t]);
        aU3[0][t] += nu[NS + t] * 0.5 * Rtot + lkb * uj[t];
        aU3[1][t] += nu[NS + t] * 0.5 * Rtot + lkb * ui[t];
      }
      const double lhR = nu[NS + D];
      double lahat0 = 0.0;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const int ph = P.phase[k];
        const bool pi = pres_i[ph], pj = pres_j[ph];
        const double yi = wget(P, Wc, P.wYrho + k, ri), yj = wget(P, Wc, P.wYrho + k, rj);
        const double kp = pi && pj ? 0.5 * (yi + yj) : (pi ? yi : (pj ? yj : 0.0));
        const double sgn = ph == 0 ? 1.0 : -1.0;
        const double lR = nu[k] + lRtot;   // R_k = -kp sgn ahat0
        const double lkp = -lR * sgn * ahat0;
        lahat0 += -lR * kp * sgn;
        if (pi && pj) {
          cYr[0][k] = 0.5 * lkp;
          cYr[1][k] = 0.5 * lkp;
        } else if (pi) {
          cYr[0][k] = lkp;
        } else if (pj) {
          cYr[1][k] = lkp;
        }
      }
#pragma unroll
      for (int ph = 0; ph < 2; ++ph) {
        const bool pi = pres_i[ph], pj = pres_j[ph];
        const double hi = wget(P, Wc, P.wHrho + ph, ri), hj = wget(P, Wc, P.wHrho + ph, rj);
        const double kh = pi && pj ? 0.5 * (hi + hj) : (pi ? hi : (pj ? hj : 0.0));
        const double sgn = ph == 0 ? 1.0 : -1.0;   // hR -= kh sgn ahat0
        const double lkh = -lhR * sgn * ahat0;
        lahat0 += -lhR * kh * sgn;
        if (pi && pj) {
          cHr[0][ph] = 0.5 * lkh;
          cHr[1][ph] = 0.5 * lkh;
        } else if (pi) {
          cHr[0][ph] = lkh;
        } else if (pj) {
          cHr[1][ph] = lkh;
        }
      }
      // ahat0 = Gamma (eps dphi - 0.25 (sech2 - sharp0) nd)
      const double ldphi = lahat0 * Gamma * ceps;
      const double lsech2 = -0.25 * Gamma * nd * lahat0;
      const double lnd = -0.25 * Gamma * (sech2 - P.sharp0) * lahat0;
      cPhi[1] = ldphi * P.inv_dx;
      cPhi[0] = -ldphi * P.inv_dx;
      // sech2 = 1/cosh^2(x), x = (psi_i + psi_j) / (4 eps)
      const double lx = lsech2 * (-2.0 * sinh(xarg) / (ch * ch * ch));
      double lpsi_i = lx * 0.25 / ceps, lpsi_j = lx * 0.25 / ceps;
      if (nact) {
        double lg[3];
        const double lgn = -lnd * g[d] / (gn * gn);
#pragma unroll
        for (int t = 0; t < 3; ++t) lg[t] = lgn * g[t] / gn;
        lg[d] += lnd / gn;
        lpsi_j += lg[d] * P.inv_dx;
        lpsi_i -= lg[d] * P.inv_dx;
        int tt = 0;
#pragma unroll
        for (int t = 0; t < D; ++t) {
          if (t == d) continue;
          const double w = lg[t] * 0.25 * P.inv_dx;
          cPsiT[tt][0] = w;
          cPsiT[tt][1] = -w;
          cPsiT[tt][2] = w;
          cPsiT[tt][3] = -w;
          ++tt;
        }
      }
      cPsi[0] = lpsi_i;
      cPsi[1] = lpsi_j;
    }
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
#pragma unroll
      for (int k = 0; k < NS; ++k) put(L.nbq(s2, L.qYr + k), cYr[s2][k]);
      put(L.nbq(s2, L.qHr), cHr[s2][0]);
      put(L.nbq(s2, L.qHr + 1), cHr[s2][1]);
      put(L.nbq(s2, L.qPhi), cPhi[s2]);
      put(L.nbq(s2, L.qPsi), cPsi[s2]);
    }
#pragma unroll
    for (int tt = 0; tt < D - 1; ++tt)
#pragma unroll
      for (int q = 0; q < 4; ++q) put(L.psi0 + 4 * tt + q, cPsiT[tt][q]);
  }

  // ---- face states and HLLC (Appendix B), built here and reversed at once
  double lTL = 0.0, lTR = 0.0, lPL = 0.0, lPR = 0.0, lYL[NS], lYR[NS], luL[3] = {0.0, 0.0, 0.0},
         luR[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    lYL[k] = 0.0;
    lYR[k] = 0.0;
  }
  if (!fallback) {
    Thermo<NS> tL, tR;
    St<NS> sL, sR;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      tL.Y[k] = YL[k];
      tR.Y[k] = YR[k];
    }
    tL.p = PL;
    tL.T = TL;
    tR.p = PR;
    tR.T = TR;
    face_state<NS>(P, tL, uL, sL);
    face_state<NS>(P, tR, uR, sR);
    StAdj<NS> gL, gR;
    gL.zero();
    gR.zero();
    hllc_rev<NS, D>(d, sL, sR, nu, gL, gR);
    face_state_rev<NS>(P, tL, sL, gL, lYL, luL, lPL, lTL);
    face_state_rev<NS>(P, tR, sR, gR, lYR, luR, lPR, lTR);
  } else {
    // first-order fallback: HLLC of the two cells' own states
    St<NS> sL, sR;
    double Ui[NV], Uj[NV];
    load_U<NS, D>(P, Uk, Uin, ri, Ui);
    load_U<NS, D>(P, Uk, Uin, rj, Uj);
    sL.rho = wget(P, Wc, P.wRho, ri);
    sR.rho = wget(P, Wc, P.wRho, rj);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      sL.rhoY[k] = Ui[k];
      sR.rhoY[k] = Uj[k];
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      sL.u[t] = t < D ? wget(P, Wc, P.wU + t, ri) * sgn_flip(ri.flip, t) : 0.0;
      sR.u[t] = t < D ? wget(P, Wc, P.wU + t, rj) * sgn_flip(rj.flip, t) : 0.0;
      sL.m[t] = t < D ? Ui[NS + t] : 0.0;
      sR.m[t] = t < D ? Uj[NS + t] : 0.0;
    }
    sL.p = Pi;
    sR.p = Pj;
    sL.E = Ui[NS + D];
    sR.E = Uj[NS + D];
    sL.a = wget(P, Wc, P.wA, ri);
    sR.a = wget(P, Wc, P.wA, rj);
    StAdj<NS> gL, gR;
    gL.zero();
    gR.zero();
    hllc_rev<NS, D>(d, sL, sR, nu, gL, gR);
    aRho[0] += gL.rho;
    aRho[1] += gR.rho;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      aU[0][k] += gL.rhoY[k];
      aU[1][k] += gR.rhoY[k];
    }
#pragma unroll
    for (int t = 0; t < D; ++t) {
      aU3[0][t] += gL.u[t];
      aU3[1][t] += gR.u[t];
      aU[0][NS + t] += gL.m[t];
      aU[1][NS + t] += gR.m[t];
    }
    aP[0] += gL.p;
    aP[1] += gR.p;
    aU[0][NS + D] += gL.E;
    aU[1][NS + D] += gR.E;
    aA[0] += gL.a;
    aA[1] += gR.a;
  }

  // ---- interpolation limiters (replayed; the Y limiter recomputed)
  if (P.pos_limiter) {
    if (fl & F_THETA_T_L) { aT[0] += lTL; lTL = 0.0; }
    if (fl & F_THETA_T_R) { aT[1] += lTR; lTR = 0.0; }
    if (fl & F_THETA_P_L) { aP[0] += lPL; lPL = 0.0; }
    if (fl & F_THETA_P_R) { aP[1] += lPR; lPR = 0.0; }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      YLim<NS> ylm;
      double tmp[NS], lin[NS], lc_[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        ylm.Yc[k] = side ? Yj[k] : Yi[k];
        tmp[k] = side ? YRp[k] : YLp[k];
        lin[k] = 0.0;
        lc_[k] = 0.0;
      }
      ylim_fwd<NS>(ylm, tmp);
      ylim_rev<NS>(ylm, side ? lYR : lYL, lin, lc_);
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        if (side) lYR[k] = lin[k];
        else lYL[k] = lin[k];
        aY[side][k] += lc_[k];
      }
    }
  }

  // ---- WENO of mass fractions and tangential velocities, reversed; slots stored
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    double gj[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) gj[j] = lYL[k] * gYL[k][j] + lYR[k] * gYR[k][5 - j];
    gj[2] += aY[0][k];
    gj[3] += aY[1][k];
#pragma unroll
    for (int j = 0; j < 6; ++j) put(L.line(j, 3 + k), gj[j]);
  }
  {
    int tt = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      if (t == d) continue;
      double gj[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) gj[j] = luL[t] * gtL[tt][j] + luR[t] * gtR[tt][5 - j];
      gj[2] += aU3[0][t];
      gj[3] += aU3[1][t];
#pragma unroll
      for (int j = 0; j < 6; ++j) put(L.line(j, 3 + NS + tt), gj[j]);
      ++tt;
    }
  }

  // ---- characteristic reconstruction, reversed: T = w1 + X (w5 + w6),
  // u = ic (w5 - w6), P = w5 + w6 back-projection; w1 = T - X P,
  // w5/6 = +-c/2 u + P/2 projection (Appendix A); slots stored
  double lX = 0.0, lc;
  {
    const double l1L = lTL, l5L = X * lTL + ic * luL[d] + lPL, l6L = X * lTL - ic * luL[d] + lPL;
    const double l1R = lTR, l5R = X * lTR + ic * luR[d] + lPR, l6R = X * lTR - ic * luR[d] + lPR;
    lX += lTL * (w5L + w6L) + lTR * (w5R + w6R);
    const double lic = luL[d] * (w5L - w6L) + luR[d] * (w5R - w6R);
    lc = -lic * ic * ic;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      // left stencil v = w[0..5], right stencil v = w[5..0]
      const double lw1 = l1L * g1L[j] + l1R * g1R[5 - j];
      const double lw5 = l5L * g5L[j] + l5R * g5R[5 - j];
      const double lw6 = l6L * g6L[j] + l6R * g6R[5 - j];
      const double Pj_ = wget(P, Wc, P.wP, cr[j]);
      const double un = wget(P, Wc, P.wU + d, cr[j]) * sgn_flip(cr[j].flip, d);
      double gT_ = lw1;
      double gP_ = -X * lw1 + 0.5 * (lw5 + lw6);
      double gu_ = 0.5 * c * (lw5 - lw6);
      lX -= Pj_ * lw1;
      lc += 0.5 * un * (lw5 - lw6);
      if (j == 2 || j == 3) {
        gT_ += aT[j - 2];
        gP_ += aP[j - 2];
        gu_ += aU3[j - 2][d];
      }
      put(L.line(j, 0), gT_);
      put(L.line(j, 1), gP_);
      put(L.line(j, 2), gu_);
    }
  }

  // ---- face-average scalars, reversed
  {
    double lUb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) lUb[v] = 0.0;
    face_avg_rev<NS, D>(P, fa, lX, lc, lUb);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      aU[0][v] += 0.5 * lUb[v];
      aU[1][v] += 0.5 * lUb[v];
    }
  }
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    put(L.nbq(s2, 0), aRho[s2]);
    put(L.nbq(s2, 1), aA[s2]);
#pragma unroll
    for (int v = 0; v < NV; ++v) put(L.nbq(s2, L.qU + v), aU[s2][v]);
  }
}

// preimages of real index c along one axis (length n, boundary codes lo/hi)
// under the boundary mapping, with the mirror sign of a wall image; the
// stencils reach three ghost layers
struct Pre {
  int g[5];
  signed char s[5];
  int n;
};

__device__ __forceinline__ Pre preimages(int c, int n, int lo, int hi) {
  Pre p;
  p.n = 0;
  p.g[p.n] = c; p.s[p.n++] = 1;
  if (lo == BC_PERIODIC) {
    if (c - n >= -3) { p.g[p.n] = c - n; p.s[p.n++] = 1; }
  } else if (lo == BC_WALL) {
    if (c <= 2) { p.g[p.n] = -1 - c; p.s[p.n++] = -1; }
  } else if (lo == BC_ZEROGRAD) {
    if (c == 0) {
      p.g[p.n] = -1; p.s[p.n++] = 1;
      p.g[p.n] = -2; p.s[p.n++] = 1;
      p.g[p.n] = -3; p.s[p.n++] = 1;
    }
  }
  if (hi == BC_PERIODIC) {
    if (c + n <= n + 2) { p.g[p.n] = c + n; p.s[p.n++] = 1; }
  } else if (hi == BC_WALL) {
    if (c >= n - 3) { p.g[p.n] = 2 * n - 1 - c; p.s[p.n++] = -1; }
  } else if (hi == BC_ZEROGRAD) {
    if (c == n - 1) {   // at most 5 entries in all: n >= 3
      p.g[p.n] = n; p.s[p.n++] = 1;
      p.g[p.n] = n + 1; p.s[p.n++] = 1;
      p.g[p.n] = n + 2; p.s[p.n++] = 1;
    }
  }
  return p;
}

// Per face of direction DIR, after k_face_adj: the reverse of the viscous
// stress and heat-conduction flux (Eq. DiffusionTerms, second-order central,
// as k_face): adds to the T and velocity line slots of the two face cells and
// writes the mu, lambda slots and the tangential neighbours' velocity slots
// (zeros where the forward pass dropped the diffusive flux).
template <int NS, int D, int DIR>
__global__ void __launch_bounds__(VJP_THREADS)
    k_face_visc_adj(const KParams P, const double* __restrict__ Wc, const double* __restrict__ scal,
                    const uint32_t* __restrict__ tape, const double* __restrict__ lamL, const double coef,
                    const int mul_dt, double* __restrict__ C) {
  constexpr int NV = NS + D + 1;
  constexpr int d = DIR;
  const int f0 = P.n[0] + (d == 0), f1 = P.n[1] + (d == 1), f2 = P.n[2] + (d == 2);
  const long long nf = (long long)f0 * f1 * f2;
  const long long fid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (fid >= nf) return;
  const Lay<NS, D> L(P.cdi, P.diffusion, P.viscous);
  int fc[3];
  unflatten(fid, f0, f1, fc);
  int ci[3] = {fc[0], fc[1], fc[2]};
  ci[d] -= 1;
  const CRef ri = map_cell_m<1u << d, false>(P, ci[0], ci[1], ci[2]);
  int cj3[3] = {ci[0], ci[1], ci[2]};
  cj3[d] += 1;
  const CRef rj = map_cell_m<1u << d, false>(P, cj3[0], cj3[1], cj3[2]);
  const double sc = (mul_dt ? coef * scal[0] : coef) * P.inv_dx;
  const bool real_i = ci[d] >= 0, real_j = ci[d] + 1 <= P.n[d] - 1;
  double nu[NV];
  bool any = false;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double a = real_j ? lamL[(long long)v * P.ncell + rj.idx] : 0.0;
    const double b = real_i ? lamL[(long long)v * P.ncell + ri.idx] : 0.0;
    nu[v] = (a - b) * sc;
    any = any || nonzero(nu[v]);
  }
  // (k_face_adj has zeroed every slot of a face whose flux adjoint is zero)
  if (!any) return;
  if (tape[fid] & F_DIFF_DROPPED) {
#pragma unroll
    for (int v = 0; v < NV; ++v) nu[v] = 0.0;
  }
  auto put = [&](int q, double v) { C[(long long)q * nf + fid] = v; };
  auto add = [&](int q, double v) { C[(long long)q * nf + fid] += v; };

  // forward values
  double gu[3][3];
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
  CRef tn[3][4];  // tangential neighbours: i + e_t, i - e_t, j + e_t, j - e_t
#pragma unroll
  for (int t = 0; t < D; ++t) {
    if (t == d) continue;
    int a0[3] = {ci[0], ci[1], ci[2]}, a1[3] = {ci[0], ci[1], ci[2]};
    a0[t] += 1;
    a1[t] -= 1;
    int b0[3] = {a0[0], a0[1], a0[2]}, b1[3] = {a1[0], a1[1], a1[2]};
    b0[d] += 1;
    b1[d] += 1;
    tn[t][0] = map_cell_dt<d, false>(P, t, a0[0], a0[1], a0[2]);
    tn[t][1] = map_cell_dt<d, false>(P, t, a1[0], a1[1], a1[2]);
    tn[t][2] = map_cell_dt<d, false>(P, t, b0[0], b0[1], b0[2]);
    tn[t][3] = map_cell_dt<d, false>(P, t, b1[0], b1[1], b1[2]);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double dip = wget(P, Wc, P.wU + i, tn[t][0]) * sgn_flip(tn[t][0].flip, i) -
                         wget(P, Wc, P.wU + i, tn[t][1]) * sgn_flip(tn[t][1].flip, i);
      const double djp = wget(P, Wc, P.wU + i, tn[t][2]) * sgn_flip(tn[t][2].flip, i) -
                         wget(P, Wc, P.wU + i, tn[t][3]) * sgn_flip(tn[t][3].flip, i);
      gu[i][t] = 0.25 * P.inv_dx * (dip + djp);
    }
  }
  double div = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) div += gu[k][k];
  const double mub = 0.5 * (wget(P, Wc, P.wMu, ri) + wget(P, Wc, P.wMu, rj));
  const double lamb = 0.5 * (wget(P, Wc, P.wLam, ri) + wget(P, Wc, P.wLam, rj));
  const double Ti = wget(P, Wc, P.wT, ri), Tj = wget(P, Wc, P.wT, rj);
  double tau[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < D; ++i) tau[i] = mub * (gu[i][d] + gu[d][i] - (i == d ? (2.0 / 3.0) * div : 0.0));

  // reverse: F_{NS+i} -= tau_i; F_E -= sum ub_i tau_i + lamb (Tj - Ti) / dx
  const double lE = nu[NS + D];
  double lgu[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) lgu[i][j] = 0.0;
  double lmub = 0.0, lui[3] = {0.0, 0.0, 0.0}, luj[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const double ub = 0.5 * (ui[i] + uj[i]);
    const double ltau = -nu[NS + i] - lE * ub;
    const double lub = -lE * tau[i];
    lui[i] += 0.5 * lub;
    luj[i] += 0.5 * lub;
    lmub += ltau * (gu[i][d] + gu[d][i] - (i == d ? (2.0 / 3.0) * div : 0.0));
    lgu[i][d] += ltau * mub;
    lgu[d][i] += ltau * mub;
    if (i == d) {
#pragma unroll
      for (int k = 0; k < D; ++k) lgu[k][k] -= (2.0 / 3.0) * ltau * mub;
    }
  }
  const double llamb = -lE * (Tj - Ti) * P.inv_dx;
  const double lTj = -lE * lamb * P.inv_dx, lTi = lE * lamb * P.inv_dx;
  // normal derivatives
#pragma unroll
  for (int i = 0; i < D; ++i) {
    lui[i] -= lgu[i][d] * P.inv_dx;
    luj[i] += lgu[i][d] * P.inv_dx;
  }
  // line slots of the two face cells (j = 2: cell i, 3: cell i+1)
  add(L.line(2, 0), lTi);
  add(L.line(3, 0), lTj);
  {
    int tt = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const int q = t == d ? 2 : 3 + NS + tt;
      if (t != d) ++tt;
      add(L.line(2, q), lui[t]);
      add(L.line(3, q), luj[t]);
    }
  }
  // mu, lambda of the two cells
  put(L.nbq(0, L.qMu), 0.5 * lmub);
  put(L.nbq(1, L.qMu), 0.5 * lmub);
  put(L.nbq(0, L.qLam), 0.5 * llamb);
  put(L.nbq(1, L.qLam), 0.5 * llamb);
  // tangential derivatives: gu[i][t] = (u_{i+t} - u_{i-t} + u_{j+t} - u_{j-t}) / (4 dx)
  {
    int tt = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      if (t == d) continue;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const double g = 0.25 * P.inv_dx * lgu[i][t];
        put(L.vel(tt, 0, i), g);
        put(L.vel(tt, 1, i), -g);
        put(L.vel(tt, 2, i), g);
        put(L.vel(tt, 3, i), -g);
      }
      ++tt;
    }
  }
}

// Per cell: sums, in a fixed order, the contributions of the faces of
// direction d whose stencils reach the cell; first != 0 writes, otherwise
// adds.  gW: cache adjoint [nW][wstride]; gU: U adjoint [NV][ncell].
template <int NS, int D, int DIR>
__global__ void __launch_bounds__(CELL_THREADS)
    k_gather(const KParams P, const double* __restrict__ C, const int first, double* __restrict__ gW,
             double* __restrict__ gU) {
  constexpr int NV = NS + D + 1;
  constexpr int d = DIR;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.ncell) return;
  const Lay<NS, D> L(P.cdi, P.diffusion, P.viscous);
  int cc[3];
  unflatten(c, P.n[0], P.n[1], cc);
  const int f0 = P.n[0] + (d == 0), f1 = P.n[1] + (d == 1), f2 = P.n[2] + (d == 2);
  const long long nf = (long long)f0 * f1 * f2;
  auto face = [&](const int* fc) { return ((long long)fc[2] * f1 + fc[1]) * f0 + fc[0]; };
  auto get = [&](int q, long long f) { return C[(long long)q * nf + f]; };
  const int n = P.n[d];
  const Pre pd = preimages(cc[d], n, P.bc_lo[d], P.bc_hi[d]);

  double aT = 0.0, aP = 0.0, aUn = 0.0, aY[NS], aUt[3] = {0.0, 0.0, 0.0}, aRho = 0.0, aA = 0.0;
  double aYr[NS], aHr[2] = {0.0, 0.0}, aPhi = 0.0, aPsi = 0.0, aXr[NS], aB[NS], aU[NV];
  double aMu = 0.0, aLam = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) { aY[k] = 0.0; aYr[k] = 0.0; aXr[k] = 0.0; aB[k] = 0.0; }
#pragma unroll
  for (int v = 0; v < NV; ++v) aU[v] = 0.0;

  for (int e = 0; e < pd.n; ++e) {
    const int g = pd.g[e];
    const double sg = pd.s[e];
    // line slots: face with low cell ci = g - j + 2, index ci + 1
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int fi = g - j + 3;
      if (fi < 0 || fi > n) continue;
      int fc[3] = {cc[0], cc[1], cc[2]};
      fc[d] = fi;
      const long long f = face(fc);
      aT += get(L.line(j, 0), f);
      aP += get(L.line(j, 1), f);
      aUn += sg * get(L.line(j, 2), f);
#pragma unroll
      for (int k = 0; k < NS; ++k) aY[k] += get(L.line(j, 3 + k), f);
#pragma unroll
      for (int tt = 0; tt < D - 1; ++tt) aUt[tt] += get(L.line(j, 3 + NS + tt), f);
    }
    // neighbour slots: s = 0 when g is the low cell (face g + 1), s = 1
    // when it is the high cell (face g)
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const int fi = s2 == 0 ? g + 1 : g;
      if (fi < 0 || fi > n) continue;
      int fc[3] = {cc[0], cc[1], cc[2]};
      fc[d] = fi;
      const long long f = face(fc);
      aRho += get(L.nbq(s2, 0), f);
      aA += get(L.nbq(s2, 1), f);
      if (P.cdi) {
#pragma unroll
        for (int k = 0; k < NS; ++k) aYr[k] += get(L.nbq(s2, L.qYr + k), f);
        aHr[0] += get(L.nbq(s2, L.qHr), f);
        aHr[1] += get(L.nbq(s2, L.qHr + 1), f);
        aPhi += get(L.nbq(s2, L.qPhi), f);
        aPsi += get(L.nbq(s2, L.qPsi), f);
      }
      if (P.diffusion) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          aXr[k] += get(L.nbq(s2, L.qXr + k), f);
          aB[k] += get(L.nbq(s2, L.qB + k), f);
        }
      }
      if (P.viscous) {
        aMu += get(L.nbq(s2, L.qMu), f);
        aLam += get(L.nbq(s2, L.qLam), f);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) aU[v] += (v == NS + d ? sg : 1.0) * get(L.nbq(s2, L.qU + v), f);
    }
  }
  // psi of the tangential neighbours of a face (interface normal, CDI)
  if (P.cdi && D > 1) {
    int tt = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      if (t == d) continue;
      const Pre pt = preimages(cc[t], P.n[t], P.bc_lo[t], P.bc_hi[t]);
      for (int e = 0; e < pd.n; ++e) {
        const int gd = pd.g[e];
        for (int h = 0; h < pt.n; ++h) {
          const int gt = pt.g[h];
          // slot q: (low cell along d, tangential offset) = (gd, gt-1), (gd, gt+1),
          // (gd-1, gt-1), (gd-1, gt+1); the face sits at low cell + 1 along d
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int cid = q < 2 ? gd : gd - 1;
            const int cit = (q & 1) ? gt + 1 : gt - 1;
            const int fi = cid + 1;
            if (fi < 0 || fi > n || cit < 0 || cit >= P.n[t]) continue;
            int fc[3] = {cc[0], cc[1], cc[2]};
            fc[d] = fi;
            fc[t] = cit;
            aPsi += get(L.psi0 + 4 * tt + q, face(fc));
          }
        }
      }
      ++tt;
    }
  }

  // velocity components of the tangential neighbours of a face (viscous
  // stress), with the wall-mirror sign of the mapping that reached the cell
  if (P.viscous && D > 1) {
    int tt = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      if (t == d) continue;
      const Pre pt = preimages(cc[t], P.n[t], P.bc_lo[t], P.bc_hi[t]);
      for (int e = 0; e < pd.n; ++e) {
        const int gd = pd.g[e];
        for (int h = 0; h < pt.n; ++h) {
          const int gt = pt.g[h];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int cid = q < 2 ? gd : gd - 1;
            const int cit = (q & 1) ? gt + 1 : gt - 1;
            const int fi = cid + 1;
            if (fi < 0 || fi > n || cit < 0 || cit >= P.n[t]) continue;
            int fc[3] = {cc[0], cc[1], cc[2]};
            fc[d] = fi;
            fc[t] = cit;
            const long long f = face(fc);
#pragma unroll
            for (int i = 0; i < D; ++i) {
              const double sgn = i == d ? pd.s[e] : (i == t ? pt.s[h] : 1.0);
              const double v = sgn * get(L.vel(tt, q, i), f);
              if (i == d) aUn += v;
              else aUt[i < d ? i : i - 1] += v;
            }
          }
        }
      }
      ++tt;
    }
  }

  const long long ws = P.wstride;
  auto out = [&](int f, double v) {
    double* p = gW + (long long)f * ws + c;
    *p = first ? v : *p + v;
  };
  out(P.wT, aT);
  out(P.wP, aP);
  out(P.wRho, aRho);
  out(P.wA, aA);
#pragma unroll
  for (int k = 0; k < NS; ++k) out(P.wY + k, aY[k]);
  {
    int tt = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) out(P.wU + t, t == d ? aUn : aUt[tt++]);
  }
  if (P.cdi) {
#pragma unroll
    for (int k = 0; k < NS; ++k) out(P.wYrho + k, aYr[k]);
    out(P.wHrho, aHr[0]);
    out(P.wHrho + 1, aHr[1]);
    out(P.wPhi0, aPhi);
    out(P.wPsi, aPsi);
  }
  if (P.diffusion) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      out(P.wXr + k, aXr[k]);
      out(P.wB + k, aB[k]);
    }
  }
  if (P.viscous) {
    out(P.wMu, aMu);
    out(P.wLam, aLam);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double* p = gU + (long long)v * P.ncell + c;
    *p = first ? aU[v] : *p + aU[v];
  }
}

// per cell: out = a x + b y + cz z + gU + (dW/dU)^T gW  (y, z nullable;
// out may alias x, y or z)
template <int NS, int D>
__global__ void __launch_bounds__(CELL_THREADS)
    k_cell_adj(const KParams P, const double* __restrict__ U, const double* __restrict__ Wc,
               const double* __restrict__ gW, const double* __restrict__ gU, double* out, const double a,
               const double* x, const double b, const double* y, const double cz, const double* z) {
  constexpr int NV = NS + D + 1;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.ncell) return;
  const long long ws = P.wstride;
  {
    // a cell whose cache adjoint is zero needs no primitive-recovery reverse
    bool any = false;
    for (int f = 0; f < P.nW; ++f) any = any || nonzero(gW[(long long)f * ws + c]);
    if (!any) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const long long i = (long long)v * P.ncell + c;
        double r = a * x[i] + gU[i];
        if (y) r += b * y[i];
        if (z) r += cz * z[i];
        out[i] = r;
      }
      return;
    }
  }
  double Uc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Uc[v] = U[(long long)v * P.ncell + c];
  double rho, Y[NS], u[3], e, vol, p, T;
  decode<NS, D>(Uc, rho, Y, u, e, vol);
  if (Wc) {
    // the primitive pass of U solved the same equations from the same
    // decode: its T and P, read back
    T = Wc[P.wT * ws + c];
    p = Wc[P.wP * ws + c];
  } else {
    pt_equilibrium<NS>(P, Y, e, vol, p, T);
  }
  Thermo<NS> th;
#pragma unroll
  for (int k = 0; k < NS; ++k) th.Y[k] = Y[k];
  th.p = p;
  th.T = T;
  thermo_fwd<NS>(P, th);

  double lT = gW[P.wT * ws + c], lp = gW[P.wP * ws + c], lrho = gW[P.wRho * ws + c], la = gW[P.wA * ws + c];
  double lY[NS], lu[3] = {0.0, 0.0, 0.0}, lU[NV];
#pragma unroll
  for (int k = 0; k < NS; ++k) lY[k] = gW[(P.wY + k) * ws + c];
#pragma unroll
  for (int d = 0; d < D; ++d) lu[d] = gW[(P.wU + d) * ws + c];
#pragma unroll
  for (int v = 0; v < NV; ++v) lU[v] = 0.0;

  if (P.cdi || P.diffusion || P.viscous) {
    double phi[2] = {0.0, 0.0}, hr[2] = {0.0, 0.0}, Yp[2] = {0.0, 0.0};
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int ph = P.phase[k];
      Yp[ph] += Y[k];
      if (nonzero(Uc[k])) {
        phi[ph] += Uc[k] * (P.Rk[k] * T * th.r[k] + P.b[k]);
        hr[ph] += Uc[k] * h_k(P, k, p, T);
      }
    }
    double lphi[2] = {0.0, 0.0}, lhr[2] = {0.0, 0.0};
    if (P.cdi) {
      lphi[0] += gW[P.wPhi0 * ws + c];
      const double lpsi = gW[P.wPsi * ws + c];
      lphi[0] += lpsi * P.cdi_eps / (phi[0] + P.psi_delta);
      lphi[1] -= lpsi * P.cdi_eps / (phi[1] + P.psi_delta);
#pragma unroll
      for (int ph = 0; ph < 2; ++ph) {
        if (!(Yp[ph] >= ABSENT)) continue;
        const double iphi = 1.0 / phi[ph];
        const double lh = gW[(P.wHrho + ph) * ws + c];
        lhr[ph] += lh * iphi;
        double lq = lh * hr[ph];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          if (P.phase[k] != ph) continue;
          const double ly = gW[(P.wYrho + k) * ws + c];
          lU[k] += ly * iphi;
          lq += ly * Uc[k];
        }
        lphi[ph] -= lq * iphi * iphi;
      }
    }
    if (P.diffusion || P.viscous) {
      // gas viscosity (Wilke) and its dependence on the gas mass fractions
      double mup[2], den[NS], lmu[2] = {0.0, 0.0};
      mup[0] = P.mu_liquid;
      double num = 0.0;
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        den[i] = 0.0;
        if (P.phase[i] != 1) continue;
#pragma unroll
        for (int j = 0; j < NS; ++j)
          if (P.phase[j] == 1) den[i] += Y[j] * P.wilke[i][j];
        if (positive(den[i])) num += Y[i] * P.mu[i] / den[i];
      }
      mup[1] = Yp[1] >= ABSENT ? num : 0.0;
      if (P.viscous) {
        // mu = phi_0 mu_l + phi_1 mu_g; lambda = phi_0 lambda_l + phi_1 lambda_g,
        // lambda_g = (mu_g / Pr) cpY / Y_g, cpY = sum_{gas} Y_k cp_k
        const double lMu = gW[P.wMu * ws + c], lLam = gW[P.wLam * ws + c];
        double cpY = 0.0;
#pragma unroll
        for (int k = 0; k < NS; ++k)
          if (P.phase[k] == 1) cpY += Y[k] * P.cp[k];
        const double lam_g = Yp[1] >= ABSENT ? mup[1] / P.prandtl * (cpY / Yp[1]) : 0.0;
        lphi[0] += lMu * mup[0] + lLam * P.lambda_liquid;
        lphi[1] += lMu * mup[1] + lLam * lam_g;
        lmu[1] += lMu * phi[1];
        if (Yp[1] >= ABSENT) {
          const double llg = lLam * phi[1];
          lmu[1] += llg * cpY / (P.prandtl * Yp[1]);
          const double lcpY = llg * mup[1] / (P.prandtl * Yp[1]);
          const double lYg = -llg * mup[1] * cpY / (P.prandtl * Yp[1] * Yp[1]);
#pragma unroll
          for (int k = 0; k < NS; ++k)
            if (P.phase[k] == 1) lY[k] += lcpY * P.cp[k] + lYg;
        }
      }
#pragma unroll
      for (int ph = 0; ph < 2; ++ph) {
        if (!P.diffusion) break;
        double sY = 0.0;
#pragma unroll
        for (int j = 0; j < NS; ++j)
          if (P.phase[j] == ph) sY += Y[j] / P.W[j];
        if (!(Yp[ph] >= ABSENT && sY >= ABSENT)) continue;
        const double rho_p = rho * Yp[ph] / phi[ph];
        double lsY = 0.0, lYp = 0.0, lrho_p = 0.0;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          if (P.phase[k] != ph) continue;
          const double lxr = gW[(P.wXr + k) * ws + c];
          const double lB = gW[(P.wB + k) * ws + c];
          // xr = (Y_k / W_k) / sY
          lY[k] += lxr / (P.W[k] * sY);
          lsY -= lxr * (Y[k] / P.W[k]) / (sY * sY);
          // B = W_k sY / Yp * mu_p / (rho_p Sc_k)
          const double WcWp = P.W[k] * sY / Yp[ph];
          const double Dk = mup[ph] / (rho_p * P.Sc[k]);
          const double lW = lB * Dk, lD = lB * WcWp;
          lsY += lW * P.W[k] / Yp[ph];
          lYp -= lW * P.W[k] * sY / (Yp[ph] * Yp[ph]);
          lmu[ph] += lD / (rho_p * P.Sc[k]);
          lrho_p -= lD * Dk / rho_p;
        }
        // sY = sum_{j in p} Y_j / W_j
#pragma unroll
        for (int j = 0; j < NS; ++j)
          if (P.phase[j] == ph) lY[j] += lsY / P.W[j];
        // rho_p = rho Yp / phi
        lrho += lrho_p * Yp[ph] / phi[ph];
        lYp += lrho_p * rho / phi[ph];
        lphi[ph] -= lrho_p * rho_p / phi[ph];
#pragma unroll
        for (int j = 0; j < NS; ++j)
          if (P.phase[j] == ph) lY[j] += lYp;
      }
      // mu_g = sum_i Y_i mu_i / den_i, den_i = sum_j Y_j wilke_ij
      if (Yp[1] >= ABSENT && nonzero(lmu[1])) {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          if (P.phase[i] != 1 || !(positive(den[i]))) continue;
          lY[i] += lmu[1] * P.mu[i] / den[i];
          const double lden = -lmu[1] * Y[i] * P.mu[i] / (den[i] * den[i]);
#pragma unroll
          for (int j = 0; j < NS; ++j)
            if (P.phase[j] == 1) lY[j] += lden * P.wilke[i][j];
        }
      }
    }
    // phi_p = sum U_k v_k(P,T), hr_p = sum U_k h_k(P,T)
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (!nonzero(Uc[k])) continue;
      const int ph = P.phase[k];
      const double r = th.r[k];
      const double vk = P.Rk[k] * T * r + P.b[k];
      lU[k] += lphi[ph] * vk + lhr[ph] * h_k(P, k, p, T);
      lT += lphi[ph] * Uc[k] * P.Rk[k] * r + lhr[ph] * Uc[k] * P.cp[k];
      lp += -lphi[ph] * Uc[k] * P.Rk[k] * T * r * r + lhr[ph] * Uc[k] * P.b[k];
    }
  }
  // sound speed
  thermo_rev<NS>(P, th, 0.0, 0.0, la, 0.0, 0.0, lY, lp, lT);
  // p-T equilibrium
  double le = 0.0, lv = 0.0;
  pt_rev<NS>(P, Y, p, T, th.r, lp, lT, lY, le, lv);
  decode_rev<NS, D>(Uc, rho, Y, u, lrho, lY, lu, le, lv, lU);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const long long i = (long long)v * P.ncell + c;
    double r = a * x[i] + gU[i] + lU[v];
    if (y) r += b * y[i];
    if (z) r += cz * z[i];
    out[i] = r;
  }
}

// reverse of k_init: lam_prim = (dU/dprim)^T lam_U per cell; prim layout
// [alpha_0..alpha_{NS-1}, u_0..u_{D-1}, P, T]
template <int NS, int D>
__global__ void __launch_bounds__(CELL_THREADS)
    k_init_vjp(const KParams P, const double* __restrict__ prim, const double* __restrict__ lamU,
               double* __restrict__ lprim, long long n) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double p = prim[(long long)(NS + D) * n + c];
  const double T = prim[(long long)(NS + D + 1) * n + c];
  double al[NS], ry[NS], rho = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    al[k] = prim[(long long)k * n + c];
    ry[k] = nonzero(al[k]) ? al[k] / v_k(P, k, p, T) : 0.0;
    rho += ry[k];
  }
  double u[3] = {0.0, 0.0, 0.0}, u2 = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    u[d] = prim[(long long)(NS + d) * n + c];
    u2 += u[d] * u[d];
  }
  const double lE = lamU[(long long)(NS + D) * n + c];
  // E = sum ry_k e_k + rho |u|^2 / 2, m_d = rho u_d
  double lrho = 0.5 * u2 * lE;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double lm = lamU[(long long)(NS + d) * n + c];
    lrho += lm * u[d];
    lprim[(long long)(NS + d) * n + c] = lm * rho + lE * rho * u[d];
  }
  double lp = 0.0, lT = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    double la = 0.0;
    if (nonzero(al[k])) {
      const double r = 1.0 / (p + P.pinf[k]);
      const double vk = P.Rk[k] * T * r + P.b[k];
      const double ek = P.cv[k] * T * (p + P.gam[k] * P.pinf[k]) * r + P.q[k];
      // e_k terms of E at fixed ry_k
      lT += lE * ry[k] * P.cv[k] * (p + P.gam[k] * P.pinf[k]) * r;
      lp += lE * ry[k] * P.cv[k] * T * (P.pinf[k] - P.gam[k] * P.pinf[k]) * r * r;
      // ry_k = alpha_k / v_k
      const double lry = lamU[(long long)k * n + c] + lrho + lE * ek;
      la = lry / vk;
      const double lv = -lry * ry[k] / vk;
      lT += lv * P.Rk[k] * r;
      lp -= lv * P.Rk[k] * T * r * r;
    }
    lprim[(long long)k * n + c] = la;
  }
  lprim[(long long)(NS + D) * n + c] = lp;
  lprim[(long long)(NS + D + 1) * n + c] = lT;
}

// the adjoint face pass of one direction with interpolation RC
template <int NS, int D, int RC>
struct AdjFaceImpl {
  static void face(const KParams& P, cudaStream_t s, int d, const double* Wc, const double* Uk, const double* Uin,
                   const double* scal, const uint32_t* tape, const double* lamL, double coef, int mul_dt,
                   double* C) {
    long long nf = 1;
    for (int e = 0; e < 3; ++e) nf *= (long long)(P.n[e] + (e == d));
    const unsigned nb = nblocks(nf, VJP_THREADS);
    if (d == 0)
      k_face_adj<NS, D, 0, RC><<<nb, VJP_THREADS, 0, s>>>(P, Wc, Uk, Uin, scal, tape, lamL, coef, mul_dt, C);
    else if (d == 1)
      k_face_adj<NS, D, (D > 1 ? 1 : 0), RC><<<nb, VJP_THREADS, 0, s>>>(P, Wc, Uk, Uin, scal, tape, lamL, coef,
                                                                        mul_dt, C);
    else
      k_face_adj<NS, D, (D > 2 ? 2 : 0), RC><<<nb, VJP_THREADS, 0, s>>>(P, Wc, Uk, Uin, scal, tape, lamL, coef,
                                                                        mul_dt, C);
  }
};

// the adjoint face pass of interpolation RC for (dimension, species count)
template <int RC>
AdjFaceFn adj_face(int dim, int ns) {
  switch (dim * 8 + ns) {
    case 9: return &AdjFaceImpl<1, 1, RC>::face;
    case 10: return &AdjFaceImpl<2, 1, RC>::face;
    case 11: return &AdjFaceImpl<3, 1, RC>::face;
    case 12: return &AdjFaceImpl<4, 1, RC>::face;
    case 17: return &AdjFaceImpl<1, 2, RC>::face;
    case 18: return &AdjFaceImpl<2, 2, RC>::face;
    case 19: return &AdjFaceImpl<3, 2, RC>::face;
    case 20: return &AdjFaceImpl<4, 2, RC>::face;
    case 25: return &AdjFaceImpl<1, 3, RC>::face;
    case 26: return &AdjFaceImpl<2, 3, RC>::face;
    case 27: return &AdjFaceImpl<3, 3, RC>::face;
    case 28: return &AdjFaceImpl<4, 3, RC>::face;
    default: return nullptr;
  }
}

template <int NS, int D>
struct AdjImpl {
  static int slots(const KParams& P) { return Lay<NS, D>(P.cdi, P.diffusion, P.viscous).total; }
  static void face(const KParams& P, cudaStream_t s, int d, const double* Wc, const double* Uk, const double* Uin,
                   const double* scal, const uint32_t* tape, const double* lamL, double coef, int mul_dt,
                   double* C) {
    AdjFaceImpl<NS, D, RC_WENO5Z>::face(P, s, d, Wc, Uk, Uin, scal, tape, lamL, coef, mul_dt, C);
  }
  static void face_visc(const KParams& P, cudaStream_t s, int d, const double* Wc, const double* scal,
                        const uint32_t* tape, const double* lamL, double coef, int mul_dt, double* C) {
    long long nf = 1;
    for (int e = 0; e < 3; ++e) nf *= (long long)(P.n[e] + (e == d));
    const unsigned nb = nblocks(nf, VJP_THREADS);
    if (d == 0)
      k_face_visc_adj<NS, D, 0><<<nb, VJP_THREADS, 0, s>>>(P, Wc, scal, tape, lamL, coef, mul_dt, C);
    else if (d == 1)
      k_face_visc_adj<NS, D, (D > 1 ? 1 : 0)><<<nb, VJP_THREADS, 0, s>>>(P, Wc, scal, tape, lamL, coef, mul_dt, C);
    else
      k_face_visc_adj<NS, D, (D > 2 ? 2 : 0)><<<nb, VJP_THREADS, 0, s>>>(P, Wc, scal, tape, lamL, coef, mul_dt, C);
  }
  static void gather(const KParams& P, cudaStream_t s, int d, const double* C, int first, double* gW, double* gU) {
    const unsigned nb = nblocks(P.ncell, CELL_THREADS);
    if (d == 0)
      k_gather<NS, D, 0><<<nb, CELL_THREADS, 0, s>>>(P, C, first, gW, gU);
    else if (d == 1)
      k_gather<NS, D, (D > 1 ? 1 : 0)><<<nb, CELL_THREADS, 0, s>>>(P, C, first, gW, gU);
    else
      k_gather<NS, D, (D > 2 ? 2 : 0)><<<nb, CELL_THREADS, 0, s>>>(P, C, first, gW, gU);
  }
  static void cell(const KParams& P, cudaStream_t s, const double* U, const double* Wc, const double* gW,
                   const double* gU, double* out, double a, const double* x, double b, const double* y, double cz,
                   const double* z) {
    k_cell_adj<NS, D><<<nblocks(P.ncell, CELL_THREADS), CELL_THREADS, 0, s>>>(P, U, Wc, gW, gU, out, a, x, b, y,
                                                                               cz, z);
  }
  static void init(const KParams& P, cudaStream_t s, const double* prim, const double* lamU, double* lprim,
                   long long n) {
    if (n > 0) k_init_vjp<NS, D><<<nblocks(n, CELL_THREADS), CELL_THREADS, 0, s>>>(P, prim, lamU, lprim, n);
  }
  static AdjOps ops() {
    AdjOps o;
    o.slots = &slots;
    o.face = &face;
    o.face_visc = &face_visc;
    o.gather = &gather;
    o.cell = &cell;
    o.init = &init;
    return o;
  }
};

}  // namespace adj
}  // namespace mpmc
