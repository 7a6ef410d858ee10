// Mixed-precision kernels of the MPMC stage: reconstruction, face EOS,
// HLLC, regularization and diffusion fluxes in FP32 with FP32 accumulation;
// the cell p-T equilibrium inversion, the positivity-limiter pseudo-updates
// and the conservative RK accumulation in FP64.
//
// Uniform fields stay exactly uniform: every stencil value is reconstructed
// as its deviation from the face's left cell (W_j - W_i, zero where P, T, u
// are uniform), and the HLLC contact speed is written as u_L plus a term
// that vanishes when P and u are continuous.
#pragma once
#include "mpmc_device.cuh"
#include "mpmc_ops.h"
#include "mpmc_narrow.h"
#include "mpmc_update.cuh"

namespace mpmc {
namespace mx {

constexpr int FACE_THREADS = 128;
constexpr int CELL_THREADS = 256;
constexpr float WENO_EPS32 = 1e-30f;   // reading: FP32 epsilon kept normal
constexpr float DELTA32 = 1e-30f;      // psi transform delta in FP32 (1e-100 underflows)
constexpr float GTOL32 = 1e-6f;        // |grad psi| threshold at FP32 round-off

// ---------------------------------------------------------------------------
// FP32 species EOS (Eq. NASG_EOS) with constants cast once
struct SpeciesF {
  float cv, gam, q, b, pinf, Rk, cp;
};

template <int NS>
__device__ __forceinline__ void load_species(const KParams& P, SpeciesF* s) {
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    s[k].cv = P.f32.cv[k];
    s[k].gam = P.f32.gam[k];
    s[k].q = P.f32.q[k];
    s[k].b = P.f32.b[k];
    s[k].pinf = P.f32.pinf[k];
    s[k].Rk = P.f32.Rk[k];
    s[k].cp = P.f32.cp[k];
  }
}

// forward EOS at (p, T, Y) in FP32: density, internal energy, sound speed
template <int NS>
__device__ __forceinline__ void eos_forward_f(const SpeciesF* s, const float* Y, float p, float T, float& rho,
                                              float& e, float& a) {
  float v = 0.f, cp = 0.f, sa = 0.f, sb = 0.f;
  e = 0.f;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (Y[k] != 0.f) {
      const float r = __frcp_rn(p + s[k].pinf);
      const float RT = s[k].Rk * T;
      v += Y[k] * (RT * r + s[k].b);
      e += Y[k] * (s[k].cv * T * (p + s[k].gam * s[k].pinf) * r + s[k].q);
      cp += Y[k] * s[k].cp;
      sa += Y[k] * s[k].Rk * r;
      sb += Y[k] * RT * r * r;
    }
  }
  rho = __frcp_rn(v);
  const float al = rho * sa, be = rho * sb;
  a = sqrtf(cp / (rho * be * cp - al * al * T));
}

// p-T equilibrium in FP32 (face average only: feeds the characteristic
// matrices, whose scalars depend on P through P + Pinf)
template <int NS>
__device__ __forceinline__ void pt_equilibrium_f(const SpeciesF* s, const float* Y, float e, float v, float& p,
                                                 float& T) {
  float Cv = 0.f, q = 0.f, b = 0.f, Rg = 0.f, Rl = 0.f, wpl = 0.f;
  float pl = -1.f;
  bool gas = false;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    Cv += Y[k] * s[k].cv;
    q += Y[k] * s[k].q;
    b += Y[k] * s[k].b;
    if (Y[k] > 0.f) {
      if (s[k].pinf > 0.f) {
        Rl += Y[k] * s[k].Rk;
        wpl += Y[k] * s[k].Rk * s[k].pinf;
        pl = 1.f;
      } else {
        gas = true;
        Rg += Y[k] * s[k].Rk;
      }
    }
  }
  const float em = e - q, Ep = em / (v - b);
  if (pl < 0.f) {
    p = Ep * Rg / Cv;
  } else {
    // several liquids merged into one with a Y-weighted Pinf (only the
    // characteristic scalars use this pressure)
    const float pe = wpl / Rl;
    const float a2 = Ep * (Rg + Rl) - pe * Cv - pe * Rl;
    if (!gas) {
      p = a2 / Cv;
    } else {
      const float a3 = Ep * pe * Rg;
      const float sq = sqrtf(a2 * a2 + 4.f * Cv * a3);
      p = a2 >= 0.f ? (a2 + sq) / (2.f * Cv) : 2.f * a3 / (sq - a2);
    }
  }
  float den = 0.f;
#pragma unroll
  for (int k = 0; k < NS; ++k)
    if (Y[k] != 0.f) den += Y[k] * s[k].cv * (p + s[k].gam * s[k].pinf) / (p + s[k].pinf);
  T = em / den;
}

// WENO5-Z in FP32 on deviations (exponent 1)
__device__ __forceinline__ float weno5z_f(float v0, float v1, float v2, float v3, float v4) {
  const float q0 = (2.f * v0 - 7.f * v1 + 11.f * v2) * (1.f / 6.f);
  const float q1 = (-v1 + 5.f * v2 + 2.f * v3) * (1.f / 6.f);
  const float q2 = (2.f * v2 + 5.f * v3 - v4) * (1.f / 6.f);
  float t = v0 - 2.f * v1 + v2, s = v0 - 4.f * v1 + 3.f * v2;
  const float b0 = (13.f / 12.f) * t * t + 0.25f * s * s;
  t = v1 - 2.f * v2 + v3;
  s = v1 - v3;
  const float b1 = (13.f / 12.f) * t * t + 0.25f * s * s;
  t = v2 - 2.f * v3 + v4;
  s = 3.f * v2 - 4.f * v3 + v4;
  const float b2 = (13.f / 12.f) * t * t + 0.25f * s * s;
  const float tau = fabsf(b0 - b2);
  // tau / (beta + eps) clamped at 1e30: with eps = 1e-30 the ratio of a
  // stencil that is flat next to a jump would overflow FP32 (in FP64 it
  // reaches 1e50 harmlessly); at 1e30 that stencil already carries all the
  // weight, so the clamp changes the weights by 1 part in 1e30.
  // The divisions are the fast reciprocal-multiply form: every denominator
  // stays far below 2^126 (smoothness indicators of these variables are
  // < 1e20, the weights' sum < 1e31), an overflowing ratio is clamped, and
  // a 2-ulp weight error moves only the deviation from the left cell, which
  // is zero where the field is uniform.
  const float a0 = 0.1f * (1.f + fminf(__fdividef(tau, b0 + WENO_EPS32), 1e30f));
  const float a1 = 0.6f * (1.f + fminf(__fdividef(tau, b1 + WENO_EPS32), 1e30f));
  const float a2 = 0.3f * (1.f + fminf(__fdividef(tau, b2 + WENO_EPS32), 1e30f));
  return __fdividef(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
}

// weno5z_f of both sides of a face, of y[0..4] and of y[5..1]: the two
// sides share two candidates (q_1 of one is q_2 of the other) and two
// second differences with their (13/12) t^2 terms
__device__ __forceinline__ float weno5z_side_f(float b0, float b1, float b2, float q0, float q1, float q2) {
  const float tau = fabsf(b0 - b2);
  const float a0 = 0.1f * (1.f + fminf(__fdividef(tau, b0 + WENO_EPS32), 1e30f));
  const float a1 = 0.6f * (1.f + fminf(__fdividef(tau, b1 + WENO_EPS32), 1e30f));
  const float a2 = 0.3f * (1.f + fminf(__fdividef(tau, b2 + WENO_EPS32), 1e30f));
  return __fdividef(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
}

__device__ __forceinline__ void weno5z_lr_f(const float* y, float& L, float& R) {
  const float t123 = y[1] - 2.f * y[2] + y[3], t234 = y[2] - 2.f * y[3] + y[4];
  const float e123 = (13.f / 12.f) * t123 * t123, e234 = (13.f / 12.f) * t234 * t234;
  const float qa = (-y[1] + 5.f * y[2] + 2.f * y[3]) * (1.f / 6.f);
  const float qb = (2.f * y[2] + 5.f * y[3] - y[4]) * (1.f / 6.f);
  {
    const float t = y[0] - 2.f * y[1] + y[2], s = y[0] - 4.f * y[1] + 3.f * y[2];
    const float s1 = y[1] - y[3], s2 = 3.f * y[2] - 4.f * y[3] + y[4];
    const float q0 = (2.f * y[0] - 7.f * y[1] + 11.f * y[2]) * (1.f / 6.f);
    L = weno5z_side_f((13.f / 12.f) * t * t + 0.25f * s * s, e123 + 0.25f * s1 * s1, e234 + 0.25f * s2 * s2, q0,
                      qa, qb);
  }
  {
    const float t = y[5] - 2.f * y[4] + y[3], s = y[5] - 4.f * y[4] + 3.f * y[3];
    const float s1 = y[4] - y[2], s2 = 3.f * y[3] - 4.f * y[2] + y[1];
    const float q0 = (2.f * y[5] - 7.f * y[4] + 11.f * y[3]) * (1.f / 6.f);
    R = weno5z_side_f((13.f / 12.f) * t * t + 0.25f * s * s, e234 + 0.25f * s1 * s1, e123 + 0.25f * s2 * s2, q0,
                      qb, qa);
  }
}

// Sec. 4.1's other ENO-type interpolations in FP32 (as the FP64 ones in
// mpmc_device.cuh; the mixed face kernel feeds them deviations from the left
// cell).  Ratios tau / (beta + eps) are clamped at 1e30 as in weno5z_f.
struct Eno3f {
  float ql, qc, qr, bl, bc, br;
};

__device__ __forceinline__ Eno3f eno3_f(float v0, float v1, float v2, float v3, float v4) {
  Eno3f e;
  e.ql = (2.f * v0 - 7.f * v1 + 11.f * v2) * (1.f / 6.f);
  e.qc = (-v1 + 5.f * v2 + 2.f * v3) * (1.f / 6.f);
  e.qr = (2.f * v2 + 5.f * v3 - v4) * (1.f / 6.f);
  float t = v0 - 2.f * v1 + v2, s = v0 - 4.f * v1 + 3.f * v2;
  e.bl = (13.f / 12.f) * t * t + 0.25f * s * s;
  t = v1 - 2.f * v2 + v3;
  s = v1 - v3;
  e.bc = (13.f / 12.f) * t * t + 0.25f * s * s;
  t = v2 - 2.f * v3 + v4;
  s = 3.f * v2 - 4.f * v3 + v4;
  e.br = (13.f / 12.f) * t * t + 0.25f * s * s;
  return e;
}

// WENO5-JS: alpha_k = d_k / (eps + beta_k)^2, eps = 1e-6
__device__ __forceinline__ float weno5js_f(float v0, float v1, float v2, float v3, float v4) {
  const Eno3f e = eno3_f(v0, v1, v2, v3, v4);
  // 1/(eps + beta)^2 stays a normal FP32 number for indicators below 1e18
  const float il = __frcp_rn(1e-6f + e.bl), ic = __frcp_rn(1e-6f + e.bc), ir = __frcp_rn(1e-6f + e.br);
  const float al = 0.1f * il * il, ac = 0.6f * ic * ic, ar = 0.3f * ir * ir;
  return (al * e.ql + ac * e.qc + ar * e.qr) / (al + ac + ar);
}

template <int K>
__device__ __forceinline__ float teno_select_f(const float* q, const float* b, const float* dk, float tau, float CT) {
  float r[K], rmax = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    r[k] = 1.f + fminf(__fdividef(tau, b[k] + WENO_EPS32), 1e30f);
    rmax = fmaxf(rmax, r[k]);
  }
  const float irm = __frcp_rn(rmax);
  float g[K], gs = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float x = r[k] * irm, x2 = x * x;
    g[k] = x2 * x2 * x2;
    gs += g[k];
  }
  float num = 0.f, den = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (!(g[k] < CT * gs)) {
      num += dk[k] * q[k];
      den += dk[k];
    }
  return num / den;
}

__device__ __forceinline__ float teno5_f(float v0, float v1, float v2, float v3, float v4) {
  const Eno3f e = eno3_f(v0, v1, v2, v3, v4);
  const float q[3] = {e.qc, e.ql, e.qr}, b[3] = {e.bc, e.bl, e.br}, dk[3] = {0.6f, 0.1f, 0.3f};
  return teno_select_f<3>(q, b, dk, fabsf(e.bl - e.br), 1e-5f);
}

__device__ __forceinline__ float teno6_f(float v0, float v1, float v2, float v3, float v4, float v5) {
  const Eno3f e = eno3_f(v0, v1, v2, v3, v4);
  const float q4 = (3.f * v2 + 13.f * v3 - 5.f * v4 + v5) * (1.f / 12.f);
  const float e0 = v0 - v2, e1 = v1 - v2, e3 = v3 - v2, e4 = v4 - v2, e5 = v5 - v2;
  const float s = 18.f * e3 - 9.f * e4 + 2.f * e5, t = -5.f * e3 + 4.f * e4 - e5, u = 3.f * e3 - 3.f * e4 + e5;
  const float b4 = (1.f / 36.f) * s * s + (13.f / 12.f) * t * t + (781.f / 720.f) * u * u;
  const float c1 = 3.f * e0 - 30.f * e1 + 60.f * e3 - 15.f * e4 + 2.f * e5;
  const float c2 = -11.f * e0 + 174.f * e1 + 174.f * e3 - 11.f * e4;
  const float c3 = -16315.f * e0 - 16831.f * e1 - 230474.f * e3 + 115237.f * e4 - 16487.f * e5;
  const float c4 = e0 - 4.f * e1 - 4.f * e3 + e4;
  const float c5 = -e0 + 5.f * e1 + 10.f * e3 - 5.f * e4 + e5;
  const float b6 = (1.f / 3600.f) * c1 * c1 + (1.f / 15600.f) * c2 * c2 + (1.f / 3967729920.f) * c3 * c3 +
                   (1421461.f / 1310400.f) * c4 * c4 + (21520059541.f / 19838649600.f) * c5 * c5;
  const float q[4] = {e.qc, e.ql, e.qr, q4}, b[4] = {e.bc, e.bl, e.br, b4}, dk[4] = {0.45f, 0.05f, 0.3f, 0.2f};
  return teno_select_f<4>(q, b, dk, fabsf(b6 - (e.bl + e.br + 4.f * e.bc) * (1.f / 6.f)), 1e-7f);
}

template <int RC>
__device__ __forceinline__ float recon_f(float v0, float v1, float v2, float v3, float v4, float v5) {
  if constexpr (RC == RC_WENO5JS) return weno5js_f(v0, v1, v2, v3, v4);
  else if constexpr (RC == RC_TENO5) return teno5_f(v0, v1, v2, v3, v4);
  else if constexpr (RC == RC_TENO6) return teno6_f(v0, v1, v2, v3, v4, v5);
  else return weno5z_f(v0, v1, v2, v3, v4);
}

// both sides of a face from the six cells y[0..5] (left: y[0..5]; right:
// y[5..0]); WENO5-Z shares the sides' common terms (weno5z_lr_f)
template <int RC>
__device__ __forceinline__ void recon_lr_f(const float* y, float& L, float& R) {
  if constexpr (RC == RC_WENO5Z) {
    weno5z_lr_f(y, L, R);
  } else {
    L = recon_f<RC>(y[0], y[1], y[2], y[3], y[4], y[5]);
    R = recon_f<RC>(y[5], y[4], y[3], y[2], y[1], y[0]);
  }
}

template <int NS>
struct StateF {
  float rho, rhoY[NS], u[3], m[3], p, E, a;
};

// HLLC (Appendix B) in FP32; the contact speed in the form
// s* = u_L + (P_R - P_L - rho_R d_R (u_R - u_L)) / (rho_L d_L - rho_R d_R),
// algebraically the printed one, exactly u where P and u are continuous
// F(S) + s (U*_S - U_S) on the side S of the contact the face lies on
template <int NS, int D>
__device__ __forceinline__ void hllc_side_f(int d, const StateF<NS>& S, float s, float sS, float dS, float ss,
                                            float* F) {
  const float f = dS / (sS - ss);
#pragma unroll
  for (int k = 0; k < NS; ++k) F[k] = S.rhoY[k] * S.u[d] + s * (f * S.rhoY[k] - S.rhoY[k]);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const float Fs = S.rho * S.u[d] * S.u[j] + (j == d ? S.p : 0.f);
    const float Us = f * S.rho * (j == d ? ss : S.u[j]);
    F[NS + j] = Fs + s * (Us - S.m[j]);
  }
  const float Fs = S.u[d] * (S.E + S.p);
  const float Us = f * (S.E + (ss - S.u[d]) * (S.rho * ss + S.p / dS));
  F[NS + D] = Fs + s * (Us - S.E);
}

template <int NS, int D>
__device__ __forceinline__ void hllc_f(int d, const StateF<NS>& L, const StateF<NS>& R, float* F) {
  const float ub = 0.5f * (L.u[d] + R.u[d]), ab = 0.5f * (L.a + R.a);
  const float sL = fminf(ub - ab, L.u[d] - L.a);
  const float sR = fmaxf(ub + ab, R.u[d] + R.a);
  const float sm = fminf(0.f, sL), sp = fmaxf(0.f, sR);
  const float dL = sL - L.u[d], dR = sR - R.u[d];
  const float ss = L.u[d] + (R.p - L.p - R.rho * dR * (R.u[d] - L.u[d])) / (L.rho * dL - R.rho * dR);
  // only the side of the contact the face lies on; sign(0) = 0 averages both
  if (ss > 0.f) {
    hllc_side_f<NS, D>(d, L, sm, sL, dL, ss, F);
  } else if (ss < 0.f) {
    hllc_side_f<NS, D>(d, R, sp, sR, dR, ss, F);
  } else {
    constexpr int NV = NS + D + 1;
    float FL[NV], FR[NV];
    hllc_side_f<NS, D>(d, L, sm, sL, dL, ss, FL);
    hllc_side_f<NS, D>(d, R, sp, sR, dR, ss, FR);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = 0.5f * FL[v] + 0.5f * FR[v];
  }
}

template <int NS>
__device__ __forceinline__ void state_from_primitive_f(const SpeciesF* s, const float* Y, const float* u, float p,
                                                       float T, StateF<NS>& st) {
  float e;
  eos_forward_f<NS>(s, Y, p, T, st.rho, e, st.a);
  float ke = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    st.u[d] = u[d];
    st.m[d] = st.rho * u[d];
    ke += u[d] * u[d];
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) st.rhoY[k] = st.rho * Y[k];
  st.p = p;
  st.E = st.rho * (e + 0.5f * ke);
}

template <int NS>
__device__ __forceinline__ bool y_limiter_f(float* Y, const float* Yc) {
  bool active = false;
#pragma unroll
  for (int k = 0; k < NS; ++k)
    if (Y[k] < 0.f) {
      Y[k] = 0.f;
      active = true;
    }
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < NS; ++k) sum += Y[k];
  // a sum within FP32 rounding of one needs no correction (correcting it
  // would move trace species by ~1e-7 absolute)
  if (fabsf(sum - 1.f) > (float)NS * 1.2e-7f) {
    const bool over = sum > 1.f;
    float dd[NS], Sig = 0.f;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      dd[k] = (over ? fminf(Y[k], Yc[k]) : fmaxf(Y[k], Yc[k])) - Y[k];
      Sig += dd[k];
    }
    if (Sig != 0.f) {
      const float f = (1.f - sum) / Sig;
#pragma unroll
      for (int k = 0; k < NS; ++k) Y[k] += f * dd[k];
      active = true;
    }
  }
  return active;
}

__device__ __forceinline__ float wgetf(const KParams& P, const float* __restrict__ Wc, int f, CRef r) {
  return Wc[(long long)f * P.wstride + r.idx];
}
__device__ __forceinline__ float sgnf(unsigned flip, int d) { return (flip >> d) & 1u ? -1.f : 1.f; }

// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ void block_max2f(float a, float b, unsigned long long* red) {
  __shared__ float sa[32], sb[32];
  a = warp_maxf(a);
  b = warp_maxf(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sa[wid] = a;
    sb[wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    a = lane < nw ? sa[lane] : 0.f;
    b = lane < nw ? sb[lane] : 0.f;
    a = warp_maxf(a);
    b = warp_maxf(b);
    if (lane == 0) {
      atomicMax(red + 0, (unsigned long long)__double_as_longlong((double)a));
      atomicMax(red + 1, (unsigned long long)__double_as_longlong((double)b));
    }
  }
}

// per cell: FP64 inversion, FP32 cache
template <int NS, int D>
__global__ void __launch_bounds__(CELL_THREADS)
    k_prim(const KParams P, const double* __restrict__ U, const double* __restrict__ Uin, float* __restrict__ Wc,
           unsigned long long* __restrict__ red, int* __restrict__ status) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float smax = 0.f, gmax = 0.f;
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
    double rho, Y[NS], u[3], e, vol;
    decode<NS, D, false>(Uc, rho, Y, u, e, vol);
    int st = positive(rho) ? ST_OK : ST_INADMISSIBLE;
#pragma unroll
    for (int k = 0; k < NS; ++k)
      if (Uc[k] < -YTOL * rho) st = ST_INADMISSIBLE;
    double pd, Td;
    const int st2 = pt_equilibrium<NS, false, true>(P, Y, e, vol, pd, Td, rho);
    if (st == ST_OK) st = st2;
    SpeciesF sp[NS];
    load_species<NS>(P, sp);
    float Yf[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) Yf[k] = narrow(Y[k]);
    const float p = narrow(pd), T = narrow(Td);
    float r2, e2, a;
    eos_forward_f<NS>(sp, Yf, p, T, r2, e2, a);
    Wc[P.wT * ws + c] = T;
    Wc[P.wP * ws + c] = p;
    Wc[P.wRho * ws + c] = narrow(rho);
    Wc[P.wA * ws + c] = a;
#pragma unroll
    for (int k = 0; k < NS; ++k) Wc[(P.wY + k) * ws + c] = Yf[k];
#pragma unroll
    for (int d = 0; d < D; ++d) Wc[(P.wU + d) * ws + c] = narrow(u[d]);
    // FP32 copies of U for the limiter's first (FP32) admissibility test;
    // the pass that computes dt and Gamma (red != null) runs on U^n
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float uf = narrow(Uc[v]);
      Wc[(P.nW + v) * ws + c] = uf;
      if (red) P.unf[v * ws + c] = uf;
    }
    float mu = 0.f, lam = 0.f;
    const float rhof = narrow(rho);
    if (P.cdi || P.diffusion || P.viscous) {
      float phi[2], Yp[2];
#pragma unroll
      for (int ph = 0; ph < 2; ++ph) {
        float f = 0.f, hr = 0.f, yp = 0.f;
#pragma unroll
        for (int k = 0; k < NS; ++k)
          if (P.phase[k] == ph) {
            yp += Yf[k];
            const float ry = narrow(Uc[k]);
            if (ry != 0.f) {
              f += ry * (sp[k].Rk * T / (p + sp[k].pinf) + sp[k].b);
              hr += ry * (sp[k].cp * T + sp[k].b * p + sp[k].q);
            }
          }
        phi[ph] = f;
        Yp[ph] = yp;
        if (P.cdi) {
          // a phase whose FP32 volume fraction underflows counts as absent
          const bool present = f > 0.f;
          Wc[(P.wHrho + ph) * ws + c] = present ? hr / f : 0.f;
#pragma unroll
          for (int k = 0; k < NS; ++k)
            if (P.phase[k] == ph) Wc[(P.wYrho + k) * ws + c] = present ? (float)Uc[k] / f : 0.f;
        }
      }
      if (P.cdi) {
        Wc[P.wPhi0 * ws + c] = phi[0];
        Wc[P.wPsi * ws + c] = P.f32.cdi_eps * __logf((phi[0] + DELTA32) / (phi[1] + DELTA32));
      }
      float mup[2] = {P.f32.mu_liquid, 0.f};
      if (P.diffusion || P.viscous) {
        float num = 0.f;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          if (P.phase[i] != 1) continue;
          float den = 0.f;
#pragma unroll
          for (int j = 0; j < NS; ++j)
            if (P.phase[j] == 1) den += Yf[j] * P.f32.wilke[i][j];
          if (den > 0.f) num += Yf[i] * P.f32.mu[i] / den;
        }
        mup[1] = Yp[1] > 0.f ? num : 0.f;
        mu = phi[0] * mup[0] + phi[1] * mup[1];
      }
      if (P.viscous) {
        float cpY = 0.f;
#pragma unroll
        for (int k = 0; k < NS; ++k)
          if (P.phase[k] == 1) cpY += Yf[k] * sp[k].cp;
        const float lam_g = Yp[1] > 0.f ? mup[1] / P.f32.prandtl * (cpY / Yp[1]) : 0.f;
        lam = phi[0] * P.f32.lambda_liquid + phi[1] * lam_g;
        Wc[P.wMu * ws + c] = mu;
        Wc[P.wLam * ws + c] = lam;
      }
      if (P.diffusion) {
#pragma unroll
        for (int ph = 0; ph < 2; ++ph) {
          float sY = 0.f;
#pragma unroll
          for (int j = 0; j < NS; ++j)
            if (P.phase[j] == ph) sY += Yf[j] / P.f32.W[j];
          const bool present = Yp[ph] > 0.f && sY > 0.f && phi[ph] > 0.f;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            if (P.phase[k] != ph) continue;
            float xr = 0.f, B = 0.f;
            if (present) {
              xr = (Yf[k] / P.f32.W[k]) / sY;
              const float WcWp = P.f32.W[k] * sY / Yp[ph];
              const float rho_p = rhof * Yp[ph] / phi[ph];
              B = WcWp * (mup[ph] / (rho_p * P.f32.Sc[k]));
            }
            Wc[(P.wXr + k) * ws + c] = xr;
            Wc[(P.wB + k) * ws + c] = B;
          }
        }
      }
    }
    if (st != ST_OK) atomicMax(status, st);
    if (c < P.ncell) {
      const float idx = P.f32.inv_dx;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float ud = fabsf(narrow(u[d]));
        smax = fmaxf(smax, (ud + a) * idx);
        gmax = fmaxf(gmax, ud);
      }
      if (P.diffusion || P.viscous) smax = fmaxf(smax, 4.f * mu / rhof * (idx * idx));
      if (P.viscous) {
        float cv = 0.f;
#pragma unroll
        for (int k = 0; k < NS; ++k) cv += Yf[k] * sp[k].cv;
        smax = fmaxf(smax, 4.f * lam / (rhof * cv) * (idx * idx));
      }
    }
  }
  if (red) block_max2f(smax, gmax, red);
}

// Admissibility (Eqs. PositivityReqs1/2, as in admissible()) of the
// pseudo-update T = rk0 Un + rk1 Uk + s lam F from FP32 copies.  Each test is
// decided only when its value clears RMARGIN times the magnitudes of its
// terms, far above FP32 rounding (~13 ulp of those magnitudes), so a
// decision equals the exact one: returns 1 (admissible), 0 (not), -1 (too
// close to call: the caller decides in FP64).
constexpr float RMARGIN = 1e-4f;

template <int NS, int D>
__device__ __forceinline__ int admissible_f(const KParams& P, const float* Unf, const float* Ukf, const float* F,
                                            float rk0, float rk1, float slam) {
  constexpr int NV = NS + D + 1;
  float T[NV], M[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float a = rk0 * Unf[v], b = rk1 * Ukf[v], f = slam * F[v];
    T[v] = a + b + f;
    M[v] = fabsf(a) + fabsf(b) + fabsf(f);
  }
  bool undecided = false;
  auto test = [&](float val, float mag) {
    if (val > RMARGIN * mag) return true;
    if (!(val < -RMARGIN * mag)) undecided = true;
    return false;
  };
  float rho = 0.f, Mrho = 0.f, sb = 0.f, Msb = 0.f, sq = 0.f, Msq = 0.f;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    rho += T[k];
    Mrho += M[k];
    const float b = P.f32.b[k], q = P.f32.q[k];
    sb += T[k] * b;
    Msb += M[k] * fabsf(b);
    sq += T[k] * q;
    Msq += M[k] * fabsf(q);
  }
  bool ok = test(rho, Mrho);
  ok = test(1.f - sb, 1.f + Msb) && ok;
  const float ytol = (float)YTOL;
#pragma unroll
  for (int k = 0; k < NS; ++k) ok = test(T[k] + ytol * rho, M[k] + ytol * Mrho) && ok;
  float mm = 0.f, Mmm = 0.f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    mm += T[NS + d] * T[NS + d];
    Mmm += M[NS + d] * M[NS + d];
  }
  ok = test(rho * T[NS + D] - 0.5f * mm - rho * sq, Mrho * M[NS + D] + 0.5f * Mmm + Mrho * Msq) && ok;
  if (ok) return 1;
  // a test decided "no" makes the state inadmissible whatever the others say
  return undecided ? -1 : 0;
}

// The FP64 test of one cell's pseudo-update T = rk0 U^n + rk1 U^(k) + s F
// (Eqs. PositivityReqs1/2, the FP64 path's admissible()), for a flux the
// FP32 test could not decide.  Streams over the components, reloading each
// from memory when it is needed again, so that only the running sums are
// held: the FP64 states of both cells kept in registers at every limiter
// test made the face kernel spill in the common path.
template <int NS, int D>
__device__ __forceinline__ bool admissible_stream(const KParams& P, const double* __restrict__ Un,
                                                  const double* __restrict__ Uk, const double* __restrict__ Uin,
                                                  const CRef r, const float* Ft, const double rk0, const double rk1,
                                                  const double s) {
  const bool ghost = r.idx >= P.ncell;
  const long long col = r.idx - P.ncell;
  // (a wall's mirror image negates the cell's momentum component d, as
  // load_U does, before the flux term is added)
  auto T = [&](int v) {
    double un = ghost ? P.gn[(long long)v * P.gstride + col] : Un[(long long)v * P.ncell + r.idx];
    double uk = ghost ? Uin[(long long)v * P.gstride + col] : Uk[(long long)v * P.ncell + r.idx];
    if (v >= NS && v < NS + D) {
      un *= sgn_flip(r.flip, v - NS);
      uk *= sgn_flip(r.flip, v - NS);
    }
    return rk0 * un + rk1 * uk + s * (double)Ft[v];
  };
  double rho = 0.0, sb = 0.0, sq = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double t = T(k);
    rho += t;
    if (P.has_b) sb += t * P.b[k];
    if (P.has_q) sq += t * P.q[k];
  }
  if (!positive(rho) || (P.has_b && !positive(1.0 - sb))) return false;
#pragma unroll
  for (int k = 0; k < NS; ++k)
    if (!(T(k) >= -YTOL * rho)) return false;
  double mm = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double t = T(NS + d);
    mm += t * t;
  }
  const double ei = rho * T(NS + D) - 0.5 * mm;
  return positive(P.has_q ? ei - rho * sq : ei);
}

// per face: FP32 pipeline; the limiter's decisions from FP32 copies of the
// states with a margin, in FP64 when a state is too close to call
// DIR: the face direction, a template parameter so that every array indexed
// by it is indexed by a constant (registers, not the stack).  Five blocks per
// SM (<= 96 registers, a small spill) hide more of the cache loads' latency
// than four with 126 registers: 6 % less time for this kernel on GB300.
// RC: the ENO-type interpolation (RC_WENO5Z or one of Sec. 4.1's others).
template <int NS, int D, int DIR, int RC>
__global__ void __launch_bounds__(FACE_THREADS, 5)
    k_face(const KParams P, const float* __restrict__ Wc, const double* __restrict__ Un,
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
  ci[d] -= 1;
  const double dt = scal[0];
  const float Gamma = (float)scal[1];
  SpeciesF sp[NS];
  load_species<NS>(P, sp);

  CRef cr[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    int cc[3] = {ci[0], ci[1], ci[2]};
    cc[d] += j - 2;
    cr[j] = map_cell_m<1u << d>(P, cc[0], cc[1], cc[2]);
  }
  const CRef ri = cr[2], rj = cr[3];
  uint32_t fl = 0u;

  // FP32 copies of the two neighbours' conserved states (wall mirror applied)
  float Uki[NV], Ukj[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float si = v >= NS && v < NS + D ? sgnf(ri.flip, v - NS) : 1.f;
    const float sj = v >= NS && v < NS + D ? sgnf(rj.flip, v - NS) : 1.f;
    Uki[v] = wgetf(P, Wc, P.nW + v, ri) * si;
    Ukj[v] = wgetf(P, Wc, P.nW + v, rj) * sj;
  }

  // characteristic scalars at the averaged state (FP32 EOS)
  float X, c, ic;
  {
    float Ub[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Ub[v] = 0.5f * (Uki[v] + Ukj[v]);
    float rho = 0.f, Y[NS], ke = 0.f;
#pragma unroll
    for (int k = 0; k < NS; ++k) rho += Ub[k];
    const float ir = __frcp_rn(rho);
#pragma unroll
    for (int k = 0; k < NS; ++k) Y[k] = Ub[k] * ir;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const float u = Ub[NS + t] * ir;
      ke += u * u;
    }
    const float e = Ub[NS + D] * ir - 0.5f * ke;
    float p, T, r2, e2, a;
    pt_equilibrium_f<NS>(sp, Y, e, ir, p, T);
    // alpha, beta at the averaged state
    float sa = 0.f, sb = 0.f, cp = 0.f;
#pragma unroll
    for (int k = 0; k < NS; ++k)
      if (Y[k] != 0.f) {
        const float r = __frcp_rn(p + sp[k].pinf);
        sa += Y[k] * sp[k].Rk * r;
        sb += Y[k] * sp[k].Rk * T * r * r;
        cp += Y[k] * sp[k].cp;
      }
    eos_forward_f<NS>(sp, Y, p, T, r2, e2, a);
    const float al = r2 * sa, be = r2 * sb;
    X = (rho * a * a * be - 1.f) / (al * a * a * rho);
    c = a * rho;
    ic = __frcp_rn(c);
  }

  // deviations from the left cell, projection, WENO5-Z, back-projection
  const float Ti = wgetf(P, Wc, P.wT, ri), Tj = wgetf(P, Wc, P.wT, rj);
  const float Pi = wgetf(P, Wc, P.wP, ri), Pj = wgetf(P, Wc, P.wP, rj);
  float YL[NS], YR[NS], uL[3] = {0.f, 0.f, 0.f}, uR[3] = {0.f, 0.f, 0.f}, PL, PR, TL, TR;
  {
    const float uni = wgetf(P, Wc, P.wU + d, ri) * sgnf(ri.flip, d);
    float w1[6], w5[6], w6[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float dT = wgetf(P, Wc, P.wT, cr[j]) - Ti;
      const float dp = wgetf(P, Wc, P.wP, cr[j]) - Pi;
      const float du = wgetf(P, Wc, P.wU + d, cr[j]) * sgnf(cr[j].flip, d) - uni;
      w1[j] = dT - X * dp;
      w5[j] = (0.5f * c) * du + 0.5f * dp;
      w6[j] = (-0.5f * c) * du + 0.5f * dp;
    }
    float w1L, w1R, w5L, w5R, w6L, w6R;
    recon_lr_f<RC>(w1, w1L, w1R);
    recon_lr_f<RC>(w5, w5L, w5R);
    recon_lr_f<RC>(w6, w6L, w6R);
    TL = Ti + (w1L + X * (w5L + w6L));
    TR = Ti + (w1R + X * (w5R + w6R));
    uL[d] = uni + ic * (w5L - w6L);
    uR[d] = uni + ic * (w5R - w6R);
    PL = Pi + (w5L + w6L);
    PR = Pi + (w5R + w6R);
  }
  float Yi[NS], Yj[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    Yi[k] = wgetf(P, Wc, P.wY + k, ri);
    Yj[k] = wgetf(P, Wc, P.wY + k, rj);
    float y[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) y[j] = wgetf(P, Wc, P.wY + k, cr[j]) - Yi[k];
    float dl, dr;
    recon_lr_f<RC>(y, dl, dr);
    YL[k] = Yi[k] + dl;
    YR[k] = Yi[k] + dr;
  }
#pragma unroll
  for (int t = 0; t < D; ++t) {
    if (t == d) continue;
    const float ut = wgetf(P, Wc, P.wU + t, ri) * sgnf(ri.flip, t);
    float y[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) y[j] = wgetf(P, Wc, P.wU + t, cr[j]) * sgnf(cr[j].flip, t) - ut;
    float dl, dr;
    recon_lr_f<RC>(y, dl, dr);
    uL[t] = ut + dl;
    uR[t] = ut + dr;
  }

  if (P.pos_limiter) {
    if (y_limiter_f<NS>(YL, Yi)) fl |= F_YLIM_L;
    if (y_limiter_f<NS>(YR, Yj)) fl |= F_YLIM_R;
    if (!(TL > 0.f)) { TL = Ti; fl |= F_THETA_T_L; }
    if (!(TR > 0.f)) { TR = Tj; fl |= F_THETA_T_R; }
    bool okL = true, okR = true;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (YL[k] > 0.f && !(PL + sp[k].pinf > 0.f)) okL = false;
      if (YR[k] > 0.f && !(PR + sp[k].pinf > 0.f)) okR = false;
    }
    if (!okL) { PL = Pi; fl |= F_THETA_P_L; }
    if (!okR) { PR = Pj; fl |= F_THETA_P_R; }
  }

  float Fx[NV];
  {
    StateF<NS> sL, sR;
    state_from_primitive_f<NS>(sp, YL, uL, PL, TL, sL);
    state_from_primitive_f<NS>(sp, YR, uR, PR, TR, sR);
    hllc_f<NS, D>(d, sL, sR, Fx);
  }

  // positivity decisions on the pseudo-updates: FP32 with a margin, FP64
  // (exact as in the FP64 path) when too close to call
  const double lam = 2.0 * D * rk2 * dt * P.inv_dx;
  float Uni[NV], Unj[NV];
  if (P.pos_limiter) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float si = v >= NS && v < NS + D ? sgnf(ri.flip, v - NS) : 1.f;
      const float sj = v >= NS && v < NS + D ? sgnf(rj.flip, v - NS) : 1.f;
      Uni[v] = P.unf[(long long)v * P.wstride + ri.idx] * si;
      Unj[v] = P.unf[(long long)v * P.wstride + rj.idx] * sj;
    }
  }
  auto passes = [&](const float* Ft) {
    const float r0 = (float)rk0, r1 = (float)rk1, lf = (float)lam;
    const int a = admissible_f<NS, D>(P, Uni, Uki, Ft, r0, r1, -lf);
    if (a == 0) return false;
    const int b = admissible_f<NS, D>(P, Unj, Ukj, Ft, r0, r1, lf);
    if (b == 0) return false;
    if (a == 1 && b == 1) return true;
    return admissible_stream<NS, D>(P, Un, Uk, Uin, ri, Ft, rk0, rk1, -lam) &&
           admissible_stream<NS, D>(P, Un, Uk, Uin, rj, Ft, rk0, rk1, lam);
  };
  if (P.pos_limiter && !passes(Fx)) {
    StateF<NS> si, sj;
    si.rho = wgetf(P, Wc, P.wRho, ri);
    sj.rho = wgetf(P, Wc, P.wRho, rj);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      si.rhoY[k] = Uki[k];
      sj.rhoY[k] = Ukj[k];
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      si.u[t] = t < D ? wgetf(P, Wc, P.wU + t, ri) * sgnf(ri.flip, t) : 0.f;
      sj.u[t] = t < D ? wgetf(P, Wc, P.wU + t, rj) * sgnf(rj.flip, t) : 0.f;
      si.m[t] = t < D ? Uki[NS + t] : 0.f;
      sj.m[t] = t < D ? Ukj[NS + t] : 0.f;
    }
    si.p = Pi;
    sj.p = Pj;
    si.E = Uki[NS + D];
    sj.E = Ukj[NS + D];
    si.a = wgetf(P, Wc, P.wA, ri);
    sj.a = wgetf(P, Wc, P.wA, rj);
    hllc_f<NS, D>(d, si, sj, Fx);
    fl |= F_HLLC_FALLBACK;
  }

  if (P.cdi && P.two_phase) {
    bool pres_i[2] = {false, false}, pres_j[2] = {false, false};
    {
      // (branches on the phase rather than ypi[P.phase[k]]: an array indexed
      // at run time would live on the stack)
      float ypi[2] = {0.f, 0.f}, ypj[2] = {0.f, 0.f};
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
        pres_i[ph] = ypi[ph] > 0.f;
        pres_j[ph] = ypj[ph] > 0.f;
      }
    }
    if ((pres_i[0] || pres_j[0]) && (pres_i[1] || pres_j[1])) {
      const float ceps = P.f32.cdi_eps, idx = P.f32.inv_dx;
      const float psi_i = wgetf(P, Wc, P.wPsi, ri), psi_j = wgetf(P, Wc, P.wPsi, rj);
      const float dphi = (wgetf(P, Wc, P.wPhi0, rj) - wgetf(P, Wc, P.wPhi0, ri)) * idx;
      float g[3] = {0.f, 0.f, 0.f};
      g[d] = (psi_j - psi_i) * idx;
#pragma unroll
      for (int t = 0; t < D; ++t) {
        if (t == d) continue;
        int a0[3] = {ci[0], ci[1], ci[2]}, a1[3] = {ci[0], ci[1], ci[2]};
        a0[t] += 1;
        a1[t] -= 1;
        int b0[3] = {a0[0], a0[1], a0[2]}, b1[3] = {a1[0], a1[1], a1[2]};
        b0[d] += 1;
        b1[d] += 1;
        const float pip = wgetf(P, Wc, P.wPsi, map_cell_dt<d>(P, t, a0[0], a0[1], a0[2]));
        const float pim = wgetf(P, Wc, P.wPsi, map_cell_dt<d>(P, t, a1[0], a1[1], a1[2]));
        const float pjp = wgetf(P, Wc, P.wPsi, map_cell_dt<d>(P, t, b0[0], b0[1], b0[2]));
        const float pjm = wgetf(P, Wc, P.wPsi, map_cell_dt<d>(P, t, b1[0], b1[1], b1[2]));
        g[t] = 0.25f * idx * ((pip - pim) + (pjp - pjm));
      }
      const float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      const float nd = gn >= GTOL32 ? g[d] / gn : 0.f;
      const float ch = coshf((0.5f * (psi_i + psi_j)) / (2.f * ceps));
      const float sech2 = __frcp_rn(ch * ch);
      const float ahat0 = Gamma * (ceps * dphi - 0.25f * (sech2 - P.f32.sharp0) * nd);
      float Fdi[NV], Rtot = 0.f, hR = 0.f;
#pragma unroll
      for (int ph = 0; ph < 2; ++ph) {
        const float ahat = ph == 0 ? ahat0 : -ahat0;
        const bool pi = pres_i[ph], pj = pres_j[ph];
        auto keep = [&](float a, float b) { return pi && pj ? 0.5f * (a + b) : (pi ? a : (pj ? b : 0.f)); };
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          if (P.phase[k] != ph) continue;
          const float R = -keep(wgetf(P, Wc, P.wYrho + k, ri), wgetf(P, Wc, P.wYrho + k, rj)) * ahat;
          Fdi[k] = R;
          Rtot += R;
        }
        hR -= keep(wgetf(P, Wc, P.wHrho + ph, ri), wgetf(P, Wc, P.wHrho + ph, rj)) * ahat;
      }
      float kb = 0.f;
#pragma unroll
      for (int t = 0; t < D; ++t) {
        const float ui = wgetf(P, Wc, P.wU + t, ri) * sgnf(ri.flip, t);
        const float uj = wgetf(P, Wc, P.wU + t, rj) * sgnf(rj.flip, t);
        kb += ui * uj;
        Fdi[NS + t] = 0.5f * (ui + uj) * Rtot;
      }
      Fdi[NS + D] = 0.5f * kb * Rtot + hR;
      float Ft[NV];
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

  // the diffusive flux passes the regularization flux's limiter (as on the
  // FP64 path; FP32 test, FP64 when too close to call)
  float Fnu[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Fnu[v] = 0.f;
  if (P.diffusion) {
    const float idx = P.f32.inv_dx;
    const float rb = 0.5f * (wgetf(P, Wc, P.wRho, ri) + wgetf(P, Wc, P.wRho, rj));
    float Jh = 0.f;
#pragma unroll
    for (int ph = 0; ph < 2; ++ph) {
      float Yp = 0.f, S = 0.f, Bf[NS], G[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        Bf[k] = 0.f;
        G[k] = 0.f;
        if (P.phase[k] != ph) continue;
        Yp += 0.5f * (Yi[k] + Yj[k]);
        Bf[k] = 0.5f * (wgetf(P, Wc, P.wB + k, ri) + wgetf(P, Wc, P.wB + k, rj));
        G[k] = (wgetf(P, Wc, P.wXr + k, rj) - wgetf(P, Wc, P.wXr + k, ri)) * idx;
        S += Bf[k] * G[k];
      }
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        if (P.phase[k] != ph) continue;
        const float J = -rb * (Yp * Bf[k] * G[k] - 0.5f * (Yi[k] + Yj[k]) * S);
        Fnu[k] = J;
        const float hi = sp[k].cp * Ti + sp[k].b * Pi + sp[k].q;
        const float hj = sp[k].cp * Tj + sp[k].b * Pj + sp[k].q;
        Jh += J * (0.5f * (hi + hj));
      }
    }
    Fnu[NS + D] = Jh;
  }

  // viscous stress and heat conduction in FP32, as the FP64 face kernel's
  // (second-order central; uniform u and T give exactly zero)
  if (P.viscous) {
    const float idx = P.f32.inv_dx;
    float gu[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) gu[i][j] = 0.f;
    float ui[3] = {0.f, 0.f, 0.f}, uj[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < D; ++i) {
      ui[i] = wgetf(P, Wc, P.wU + i, ri) * sgnf(ri.flip, i);
      uj[i] = wgetf(P, Wc, P.wU + i, rj) * sgnf(rj.flip, i);
      gu[i][d] = (uj[i] - ui[i]) * idx;
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
        const float dip = wgetf(P, Wc, P.wU + i, ip) * sgnf(ip.flip, i) - wgetf(P, Wc, P.wU + i, im) * sgnf(im.flip, i);
        const float djp = wgetf(P, Wc, P.wU + i, jp) * sgnf(jp.flip, i) - wgetf(P, Wc, P.wU + i, jm) * sgnf(jm.flip, i);
        gu[i][t] = 0.25f * idx * (dip + djp);
      }
    }
    float div = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) div += gu[k][k];
    const float mub = 0.5f * (wgetf(P, Wc, P.wMu, ri) + wgetf(P, Wc, P.wMu, rj));
    const float lamb = 0.5f * (wgetf(P, Wc, P.wLam, ri) + wgetf(P, Wc, P.wLam, rj));
    float work = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float tau = mub * (gu[i][d] + gu[d][i] - (i == d ? (2.f / 3.f) * div : 0.f));
      Fnu[NS + i] = -tau;
      work += 0.5f * (ui[i] + uj[i]) * tau;
    }
    Fnu[NS + D] -= work + lamb * (Tj - Ti) * idx;
  }
  if (P.diffusion || P.viscous) {
    float Ft[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Ft[v] = Fx[v] + Fnu[v];
    if (P.pos_limiter && !passes(Ft)) {
      fl |= F_DIFF_DROPPED;
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) Fx[v] = Ft[v];
    }
  }

  // stored widened to FP64 (exact): the update then takes every flux with
  // the same FP64 value in its two cells, and the widening happens once per
  // face, here, where the FP64 pipe is otherwise idle
  for (int v = 0; v < NV; ++v) F[(long long)v * nf + fid] = (double)Fx[v];
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

// divergence and RK combination in FP64 (the FP64 path's, on the widened fluxes)
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

inline unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// the mixed face pass of one direction with interpolation RC
template <int NS, int D, int RC>
struct FaceImpl {
  static void face(const KParams& P, cudaStream_t s, int d, const double* Wc, const double* Un, const double* Uk,
                   const double* Uin, const double* scal, double rk0, double rk1, double rk2, double* F,
                   uint32_t* flags, unsigned long long* stats) {
    long long nf = 1;
    for (int e = 0; e < 3; ++e) nf *= (long long)(P.n[e] + (e == d));
    const unsigned nb = nblocks(nf, FACE_THREADS);
    const float* W = reinterpret_cast<const float*>(Wc);
    if (d == 0)
      k_face<NS, D, 0, RC><<<nb, FACE_THREADS, 0, s>>>(P, W, Un, Uk, Uin, scal, rk0, rk1, rk2, F, flags, stats);
    else if (d == 1)
      k_face<NS, D, (D > 1 ? 1 : 0), RC><<<nb, FACE_THREADS, 0, s>>>(P, W, Un, Uk, Uin, scal, rk0, rk1, rk2, F,
                                                                     flags, stats);
    else
      k_face<NS, D, (D > 2 ? 2 : 0), RC><<<nb, FACE_THREADS, 0, s>>>(P, W, Un, Uk, Uin, scal, rk0, rk1, rk2, F,
                                                                     flags, stats);
  }
};

// the mixed face pass of interpolation RC for (dimension, species count)
template <int RC>
FaceFn face_mixed(int dim, int ns) {
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
  static void prim(const KParams& P, cudaStream_t s, const double* U, const double* Uin, double* Wc,
                   unsigned long long* red, int* status) {
    k_prim<NS, D><<<nblocks(P.ncell + P.nextra, CELL_THREADS), CELL_THREADS, 0, s>>>(
        P, U, Uin, reinterpret_cast<float*>(Wc), red, status);
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
};

}  // namespace mx
}  // namespace mpmc
