/*
 * CPU oracle for the four-equation multi-phase multi-component (MPMC)
 * finite-volume right-hand side and its SSP-RK3 stages (arXiv 2504.14063).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or helper with the GPU library: everything below is
 * written plainly, in FP64, following the paper's equations in the paper's
 * order, with face fluxes stored in arrays (each face computed once) and
 * one sweep per direction.  Nothing is blocked, fused or reordered.
 *
 * Layout of every field array handed to this API: structure of arrays,
 * [component][nz][ny][nx], x fastest, interior cells only (no ghosts).
 *   conserved U : [rhoY_0..rhoY_{ns-1}, m_0..m_{dim-1}, E]      (ns+dim+1)
 *   primitive   : [alpha_0..alpha_{ns-1}, u_0..u_{dim-1}, P, T] (ns+dim+2)
 * alpha_k are species volume fractions (Amagat: each species occupies its
 * own volume at the common P and T), so rhoY_k = alpha_k / v_k(P, T).
 */
#ifndef MPMC_ORACLE_H
#define MPMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXS 8

/* boundary codes */
#define ORC_BC_PERIODIC 0
#define ORC_BC_WALL 1      /* reflecting slip wall: mirror, normal velocity negated */
#define ORC_BC_ZEROGRAD 2  /* copy of the boundary cell */
#define ORC_BC_INFLOW 3    /* Dirichlet: fixed primitive state `inflow` */
#define ORC_BC_CHAR 4      /* characteristic non-reflecting inflow/outflow towards the far-field
                              state `inflow` (Sec. 3.5); direction 0 only */

/* per-face flag bits written by orc_stage (same meaning as the GPU tape bits,
 * defined independently there) */
#define ORC_F_THETA_T_L (1u << 0)
#define ORC_F_THETA_T_R (1u << 1)
#define ORC_F_THETA_P_L (1u << 2)
#define ORC_F_THETA_P_R (1u << 3)
#define ORC_F_HLLC_FALLBACK (1u << 4)
#define ORC_F_CDI_DROPPED (1u << 5)
#define ORC_F_YLIM_L (1u << 6)
#define ORC_F_YLIM_R (1u << 7)
#define ORC_F_DIFF_DROPPED (1u << 8)

typedef struct {
  /* grid */
  int dim;          /* 1, 2 or 3 */
  int n[3];         /* cells per direction; inactive directions = 1 */
  double dx;        /* isotropic spacing (Section 3.1) */
  int bc_lo[3], bc_hi[3];
  double inflow[ORC_MAXS + 5]; /* primitive inflow state, same layout as a primitive cell */
  /* species (Eq. NASG_EOS), phase 0 = liquid, phase 1 = gas */
  int ns;
  int phase[ORC_MAXS];
  double cv[ORC_MAXS], gamma[ORC_MAXS], q[ORC_MAXS], b[ORC_MAXS], pinf[ORC_MAXS];
  double W[ORC_MAXS], mu[ORC_MAXS], Sc[ORC_MAXS];
  /* model */
  double weno_eps;   /* WENO5-Z epsilon */
  int cdi;           /* interface regularization on/off */
  int diffusion;     /* species diffusion on/off */
  int pos_limiter;   /* interpolation + flux limiters on/off */
  double cdi_eps;    /* CDI length scale epsilon */
  double cdi_gamma;  /* > 0: fixed velocity scale Gamma; <= 0: Gamma = max |u_d| */
  double phi_min;    /* CDI volume-fraction floor */
  double psi_delta;  /* delta of the psi transform */
  double cfl;
  double mu_liquid;  /* liquid-phase viscosity (constant) */
  int recon_basis;   /* 0: characteristic [T, Y, u, P] (the method);
                        1: component-wise [rhoY, u, P] (negative control, test only) */
  int eos_iterative; /* 1: force the iterative p-T solve even when the closed form applies */
  int nthreads;      /* OpenMP threads, <= 0: library default */
  int recon;         /* ENO-type interpolation: 0 WENO5-Z (the method's default),
                        1 WENO5-JS, 2 TENO5, 3 TENO6 (Sec. 4.1's other schemes) */
  int viscous;       /* viscous stress and heat conduction on/off */
  double prandtl;    /* gas-phase Prandtl number (lambda_g = mu_g cp_g / Pr) */
  double lambda_liquid; /* liquid-phase heat conductivity [W/(m K)] */
} orc_params;

/* status codes */
#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_INADMISSIBLE 3
#define ORC_EOS_NO_CONVERGE 4

int orc_nvars(const orc_params* p);
int orc_init_state(const orc_params* p, const double* prim, double* U);
/* per-cell diagnostics: out = [P, T, a, rho, phi_0, phi_1, psi_0, psi_1] x ncells */
int orc_primitives(const orc_params* p, const double* U, double* out);
/* CFL time step and CDI velocity scale from U (Section 3.4, Section 3.2) */
int orc_dt_gamma(const orc_params* p, const double* U, double* dt, double* Gamma);
/* One SSP-RK stage: L = L(U_k) with the limiters using U_n, rk0..rk2 and dt;
 * U_out = rk0*U_n + rk1*U_k + rk2*dt*L.  dUdt, U_out, flags may be NULL.
 * flags: per face, [dim][faces of that direction], faces of direction d
 * laid out like cells with n_d+1 entries along d. */
int orc_stage(const orc_params* p, const double* U_n, const double* U_k,
              double rk0, double rk1, double rk2, double dt, double Gamma,
              double* U_out, double* dUdt, uint32_t* flags);
/* Face fluxes of one stage evaluation, [dim][nv][faces of that direction]. */
int orc_face_fluxes(const orc_params* p, const double* U_n, const double* U_k,
                    double rk0, double rk1, double rk2, double dt, double Gamma,
                    double* F);
/* One SSP-RK3 step in place. dt <= 0: CFL step from U^n. Returns dt used. */
int orc_rk_step(const orc_params* p, double* U, double dt, double* dt_used);
/* n steps (or until t_end > 0 is reached, last step clipped). */
int orc_run(const orc_params* p, double* U, int nsteps, double t_end, double* t_out, int* steps_out);

/* --- point functions exposed for pins ------------------------------------ */
/* p-T equilibrium (Eqs. NASG_T1, NASG_T2, NASG_P): Y[ns], e, v -> P, T */
int orc_eos_pt(const orc_params* p, const double* Y, double e, double v, double* P, double* T);
/* forward EOS at (P, T, Y): out = [rho, e, a, alpha, beta, cp] */
int orc_eos_forward(const orc_params* p, const double* Y, double P, double T, double* out);
double orc_weno5z(const double* v5, double eps);
/* the interpolation of kind 0..3 (see orc_params.recon) at the right face of
 * cell i from the cells i-2..i+3 */
double orc_reconstruct(int kind, const double* v6, double eps);
/* candidate polynomial of the n cells starting at offset (relative to cell
 * i = v6[2]) fitted to the cell averages: its value at the right face of
 * cell i and its Jiang-Shu smoothness indicator on cell i */
void orc_candidate(const double* v6, int offset, int n, double* value, double* beta);
/* the mass-fraction limiter of Sec. 3.3.1 on one face side: Y[ns] (in/out)
 * the reconstructed mass fractions, Yc[ns] the adjacent cell's; returns 1 if
 * it changed Y, 0 if not, -1 on invalid parameters */
int orc_y_limiter(const orc_params* p, double* Y, const double* Yc);
/* face states of the face (i, j, k) of direction d of U (interior cells,
 * ghosts filled as in orc_stage; the face's low cell is i-1 along d):
 * W = [Y_0..Y_{ns-1}, u_0, u_1, u_2, P, T] of each side after the
 * interpolation limiters of Sec. 3.3.1 (before them when pos_limiter = 0);
 * flags receives their ORC_F_THETA_* / ORC_F_YLIM_* bits */
int orc_face_states(const orc_params* p, const double* U, int d, int i, int j, int k, double* WL,
                    double* WR, uint32_t* flags);
/* characteristic matrices of direction d at the conserved state Ubar:
 * Sinv, S dense nc x nc row-major, nc = ns + dim + 1; scal = [rho, a, alpha, beta, X, rho*a] */
int orc_char_matrices(const orc_params* p, int d, const double* Ubar, double* Sinv, double* S, double* scal);
/* HLLC flux (Appendix B) between two primitive states W = [Y_0..Y_{ns-1}, u_0, u_1, u_2, P, T] */
int orc_hllc_prim(const orc_params* p, int d, const double* WL, const double* WR, double* F);
int orc_physical_flux(const orc_params* p, int d, const double* W, double* F);
/* conserved vector of a primitive point state W (layout as in orc_hllc_prim) */
int orc_cons_from_point(const orc_params* p, const double* W, double* U);

/* Forward-mode tangents (directional derivatives of the discrete map, its
 * branches taken on values; dt and Gamma frozen), the CPU reference for the
 * discrete adjoint.  Each returns the primal outputs as well. */
int orc_stage_jvp(const orc_params* p, const double* U_n, const double* U_k, const double* dU_k,
                  double rk0, double rk1, double rk2, double dt, double Gamma, double* dUdt,
                  double* d_dUdt);
/* one SSP-RK3 step with the given dt > 0 and Gamma >= 0 */
int orc_rk_step_jvp(const orc_params* p, const double* U, const double* dU, double dt, double Gamma,
                    double* U_out, double* dU_out);
/* the eight fields of orc_primitives and their tangents */
int orc_primitives_jvp(const orc_params* p, const double* U, const double* dU, double* out, double* dout);
int orc_init_state_jvp(const orc_params* p, const double* prim, const double* dprim, double* U, double* dU);
/* WENO5-Z value and tangent (ideal weights on a stencil flat to 1e-10) */
double orc_weno5z_jvp(const double* v5, const double* dv5, double eps, double* dout);

#ifdef __cplusplus
}
#endif
#endif
