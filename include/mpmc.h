/*
 * mpmc.h -- C ABI of the GB300 library for the hot path of the four-equation
 * multi-phase multi-component (MPMC) solver of arXiv 2504.14063: the
 * finite-volume right-hand side evaluated at every stage of the explicit
 * SSP-RK3 scheme, with the stage update fused in.
 *
 * Method (all section / equation names are the paper's):
 *   - conserved U = [rhoY_k, rho u, E] -> primitives through the p-T
 *     equilibrium closure of the NASG mixture (Sec. 2.2-2.3, Eqs. NASG_EOS,
 *     NASG_T1, NASG_T2, NASG_P);
 *   - per face: characteristic projection of W = [T, Y, u, P] (Sec. 3.1.2,
 *     Appendix A), WENO5-Z interpolation (Sec. 4), interpolation limiters
 *     (Sec. 3.3.1), face EOS, HLLC (Appendix B), flux limiter (Sec. 3.3.2),
 *     KEEP-split CDI regularization flux (Sec. 3.2, Eqs. MPMC_ACDI,
 *     SkewSymmetricSplitting_Regularization*) with its limiter, and the
 *     phase-confined species diffusion flux (Eq. SpeciesMassDiffusion);
 *   - per cell: divergence and SSP-RK3 combination (Eq. SSPRK3) with the
 *     CFL step of Sec. 3.4 computed on the device.
 *
 * Conventions
 *   - Every array argument is a DEVICE pointer unless its name ends in
 *     `_host`.  Arrays are structure-of-arrays, [component][nz][ny][nx], x
 *     fastest, FP64, interior cells only (no ghost layers; boundary ghosts are
 *     produced by index mapping inside the kernels).
 *       conserved U : ns + dim + 1 components [rhoY_0..rhoY_{ns-1}, m_0..m_{dim-1}, E]
 *       primitive   : ns + dim + 2 components [alpha_0..alpha_{ns-1}, u_0..u_{dim-1}, P, T]
 *     alpha_k are species volume fractions (Amagat): rhoY_k = alpha_k / v_k(P, T).
 *   - The caller owns every array it passes; the context owns its scratch
 *     (primitive cache, face fluxes, RK stage registers, reduction scalars,
 *     tape workspace), allocated in mpmc_create and freed in mpmc_destroy.
 *   - All work is enqueued on the context's CUDA stream (a cudaStream_t
 *     passed as void*; NULL = the legacy default stream).  mpmc_rhs,
 *     mpmc_rk_step and mpmc_step_n never synchronize the host.
 *   - Every call returns an int status (MPMC_OK = 0).  Errors detected on the
 *     device (an inadmissible cell, an equation-of-state solve that did not
 *     converge) are latched in a device status word and returned by
 *     mpmc_get_status or the next synchronizing call.  No device traps.
 */
#ifndef MPMC_H
#define MPMC_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPMC_MAXS 4 /* species supported by the kernels */

/* status codes */
#define MPMC_OK 0
#define MPMC_INVALID_ARG 1
#define MPMC_CUDA_ERROR 2
#define MPMC_INADMISSIBLE 3    /* a cell violates Eqs. PositivityReqs1/2 */
#define MPMC_EOS_NO_CONVERGE 4 /* iterative p-T equilibrium hit its iteration cap */
#define MPMC_OUT_OF_MEMORY 5

/* boundary conditions of the ghost layers */
#define MPMC_BC_PERIODIC 0
#define MPMC_BC_WALL 1     /* reflecting slip wall: mirror image, normal velocity negated */
#define MPMC_BC_ZEROGRAD 2 /* copy of the boundary cell */
#define MPMC_BC_INFLOW 3   /* Dirichlet: the fixed primitive state mpmc_grid.inflow */
#define MPMC_BC_CHAR 4     /* characteristic non-reflecting inflow / outflow (Sec. 3.5, the conditions
                              of Thompson and of Poinsot & Lele in their locally one-dimensional
                              inviscid form): per boundary cell, the characteristic fields of
                              Appendix A that leave the domain keep the cell's values and those that
                              enter take the far-field state mpmc_grid.inflow.  x boundaries only
                              (MPMC_INVALID_ARG on y or z); forward paths only: the adjoint entries
                              and mpmc_rhs_noalloc refuse it (MPMC_INVALID_ARG) */

/* ENO-type interpolation of the face states (Sec. 3.1.3; Sec. 4.1 runs all
 * four).  WENO5-Z (Borges et al. 2008) is the method's; the others follow
 * their cited definitions (Jiang & Shu 1996; Fu, Hu & Adams 2016), on FP64
 * and mixed contexts (FP32 there) and in the adjoint (TENO differentiated
 * with its candidate selection replayed). */
#define MPMC_RECON_WENO5Z 0
#define MPMC_RECON_WENO5JS 1 /* eps 1e-6, exponent 2 */
#define MPMC_RECON_TENO5 2   /* C = 1, q = 6, CT = 1e-5 */
#define MPMC_RECON_TENO6 3   /* C = 1, q = 6, CT = 1e-7, six-cell stencil i-2..i+3 */

/* precision of the hot path */
#define MPMC_FP64 0
#define MPMC_MIXED 1 /* reconstruction, fluxes, diffusion in FP32; EOS inversion,
                        positivity bounds and RK accumulation in FP64 */

/* per-face tape bits (mpmc_rk_step tape, mpmc_rhs flags) */
#define MPMC_F_THETA_T_L (1u << 0) /* left T fell back to the cell value (Sec. 3.3.1) */
#define MPMC_F_THETA_T_R (1u << 1)
#define MPMC_F_THETA_P_L (1u << 2)
#define MPMC_F_THETA_P_R (1u << 3)
#define MPMC_F_HLLC_FALLBACK (1u << 4) /* first-order HLLC of the cell states (Sec. 3.3.2) */
#define MPMC_F_CDI_DROPPED (1u << 5)   /* regularization flux not added (Sec. 3.3.2, last paragraph) */
#define MPMC_F_YLIM_L (1u << 6)        /* mass-fraction limiter changed the left state */
#define MPMC_F_YLIM_R (1u << 7)
#define MPMC_F_DIFF_DROPPED (1u << 8) /* diffusive flux (species diffusion, viscous stress, conduction) not
                                         added: the regularization flux's limiter applied to it */

/* Grid (Sec. 3.1: isotropic Cartesian cells). n[d] = 1 for inactive
 * directions; active directions need n[d] >= 3. */
typedef struct {
  int dim;
  int n[3];
  double dx;
  int bc_lo[3], bc_hi[3];
  double inflow[MPMC_MAXS + 5]; /* primitive inflow state [alpha(ns), u(dim), P, T]; also the
                                   far-field state of MPMC_BC_CHAR boundaries */
} mpmc_grid;

/* Species table (Eq. NASG_EOS per species; Table NASGMaterialParamters).
 * phase 0 = liquid, 1 = gas.  W: molar mass; mu: viscosity (gas species,
 * mixed by Wilke's rule, Sec. 2.2.2); Sc: Schmidt number (Sec. 2.2.3). */
typedef struct {
  int n_species;
  int phase[MPMC_MAXS];
  double cv[MPMC_MAXS], gamma[MPMC_MAXS], q[MPMC_MAXS], b[MPMC_MAXS], pinf[MPMC_MAXS];
  double W[MPMC_MAXS], mu[MPMC_MAXS], Sc[MPMC_MAXS];
} mpmc_eos;

/* Model coefficients (Sec. 3.2: Gamma, epsilon, phi_min, delta; Sec. 3.4: CFL) */
typedef struct {
  double weno_eps;  /* WENO5-Z epsilon (1e-40) */
  int cdi;          /* interface regularization on/off */
  int diffusion;    /* species diffusion on/off */
  int pos_limiter;  /* interpolation and flux limiters on/off */
  double cdi_eps;   /* CDI length scale epsilon [m] */
  double cdi_gamma; /* > 0: fixed Gamma [m/s]; <= 0: Gamma = max |u_d| of U^n each step */
  double phi_min;   /* 1e-8 */
  double psi_delta; /* 1e-100 */
  double cfl;       /* 0.5 */
  double mu_liquid; /* liquid-phase viscosity [Pa s] */
  int precision;    /* MPMC_FP64 or MPMC_MIXED */
  int recon;        /* MPMC_RECON_*; 0 (WENO5-Z) is the default.  Another value
                       is refused by mpmc_rhs_noalloc (MPMC_INVALID_ARG) */
  int viscous;      /* viscous stress and heat conduction (Eq. DiffusionTerms:
                       tau = mu (grad u + grad u^T - 2/3 div u I),
                       q = -lambda grad T + sum J h), second-order central on
                       the faces (FP32 on mixed contexts); reversed by the
                       adjoint entries too */
  double prandtl;   /* gas-phase Prandtl number: lambda_g = mu_g cp_g / Pr
                       (> 0 when viscous) */
  double lambda_liquid; /* liquid-phase heat conductivity [W/(m K)] (>= 0) */
} mpmc_model;

/* One SSP-RK stage: U^(k+1) = rk0 U^n + rk1 U^(k) + rk2 dt L(U^(k)).
 * The flux limiter of Sec. 3.3.2 tests pseudo-updates built from these.
 * dt <= 0: CFL step from U_n; Gamma < 0: max |u_d| of U_n. */
typedef struct {
  const double* U_n; /* device */
  double rk0, rk1, rk2, dt, Gamma;
} mpmc_stage;

typedef struct {
  uint64_t faces;          /* faces evaluated since the last reset */
  uint64_t hllc_fallback;  /* faces that took the first-order flux */
  uint64_t cdi_dropped;    /* faces whose regularization flux was dropped */
  uint64_t theta_p, theta_t, ylim; /* interpolation-limiter activations (face sides) */
  uint64_t diff_dropped;   /* faces whose diffusive flux was dropped (MPMC_F_DIFF_DROPPED) */
} mpmc_stats;

typedef struct mpmc_ctx mpmc_ctx;

/* Creates a context for one grid / species table / model on the current
 * CUDA device; allocates all scratch sized by the grid.  stream: cudaStream_t
 * or NULL.  Returns MPMC_INVALID_ARG for unsupported sizes (ns > MPMC_MAXS,
 * dim outside 1..3, an active n[d] < 3, dx <= 0, 2^31 - 1 or more cells or
 * faces in one direction: the kernels index them in 32 bits, and no such
 * grid's state and scratch fit in one GPU's memory), MPMC_OUT_OF_MEMORY if an
 * allocation fails.  *out is NULL on failure. */
int mpmc_create(const mpmc_grid* grid, const mpmc_eos* eos, const mpmc_model* model, void* stream,
                mpmc_ctx** out);
void mpmc_destroy(mpmc_ctx* ctx);
int mpmc_set_stream(mpmc_ctx* ctx, void* stream);
/* Number of conserved components ns + dim + 1 and of cells. */
int mpmc_nvars(const mpmc_ctx* ctx);
size_t mpmc_ncells(const mpmc_ctx* ctx);
/* Doubles of one primitive cache (the per-cell fields of Sec. 3.1.3's
 * step 1 that the face pass reads, with the boundary slots): the unit of
 * the W_stages buffers of mpmc_rk_step_record / mpmc_rk_step_adjoint.  0
 * for a null context. */
size_t mpmc_cache_doubles(const mpmc_ctx* ctx);

/* Conserved state from primitive fields (Eq. NASG_EOS with Amagat mixing,
 * Sec. 2.2.1): rhoY_k = alpha_k / v_k(P,T), m = rho u,
 * E = sum_k rhoY_k e_k(P,T) + rho |u|^2 / 2.  prim, U: device. */
int mpmc_init_state(mpmc_ctx* ctx, const double* prim, double* U);

/* Right-hand side L(U) of Eq. DiscreteGoverningEquations (convective HLLC
 * flux with the limiters, regularization and diffusion fluxes).  The flux
 * limiter is stage-aware (Sec. 3.3.2): stage = NULL means a forward-Euler
 * stage from U with the CFL step and Gamma of U.  dUdt: device, same layout
 * as U.  flags (nullable, device): per face, all faces of direction 0, then
 * 1, then 2, each laid out like cells with n[d]+1 entries along d. */
int mpmc_rhs(mpmc_ctx* ctx, const double* U, double* dUdt, const mpmc_stage* stage, uint32_t* flags);

/* One SSP-RK3 step (Eq. SSPRK3) in place on device array U.  dt > 0: fixed
 * step; dt <= 0: CFL step (Sec. 3.4) from U^n computed on the device.  tape
 * (nullable, device, 3 x faces uint32): per stage and face the flag bits
 * above, for replay by the adjoint. */
int mpmc_rk_step(mpmc_ctx* ctx, double* U, double dt, uint32_t* tape);

/* n SSP-RK3 steps in place (replayed as a CUDA graph); each step takes its
 * CFL step (Sec. 3.4) from its own U^n on the device.  t_end > 0: the run
 * stops at physical time t_end — the step that would pass it is clipped to
 * it and any later step has zero length (U unchanged), all decided on the
 * device; t_end <= 0: no end time.  dt_dev_out (nullable, device): receives
 * the n step sizes (their sum is the time advanced).  Asynchronous, like
 * mpmc_rk_step: the call returns once the steps are enqueued on the
 * context's stream (the host does not wait for them); mpmc_get_status
 * synchronizes. */
int mpmc_step_n(mpmc_ctx* ctx, double* U, int n, double t_end, double* dt_dev_out);

/* Host-buffer entry: copies U_host (nv x ncells FP64, pinned or pageable)
 * to the device, runs n steps, copies the state back; synchronizes.  The
 * device copy lives in the context. */
int mpmc_step_n_host(mpmc_ctx* ctx, double* U_host, int n);

/* CFL step and regularization velocity scale of U (Sec. 3.4, Sec. 3.2):
 * writes [dt, Gamma] to out_dev (2 doubles, device). */
int mpmc_dt_gamma(mpmc_ctx* ctx, const double* U, double* out_dev);

/* ---- Discrete adjoint (FP64 contexts; MPMC_INVALID_ARG on a mixed one) ----
 * The adjoint of the discrete map itself: every discrete decision of the
 * forward pass (interpolation limiters theta_T / theta_P of Sec. 3.3.1,
 * first-order fallback of the flux limiter of Sec. 3.3.2, dropped
 * regularization flux) is replayed from its flag bits, the Y limiter of
 * Sec. 3.3.1 is differentiated on the branch the forward took, and dt and
 * Gamma (Sec. 3.4, Sec. 3.2) are frozen at the forward values.  A species
 * with Y_k = 0 exactly contributes no sensitivity (the forward omits it).
 * Adjoint scratch (cache adjoint, two state-sized buffers, one step of flags)
 * is allocated on the first call; MPMC_OUT_OF_MEMORY if that fails.
 *
 * lam_U += (dL/dU)^T lam_dUdt for the stage of mpmc_rhs at U.  stage: as for
 * mpmc_rhs (nullable; dt <= 0 / Gamma < 0 are recomputed from U_n exactly as
 * the forward did); tape: that call's flags (nullable: the decisions are
 * recomputed); lam_dUdt, lam_U: device, layout of U. */
int mpmc_rhs_adjoint(mpmc_ctx* ctx, const double* U, const mpmc_stage* stage, const uint32_t* tape,
                     const double* lam_dUdt, double* lam_U);

/* One SSP-RK3 step like mpmc_rk_step that also keeps what its reverse needs:
 * U_stages (device, 2 x nv x ncells, caller-owned) receives the stage states
 * U^(1) and U^(2); tape (nullable, device, 3 x faces uint32) the flags;
 * W_stages (nullable, device, 3 x mpmc_cache_doubles, caller-owned; FP64
 * contexts only, else MPMC_INVALID_ARG) the primitive caches of U^n, U^(1)
 * and U^(2), which spare the reverse step their recomputation. */
int mpmc_rk_step_record(mpmc_ctx* ctx, double* U, double dt, uint32_t* tape, double* U_stages, double* W_stages);

/* Reverse of one SSP-RK3 step (Eq. SSPRK3) from U_n:
 *   lam_n = (dU^{n+1}/dU^n)^T lam_next.
 * dt: as passed to mpmc_rk_step (<= 0: the CFL step of U_n, recomputed
 * bit-identically).  U_stages (nullable): the step's stage states from
 * mpmc_rk_step_record; recomputed from U_n when null.  W_stages (nullable;
 * only with U_stages): that call's primitive caches, used instead of
 * recomputing them (the result is the same bit for bit).  tape: that step's
 * 3 x faces flags (nullable: recomputed).  lam_n may equal lam_next (in
 * place).  Device arrays, layout of U.  The result does not depend on the
 * order in which the GPU runs threads (no atomic accumulation). */
int mpmc_rk_step_adjoint(mpmc_ctx* ctx, const double* U_n, const double* U_stages, const double* W_stages, double dt,
                         const uint32_t* tape, const double* lam_next, double* lam_n);

/* Reverse of mpmc_init_state: lam_prim = (dU/dprim)^T lam_U, layouts as for
 * mpmc_init_state (prim: the forward's input). */
int mpmc_init_state_adjoint(mpmc_ctx* ctx, const double* prim, const double* lam_U, double* lam_prim);

/* Primitive variables of U (Sec. 2.2-2.3): out (device, (4 + ns + dim) x
 * ncells FP64) = [T, P, rho, a, Y_0..Y_{ns-1}, u_0..u_{dim-1}], each a row of
 * ncells in the cell order of U.  FP64 contexts. */
int mpmc_primitives(mpmc_ctx* ctx, const double* U, double* out);

/* lam_U += (dW/dU)^T lam_W for W = mpmc_primitives(U); lam_W in that layout. */
int mpmc_primitives_adjoint(mpmc_ctx* ctx, const double* U, const double* lam_W, double* lam_U);

/* Statistics of the limiters since the last reset (synchronizes). */
int mpmc_get_stats(mpmc_ctx* ctx, mpmc_stats* out, int reset);
/* Device status word (synchronizes): MPMC_OK, MPMC_INADMISSIBLE or
 * MPMC_EOS_NO_CONVERGE.  reset != 0 clears it. */
int mpmc_get_status(mpmc_ctx* ctx, int reset);
/* Kernel timing: with profiling enabled the context records CUDA events on
 * its stream around every launch it makes outside graph capture (no host
 * synchronization).  mpmc_get_profile synchronizes and returns, per kernel
 * family, the summed device time in ms and the launch count:
 * [0] primitive recovery, [1] face fluxes, [2] divergence + RK update,
 * [3] time-step scalars, [4] adjoint face kernels, [5] adjoint primitive
 * kernels: ms and launches must hold 6 entries.  reset != 0 clears the sums. */
int mpmc_set_profiling(mpmc_ctx* ctx, int enable);
int mpmc_get_profile(mpmc_ctx* ctx, double* ms, uint64_t* launches, int reset);

/* Right-hand side without allocation, for callers that cannot allocate
 * device memory: code running inside another framework's memory pool or
 * arena that owns the device, real-time or embedded host loops that must not
 * block on the allocator, or setups where no allocator exists yet.  The paper
 * has no counterpart; this is a deployment variant of mpmc_rhs.
 *   - Same result as mpmc_rhs(U, dUdt, stage, NULL) for the same grid, species
 *     table and model (FP64 only: model->precision must be MPMC_FP64); no
 *     context is needed, the structs are passed directly.
 *   - Scratch (primitive cache, face fluxes, reduction scalars) lives in one
 *     fixed device array of MPMC_NOALLOC_SCRATCH_BYTES that every GPU which
 *     loads the library holds until the process exits.  No cudaMalloc,
 *     cudaFree or allocating library routine is called.
 *   - A grid whose scratch exceeds that size is rejected with
 *     MPMC_INVALID_ARG before any GPU work; *scratch_bytes (nullable) receives
 *     the bytes the grid needs.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) and keeps it for the process; make that first
 *     call before any stream capture.  A device reset (cudaDeviceReset)
 *     invalidates the kept address: do not call this entry on a device
 *     after resetting it in the same process.
 *   - If an error from earlier work is pending on the calling thread
 *     (cudaPeekAtLastError), the call returns MPMC_CUDA_ERROR before any
 *     work and leaves that error in place for its owner.
 *   - Every call uses the same array and leaves its contents behind; calls
 *     whose work overlaps on the GPU (different streams without ordering)
 *     race.  Serialize them on one stream.
 *   - Work is enqueued on `stream` without host synchronization; errors found
 *     on the device (inadmissible cells) are not reported by this entry.
 * U, dUdt and stage->U_n are device arrays in the layout of mpmc_rhs. */
#define MPMC_NOALLOC_SCRATCH_BYTES (32u << 20)
int mpmc_rhs_noalloc(const mpmc_grid* grid, const mpmc_eos* eos, const mpmc_model* model, void* stream,
                     const double* U, double* dUdt, const mpmc_stage* stage, size_t* scratch_bytes);

/* Arithmetic-rate probe (a measurement utility; the paper has no counterpart):
 * one launch of `blocks` x 256 threads, each running eight independent
 * fused-multiply-add chains for `iters` rounds in FP64 (fp64 != 0) or FP32,
 * i.e. 16 x iters x blocks x 256 floating-point operations, on `stream`
 * (cudaStream_t or NULL).  Timed by the caller, it gives the measured peak
 * of the pipe that bounds the face-flux kernels.  out: device array of at
 * least blocks x 256 elements of that precision (each thread writes the sum
 * of its chains); MPMC_INVALID_ARG if it is smaller or an argument is not
 * positive. */
int mpmc_fma_probe(int fp64, int blocks, int iters, void* out, size_t out_elems, void* stream);

/* Text of the last error on this context (static storage of the context). */
const char* mpmc_last_error(const mpmc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
