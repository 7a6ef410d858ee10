// C ABI of the MPMC hot path (declared in include/mpmc.h): context,
// scratch, stage sequencing of Eq. SSPRK3, CUDA-graph replay of steps.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mpmc.h"
#include "mpmc_device.cuh"
#include "mpmc_params.h"
#include "mpmc_ops.h"

using namespace mpmc;

static constexpr int NFAM_MAX = 6;

struct mpmc_ctx {
  KParams P;
  Ops ops;
  AdjOps aops;
  int precision;
  cudaStream_t stream;
  cudaStream_t cap;  // internal stream used only to capture graphs
  int device;
  double* Wc = nullptr;
  double* F[3] = {nullptr, nullptr, nullptr};
  long long nface[3] = {0, 0, 0};
  long long nface_total = 0;
  double* U1 = nullptr;
  double* U2 = nullptr;
  double* Ud = nullptr;   // device state of the host-buffer entry
  // ghost buffers [nv][gstride]: column 0 the inflow (far-field) state,
  // then the characteristic ghosts; Uin for U^n (KParams.gn), Gk for the
  // stage states (Gk == Uin without characteristic boundaries)
  double* Uin = nullptr;
  double* Gk = nullptr;
  double* scal = nullptr; // [dt, Gamma]
  unsigned long long* red = nullptr;
  int* status = nullptr;
  unsigned long long* stats = nullptr;
  int* counter = nullptr;
  // adjoint scratch (allocated on first use): per-face slot buffer of one
  // direction, cache adjoint, U adjoint, two stage adjoints, an internal
  // tape of one step
  double* Cslots = nullptr;
  double* gW = nullptr;
  double* gU = nullptr;
  double* lamA = nullptr;
  double* lamB = nullptr;
  uint32_t* tape_int = nullptr;
  float* unf = nullptr;   // mixed precision: FP32 copy of U^n
  // graph of one SSP-RK3 step for step_n
  cudaGraphExec_t gexec = nullptr;
  const double* g_U = nullptr;
  double* g_hist = nullptr;
  unsigned long long faces_done = 0;
  // optional kernel timing
  bool profiling = false;
  bool capturing = false;
  struct Mark {
    int fam;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
  double prof_ms[NFAM_MAX] = {};
  unsigned long long prof_n[NFAM_MAX] = {};
  char err[256];
};

enum { FAM_PRIM = 0, FAM_FACE = 1, FAM_UPDATE = 2, FAM_DT = 3, FAM_ADJ_FACE = 4, FAM_ADJ_PRIM = 5, NFAM = 6 };

static cudaEvent_t take_event(mpmc_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// brackets one launch of family `fam` with events on stream s
struct ProfScope {
  mpmc_ctx* c;
  int fam;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(mpmc_ctx* c_, int fam_, cudaStream_t s_) : c(c_), fam(fam_), s(s_) {
    if (c->profiling && !c->capturing) {
      a = take_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, s);
      c->marks.push_back({fam, a, b});
    }
  }
};

namespace mpmc {
// the run clock and end time of a step_n call (scal[2], scal[3]), set in
// stream order from kernel arguments: a host copy from pageable memory
// would block the caller until the work queued before it had finished
__global__ void k_set_run_time(double* scal, double t_end) {
  scal[2] = 0.0;
  scal[3] = t_end;
}

__global__ void k_dt(const KParams P, unsigned long long* red, double* scal, double dt_fixed, double gamma_fixed,
                     double* dt_hist, int* counter) {
  const double smax = __longlong_as_double((long long)red[0]);
  const double gmax = __longlong_as_double((long long)red[1]);
  double dt = dt_fixed > 0.0 ? dt_fixed : P.cfl / smax;
  const double G = gamma_fixed >= 0.0 ? gamma_fixed : (P.cdi_gamma > 0.0 ? P.cdi_gamma : gmax);
  // scal[2]: elapsed time of the run; scal[3] > 0: its end time, the last
  // step clipped to it and any later step of zero length
  if (scal[3] > 0.0) dt = fmin(dt, fmax(scal[3] - scal[2], 0.0));
  scal[2] += dt;
  scal[0] = dt;
  scal[1] = G;
  red[0] = 0ull;
  red[1] = 0ull;
  if (dt_hist) {
    dt_hist[*counter] = dt;
    *counter += 1;
  }
}
}  // namespace mpmc

static int fail(mpmc_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

static int check_launch(mpmc_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, MPMC_CUDA_ERROR, "%s: %s", where, cudaGetErrorString(e));
  return MPMC_OK;
}

static void free_all(mpmc_ctx* c) {
  // g_U and g_hist are caller-owned and never freed here
  void* ptrs[] = {c->Wc,   c->F[0],  c->F[1],    c->F[2],   c->U1,   c->U2,   c->Ud,   c->Uin,
                  c->scal, c->red,   c->status,  c->stats,  c->counter, c->gW, c->lamA, c->lamB,
                  c->tape_int, c->Cslots, c->gU, c->unf, c->Gk != c->Uin ? c->Gk : nullptr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (auto& m : c->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  c->marks.clear();
  c->pool.clear();
}

static int alloc(mpmc_ctx* c, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes < 16 ? 16 : bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, MPMC_OUT_OF_MEMORY, "cudaMalloc of %zu bytes failed", bytes);
  }
  return MPMC_OK;
}

extern "C" int mpmc_create(const mpmc_grid* g, const mpmc_eos* eos, const mpmc_model* m, void* stream,
                           mpmc_ctx** out) {
  if (!out) return MPMC_INVALID_ARG;
  *out = nullptr;
  KParams P0;
  const int prc = build_params(g, eos, m, P0);
  if (prc) return prc;
  mpmc_ctx* c = new (std::nothrow) mpmc_ctx();
  if (!c) return MPMC_OUT_OF_MEMORY;
  c->err[0] = 0;
  c->P = P0;
  KParams& P = c->P;
  const int ns = P.ns, D = P.dim;
  c->precision = m->precision;

  const bool mixed = m->precision == MPMC_MIXED;
  switch (D) {
    case 1: c->ops = mixed ? ops_mixed_d1(ns) : ops_fp64_d1(ns); break;
    case 2: c->ops = mixed ? ops_mixed_d2(ns) : ops_fp64_d2(ns); break;
    default: c->ops = mixed ? ops_mixed_d3(ns) : ops_fp64_d3(ns); break;
  }
  switch (D) {
    case 1: c->aops = adj_ops_d1(ns); break;
    case 2: c->aops = adj_ops_d2(ns); break;
    default: c->aops = adj_ops_d3(ns); break;
  }
  if (P.recon == MPMC_RECON_WENO5JS) {
    c->ops.face = mixed ? face_mixed_weno5js(D, ns) : face_fp64_weno5js(D, ns);
    c->aops.face = adj_face_weno5js(D, ns);
  } else if (P.recon == MPMC_RECON_TENO5) {
    c->ops.face = mixed ? face_mixed_teno5(D, ns) : face_fp64_teno5(D, ns);
    c->aops.face = adj_face_teno5(D, ns);
  } else if (P.recon == MPMC_RECON_TENO6) {
    c->ops.face = mixed ? face_mixed_teno6(D, ns) : face_fp64_teno6(D, ns);
    c->aops.face = adj_face_teno6(D, ns);
  }
  if (!c->ops.face || !c->aops.face) {
    delete c;
    return MPMC_INVALID_ARG;
  }
  cudaGetDevice(&c->device);
  c->stream = (cudaStream_t)stream;
  int rc = MPMC_OK;
  const size_t st_bytes = (size_t)P.nv * P.ncell * sizeof(double);
  rc = rc ? rc : alloc(c, (void**)&c->Wc, (size_t)P.nW * P.wstride * sizeof(double));
  for (int d = 0; d < D && !rc; ++d) {
    long long nf = 1;
    for (int e = 0; e < 3; ++e) nf *= (long long)(P.n[e] + (e == d));
    c->nface[d] = nf;
    c->nface_total += nf;
    rc = alloc(c, (void**)&c->F[d], (size_t)P.nv * nf * sizeof(double));
  }
  if (!rc && mixed) {
    // FP32 copy of U^n for the mixed path's limiter (read by its face kernel)
    rc = alloc(c, (void**)&c->unf, (size_t)P.nv * P.wstride * sizeof(float));
    P.unf = c->unf;
  }
  rc = rc ? rc : alloc(c, (void**)&c->U1, st_bytes);
  rc = rc ? rc : alloc(c, (void**)&c->U2, st_bytes);
  const size_t gbytes = (size_t)P.nv * P.gstride * sizeof(double);
  rc = rc ? rc : alloc(c, (void**)&c->Uin, gbytes < 32 * sizeof(double) ? 32 * sizeof(double) : gbytes);
  if (!rc && P.nslots) rc = alloc(c, (void**)&c->Gk, gbytes);
  if (!rc && !P.nslots) c->Gk = c->Uin;
  P.gn = c->Uin;
  rc = rc ? rc : alloc(c, (void**)&c->scal, 8 * sizeof(double));
  rc = rc ? rc : alloc(c, (void**)&c->red, 4 * sizeof(unsigned long long));
  rc = rc ? rc : alloc(c, (void**)&c->status, 4 * sizeof(int));
  rc = rc ? rc : alloc(c, (void**)&c->stats, 8 * sizeof(unsigned long long));
  rc = rc ? rc : alloc(c, (void**)&c->counter, 4 * sizeof(int));
  if (!rc && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
    rc = fail(c, MPMC_CUDA_ERROR, "stream creation failed");
  if (rc) {
    free_all(c);
    delete c;
    return rc;
  }
  cudaMemsetAsync(c->red, 0, 4 * sizeof(unsigned long long), c->stream);
  cudaMemsetAsync(c->status, 0, 4 * sizeof(int), c->stream);
  cudaMemsetAsync(c->stats, 0, 8 * sizeof(unsigned long long), c->stream);
  cudaMemsetAsync(c->scal, 0, 8 * sizeof(double), c->stream);
  cudaMemsetAsync(c->Uin, 0, gbytes < 32 * sizeof(double) ? 32 * sizeof(double) : gbytes, c->stream);
  if (c->Gk != c->Uin) cudaMemsetAsync(c->Gk, 0, gbytes, c->stream);
  if (P.has_inflow) {
    // inflow state: primitive -> conserved on the device (1 cell), then into
    // column 0 of each ghost buffer
    double* tmp = nullptr;
    rc = alloc(c, (void**)&tmp, 64 * sizeof(double));
    if (!rc) {
      double w[32] = {0};
      for (int v = 0; v < ns + D + 2; ++v) w[v] = g->inflow[v];
      cudaMemcpy(tmp, w, sizeof(w), cudaMemcpyHostToDevice);
      c->ops.init(P, c->stream, tmp, tmp + 32, 1);
      for (int v = 0; v < P.nv; ++v) {
        cudaMemcpyAsync(c->Uin + (size_t)v * P.gstride, tmp + 32 + v, sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream);
        if (c->Gk != c->Uin)
          cudaMemcpyAsync(c->Gk + (size_t)v * P.gstride, tmp + 32 + v, sizeof(double), cudaMemcpyDeviceToDevice,
                          c->stream);
      }
      cudaStreamSynchronize(c->stream);
      cudaFree(tmp);
    }
  }
  if (!rc) rc = check_launch(c, "create");
  if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = fail(c, MPMC_CUDA_ERROR, "create sync");
  if (rc) {
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return MPMC_OK;
}

extern "C" void mpmc_destroy(mpmc_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

extern "C" int mpmc_set_stream(mpmc_ctx* c, void* stream) {
  if (!c) return MPMC_INVALID_ARG;
  c->stream = (cudaStream_t)stream;
  return MPMC_OK;
}

extern "C" int mpmc_nvars(const mpmc_ctx* c) { return c ? c->P.nv : 0; }
extern "C" size_t mpmc_ncells(const mpmc_ctx* c) { return c ? (size_t)c->P.ncell : 0; }
extern "C" size_t mpmc_cache_doubles(const mpmc_ctx* c) { return c ? (size_t)c->P.nW * c->P.wstride : 0; }
extern "C" const char* mpmc_last_error(const mpmc_ctx* c) { return c ? c->err : "null context"; }

extern "C" int mpmc_init_state(mpmc_ctx* c, const double* prim, double* U) {
  if (!c || !prim || !U) return fail(c, MPMC_INVALID_ARG, "init_state: null argument");
  c->ops.init(c->P, c->stream, prim, U, c->P.ncell);
  return check_launch(c, "init_state");
}

// ---------------------------------------------------------------------------
// one stage: faces of every direction from the primitive cache of Uk, then
// the fused divergence / RK combination
static void stage(mpmc_ctx* c, cudaStream_t s, const double* Un, const double* Uk, double rk0, double rk1, double rk2,
                  double* Uout, double* dUdt, uint32_t* flags) {
  const KParams& P = c->P;
  long long off = 0;
  const double* Gk = Uk == Un ? c->Uin : c->Gk;   // the ghost buffer of U^(k)
  for (int d = 0; d < P.dim; ++d) {
    ProfScope ps(c, FAM_FACE, s);
    c->ops.face(P, s, d, c->Wc, Un, Uk, Gk, c->scal, rk0, rk1, rk2, c->F[d], flags ? flags + off : nullptr,
                c->stats);
    off += c->nface[d];
  }
  ProfScope ps(c, FAM_UPDATE, s);
  c->ops.update(P, s, Un, Uk, c->F, c->scal, rk0, rk1, rk2, Uout, dUdt, c->status);
}

// primitive cache of U; the pass that computes dt and Gamma (red != null)
// is the one of U^n, every other one of a stage state: each first fills its
// ghost buffer's characteristic ghosts
static void prim(mpmc_ctx* c, cudaStream_t s, const double* U, unsigned long long* red) {
  ProfScope ps(c, FAM_PRIM, s);
  double* G = red ? c->Uin : c->Gk;
  if (c->P.nslots) c->ops.ghost(c->P, s, U, G);
  c->ops.prim(c->P, s, U, G, c->Wc, red, c->status);
}

// dt and Gamma from U (prim pass with the block maxima), then k_dt
static void dt_gamma(mpmc_ctx* c, cudaStream_t s, const double* U, double dt_fixed, double gamma_fixed,
                     double* hist) {
  prim(c, s, U, c->red);
  ProfScope ps(c, FAM_DT, s);
  k_dt<<<1, 1, 0, s>>>(c->P, c->red, c->scal, dt_fixed, gamma_fixed, hist, c->counter);
}

// Eq. SSPRK3 with U^n = U, result written back to U
static void rk3(mpmc_ctx* c, cudaStream_t s, double* U, double dt, uint32_t* tape, double* hist) {
  dt_gamma(c, s, U, dt, -1.0, hist);
  const long long nf = c->nface_total;
  stage(c, s, U, U, 1.0, 0.0, 1.0, c->U1, nullptr, tape);
  prim(c, s, c->U1, nullptr);
  stage(c, s, U, c->U1, 0.75, 0.25, 0.25, c->U2, nullptr, tape ? tape + nf : nullptr);
  prim(c, s, c->U2, nullptr);
  stage(c, s, U, c->U2, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, U, nullptr, tape ? tape + 2 * nf : nullptr);
}

extern "C" int mpmc_rhs(mpmc_ctx* c, const double* U, double* dUdt, const mpmc_stage* st, uint32_t* flags) {
  if (!c || !U || !dUdt) return fail(c, MPMC_INVALID_ARG, "rhs: null argument");
  const double* Un = st && st->U_n ? st->U_n : U;
  const double rk0 = st ? st->rk0 : 1.0, rk1 = st ? st->rk1 : 0.0, rk2 = st ? st->rk2 : 1.0;
  const double dt = st ? st->dt : 0.0, G = st ? st->Gamma : -1.0;
  cudaStream_t s = c->stream;
  // dt / Gamma from U^n (always run so that the prim pass of U_n also
  // validates it); then the primitive cache of U
  dt_gamma(c, s, Un, dt, G, nullptr);
  if (Un != U) prim(c, s, U, nullptr);
  stage(c, s, Un, U, rk0, rk1, rk2, nullptr, dUdt, flags);
  c->faces_done += c->nface_total;
  return check_launch(c, "rhs");
}

extern "C" int mpmc_rk_step(mpmc_ctx* c, double* U, double dt, uint32_t* tape) {
  if (!c || !U) return fail(c, MPMC_INVALID_ARG, "rk_step: null argument");
  rk3(c, c->stream, U, dt, tape, nullptr);
  c->faces_done += 3ull * c->nface_total;
  return check_launch(c, "rk_step");
}

extern "C" int mpmc_step_n(mpmc_ctx* c, double* U, int n, double t_end, double* dt_out) {
  if (!c || !U || n < 0) return fail(c, MPMC_INVALID_ARG, "step_n: bad argument");
  if (n == 0) return MPMC_OK;
  cudaStream_t s = c->stream;
  // run clock and end time (scal[2], scal[3]) for the steps of this call
  k_set_run_time<<<1, 1, 0, s>>>(c->scal, t_end > 0.0 ? t_end : 0.0);
  if (!c->gexec || c->g_U != U || c->g_hist != dt_out) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fail(c, MPMC_CUDA_ERROR, "step_n: capture begin failed");
    c->capturing = true;
    rk3(c, c->cap, U, 0.0, nullptr, dt_out);
    c->capturing = false;
    if (cudaStreamEndCapture(c->cap, &graph) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, MPMC_CUDA_ERROR, "step_n: capture failed");
    }
    cudaError_t e = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->gexec = nullptr;
      return fail(c, MPMC_CUDA_ERROR, "step_n: instantiate: %s", cudaGetErrorString(e));
    }
    c->g_U = U;
    c->g_hist = dt_out;
  }
  if (dt_out) cudaMemsetAsync(c->counter, 0, sizeof(int), s);
  for (int i = 0; i < n; ++i) {
    cudaError_t e = cudaGraphLaunch(c->gexec, s);
    if (e != cudaSuccess) return fail(c, MPMC_CUDA_ERROR, "step_n: graph launch: %s", cudaGetErrorString(e));
  }
  c->faces_done += 3ull * c->nface_total * (unsigned long long)n;
  // later single steps are not clipped
  k_set_run_time<<<1, 1, 0, s>>>(c->scal, 0.0);
  return check_launch(c, "step_n");
}

extern "C" int mpmc_step_n_host(mpmc_ctx* c, double* U_host, int n) {
  if (!c || !U_host || n < 0) return fail(c, MPMC_INVALID_ARG, "step_n_host: bad argument");
  const size_t bytes = (size_t)c->P.nv * c->P.ncell * sizeof(double);
  if (!c->Ud) {
    int rc = alloc(c, (void**)&c->Ud, bytes);
    if (rc) return rc;
  }
  cudaStream_t s = c->stream;
  if (cudaMemcpyAsync(c->Ud, U_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(c, MPMC_CUDA_ERROR, "step_n_host: copy in");
  int rc = mpmc_step_n(c, c->Ud, n, 0.0, nullptr);
  if (rc) return rc;
  if (cudaMemcpyAsync(U_host, c->Ud, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return fail(c, MPMC_CUDA_ERROR, "step_n_host: copy out");
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(c, MPMC_CUDA_ERROR, "step_n_host: sync");
  return MPMC_OK;
}

extern "C" int mpmc_dt_gamma(mpmc_ctx* c, const double* U, double* out_dev) {
  if (!c || !U || !out_dev) return fail(c, MPMC_INVALID_ARG, "dt_gamma: null argument");
  dt_gamma(c, c->stream, U, 0.0, -1.0, nullptr);
  cudaMemcpyAsync(out_dev, c->scal, 2 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  return check_launch(c, "dt_gamma");
}

// ---------------------------------------------------------------------------
// discrete adjoint (FP64 contexts)
static int ensure_adjoint(mpmc_ctx* c) {
  if (c->precision != MPMC_FP64) return fail(c, MPMC_INVALID_ARG, "adjoint: needs an FP64 context");
  if (c->P.nslots) return fail(c, MPMC_INVALID_ARG, "adjoint: characteristic boundaries are not differentiated");
  const KParams& P = c->P;
  int rc = MPMC_OK;
  const size_t st_bytes = (size_t)P.nv * P.ncell * sizeof(double);
  long long nfmax = 0;
  for (int d = 0; d < P.dim; ++d) nfmax = c->nface[d] > nfmax ? c->nface[d] : nfmax;
  if (!c->Cslots) rc = alloc(c, (void**)&c->Cslots, (size_t)c->aops.slots(P) * nfmax * sizeof(double));
  if (!rc && !c->gW) rc = alloc(c, (void**)&c->gW, (size_t)P.nW * P.wstride * sizeof(double));
  if (!rc && !c->gU) rc = alloc(c, (void**)&c->gU, st_bytes);
  if (!rc && !c->lamA) rc = alloc(c, (void**)&c->lamA, st_bytes);
  if (!rc && !c->lamB) rc = alloc(c, (void**)&c->lamB, st_bytes);
  if (!rc && !c->tape_int) rc = alloc(c, (void**)&c->tape_int, 3 * (size_t)c->nface_total * sizeof(uint32_t));
  return rc;
}

// face fluxes of one stage for their flags only (no divergence / update)
static void faces_only(mpmc_ctx* c, cudaStream_t s, const double* Un, const double* Uk, double rk0, double rk1,
                       double rk2, uint32_t* flags) {
  long long off = 0;
  const double* Gk = Uk == Un ? c->Uin : c->Gk;
  for (int d = 0; d < c->P.dim; ++d) {
    ProfScope ps(c, FAM_FACE, s);
    c->ops.face(c->P, s, d, c->Wc, Un, Uk, Gk, c->scal, rk0, rk1, rk2, c->F[d], flags + off, nullptr);
    off += c->nface[d];
  }
}

// out = a x + b y + cz z + coef (dt) (dL/dU)^T lamL at U (whose primitive
// cache is in Wc): per direction the faces' slots, their gather, then the
// per-cell primitive-recovery reverse fused with the combination
static void stage_vjp(mpmc_ctx* c, cudaStream_t s, const double* U, const double* Wc, const uint32_t* tape,
                      const double* lamL, double coef, int mul_dt, double* out, double a, const double* x, double b,
                      const double* y, double cz, const double* z) {
  const KParams& P = c->P;
  long long off = 0;
  for (int d = 0; d < P.dim; ++d) {
    {
      ProfScope ps(c, FAM_ADJ_FACE, s);
      c->aops.face(P, s, d, Wc, U, c->Uin, c->scal, tape + off, lamL, coef, mul_dt, c->Cslots);
      if (P.viscous) c->aops.face_visc(P, s, d, Wc, c->scal, tape + off, lamL, coef, mul_dt, c->Cslots);
    }
    ProfScope ps(c, FAM_ADJ_PRIM, s);
    c->aops.gather(P, s, d, c->Cslots, d == 0, c->gW, c->gU);
    off += c->nface[d];
  }
  ProfScope ps(c, FAM_ADJ_PRIM, s);
  c->aops.cell(P, s, U, Wc, c->gW, c->gU, out, a, x, b, y, cz, z);
}

extern "C" int mpmc_rhs_adjoint(mpmc_ctx* c, const double* U, const mpmc_stage* st, const uint32_t* tape,
                                const double* lam_dUdt, double* lam_U) {
  if (!c || !U || !lam_dUdt || !lam_U) return fail(c, MPMC_INVALID_ARG, "rhs_adjoint: null argument");
  int rc = ensure_adjoint(c);
  if (rc) return rc;
  const double* Un = st && st->U_n ? st->U_n : U;
  const double rk0 = st ? st->rk0 : 1.0, rk1 = st ? st->rk1 : 0.0, rk2 = st ? st->rk2 : 1.0;
  const double dt = st ? st->dt : 0.0, G = st ? st->Gamma : -1.0;
  cudaStream_t s = c->stream;
  // the same dt / Gamma and primitive cache as mpmc_rhs
  dt_gamma(c, s, Un, dt, G, nullptr);
  if (Un != U) prim(c, s, U, nullptr);
  if (!tape) {
    faces_only(c, s, Un, U, rk0, rk1, rk2, c->tape_int);
    tape = c->tape_int;
  }
  stage_vjp(c, s, U, (const double*)c->Wc, tape, lam_dUdt, 1.0, 0, lam_U, 1.0, lam_U, 0.0, nullptr, 0.0, nullptr);
  return check_launch(c, "rhs_adjoint");
}

extern "C" int mpmc_rk_step_record(mpmc_ctx* c, double* U, double dt, uint32_t* tape, double* U_stages,
                                   double* W_stages) {
  if (!c || !U || !U_stages) return fail(c, MPMC_INVALID_ARG, "rk_step_record: null argument");
  if (W_stages && c->precision != MPMC_FP64)
    return fail(c, MPMC_INVALID_ARG, "rk_step_record: W_stages needs an FP64 context");
  const KParams& P = c->P;
  const long long n = (long long)P.nv * P.ncell, nf = c->nface_total;
  const size_t nw = mpmc_cache_doubles(c);
  double* U1 = U_stages;
  double* U2 = U_stages + n;
  cudaStream_t s = c->stream;
  // the primitive cache just computed, kept as stage k's
  auto keep = [&](int k) {
    return !W_stages || cudaMemcpyAsync(W_stages + k * nw, c->Wc, nw * sizeof(double), cudaMemcpyDeviceToDevice,
                                        s) == cudaSuccess;
  };
  dt_gamma(c, s, U, dt, -1.0, nullptr);
  if (!keep(0)) return fail(c, MPMC_CUDA_ERROR, "rk_step_record: cache copy");
  stage(c, s, U, U, 1.0, 0.0, 1.0, U1, nullptr, tape);
  prim(c, s, U1, nullptr);
  if (!keep(1)) return fail(c, MPMC_CUDA_ERROR, "rk_step_record: cache copy");
  stage(c, s, U, U1, 0.75, 0.25, 0.25, U2, nullptr, tape ? tape + nf : nullptr);
  prim(c, s, U2, nullptr);
  if (!keep(2)) return fail(c, MPMC_CUDA_ERROR, "rk_step_record: cache copy");
  stage(c, s, U, U2, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, U, nullptr, tape ? tape + 2 * nf : nullptr);
  c->faces_done += 3ull * c->nface_total;
  return check_launch(c, "rk_step_record");
}

extern "C" int mpmc_rk_step_adjoint(mpmc_ctx* c, const double* U_n, const double* U_stages, const double* W_stages,
                                    double dt, const uint32_t* tape, const double* lam_next, double* lam_n) {
  if (!c || !U_n || !lam_next || !lam_n) return fail(c, MPMC_INVALID_ARG, "rk_step_adjoint: null argument");
  if (W_stages && !U_stages) return fail(c, MPMC_INVALID_ARG, "rk_step_adjoint: W_stages without U_stages");
  int rc = ensure_adjoint(c);
  if (rc) return rc;
  const KParams& P = c->P;
  const long long nf = c->nface_total, n = (long long)P.nv * P.ncell;
  cudaStream_t s = c->stream;
  dt_gamma(c, s, U_n, dt, -1.0, nullptr);
  const double* U1 = U_stages ? U_stages : c->U1;
  const double* U2 = U_stages ? U_stages + n : c->U2;
  uint32_t* tp = tape ? nullptr : c->tape_int;
  if (!U_stages) {
    // forward recomputation of the stage states (and of the flags if no tape)
    stage(c, s, U_n, U_n, 1.0, 0.0, 1.0, c->U1, nullptr, tp);
    prim(c, s, c->U1, nullptr);
    stage(c, s, U_n, c->U1, 0.75, 0.25, 0.25, c->U2, nullptr, tp ? tp + nf : nullptr);
    prim(c, s, c->U2, nullptr);
    if (tp) faces_only(c, s, U_n, c->U2, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, tp + 2 * nf);
  } else if (tp) {
    // stage states given, flags recomputed
    faces_only(c, s, U_n, U_n, 1.0, 0.0, 1.0, tp);
    prim(c, s, U1, nullptr);
    faces_only(c, s, U_n, U1, 0.75, 0.25, 0.25, tp + nf);
    prim(c, s, U2, nullptr);
    faces_only(c, s, U_n, U2, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, tp + 2 * nf);
  } else if (!W_stages) {
    prim(c, s, U2, nullptr);
  }
  const uint32_t* T = tape ? tape : c->tape_int;
  // the primitive cache of each stage state: kept by mpmc_rk_step_record, or
  // recomputed into the context's cache just before its use
  const size_t nw = mpmc_cache_doubles(c);
  const double* Wc = c->Wc;
  // Eq. SSPRK3 reversed:
  //   lam2 = 2/3 lam3 + 2/3 dt L(U2)^T lam3
  //   lam1 = 1/4 lam2 + 1/4 dt L(U1)^T lam2
  //   lamn = 1/3 lam3 + 3/4 lam2 + lam1 + dt L(Un)^T lam1
  double* l2 = c->lamB;
  double* l1 = c->lamA;
  stage_vjp(c, s, U2, W_stages ? W_stages + 2 * nw : Wc, T + 2 * nf, lam_next, 2.0 / 3.0, 1, l2, 2.0 / 3.0,
            lam_next, 0.0, nullptr, 0.0, nullptr);
  if (!W_stages) prim(c, s, U1, nullptr);
  stage_vjp(c, s, U1, W_stages ? W_stages + nw : Wc, T + nf, l2, 0.25, 1, l1, 0.25, l2, 0.0, nullptr, 0.0,
            nullptr);
  if (!W_stages) prim(c, s, U_n, nullptr);
  stage_vjp(c, s, U_n, W_stages ? W_stages : Wc, T, l1, 1.0, 1, lam_n, 1.0 / 3.0, lam_next, 0.75, l2, 1.0, l1);
  return check_launch(c, "rk_step_adjoint");
}

extern "C" int mpmc_init_state_adjoint(mpmc_ctx* c, const double* prim_in, const double* lam_U, double* lam_prim) {
  if (!c || !prim_in || !lam_U || !lam_prim) return fail(c, MPMC_INVALID_ARG, "init_state_adjoint: null argument");
  c->aops.init(c->P, c->stream, prim_in, lam_U, lam_prim, c->P.ncell);
  return check_launch(c, "init_state_adjoint");
}

static int nprim_fields(const KParams& P) { return 4 + P.ns + P.dim; }

extern "C" int mpmc_primitives(mpmc_ctx* c, const double* U, double* out) {
  if (!c || !U || !out) return fail(c, MPMC_INVALID_ARG, "primitives: null argument");
  if (c->precision != MPMC_FP64) return fail(c, MPMC_INVALID_ARG, "primitives: needs an FP64 context");
  const KParams& P = c->P;
  prim(c, c->stream, U, nullptr);
  if (cudaMemcpy2DAsync(out, (size_t)P.ncell * sizeof(double), c->Wc, (size_t)P.wstride * sizeof(double),
                        (size_t)P.ncell * sizeof(double), (size_t)nprim_fields(P), cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess)
    return fail(c, MPMC_CUDA_ERROR, "primitives: copy");
  return check_launch(c, "primitives");
}

extern "C" int mpmc_primitives_adjoint(mpmc_ctx* c, const double* U, const double* lam_W, double* lam_U) {
  if (!c || !U || !lam_W || !lam_U) return fail(c, MPMC_INVALID_ARG, "primitives_adjoint: null argument");
  int rc = ensure_adjoint(c);
  if (rc) return rc;
  const KParams& P = c->P;
  cudaStream_t s = c->stream;
  cudaMemsetAsync(c->gW, 0, (size_t)P.nW * P.wstride * sizeof(double), s);
  cudaMemsetAsync(c->gU, 0, (size_t)P.nv * P.ncell * sizeof(double), s);
  if (cudaMemcpy2DAsync(c->gW, (size_t)P.wstride * sizeof(double), lam_W, (size_t)P.ncell * sizeof(double),
                        (size_t)P.ncell * sizeof(double), (size_t)nprim_fields(P), cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
    return fail(c, MPMC_CUDA_ERROR, "primitives_adjoint: copy");
  ProfScope ps(c, FAM_ADJ_PRIM, s);
  c->aops.cell(P, s, U, nullptr, c->gW, c->gU, lam_U, 1.0, lam_U, 0.0, nullptr, 0.0, nullptr);
  return check_launch(c, "primitives_adjoint");
}

extern "C" int mpmc_get_status(mpmc_ctx* c, int reset) {
  if (!c) return MPMC_INVALID_ARG;
  int st = 0;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, MPMC_CUDA_ERROR, "get_status: sync");
  cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (reset) cudaMemset(c->status, 0, sizeof(int));
  return st;
}

extern "C" int mpmc_get_stats(mpmc_ctx* c, mpmc_stats* out, int reset) {
  if (!c || !out) return MPMC_INVALID_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, MPMC_CUDA_ERROR, "get_stats: sync");
  unsigned long long s[8];
  cudaMemcpy(s, c->stats, sizeof(s), cudaMemcpyDeviceToHost);
  out->faces = c->faces_done;
  out->hllc_fallback = s[1];
  out->cdi_dropped = s[2];
  out->theta_p = s[3];
  out->theta_t = s[4];
  out->ylim = s[5];
  out->diff_dropped = s[6];
  if (reset) {
    cudaMemset(c->stats, 0, sizeof(s));
    c->faces_done = 0;
  }
  return MPMC_OK;
}

extern "C" int mpmc_set_profiling(mpmc_ctx* c, int enable) {
  if (!c) return MPMC_INVALID_ARG;
  c->profiling = enable != 0;
  return MPMC_OK;
}

extern "C" int mpmc_get_profile(mpmc_ctx* c, double* ms, uint64_t* launches, int reset) {
  if (!c) return MPMC_INVALID_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, MPMC_CUDA_ERROR, "get_profile: sync");
  for (auto& m : c->marks) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) {
      c->prof_ms[m.fam] += t;
      c->prof_n[m.fam] += 1;
    }
    c->pool.push_back(m.a);
    c->pool.push_back(m.b);
  }
  c->marks.clear();
  for (int f = 0; f < NFAM; ++f) {
    if (ms) ms[f] = c->prof_ms[f];
    if (launches) launches[f] = c->prof_n[f];
    if (reset) {
      c->prof_ms[f] = 0.0;
      c->prof_n[f] = 0;
    }
  }
  return MPMC_OK;
}
