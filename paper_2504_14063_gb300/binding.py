"""Thin ctypes binding of libmpmc.so (include/mpmc.h).

Argument marshalling only: torch CUDA tensors are passed by data pointer and
every step of the path runs in the library's kernels.  If the library is
missing the import of this module raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import workloads as _wl

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpmc.so")
MAXS = 4

OK, INVALID_ARG, CUDA_ERROR, INADMISSIBLE, EOS_NO_CONVERGE, OUT_OF_MEMORY = 0, 1, 2, 3, 4, 5
FP64, MIXED = 0, 1
F_THETA_T_L, F_THETA_T_R, F_THETA_P_L, F_THETA_P_R = 1, 2, 4, 8
F_HLLC_FALLBACK, F_CDI_DROPPED, F_YLIM_L, F_YLIM_R, F_DIFF_DROPPED = 16, 32, 64, 128, 256


class MpmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mpmc error {code}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double),
                ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3),
                ("inflow", ctypes.c_double * (MAXS + 5))]


class Eos(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int), ("phase", ctypes.c_int * MAXS)] + [
        (f, ctypes.c_double * MAXS) for f in ("cv", "gamma", "q", "b", "pinf", "W", "mu", "Sc")]


class ModelC(ctypes.Structure):
    _fields_ = [("weno_eps", ctypes.c_double), ("cdi", ctypes.c_int), ("diffusion", ctypes.c_int),
                ("pos_limiter", ctypes.c_int), ("cdi_eps", ctypes.c_double), ("cdi_gamma", ctypes.c_double),
                ("phi_min", ctypes.c_double), ("psi_delta", ctypes.c_double), ("cfl", ctypes.c_double),
                ("mu_liquid", ctypes.c_double), ("precision", ctypes.c_int), ("recon", ctypes.c_int),
                ("viscous", ctypes.c_int), ("prandtl", ctypes.c_double), ("lambda_liquid", ctypes.c_double)]


class StageC(ctypes.Structure):
    _fields_ = [("U_n", ctypes.c_void_p), ("rk0", ctypes.c_double), ("rk1", ctypes.c_double),
                ("rk2", ctypes.c_double), ("dt", ctypes.c_double), ("Gamma", ctypes.c_double)]


class StatsC(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("faces", "hllc_fallback", "cdi_dropped", "theta_p", "theta_t", "ylim",
                                                     "diff_dropped")]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmpmc.so not found at {LIB_PATH}: build it with paper_2504_14063_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "mpmc_create": (i, [ctypes.POINTER(Grid), ctypes.POINTER(Eos), ctypes.POINTER(ModelC), vp,
                            ctypes.POINTER(vp)]),
        "mpmc_destroy": (None, [vp]),
        "mpmc_set_stream": (i, [vp, vp]),
        "mpmc_nvars": (i, [vp]),
        "mpmc_ncells": (ctypes.c_size_t, [vp]),
        "mpmc_cache_doubles": (ctypes.c_size_t, [vp]),
        "mpmc_init_state": (i, [vp, vp, vp]),
        "mpmc_rhs": (i, [vp, vp, vp, ctypes.POINTER(StageC), vp]),
        "mpmc_rk_step": (i, [vp, vp, d, vp]),
        "mpmc_step_n": (i, [vp, vp, i, d, vp]),
        "mpmc_step_n_host": (i, [vp, vp, i]),
        "mpmc_dt_gamma": (i, [vp, vp, vp]),
        "mpmc_rhs_adjoint": (i, [vp, vp, ctypes.POINTER(StageC), vp, vp, vp]),
        "mpmc_rk_step_record": (i, [vp, vp, d, vp, vp, vp]),
        "mpmc_rk_step_adjoint": (i, [vp, vp, vp, vp, d, vp, vp, vp]),
        "mpmc_init_state_adjoint": (i, [vp, vp, vp, vp]),
        "mpmc_primitives": (i, [vp, vp, vp]),
        "mpmc_primitives_adjoint": (i, [vp, vp, vp, vp]),
        "mpmc_get_stats": (i, [vp, ctypes.POINTER(StatsC), i]),
        "mpmc_get_status": (i, [vp, i]),
        "mpmc_last_error": (ctypes.c_char_p, [vp]),
        "mpmc_set_profiling": (i, [vp, i]),
        "mpmc_get_profile": (i, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64), i]),
        "mpmc_fma_probe": (i, [i, i, i, vp, ctypes.c_size_t, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    assert t.is_cuda and t.is_contiguous(), "expects a contiguous CUDA tensor"
    return t.data_ptr()


def _dev(t):
    assert t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()
    return t.data_ptr()


def fma_probe(fp64, blocks, iters, out, stream=None):
    """One launch of mpmc_fma_probe on `stream` (torch's current stream if
    None); out: CUDA tensor of >= blocks x 256 elements of that precision.
    Returns the launch's floating-point operation count."""
    assert out.is_cuda and out.is_contiguous() and out.dtype == (torch.float64 if fp64 else torch.float32)
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = lib.mpmc_fma_probe(1 if fp64 else 0, int(blocks), int(iters), out.data_ptr(), out.numel(), s)
    if rc != OK:
        raise MpmcError(rc, "fma_probe")
    return 16 * int(iters) * int(blocks) * 256


def structs_from_problem(problem, precision=FP64):
    """Library structs from a workloads.Problem (same fields as the paper's
    species table and model coefficients)."""
    g = Grid()
    g.dim = problem.dim
    for d in range(3):
        g.n[d] = problem.n[d]
        g.bc_lo[d] = problem.bc_lo[d]
        g.bc_hi[d] = problem.bc_hi[d]
    g.dx = problem.dx
    if problem.inflow is not None:
        for q, v in enumerate(problem.inflow):
            g.inflow[q] = float(v)
    e = Eos()
    e.n_species = problem.ns
    for k, s in enumerate(problem.species):
        e.phase[k] = s.phase
        for f in ("cv", "gamma", "q", "b", "pinf", "W", "mu", "Sc"):
            getattr(e, f)[k] = getattr(s, f)
    m = ModelC()
    pm = problem.model
    for f in ("weno_eps", "cdi", "diffusion", "pos_limiter", "cdi_eps", "cdi_gamma", "phi_min", "psi_delta",
              "cfl", "mu_liquid", "recon", "viscous", "prandtl", "lambda_liquid"):
        setattr(m, f, getattr(pm, f))
    m.precision = precision
    return g, e, m


class Context:
    """One grid / species table / model on the current CUDA device."""

    def __init__(self, problem, precision=FP64, stream=None):
        self.problem = problem
        self.precision = precision
        g, e, m = structs_from_problem(problem, precision)
        self._structs = (g, e, m)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        h = ctypes.c_void_p()
        rc = lib.mpmc_create(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), ctypes.c_void_p(s.cuda_stream),
                             ctypes.byref(h))
        if rc != OK:
            raise MpmcError(rc, "mpmc_create failed")
        self.h = h
        self.nv = lib.mpmc_nvars(h)
        self.ncells = lib.mpmc_ncells(h)
        self.cache_doubles = lib.mpmc_cache_doubles(h)
        self.shape = (self.nv, problem.n[2], problem.n[1], problem.n[0])
        self.device = torch.device("cuda", torch.cuda.current_device())

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and lib is not None:
            lib.mpmc_destroy(h)
            self.h = None

    def _check(self, rc):
        if rc != OK:
            raise MpmcError(rc, lib.mpmc_last_error(self.h).decode())

    def nfaces(self, d):
        n = list(self.problem.n)
        n[d] += 1
        return n[0] * n[1] * n[2]

    @property
    def nfaces_total(self):
        return sum(self.nfaces(d) for d in range(self.problem.dim))

    def empty_state(self):
        return torch.empty(self.shape, dtype=torch.float64, device=self.device)

    # ---- the five entry points ---------------------------------------------
    def init_state(self, prim, U=None):
        prim = prim.to(self.device, torch.float64).contiguous() if torch.is_tensor(prim) else \
            torch.as_tensor(prim, dtype=torch.float64, device=self.device).contiguous()
        U = self.empty_state() if U is None else U
        self._check(lib.mpmc_init_state(self.h, _dev(prim), _dev(U)))
        return U

    def rhs(self, U, dUdt=None, stage=None, flags=None):
        """stage: None or dict(U_n=tensor, rk=(rk0, rk1, rk2), dt=float, Gamma=float)."""
        dUdt = torch.empty_like(U) if dUdt is None else dUdt
        sp = None
        if stage is not None:
            sc = StageC()
            sc.U_n = _dev(stage["U_n"]) if stage.get("U_n") is not None else None
            sc.rk0, sc.rk1, sc.rk2 = stage.get("rk", (1.0, 0.0, 1.0))
            sc.dt = stage.get("dt", 0.0)
            sc.Gamma = stage.get("Gamma", -1.0)
            sp = ctypes.byref(sc)
        self._check(lib.mpmc_rhs(self.h, _dev(U), _dev(dUdt), sp, _ptr(flags)))
        return dUdt

    def rk_step(self, U, dt=0.0, tape=None):
        self._check(lib.mpmc_rk_step(self.h, _dev(U), float(dt), _ptr(tape)))
        return U

    def step_n(self, U, n, dt_out=None, t_end=0.0):
        """n SSP-RK3 steps in place; t_end > 0 stops at that physical time
        (later steps have zero length); dt_out (n doubles, device) receives
        the step sizes."""
        self._check(lib.mpmc_step_n(self.h, _dev(U), int(n), float(t_end), _ptr(dt_out)))
        return U

    def step_n_host(self, U_host, n):
        """U_host: CPU float64 tensor (pinned for overlap), updated in place."""
        assert U_host.dtype == torch.float64 and not U_host.is_cuda and U_host.is_contiguous()
        self._check(lib.mpmc_step_n_host(self.h, U_host.data_ptr(), int(n)))
        return U_host

    def dt_gamma(self, U):
        out = torch.empty(2, dtype=torch.float64, device=self.device)
        self._check(lib.mpmc_dt_gamma(self.h, _dev(U), _dev(out)))
        return out

    @staticmethod
    def _stage(stage):
        if stage is None:
            return None
        sc = StageC()
        sc.U_n = _dev(stage["U_n"]) if stage.get("U_n") is not None else None
        sc.rk0, sc.rk1, sc.rk2 = stage.get("rk", (1.0, 0.0, 1.0))
        sc.dt = stage.get("dt", 0.0)
        sc.Gamma = stage.get("Gamma", -1.0)
        return sc

    # ---- discrete adjoint (FP64 contexts) ------------------------------------
    def rhs_adjoint(self, U, stage, tape, lam_dUdt, lam_U=None):
        """lam_U += (dL/dU)^T lam_dUdt with the decisions of the forward stage
        (tape from rhs(flags=...), or None to recompute them)."""
        lam_U = torch.zeros_like(U) if lam_U is None else lam_U
        sc = self._stage(stage)
        self._check(lib.mpmc_rhs_adjoint(self.h, _dev(U), ctypes.byref(sc) if sc is not None else None, _ptr(tape),
                                         _dev(lam_dUdt), _dev(lam_U)))
        return lam_U

    def _wstages(self, w):
        """Device pointer of a stage-cache buffer (3 x cache_doubles FP64), or None."""
        if w is None:
            return None
        if not (w.dtype == torch.float64 and w.is_cuda and w.is_contiguous() and w.numel() >= 3 * self.cache_doubles):
            raise ValueError("wstages: a contiguous CUDA float64 tensor of at least 3 x cache_doubles elements")
        return w.data_ptr()

    def rk_step_record(self, U, dt=0.0, tape=None, stages=None, wstages=None):
        """One SSP-RK3 step in place that also returns its stage states
        (2 x state: U^(1), U^(2)) and fills `tape` (3 x faces uint32) and
        `wstages` (3 x cache_doubles FP64: the primitive caches of U^n, U^(1),
        U^(2)) if given."""
        stages = torch.empty((2,) + tuple(U.shape), dtype=U.dtype, device=U.device) if stages is None else stages
        self._check(lib.mpmc_rk_step_record(self.h, _dev(U), float(dt), _ptr(tape), _dev(stages),
                                            self._wstages(wstages)))
        return stages

    def rk_step_adjoint(self, U_n, lam_next, dt=0.0, tape=None, lam_n=None, stages=None, wstages=None):
        """lam_n = (dU^{n+1}/dU^n)^T lam_next for the SSP-RK3 step from U_n
        (dt and Gamma frozen; dt <= 0: the CFL step of U_n).  stages/tape/
        wstages: from rk_step_record (recomputed when None).  lam_n may be
        lam_next (in place)."""
        lam_n = torch.empty_like(lam_next) if lam_n is None else lam_n
        self._check(lib.mpmc_rk_step_adjoint(self.h, _dev(U_n), _ptr(stages), self._wstages(wstages), float(dt),
                                             _ptr(tape), _dev(lam_next), _dev(lam_n)))
        return lam_n

    def init_state_adjoint(self, prim, lam_U):
        prim = prim.to(self.device, torch.float64).contiguous()
        lam_prim = torch.empty_like(prim)
        self._check(lib.mpmc_init_state_adjoint(self.h, _dev(prim), _dev(lam_U), _dev(lam_prim)))
        return lam_prim

    @property
    def prim_fields(self):
        ns, D = self.problem.ns, self.problem.dim
        return ["T", "P", "rho", "a"] + [f"Y{k}" for k in range(ns)] + [f"u{d}" for d in range(D)]

    def primitives(self, U, out=None):
        """[T, P, rho, a, Y_k, u_d] per cell, shape (4 + ns + D, nz, ny, nx)."""
        if out is None:
            out = torch.empty((len(self.prim_fields),) + self.shape[1:], dtype=torch.float64, device=self.device)
        self._check(lib.mpmc_primitives(self.h, _dev(U), _dev(out)))
        return out

    def primitives_adjoint(self, U, lam_W, lam_U=None):
        """lam_U += (dW/dU)^T lam_W, W as returned by primitives()."""
        lam_U = torch.zeros_like(U) if lam_U is None else lam_U
        self._check(lib.mpmc_primitives_adjoint(self.h, _dev(U), _dev(lam_W.contiguous()), _dev(lam_U)))
        return lam_U

    def set_profiling(self, enable=True):
        self._check(lib.mpmc_set_profiling(self.h, 1 if enable else 0))

    def profile(self, reset=False):
        """{family: (ms, launches)} for prim, face, update, dt and the adjoint's
        face and prim kernels."""
        ms = (ctypes.c_double * 6)()
        n = (ctypes.c_uint64 * 6)()
        self._check(lib.mpmc_get_profile(self.h, ms, n, 1 if reset else 0))
        return {k: (ms[i], n[i]) for i, k in enumerate(("prim", "face", "update", "dt", "adj_face", "adj_prim"))}

    def status(self, reset=False):
        return lib.mpmc_get_status(self.h, 1 if reset else 0)

    def stats(self, reset=False):
        s = StatsC()
        self._check(lib.mpmc_get_stats(self.h, ctypes.byref(s), 1 if reset else 0))
        return {f: getattr(s, f) for f, _ in StatsC._fields_}


# module-level names mirroring the C ABI
def create(problem, precision=FP64, stream=None):
    return Context(problem, precision, stream)


def init_state(ctx, prim, U=None):
    return ctx.init_state(prim, U)


def rhs(ctx, U, dUdt=None, stage=None, flags=None):
    return ctx.rhs(U, dUdt, stage, flags)


def rk_step(ctx, U, dt=0.0, tape=None):
    return ctx.rk_step(U, dt, tape)


def step_n(ctx, U, n, dt_out=None, t_end=0.0):
    return ctx.step_n(U, n, dt_out, t_end)


def rhs_adjoint(ctx, U, stage, tape, lam_dUdt, lam_U=None):
    return ctx.rhs_adjoint(U, stage, tape, lam_dUdt, lam_U)


def rk_step_record(ctx, U, dt=0.0, tape=None, stages=None, wstages=None):
    return ctx.rk_step_record(U, dt, tape, stages, wstages)


def rk_step_adjoint(ctx, U_n, lam_next, dt=0.0, tape=None, lam_n=None, stages=None, wstages=None):
    return ctx.rk_step_adjoint(U_n, lam_next, dt, tape, lam_n, stages, wstages)


def init_state_adjoint(ctx, prim, lam_U):
    return ctx.init_state_adjoint(prim, lam_U)


def primitives(ctx, U, out=None):
    return ctx.primitives(U, out)


def primitives_adjoint(ctx, U, lam_W, lam_U=None):
    return ctx.primitives_adjoint(U, lam_W, lam_U)


workloads = _wl
