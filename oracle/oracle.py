"""ctypes front end of the CPU oracle (test infrastructure only).

`build()` compiles mpmc_oracle.cpp with the host C++ compiler (plain FP64,
no FMA contraction so that x86 and Arm hosts agree bit for bit), and a
rounding twin of the same source with fused multiply-add contraction whose
results differ from the plain build's only by rounding: the parity tests
read their differences as the method's own rounding noise.  `Oracle` wraps
one problem (grid, species, model) and exposes init_state, stage, rk_step,
run and the point functions used by the pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = [os.path.join(HERE, "mpmc_oracle.cpp")]
HDR = [os.path.join(HERE, "mpmc_oracle.h"), os.path.join(HERE, "oracle_scalar.hpp")]
MAXS = 8

_lock = threading.Lock()
_lib = None
_lib_fma = None


def lib_path(fma=False):
    return os.path.join(HERE, "liboracle_fma.so" if fma else "liboracle.so")


def _fma_flags():
    # fused multiply-adds wherever the compiler contracts (x86-64 needs the
    # FMA instructions named; AArch64 has them in its base set)
    import platform
    return ["-ffp-contract=fast"] + (["-mfma"] if platform.machine() in ("x86_64", "AMD64") else [])


def build(force=False, verbose=False):
    """Compile the oracle shared library if it is missing or stale, and its
    rounding twin: the same source with fused multiply-add contraction
    (liboracle_fma.so), whose differences from the plain build measure the
    method's own rounding noise in the parity tests."""
    newest = max(os.path.getmtime(f) for f in SRC + HDR)
    jobs = []
    for fma in (False, True):
        out = lib_path(fma)
        if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
            jobs.append((out, fma))
    procs = []
    for out, fma in jobs:
        flags = _fma_flags() if fma else ["-ffp-contract=off"]
        cmd = ["g++", "-O2", "-std=c++17"] + flags + ["-fopenmp", "-fPIC", "-shared", "-o", out + ".tmp"] + SRC
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((out, subprocess.Popen(cmd)))
    for out, p in procs:
        if p.wait() != 0:
            raise RuntimeError("oracle build failed: " + out)
        os.replace(out + ".tmp", out)
    return lib_path(False)


def _load(fma=False):
    global _lib, _lib_fma
    with _lock:
        if (_lib_fma if fma else _lib) is None:
            build()
            L = ctypes.CDLL(lib_path(fma))
            _declare(L)
            if fma:
                _lib_fma = L
            else:
                _lib = L
    return _lib_fma if fma else _lib


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double),
        ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3),
        ("inflow", ctypes.c_double * (MAXS + 5)),
        ("ns", ctypes.c_int), ("phase", ctypes.c_int * MAXS),
        ("cv", ctypes.c_double * MAXS), ("gamma", ctypes.c_double * MAXS), ("q", ctypes.c_double * MAXS),
        ("b", ctypes.c_double * MAXS), ("pinf", ctypes.c_double * MAXS),
        ("W", ctypes.c_double * MAXS), ("mu", ctypes.c_double * MAXS), ("Sc", ctypes.c_double * MAXS),
        ("weno_eps", ctypes.c_double), ("cdi", ctypes.c_int), ("diffusion", ctypes.c_int),
        ("pos_limiter", ctypes.c_int), ("cdi_eps", ctypes.c_double), ("cdi_gamma", ctypes.c_double),
        ("phi_min", ctypes.c_double), ("psi_delta", ctypes.c_double), ("cfl", ctypes.c_double),
        ("mu_liquid", ctypes.c_double), ("recon_basis", ctypes.c_int), ("eos_iterative", ctypes.c_int),
        ("nthreads", ctypes.c_int), ("recon", ctypes.c_int), ("viscous", ctypes.c_int),
        ("prandtl", ctypes.c_double), ("lambda_liquid", ctypes.c_double),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def _declare(L):
    P = ctypes.POINTER(OrcParams)
    d, i = ctypes.c_double, ctypes.c_int
    sig = {
        "orc_init_state": [P, _dp, _dp],
        "orc_primitives": [P, _dp, _dp],
        "orc_dt_gamma": [P, _dp, _dp, _dp],
        "orc_stage": [P, _dp, _dp, d, d, d, d, d, _dp, _dp, _u32p],
        "orc_face_fluxes": [P, _dp, _dp, d, d, d, d, d, _dp],
        "orc_rk_step": [P, _dp, d, _dp],
        "orc_run": [P, _dp, i, d, _dp, ctypes.POINTER(i)],
        "orc_eos_pt": [P, _dp, d, d, _dp, _dp],
        "orc_eos_forward": [P, _dp, d, d, _dp],
        "orc_char_matrices": [P, i, _dp, _dp, _dp, _dp],
        "orc_hllc_prim": [P, i, _dp, _dp, _dp],
        "orc_physical_flux": [P, i, _dp, _dp],
        "orc_cons_from_point": [P, _dp, _dp],
        "orc_stage_jvp": [P, _dp, _dp, _dp, d, d, d, d, d, _dp, _dp],
        "orc_rk_step_jvp": [P, _dp, _dp, d, d, _dp, _dp],
        "orc_primitives_jvp": [P, _dp, _dp, _dp, _dp],
        "orc_init_state_jvp": [P, _dp, _dp, _dp, _dp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.orc_weno5z.argtypes = [_dp, d]
    L.orc_weno5z.restype = d
    L.orc_reconstruct.argtypes = [ctypes.c_int, _dp, d]
    L.orc_reconstruct.restype = d
    L.orc_candidate.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp]
    L.orc_candidate.restype = None
    L.orc_weno5z_jvp.argtypes = [_dp, _dp, d, _dp]
    L.orc_weno5z_jvp.restype = d
    L.orc_y_limiter.argtypes = [P, _dp, _dp]
    L.orc_y_limiter.restype = ctypes.c_int
    L.orc_face_states.argtypes = [P, _dp, i, i, i, i, _dp, _dp, _u32p]
    L.orc_face_states.restype = ctypes.c_int


def _ptr(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.uint32:
        return a.ctypes.data_as(_u32p)
    assert a.dtype == np.float64
    return a.ctypes.data_as(_dp)


class Oracle:
    """One problem on the CPU oracle.  Arrays are numpy float64 SoA
    [var, nz, ny, nx] of interior cells."""

    def __init__(self, problem, nthreads=0, recon_basis=0, eos_iterative=0, fma=False, **model_overrides):
        """fma: the rounding twin (same source, fused multiply-adds), for
        estimating rounding noise only"""
        self.lib = _load(fma)
        self.problem = problem
        p = OrcParams()
        pr = problem
        p.dim = pr.dim
        for d in range(3):
            p.n[d] = pr.n[d]
            p.bc_lo[d] = pr.bc_lo[d]
            p.bc_hi[d] = pr.bc_hi[d]
        p.dx = pr.dx
        if pr.inflow is not None:
            for q, v in enumerate(pr.inflow):
                p.inflow[q] = float(v)
        p.ns = pr.ns
        for k, s in enumerate(pr.species):
            p.phase[k] = s.phase
            p.cv[k], p.gamma[k], p.q[k], p.b[k], p.pinf[k] = s.cv, s.gamma, s.q, s.b, s.pinf
            p.W[k], p.mu[k], p.Sc[k] = s.W, s.mu, s.Sc
        m = pr.model
        fields = dict(weno_eps=m.weno_eps, cdi=m.cdi, diffusion=m.diffusion, pos_limiter=m.pos_limiter,
                      cdi_eps=m.cdi_eps, cdi_gamma=m.cdi_gamma, phi_min=m.phi_min, psi_delta=m.psi_delta,
                      cfl=m.cfl, mu_liquid=m.mu_liquid, recon=m.recon, viscous=m.viscous,
                      prandtl=m.prandtl, lambda_liquid=m.lambda_liquid)
        fields.update(model_overrides)
        for k, v in fields.items():
            setattr(p, k, v)
        p.recon_basis = recon_basis
        p.eos_iterative = eos_iterative
        p.nthreads = nthreads
        self.p = p
        self.pp = ctypes.byref(p)
        self.nv = pr.nvars
        self.shape = (pr.n[2], pr.n[1], pr.n[0])

    # ---- grid-level -------------------------------------------------------
    def init_state(self, prim=None):
        prim = np.ascontiguousarray(self.problem.prim if prim is None else prim, dtype=np.float64)
        U = np.zeros((self.nv,) + self.shape)
        st = self.lib.orc_init_state(self.pp, _ptr(prim), _ptr(U))
        assert st == 0, st
        return U

    def primitives(self, U):
        out = np.zeros((8,) + self.shape)
        st = self.lib.orc_primitives(self.pp, _ptr(np.ascontiguousarray(U)), _ptr(out))
        return dict(P=out[0], T=out[1], a=out[2], rho=out[3], phi0=out[4], phi1=out[5],
                    psi0=out[6], psi1=out[7], status=st)

    def dt_gamma(self, U):
        dt, G = ctypes.c_double(), ctypes.c_double()
        st = self.lib.orc_dt_gamma(self.pp, _ptr(np.ascontiguousarray(U)), ctypes.byref(dt), ctypes.byref(G))
        return dt.value, G.value, st

    def nfaces(self, d):
        n = list(self.problem.n)
        n[d] += 1
        return n[0] * n[1] * n[2]

    def stage(self, U_n, U_k, rk=(1.0, 0.0, 1.0), dt=None, Gamma=None, flags=False):
        """Returns (U_out, dUdt, flags or None, status)."""
        U_n = np.ascontiguousarray(U_n)
        U_k = np.ascontiguousarray(U_k)
        if dt is None or Gamma is None:
            dtc, Gc, _ = self.dt_gamma(U_n)
            dt = dtc if dt is None else dt
            Gamma = Gc if Gamma is None else Gamma
        Uo = np.zeros_like(U_k)
        L = np.zeros_like(U_k)
        fl = np.zeros(sum(self.nfaces(d) for d in range(self.problem.dim)), dtype=np.uint32) if flags else None
        st = self.lib.orc_stage(self.pp, _ptr(U_n), _ptr(U_k), rk[0], rk[1], rk[2], dt, Gamma,
                                _ptr(Uo), _ptr(L), _ptr(fl))
        return Uo, L, fl, st

    def face_fluxes(self, U_n, U_k, rk=(1.0, 0.0, 1.0), dt=0.0, Gamma=0.0):
        tot = sum(self.nfaces(d) for d in range(self.problem.dim)) * self.nv
        F = np.zeros(tot)
        st = self.lib.orc_face_fluxes(self.pp, _ptr(np.ascontiguousarray(U_n)), _ptr(np.ascontiguousarray(U_k)),
                                      rk[0], rk[1], rk[2], dt, Gamma, _ptr(F))
        out, off = [], 0
        for d in range(self.problem.dim):
            n = list(self.problem.n)
            n[d] += 1
            sz = self.nv * n[0] * n[1] * n[2]
            out.append(F[off:off + sz].reshape(self.nv, n[2], n[1], n[0]))
            off += sz
        return out, st

    def rk_step(self, U, dt=0.0):
        U = np.ascontiguousarray(U).copy()
        used = ctypes.c_double()
        st = self.lib.orc_rk_step(self.pp, _ptr(U), dt, ctypes.byref(used))
        return U, used.value, st

    # ---- forward-mode tangents (dt and Gamma frozen) ----------------------------
    def stage_jvp(self, U_n, U_k, dU_k, rk, dt, Gamma):
        """(dUdt, d(dUdt)) of the stage at U_k in direction dU_k."""
        U_n, U_k, dU_k = (np.ascontiguousarray(a, dtype=np.float64) for a in (U_n, U_k, dU_k))
        L, dL = np.zeros_like(U_k), np.zeros_like(U_k)
        st = self.lib.orc_stage_jvp(self.pp, _ptr(U_n), _ptr(U_k), _ptr(dU_k), rk[0], rk[1], rk[2], dt, Gamma,
                                    _ptr(L), _ptr(dL))
        return L, dL, st

    def rk_step_jvp(self, U, dU, dt, Gamma):
        U, dU = (np.ascontiguousarray(a, dtype=np.float64) for a in (U, dU))
        Uo, dUo = np.zeros_like(U), np.zeros_like(U)
        st = self.lib.orc_rk_step_jvp(self.pp, _ptr(U), _ptr(dU), dt, Gamma, _ptr(Uo), _ptr(dUo))
        return Uo, dUo, st

    def primitives_jvp(self, U, dU):
        U, dU = (np.ascontiguousarray(a, dtype=np.float64) for a in (U, dU))
        out, dout = np.zeros((8,) + self.shape), np.zeros((8,) + self.shape)
        st = self.lib.orc_primitives_jvp(self.pp, _ptr(U), _ptr(dU), _ptr(out), _ptr(dout))
        names = ("P", "T", "a", "rho", "phi0", "phi1", "psi0", "psi1")
        return {k: out[i] for i, k in enumerate(names)}, {k: dout[i] for i, k in enumerate(names)}, st

    def weno5z_jvp(self, v5, dv5, eps=None):
        v5 = np.ascontiguousarray(v5, dtype=np.float64)
        dv5 = np.ascontiguousarray(dv5, dtype=np.float64)
        out = ctypes.c_double()
        val = self.lib.orc_weno5z_jvp(_ptr(v5), _ptr(dv5), self.p.weno_eps if eps is None else eps,
                                      ctypes.byref(out))
        return val, out.value

    def init_state_jvp(self, prim, dprim):
        prim, dprim = (np.ascontiguousarray(a, dtype=np.float64) for a in (prim, dprim))
        U, dU = np.zeros((self.nv,) + self.shape), np.zeros((self.nv,) + self.shape)
        st = self.lib.orc_init_state_jvp(self.pp, _ptr(prim), _ptr(dprim), _ptr(U), _ptr(dU))
        return U, dU, st

    def run(self, U, nsteps, t_end=0.0):
        U = np.ascontiguousarray(U).copy()
        t = ctypes.c_double()
        ns = ctypes.c_int()
        st = self.lib.orc_run(self.pp, _ptr(U), nsteps, t_end, ctypes.byref(t), ctypes.byref(ns))
        return U, t.value, ns.value, st

    # ---- point functions --------------------------------------------------
    def eos_pt(self, Y, e, v):
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        P, T = ctypes.c_double(), ctypes.c_double()
        st = self.lib.orc_eos_pt(self.pp, _ptr(Y), e, v, ctypes.byref(P), ctypes.byref(T))
        return P.value, T.value, st

    def eos_forward(self, Y, P, T):
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        out = np.zeros(6)
        self.lib.orc_eos_forward(self.pp, _ptr(Y), P, T, _ptr(out))
        return dict(rho=out[0], e=out[1], a=out[2], alpha=out[3], beta=out[4], cp=out[5])

    def weno5z(self, v5, eps=None):
        v = np.ascontiguousarray(v5, dtype=np.float64)
        return self.lib.orc_weno5z(_ptr(v), self.p.weno_eps if eps is None else eps)

    def reconstruct(self, kind, v6, eps=None):
        """value at the right face of cell i from cells i-2..i+3 (kind: the
        workloads RECON_* constants)"""
        v = np.ascontiguousarray(v6, dtype=np.float64)
        assert v.shape == (6,)
        return self.lib.orc_reconstruct(int(kind), _ptr(v), self.p.weno_eps if eps is None else eps)

    def candidate(self, v6, offset, n):
        """(value at the right face of cell i, Jiang-Shu indicator) of the
        polynomial fitted to the n cell averages starting at offset from cell i"""
        v = np.ascontiguousarray(v6, dtype=np.float64)
        val, beta = ctypes.c_double(), ctypes.c_double()
        self.lib.orc_candidate(_ptr(v), int(offset), int(n), ctypes.byref(val), ctypes.byref(beta))
        return val.value, beta.value

    def y_limiter(self, Y, Yc):
        """The mass-fraction limiter of Sec. 3.3.1 on one face side: returns
        (limited Y, whether it changed Y)."""
        Y = np.array(Y, dtype=np.float64)
        Yc = np.ascontiguousarray(Yc, dtype=np.float64)
        assert Y.shape == (self.problem.ns,) and Yc.shape == Y.shape
        r = self.lib.orc_y_limiter(self.pp, _ptr(Y), _ptr(Yc))
        assert r in (0, 1)
        return Y, bool(r)

    def face_states(self, U, d, face):
        """Face states of the face `face` = (i, j, k) of direction d (its low
        cell is i - 1 along d) after the interpolation limiters: (WL, WR,
        flags, status), W = dict(Y, u, P, T)."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        ns = self.problem.ns
        WL, WR = np.zeros(ns + 5), np.zeros(ns + 5)
        fl = np.zeros(1, dtype=np.uint32)
        i, j, k = (list(face) + [0, 0])[:3]
        st = self.lib.orc_face_states(self.pp, _ptr(U), int(d), int(i), int(j), int(k), _ptr(WL), _ptr(WR),
                                      _ptr(fl))
        assert st != 1, "invalid face"
        split = lambda w: dict(Y=w[:ns].copy(), u=w[ns:ns + 3].copy(), P=float(w[ns + 3]), T=float(w[ns + 4]))
        return split(WL), split(WR), int(fl[0]), st

    def char_matrices(self, d, Ubar):
        nc = self.problem.ns + self.problem.dim + 1
        Sinv = np.zeros((nc, nc))
        S = np.zeros((nc, nc))
        sc = np.zeros(6)
        Ubar = np.ascontiguousarray(Ubar, dtype=np.float64)
        st = self.lib.orc_char_matrices(self.pp, d, _ptr(Ubar), _ptr(Sinv), _ptr(S), _ptr(sc))
        return Sinv, S, dict(rho=sc[0], a=sc[1], alpha=sc[2], beta=sc[3], X=sc[4], rhoa=sc[5]), st

    def _point(self, Y, u, P, T):
        W = np.zeros(self.problem.ns + 5)
        W[:self.problem.ns] = Y
        W[self.problem.ns:self.problem.ns + 3] = list(u) + [0.0] * (3 - len(u))
        W[self.problem.ns + 3] = P
        W[self.problem.ns + 4] = T
        return W

    def hllc(self, d, left, right):
        F = np.zeros(self.nv)
        self.lib.orc_hllc_prim(self.pp, d, _ptr(self._point(*left)), _ptr(self._point(*right)), _ptr(F))
        return F

    def physical_flux(self, d, state):
        F = np.zeros(self.nv)
        self.lib.orc_physical_flux(self.pp, d, _ptr(self._point(*state)), _ptr(F))
        return F

    def cons_from_point(self, state):
        U = np.zeros(self.nv)
        self.lib.orc_cons_from_point(self.pp, _ptr(self._point(*state)), _ptr(U))
        return U
