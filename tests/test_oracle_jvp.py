"""Pins of the oracle's forward-mode tangents (Dual<1> evaluation of its own
arithmetic), the CPU reference for the discrete adjoint:
  * the primal part of a Dual evaluation equals the plain FP64 evaluation bit
    for bit (the same operations on the same values);
  * the tangent equals central differences of the plain FP64 oracle, with dt
    and Gamma held fixed, for directions whose +-h perturbations leave every
    discrete decision (the per-face flag bits) unchanged.
A wrong derivative rule in the dual type or a branch that drops a tangent
fails the second check."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W

H = 1e-7   # larger steps cross unflagged kinks (wave-speed min/max, |b0 - b2| of WENO-Z)


def _smooth(rng, shape):
    nz, ny, nx = shape
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    f = np.zeros_like(X)
    for kx in range(3):
        for ky in range(3 if ny > 1 else 1):
            a, ph = rng.standard_normal(), rng.uniform(0, 2 * np.pi)
            f += a * np.cos(2 * np.pi * (kx * X + ky * Y) + ph)
    return f[None] / np.abs(f).max()


def _state_and_dir(o, p, rng):
    """U = init(prim) and a direction dU = (dU/dprim) dprim with a smooth
    dprim: relative changes of the volume fractions, P and T, velocity
    changes of 10 m/s.  Smooth, because on a stencil that is flat to rounding
    a difference quotient measures WENO-Z applied to the direction itself;
    primitive, because a relative change of a stiff liquid's energy moves
    its pressure by gamma Pinf / P times as much and leaves the linear regime
    of the difference quotient early."""
    ns, D = p.ns, p.dim
    prim = p.prim
    dprim = np.zeros_like(prim)
    for k in range(ns):
        dprim[k] = prim[k] * _smooth(rng, prim.shape[1:])
    for d in range(D):
        dprim[ns + d] = 10.0 * _smooth(rng, prim.shape[1:])
    for q in (ns + D, ns + D + 1):
        dprim[q] = prim[q] * _smooth(rng, prim.shape[1:])
    U, dU, st = o.init_state_jvp(prim, dprim)
    assert st == 0
    return U, dU


def _modulated(p, amp=0.01, du=1.0):
    """The same problem with smooth P, T and velocity modulations, so that no
    stencil is flat to rounding (where WENO-Z has no linear derivative, see
    test_weno_tangent_flat_stencil_is_the_linear_scheme)."""
    nz, ny, nx = p.prim.shape[1:]
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    ns, D = p.ns, p.dim
    p.prim[ns + D] *= (1.0 + amp * np.sin(2 * np.pi * (X + 0.3 * Y) + 0.4))[None]
    p.prim[ns + D + 1] *= (1.0 + amp * np.cos(2 * np.pi * (X - 0.2 * Y) + 1.1))[None]
    for d in range(D):
        p.prim[ns + d] += (du * np.sin(2 * np.pi * (X + (d + 1) * 0.4 * Y) + 0.7 * d))[None]
    return p


# (name, problem, difference step, tolerance).  The step is each case's best:
# truncation error falls as h^2 until round-off takes over.  A stiff liquid
# with a trace of gas is strongly curved (the pressure root of Eq. NASG_P
# moves by gamma Pinf / P times the relative energy change), which takes
# the slab's best agreement to ~1e-5.
def _cases():
    return [
        ("smooth_2d_cdi_diff", lambda: W.random_smooth_2d(16, 12, seed=3, cdi=1, diffusion=1), 1e-6, 1e-6),
        ("slab_1d_cdi", lambda: _modulated(W.interface_advection_1d(n=47, cdi=1)), 1e-9, 1e-4),
        ("shock_bubble_2d", lambda: _modulated(W.shock_bubble_2d(nx=40, ny=24, seed=1)), 1e-8, 1e-4),
    ]


def _switch_mask(o, fl_a, fl_b, shape):
    """Cells next to a face whose flag bits differ between two evaluations
    (its flux jumps there: a discrete decision switched)."""
    mask = np.zeros(shape, dtype=bool)
    off = 0
    for d in range(o.problem.dim):
        n = list(o.problem.n)
        n[d] += 1
        nf = n[0] * n[1] * n[2]
        ch = ((fl_a[off:off + nf] ^ fl_b[off:off + nf]) & 0x13F).reshape(n[2], n[1], n[0]) != 0
        off += nf
        ax = 2 - d
        low = [slice(None)] * 3
        high = [slice(None)] * 3
        low[ax] = slice(0, -1)    # face c: the low face of cell c
        high[ax] = slice(1, None)  # face c + 1: its high face
        mask |= ch[tuple(low)] | ch[tuple(high)]
    return mask


def _rel(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("name,make,h,tol", _cases())
def test_stage_tangent_matches_central_differences(name, make, h, tol):
    p = make()
    o = Oracle(p, nthreads=4)
    U, dU = _state_and_dir(o, p, np.random.default_rng(7))
    dt, G, _ = o.dt_gamma(U)
    rk = (1.0, 0.0, 1.0)
    L0, dL, st = o.stage_jvp(U, U, dU, rk, dt, G)
    assert st == 0
    _, Lp, fp, _ = o.stage(U, U + h * dU, rk, dt, G, flags=True)
    _, Lm, fm, _ = o.stage(U, U - h * dU, rk, dt, G, flags=True)
    _, Lr, fr, _ = o.stage(U, U, rk, dt, G, flags=True)
    # the primal of the dual evaluation is the FP64 evaluation itself
    assert np.array_equal(L0, Lr)
    # cells next to a face whose decisions switched within +-h are excluded
    keep = ~(_switch_mask(o, fp, fr, U.shape[1:]) | _switch_mask(o, fm, fr, U.shape[1:]))
    assert keep.mean() > 0.95
    fd = (Lp - Lm) / (2 * h)
    err = max(_rel(dL[v][keep], fd[v][keep]) for v in range(o.nv))
    print(f"stage tangent {name}: worst per-variable rel L1 vs central differences {err:.2e} "
          f"({(~keep).sum()} cells excluded)")
    assert err < tol


@pytest.mark.parametrize("name,make,h,tol", _cases()[:2])
def test_rk_step_tangent_matches_central_differences(name, make, h, tol):
    p = make()
    o = Oracle(p, nthreads=4)
    U, dU = _state_and_dir(o, p, np.random.default_rng(11))
    dt, G, _ = o.dt_gamma(U)
    of = Oracle(p, nthreads=4, cdi_gamma=G)   # Gamma frozen for the differences
    U1, dU1, st = o.rk_step_jvp(U, dU, dt, G)
    assert st == 0
    assert np.array_equal(U1, of.rk_step(U, dt)[0])
    fd = (of.rk_step(U + h * dU, dt)[0] - of.rk_step(U - h * dU, dt)[0]) / (2 * h)
    dif = dU1 - fd
    # the change over one step, not the state, is what the tangent resolves
    err = max(np.abs(dif[v]).sum() / np.abs(dU1[v] - dU[v]).sum() for v in range(o.nv))
    print(f"rk step tangent {name}: worst per-variable rel L1 of the step's change {err:.2e}")
    assert err < tol


def test_primitives_and_init_tangents_match_central_differences():
    p = W.random_smooth_2d(16, 12, seed=5, cdi=1, diffusion=1)
    o = Oracle(p, nthreads=4)
    rng = np.random.default_rng(2)
    prim = p.prim
    dprim = prim * rng.standard_normal(prim.shape)
    U, dU, st = o.init_state_jvp(prim, dprim)
    assert st == 0 and np.array_equal(U, o.init_state(prim))
    fd = (o.init_state(prim + H * dprim) - o.init_state(prim - H * dprim)) / (2 * H)
    assert _rel(dU, fd) < 1e-7
    _, dV = _state_and_dir(o, p, rng)
    out, dout, st = o.primitives_jvp(U, dV)
    assert st == 0
    ref = o.primitives(U)
    for k in ("P", "T", "a", "rho", "phi0"):
        assert np.array_equal(out[k], ref[k])
        fd = (o.primitives(U + H * dV)[k] - o.primitives(U - H * dV)[k]) / (2 * H)
        err = _rel(dout[k], fd)
        print(f"primitive {k}: rel L1 vs central differences {err:.2e}")
        assert err < 1e-6


def test_weno_tangent_flat_stencil_is_the_linear_scheme():
    """On a stencil flat to rounding the tangent is the linear fifth-order
    scheme (weights 1/10, 6/10, 3/10); elsewhere it is the derivative of the
    nonlinear weights as well (checked against central differences)."""
    p = W.interface_advection_1d(n=8)
    o = Oracle(p)
    rng = np.random.default_rng(4)
    lin = np.array([1 / 30, -13 / 60, 47 / 60, 27 / 60, -1 / 20])
    for base in (300.0, -2.5e7, 1e-3):
        v = base * (1.0 + 1e-14 * rng.standard_normal(5))   # rounding-level noise
        dv = rng.standard_normal(5)
        val, dval = o.weno5z_jvp(v, dv)
        assert abs(val - base) <= 1e-13 * abs(base)
        assert dval == pytest.approx(lin @ dv, rel=1e-12, abs=1e-15)
    v = np.array([1.0, 1.3, 0.7, 2.0, 1.1])
    dv = rng.standard_normal(5)
    val, dval = o.weno5z_jvp(v, dv)
    h = 1e-7
    fd = (o.weno5z(v + h * dv) - o.weno5z(v - h * dv)) / (2 * h)
    assert dval == pytest.approx(fd, rel=1e-7)
    assert abs(dval - lin @ dv) > 1e-3 * abs(fd)    # the nonlinear weights do contribute here
