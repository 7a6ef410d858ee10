"""Viscous stress and heat conduction (Eq. DiffusionTerms; row f2) on the
FP64 GPU path, through the C ABI: the stage right-hand side against the
oracle with walls (mirrored tangential gradients), periodic and 3D
boundaries (same bound as the inviscid parity tests), 100 steps, and the
shear wave's decay against the exact SSP-RK3 factor of the discrete
Laplacian; the mixed path's FP32 viscous fluxes within the mixed-precision
bound; the discrete adjoint with its viscous reverse (dot products against
the oracle's forward-mode tangent)."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W
from tests.test_gpu_adjoint import _dot_check
from tests.test_gpu_parity import NTH, _cuda, _gross, _steps_parity, rhs_parity
from tests.test_oracle_jvp import _modulated, _state_and_dir

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_2504_14063_gb300 import binding
    return binding


def _viscous(p, mu_scale=1.0):
    p.model.viscous = 1
    if mu_scale != 1.0:
        p.model.mu_liquid *= mu_scale
        p.model.lambda_liquid *= mu_scale
        for s in p.species:
            s.mu *= mu_scale
    return p


CASES = {
    # the viscous terms scaled up so that they are a visible part of L
    "slab_1d": (lambda: _viscous(W.interface_advection_1d(n=400, cdi=1), 1e4), 3),
    "shock_bubble_2d_walls": (lambda: _viscous(W.shock_bubble_2d(nx=100, ny=52, seed=1), 1e3), 60),
    "periodic_cdi_diffusion_2d": (lambda: _viscous(W.random_smooth_2d(41, 35, seed=5, cdi=1, diffusion=1), 1e3), 2),
    "droplet_field_3d": (lambda: _viscous(W.droplet_field_3d(n=22, ndrops=4, seed=2, rmin=3.0, rmax=5.0), 1e2), 2),
    "shock_droplet_3d": (lambda: _viscous(W.shock_droplet_3d(n=24, seed=4), 1e2), 2),
}


@pytest.mark.parametrize("case", list(CASES))
def test_rhs_parity_viscous(mp, case):
    make, pre = CASES[case]
    rhs_parity(mp, make(), pre_steps=pre)


def test_100_steps_shock_bubble_viscous(mp):
    p = _viscous(W.shock_bubble_2d(nx=72, ny=40, seed=0, liquid_cols=24), 1e3)
    _steps_parity(mp, p, 100, conditioned=False)


def test_shear_wave_decay_on_gpu(mp):
    """u_y = A sin(kx), gas at rest, periodic: after n steps of length dt
    the amplitude is A (1 - z + z^2/2 - z^3/6)^n, z = nu (2 - 2 cos k dx)
    dt / dx^2 (the three-point Laplacian that the face gradients make)."""
    nx, A, dx = 16, 1e-3, 1e-7
    prim = np.zeros((5, 1, 4, nx))
    x = (np.arange(nx) + 0.5) * dx
    prim[0] = 1.0
    prim[2] = A * np.sin(2 * np.pi * x / (nx * dx))[None, None, :]
    prim[3] = 1e5
    prim[4] = 300.0
    p = W.Problem("shear", 2, (nx, 4, 1), dx, [W.AIR], W.Model(), prim,
                  bc_lo=(W.BC_PERIODIC,) * 3, bc_hi=(W.BC_PERIODIC,) * 3)
    p.model.viscous = 1
    ctx = mp.Context(p)
    U = ctx.init_state(torch.from_numpy(prim))
    rho = float(U[0].mean())
    nu = W.AIR.mu / rho
    a = np.sqrt(W.AIR.gamma * (W.AIR.gamma - 1) * W.AIR.cv * 300.0)
    dt = min(0.4 * dx / a, 0.1 * dx * dx / nu)
    n = 40
    for _ in range(n):
        ctx.rk_step(U, dt)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    z = nu * (2 - 2 * np.cos(2 * np.pi / nx)) * dt / dx ** 2
    factor = (1 - z + z * z / 2 - z ** 3 / 6) ** n
    uy = (U[2] / U[0]).cpu().numpy()[0, 0]
    s = np.sin(2 * np.pi * (np.arange(nx) + 0.5) / nx)
    amp = (uy * s).sum() / (s * s).sum()
    print(f"GPU shear wave after {n} steps: amplitude ratio {amp / A:.12f}, discrete factor {factor:.12f}")
    assert amp / A == pytest.approx(factor, rel=1e-9)


@pytest.mark.parametrize("case", ["shock_bubble_2d_walls", "periodic_cdi_diffusion_2d", "shock_droplet_3d"])
def test_mixed_rhs_viscous_close_to_oracle(mp, case):
    """The mixed path's FP32 viscous fluxes: the stage right-hand side within
    the mixed-precision bound of tests/test_gpu_mixed.py (1e-4 of the
    oracle's L1 + 1e-7 of the gross flux + 10 x the oracle's own change
    under a 2^-24 perturbation of its input)."""
    make, pre = CASES[case]
    p = make()
    o = Oracle(p, nthreads=NTH)
    Un = o.run(o.init_state(), pre)[0]
    dt, G, _ = o.dt_gamma(Un)
    Uk = o.stage(Un, Un, (1.0, 0.0, 1.0), dt, G)[0]
    rk = (0.75, 0.25, 0.25)
    _, Lo, _, st = o.stage(Un, Uk, rk, dt, G)
    assert st == 0
    F, _ = o.face_fluxes(Un, Uk, rk, dt, G)
    ctx = mp.Context(p, precision=mp.MIXED)
    Lg = ctx.rhs(_cuda(Uk), stage=dict(U_n=_cuda(Un), rk=rk, dt=dt, Gamma=G)).cpu().numpy()
    assert ctx.status() == 0
    rng = np.random.default_rng(1)
    jit = lambda A: A * (1.0 + 2.0 ** -24 * rng.standard_normal(A.shape))
    _, Lt, _, _ = o.stage(jit(Un), jit(Uk), rk, dt, G)
    T32 = np.abs(Lt - Lo).sum(axis=(1, 2, 3))
    num = np.abs(Lg - Lo).sum(axis=(1, 2, 3))
    ref = np.abs(Lo).sum(axis=(1, 2, 3))
    bound = 1e-4 * ref + 1e-7 * _gross(p, F) + 10.0 * T32
    print(f"mixed viscous rhs {case}: rel err {np.array2string(num / ref, precision=2)}, err/bound "
          f"{np.array2string(num / bound, precision=2)}")
    assert np.all(num <= bound)


ADJ_CASES = {
    "smooth_2d_cdi_diff": lambda: _viscous(W.random_smooth_2d(24, 20, seed=3, cdi=1, diffusion=1), 1e3),
    "shock_bubble_2d_walls": lambda: _viscous(_modulated(W.shock_bubble_2d(nx=48, ny=28, seed=1)), 1e3),
    "droplet_3d": lambda: _viscous(_modulated(W.droplet_field_3d(n=14, ndrops=2, seed=2, rmin=2.5, rmax=3.5)),
                                   1e2),
}


@pytest.mark.parametrize("case", list(ADJ_CASES))
def test_viscous_rhs_adjoint_dot_product(mp, case):
    """<lam, J dU> (oracle forward-mode tangent through the viscous terms) =
    <J^T lam, dU> (GPU adjoint with its viscous reverse kernel), within 1e-9
    of the gross sum."""
    p = ADJ_CASES[case]()
    o = Oracle(p, nthreads=NTH)
    U, dU = _state_and_dir(o, p, np.random.default_rng(5))
    dt, G, _ = o.dt_gamma(U)
    rk = (0.75, 0.25, 0.25)
    Un = o.rk_step(U, 0.3 * dt)[0]
    _, dL, st = o.stage_jvp(Un, U, dU, rk, dt, G)
    assert st == 0
    lam = np.random.default_rng(9).standard_normal(U.shape)
    ctx = mp.Context(p)
    lamU = ctx.rhs_adjoint(_cuda(U), dict(U_n=_cuda(Un), rk=rk, dt=dt, Gamma=G), None, _cuda(lam)).cpu().numpy()
    assert ctx.status() == 0
    _dot_check((lam * dL).sum(), (lamU * dU).sum(), np.abs(lam * dL).sum(), f"viscous rhs {case}")


def test_viscous_rk_step_adjoint_dot_product(mp):
    p = ADJ_CASES["shock_bubble_2d_walls"]()
    o = Oracle(p, nthreads=NTH)
    U, dU = _state_and_dir(o, p, np.random.default_rng(6))
    ctx = mp.Context(p)
    dt, G = (float(x) for x in ctx.dt_gamma(_cuda(U)).cpu())
    _, dU1, st = o.rk_step_jvp(U, dU, dt, G)
    assert st == 0
    lam = np.random.default_rng(10).standard_normal(U.shape)
    lam_n = ctx.rk_step_adjoint(_cuda(U), _cuda(lam), dt=dt).cpu().numpy()
    assert ctx.status() == 0
    _dot_check((lam * dU1).sum(), (lam_n * dU).sum(), np.abs(lam * dU1).sum(), "viscous rk step")
