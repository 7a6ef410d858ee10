"""Pins of the oracle's viscous stress and heat conduction (Eq. DiffusionTerms,
the stress tensor and heat flux of Sec. 2.1, the mixture rules of Sec. 2.2.2,
second-order central face discretization of Sec. 3.1):
  * on a linear velocity field the face stress equals the closed-form tensor
    (the central differences are exact there), with its -2/3 div u part;
  * on a linear temperature field the face heat flux is -lambda dT/dx with
    lambda = (mu_g / Pr) sum_c (Y^c / Y_g) Cp^c, Wilke's mu_g;
  * a shear wave u_y = A sin(kx) decays by exactly the SSP-RK3 amplification
    factor of the discrete Laplacian's eigenvalue nu (2 - 2 cos k dx)/dx^2;
  * mass, momentum and energy are conserved with viscosity and conduction
    on a periodic two-phase field."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W


def _gas_problem(n, dim, species, prim_fn, viscous=1, bc=W.BC_ZEROGRAD, dx=1e-3):
    nn = tuple(n) + (1,) * (3 - len(n))
    ns = len(species)
    prim = np.zeros((ns + dim + 2, nn[2], nn[1], nn[0]))
    z, y, x = np.meshgrid(*[(np.arange(nn[a]) + 0.5) * dx for a in (2, 1, 0)], indexing="ij")
    prim_fn(prim, x, y, z)
    p = W.Problem("visc", dim, nn, dx, list(species), W.Model(), prim,
                  bc_lo=(bc,) * 3, bc_hi=(bc,) * 3)
    p.model.viscous = viscous
    return p


def _viscous_part(p, U):
    """face fluxes with viscosity and conduction minus those without, and the
    rounding floor of that difference per direction and row (a few ulps of
    the fluxes it is taken from: the pressure ~1e5 in the normal momentum
    row, u (E + P) in the energy row)"""
    o1 = Oracle(p, nthreads=2)
    F1, st1 = o1.face_fluxes(U, U)
    p.model.viscous = 0
    o0 = Oracle(p, nthreads=2)
    F0, st0 = o0.face_fluxes(U, U)
    p.model.viscous = 1
    assert st0 == 0 and st1 == 0
    floor = [8 * np.finfo(float).eps * np.abs(b).reshape(b.shape[0], -1).max(1) for b in F0]
    return [a - b for a, b in zip(F1, F0)], floor


def _wilke_mu(species, Y):
    """Wilke's rule for the gas phase in mass fractions (the textbook form)"""
    g = [k for k, s in enumerate(species) if s.phase == W.GAS]
    Yg = sum(Y[k] for k in g)
    mu = 0.0
    for i in g:
        den = 0.0
        for j in g:
            Wi, Wj = species[i].W, species[j].W
            phi = (1 + (species[i].mu / species[j].mu) ** 0.5 * (Wj / Wi) ** 0.25) ** 2 / (8 * (1 + Wi / Wj)) ** 0.5
            den += (Y[j] / Yg) * (Wi / Wj) * phi
        mu += (Y[i] / Yg) * species[i].mu / den
    return mu


@pytest.mark.parametrize("dim", [2, 3])
def test_stress_of_a_linear_velocity_field(dim):
    """u_i = sum_j A_ij x_j: tau = mu (A + A^T - 2/3 tr(A) I) on every interior
    face, momentum rows -tau_{d.}, energy row -u_face . tau_{d.}."""
    rng = np.random.default_rng(dim)
    A = rng.normal(size=(3, 3)) * 50.0
    A[dim:, :] = 0.0
    A[:, dim:] = 0.0
    n = (8, 7, 6)[:dim]

    def prim_fn(pr, x, y, z):
        pr[0] = 1.0
        X = (x, y, z)
        for i in range(dim):
            pr[1 + i] = sum(A[i, j] * X[j] for j in range(dim)) + 10.0 * (i + 1)
        pr[1 + dim] = 1e5
        pr[2 + dim] = 300.0

    p = _gas_problem(n, dim, [W.AIR], prim_fn)
    o = Oracle(p, nthreads=2)
    U = o.init_state()
    Fv, floor = _viscous_part(p, U)
    mu = W.AIR.mu
    tau = mu * (A + A.T - (2.0 / 3.0) * np.trace(A) * np.eye(3))
    dx = p.dx
    for d in range(dim):
        F = Fv[d]
        # interior faces only (two cells from every boundary) of the active axes
        sl = [slice(2, -2) if 2 - ax < dim else slice(None) for ax in range(3)]
        sub = F[(slice(None),) + tuple(sl)]
        assert sub[0].size > 0
        for i in range(dim):
            assert np.allclose(sub[1 + i], -tau[d, i], rtol=1e-12, atol=floor[d][1 + i])
        # the face position along d is a cell boundary: u there is linear
        face_shape = sub.shape[1:]
        idx = np.indices(face_shape).astype(float)           # [z, y, x] indices of the sub-block
        pos = [None] * 3
        for a in range(3):
            # face f along d sits at f dx; cell centres at (i + 1/2) dx
            start = 2.0 if a < dim else 0.0
            pos[a] = (idx[2 - a] + start + (0.0 if a == d else 0.5)) * dx
        uf = [sum(A[i, j] * pos[j] for j in range(dim)) + 10.0 * (i + 1) for i in range(dim)]
        work = sum(uf[i] * tau[d, i] for i in range(dim))
        assert np.allclose(sub[1 + dim], -work, rtol=1e-12, atol=floor[d][1 + dim])


def test_heat_flux_of_a_linear_temperature_field():
    """T = T0 + g x at uniform P (two gas species): q = -lambda g with
    lambda = (mu_g / Pr) sum (Y^c/Y_g) Cp^c; no momentum flux."""
    g = 2e4
    species = [W.AIR, W.HELIUM]

    def prim_fn(pr, x, y, z):
        pr[0] = 0.7
        pr[1] = 0.3
        pr[4] = 1e5
        pr[5] = 300.0 + g * x

    p = _gas_problem((10, 5), 2, species, prim_fn)
    o = Oracle(p, nthreads=2)
    U = o.init_state()
    Fv, floor = _viscous_part(p, U)
    rho = U[:2].sum(0)
    Y = U[:2] / rho
    cp = [s.gamma * s.cv for s in species]
    Yc = Y[:, 0, 2, 2]
    mu = _wilke_mu(species, Yc)
    lam = mu / p.model.prandtl * (Yc[0] * cp[0] + Yc[1] * cp[1])
    sub = Fv[0][:, :, 1:-1, 2:-2]
    assert np.all(np.abs(sub[2]) <= floor[0][2]) and np.all(np.abs(sub[3]) <= floor[0][3])
    assert np.allclose(sub[4], -lam * g, rtol=1e-12, atol=floor[0][4])   # q = -lambda dT/dx


def test_shear_wave_decays_by_the_discrete_ssprk3_factor():
    """u_y = A sin(k x) in a uniform gas at rest (periodic): only the shear
    stress acts, and the discrete scheme is the 3-point Laplacian, so after n
    steps of length dt the amplitude is (1 - z + z^2/2 - z^3/6)^n with
    z = nu (2 - 2 cos(k dx)) dt / dx^2."""
    # cells at the viscous scale (cell Reynolds number a dx / nu ~ 2), so that
    # the decay is resolved within the acoustic time-step limit
    nx, A = 16, 1e-3
    dx = 1e-7

    def prim_fn(pr, x, y, z):
        pr[0] = 1.0
        pr[1] = 0.0
        pr[2] = A * np.sin(2 * np.pi * x / (nx * dx))
        pr[3] = 1e5
        pr[4] = 300.0

    p = _gas_problem((nx, 4), 2, [W.AIR], prim_fn, bc=W.BC_PERIODIC, dx=dx)
    o = Oracle(p, nthreads=1)
    U = o.init_state()
    rho = U[0].mean()
    nu = W.AIR.mu / rho
    k = 2 * np.pi / (nx * dx)
    a = np.sqrt(W.AIR.gamma * (W.AIR.gamma - 1) * W.AIR.cv * 300.0)
    dt = min(0.4 * dx / a, 0.1 * dx * dx / nu)
    nsteps = 40
    for _ in range(nsteps):
        U, used, st = o.rk_step(U, dt)
        assert st == 0
    z = nu * (2 - 2 * np.cos(k * dx)) * dt / dx ** 2
    factor = (1 - z + z * z / 2 - z ** 3 / 6) ** nsteps
    uy = U[2] / U[0]
    amp = 2 * np.mean(uy[0, 0] * np.sin(2 * np.pi * (np.arange(nx) + 0.5) / nx))
    exact_discrete = 2 * np.mean(A * np.sin(2 * np.pi * (np.arange(nx) + 0.5) / nx) ** 2) * factor
    print(f"shear wave after {nsteps} steps: amplitude ratio {amp / A:.12f}, discrete factor {factor:.12f}")
    assert amp == pytest.approx(exact_discrete, rel=1e-9)
    assert factor < 0.9    # the decay is well resolved, not round-off


def test_conservation_with_viscosity_and_conduction():
    p = W.random_smooth_2d(24, 18, seed=3, cdi=1, diffusion=1)
    p.model.viscous = 1
    o = Oracle(p, nthreads=2)
    U0 = o.init_state()
    U, t, n, st = o.run(U0, 20)
    assert st == 0
    for v in range(U.shape[0]):
        scale = np.abs(U0[v]).sum() + 1e-300
        assert abs(U[v].sum() - U0[v].sum()) <= 1e-13 * scale, v


def test_viscous_stage_tangent_matches_central_differences():
    """The oracle's forward-mode tangent through the viscous terms (the
    reference gradient of the GPU adjoint) against central differences along
    a smooth primitive-space direction."""
    from tests.test_oracle_jvp import _state_and_dir
    p = W.random_smooth_2d(16, 12, seed=3, cdi=1, diffusion=1)
    p.model.viscous = 1
    p.model.mu_liquid *= 1e3
    p.model.lambda_liquid *= 1e3
    for s in p.species:
        s.mu *= 1e3
    o = Oracle(p, nthreads=2)
    U, dU = _state_and_dir(o, p, np.random.default_rng(5))
    dt, G, _ = o.dt_gamma(U)
    rk = (0.75, 0.25, 0.25)
    Un = o.rk_step(U, 0.3 * dt)[0]
    _, dL, st = o.stage_jvp(Un, U, dU, rk, dt, G)
    assert st == 0
    h = 1e-6
    Lp = o.stage(Un, U + h * dU, rk, dt, G)[1]
    Lm = o.stage(Un, U - h * dU, rk, dt, G)[1]
    err = np.abs((Lp - Lm) / (2 * h) - dL).sum() / np.abs(dL).sum()
    print(f"viscous stage tangent vs central differences {err:.2e}")
    assert err < 1e-6
