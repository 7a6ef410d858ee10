"""Pins of WENO5-Z, of the characteristic matrices of Appendix A and of the
HLLC flux of Appendix B."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W


def _problem(species, dim=2):
    n = (4, 4 if dim > 1 else 1, 4 if dim > 2 else 1)
    pr = np.zeros((len(species) + dim + 2, n[2], n[1], n[0]))
    pr[0] = 1.0
    pr[-2] = 1e5
    pr[-1] = 300.0
    return W.Problem("pt", dim, n, 1e-3, list(species), W.Model(), pr)


@pytest.fixture(scope="module")
def o2():
    return Oracle(_problem([W.AIR, W.HELIUM, W.LIQUID_SG], 2))


# ------------------------------------------------------------------ WENO5-Z
def _cell_averages(F, x_faces):
    h = np.diff(x_faces)
    return (F(x_faces[1:]) - F(x_faces[:-1])) / h


def test_weno_exact_for_quadratics(o2):
    """Every candidate stencil is exact for polynomials of degree <= 2, so any
    convex combination is: the face value of a quadratic from its cell
    averages is exact."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        a, b, c = rng.normal(size=3)
        h = rng.uniform(0.1, 2.0)
        x0 = rng.normal()
        xf = x0 + h * np.arange(-2, 4)  # faces of cells i-2..i+2
        F = lambda x: a * x ** 3 / 3 + b * x ** 2 / 2 + c * x  # antiderivative
        v = _cell_averages(F, xf)
        xr = xf[3]   # right face of cell i
        exact = a * xr ** 2 + b * xr + c
        assert o2.weno5z(v) == pytest.approx(exact, rel=1e-12, abs=1e-12)


def test_weno_fifth_order_and_linear_limit(o2):
    """Smooth data: error ~ h^5, and the value approaches the linear
    fifth-order upwind formula (2, -13, 47, 27, -3)/60."""
    errs = []
    for n in (10, 20, 40, 80):
        h = 1.0 / n
        x0 = 0.3
        xf = x0 + h * np.arange(-2, 4)
        F = lambda x: -np.cos(2 * np.pi * x) / (2 * np.pi)
        v = _cell_averages(F, xf)
        exact = np.sin(2 * np.pi * xf[3])
        w = o2.weno5z(v)
        lin = (2 * v[0] - 13 * v[1] + 47 * v[2] + 27 * v[3] - 3 * v[4]) / 60.0
        errs.append(abs(w - exact))
        assert abs(w - lin) <= 0.5 * abs(lin - exact) + 1e-15
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 4.5


def test_weno_step_is_essentially_non_oscillatory(o2):
    """Across a jump the reconstruction stays within the data range up to a
    small fraction of the jump."""
    for k in range(5):
        v = np.array([0.0] * (4 - k) + [1.0] * (k + 1))[:5]
        w = o2.weno5z(v)
        assert -1e-3 <= w <= 1.0 + 1e-3


def test_weno_constants(o2):
    for c in (0.0, 1.0, -3.7, 1e5, 6e8):
        assert o2.weno5z([c] * 5) == pytest.approx(c, rel=4e-16, abs=0)


# ---------------------------------------------------- characteristic matrices
def _random_state(o, rng, u_scale=200.0):
    ns = o.problem.ns
    Y = rng.dirichlet(np.ones(ns))
    u = rng.normal(size=3) * u_scale
    u[o.problem.dim:] = 0.0
    return Y, u, rng.uniform(5e4, 2e6), rng.uniform(250.0, 600.0)


def _paper_A(ns, D, d, u, rho, a, alpha, beta):
    """Appendix A, the primitive-variable matrices A, B, C in the ordering
    W = [T, Y_0..Y_{ns-2}, u_0..u_{D-1}, P]."""
    nc = ns + D + 1
    A = np.diag(np.full(nc, u[d]))
    iu, iP = ns, ns + D
    A[0, iu + d] = (rho * a * a * beta - 1.0) / alpha
    A[iu + d, iP] = 1.0 / rho
    A[iP, iu + d] = rho * a * a
    return A


def _fd_A(o, d, Y, u, P, T):
    """A = (dU/dW)^-1 dF/dW by central differences of the conserved vector and
    of the physical flux, W = [T, Y_0..Y_{ns-2}, u, P] (Y_last = 1 - sum)."""
    ns, D = o.problem.ns, o.problem.dim
    nc = ns + D + 1
    w0 = np.concatenate([[T], Y[:-1], u[:D], [P]])

    def split(w):
        Yf = np.concatenate([w[1:ns], [1.0 - w[1:ns].sum()]])
        uf = np.zeros(3)
        uf[:D] = w[ns:ns + D]
        return (Yf, uf, w[-1], w[0])

    JU = np.zeros((nc, nc))
    JF = np.zeros((nc, nc))
    for j in range(nc):
        h = 1e-6 * max(abs(w0[j]), 1.0)
        wp, wm = w0.copy(), w0.copy()
        wp[j] += h
        wm[j] -= h
        JU[:, j] = (o.cons_from_point(split(wp)) - o.cons_from_point(split(wm))) / (2 * h)
        JF[:, j] = (o.physical_flux(d, split(wp)) - o.physical_flux(d, split(wm))) / (2 * h)
    return np.linalg.solve(JU, JF)


@pytest.mark.parametrize("species,dim", [([W.AIR, W.HELIUM, W.LIQUID_SG], 2),
                                         ([W.LIQUID_SG, W.LIQUID_B, W.AIR, W.HELIUM], 3),
                                         ([W.WATER_NASG, W.AIR_TABLE], 1)])
def test_char_matrices_diagonalize_primitive_jacobian(species, dim):
    """The paper's A (built from rho, a, alpha, beta) equals the primitive-form
    flux Jacobian obtained by finite differences of U(W) and F(W); the
    oracle's S, S^-1 are mutually inverse and S^-1 A S = diag(u, .., u, u+a, u-a)."""
    o = Oracle(_problem(species, dim))
    rng = np.random.default_rng(7)
    ns, D = o.problem.ns, dim
    for _ in range(10):
        Y, u, P, T = _random_state(o, rng)
        Ub = o.cons_from_point((Y, u, P, T))
        for d in range(D):
            Sinv, S, sc, st = o.char_matrices(d, Ub)
            assert st == 0
            nc = Sinv.shape[0]
            assert np.abs(S @ Sinv - np.eye(nc)).max() < 1e-13 * max(1.0, sc["rhoa"], 1 / sc["rhoa"])
            A = _paper_A(ns, D, d, u, sc["rho"], sc["a"], sc["alpha"], sc["beta"])
            Afd = _fd_A(o, d, Y, u, P, T)
            scale = np.abs(A).max(axis=1, keepdims=True) + 1e-300
            assert np.abs((A - Afd) / scale).max() < 1e-5
            Lam = Sinv @ A @ S
            lam = np.full(nc, u[d])
            lam[-2] += sc["a"]
            lam[-1] -= sc["a"]
            assert np.abs(Lam - np.diag(lam)).max() < 1e-9 * (abs(u[d]) + sc["a"])


# --------------------------------------------------------------------- HLLC
def test_hllc_consistency(o2):
    rng = np.random.default_rng(8)
    for _ in range(50):
        s = _random_state(o2, rng)
        for d in range(2):
            F = o2.hllc(d, s, s)
            Fp = o2.physical_flux(d, s)
            assert np.allclose(F, Fp, rtol=1e-12, atol=1e-9 * np.abs(Fp).max())


def test_hllc_supersonic_upwinding(o2):
    rng = np.random.default_rng(9)
    for _ in range(20):
        L = list(_random_state(o2, rng))
        R = list(_random_state(o2, rng))
        L[1] = np.array([3000.0, 10.0, 0.0])
        R[1] = np.array([3000.0, -5.0, 0.0])
        L[0] = R[0] = np.array([0.6, 0.4, 0.0])
        assert np.allclose(o2.hllc(0, L, R), o2.physical_flux(0, L), rtol=1e-12)
        L[1], R[1] = -L[1], -R[1]
        assert np.allclose(o2.hllc(0, L, R), o2.physical_flux(0, R), rtol=1e-12)


def test_hllc_uniform_pressure_velocity_contact(o2):
    """Uniform P and u across a material contact: s* = u, the mass flux is
    the upwind partial density times u and the momentum flux is exact."""
    rng = np.random.default_rng(10)
    for _ in range(20):
        u = np.array([rng.uniform(-80, 80), rng.uniform(-20, 20), 0.0])
        P, T = 1e5, 300.0
        L = (np.array([0.9, 0.1, 0.0]), u, P, T)
        R = (np.array([0.0, 0.0, 1.0]), u, P, T)
        F = o2.hllc(0, L, R)
        up = L if u[0] > 0 else R
        Fup = o2.physical_flux(0, up)
        assert np.allclose(F[:3], Fup[:3], rtol=1e-12, atol=1e-12)
        assert F[3] == pytest.approx(Fup[3], rel=1e-12)
        assert F[4] == pytest.approx(Fup[4], rel=1e-9, abs=1e-6)


def _toro_hllc(o, d, L, R):
    """Toro's four-region HLLC (Sec. 10.4) with the same wave-speed estimates:
    F_L | F_L + S_L (U*L - U_L) | F_R + S_R (U*R - U_R) | F_R."""
    ns, D = o.problem.ns, o.problem.dim
    def prims(s):
        U = o.cons_from_point(s)
        rho = U[:ns].sum()
        f = o.eos_forward(np.asarray(s[0], float), s[2], s[3])
        return U, rho, s[1][d], s[2], f["a"]
    UL, rL, uL, pL, aL = prims(L)
    UR, rR, uR, pR, aR = prims(R)
    ub, ab = 0.5 * (uL + uR), 0.5 * (aL + aR)
    SL, SR = min(ub - ab, uL - aL), max(ub + ab, uR + aR)
    Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))
    FL, FR = o.physical_flux(d, L), o.physical_flux(d, R)

    def ustar(U, rho, uK, pK, SK):
        c = rho * (SK - uK) / (SK - Ss)
        Us = U * 0
        Us[:ns] = U[:ns] / rho * c
        for j in range(D):
            Us[ns + j] = c * (Ss if j == d else U[ns + j] / rho)
        E = U[ns + D]
        Us[ns + D] = c * (E / rho + (Ss - uK) * (Ss + pK / (rho * (SK - uK))))
        return Us
    if SL >= 0:
        return FL
    if Ss >= 0:
        return FL + SL * (ustar(UL, rL, uL, pL, SL) - UL)
    if SR > 0:
        return FR + SR * (ustar(UR, rR, uR, pR, SR) - UR)
    return FR


def test_hllc_matches_four_region_form(o2):
    rng = np.random.default_rng(11)
    for _ in range(100):
        L, R = _random_state(o2, rng, 300.0), _random_state(o2, rng, 300.0)
        for d in range(2):
            F = o2.hllc(d, L, R)
            Ft = _toro_hllc(o2, d, L, R)
            assert np.allclose(F, Ft, rtol=1e-10, atol=1e-9 * np.abs(Ft).max())
