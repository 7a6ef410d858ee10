"""Pins of the oracle's interpolation limiters (Sec. 3.3.1) and of the size
of its interface-regularization flux (Sec. 3.2, Eq. MPMC_ACDI with the KEEP
split of Eqs. SkewSymmetricSplitting_Regularization*).

  * mass-fraction limiter, reading C9/C34: hand-worked cases whose results
    are written out below (sum of Y above one, below one, a negative Y, a
    sum that is one to rounding), and the properties the method fixes for
    random inputs: the limited Y sum to one and each lies between its
    clipped reconstruction and the cell value;
  * theta_T / theta_P fallbacks, reading C10: stencils on which WENO5-Z
    undershoots below zero (premise checked with the limiters off) must give
    the cell's T (P) on that side, with the flag bit set, and leave the
    other quantities alone;
  * the regularization flux on phi = (1 + tanh(x / 2w)) / 2 with phi_min = 0,
    where psi = eps x / w and the continuous regularization velocity is
        a = Gamma sech^2(x / 2w) (eps / (4 w) - 1/4)
    (zero on the equilibrium profile w = eps): the discrete face flux of each
    phase's partial density and of the energy against that closed form, with
    second-order convergence under refinement, so that a wrong factor on
    Gamma, eps, the 1/4 term, the phase density or the enthalpy fails.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W


def _three_species_oracle():
    p = W.shock_bubble_2d(nx=16, ny=8, seed=0)
    assert p.ns == 3
    return Oracle(p)


# ----------------------------------------------------------------------------
# mass-fraction limiter (reading C9: eps_k = ((1 - sum Y) / Sigma) (m_k - Y_k),
# m_k = min(Y_k, Yc_k) when sum Y > 1 and max(Y_k, Yc_k) when sum Y < 1,
# Sigma = sum_k (m_k - Y_k), after clipping Y_k at zero)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("Y, Yc, expected, active", [
    # sum 1.2: m - Y = (-0.2, -0.3, 0), Sigma = -0.5, factor 0.4
    ([0.5, 0.6, 0.1], [0.3, 0.3, 0.4], [0.42, 0.48, 0.1], True),
    # sum 0.6: m - Y = (0.3, 0, 0.2), Sigma = 0.5, factor 0.8
    ([0.2, 0.3, 0.1], [0.5, 0.2, 0.3], [0.44, 0.3, 0.26], True),
    # Y_0 < 0 clipped to 0, then sum 1.2: m - Y = (0, -0.2, -0.1), factor 2/3
    ([-0.1, 0.7, 0.5], [0.1, 0.5, 0.4], [0.0, 0.7 - 0.2 * 2 / 3, 0.5 - 0.1 * 2 / 3], True),
    # Y_0 < 0 clipped to 0 leaves a sum of exactly one: only the clip acts
    ([-0.1, 0.6, 0.4], [0.1, 0.5, 0.4], [0.0, 0.6, 0.4], True),
    # sum one to rounding: unchanged (reading C34)
    ([0.3, 0.3, 0.4 + 2.0 ** -54], [0.1, 0.5, 0.4], [0.3, 0.3, 0.4 + 2.0 ** -54], False),
])
def test_y_limiter_hand_worked_cases(Y, Yc, expected, active):
    o = _three_species_oracle()
    out, act = o.y_limiter(Y, Yc)
    assert act == active
    np.testing.assert_allclose(out, expected, rtol=0, atol=4e-16)
    if active:
        assert abs(out.sum() - 1.0) <= 4e-16


def test_y_limiter_sums_to_one_between_reconstruction_and_cell():
    """For reconstructions off the simplex (some Y < 0 or > 1, any sum), the
    limited values sum to one and each Y_k lies between max(Y_k, 0) and the
    cell value Yc_k."""
    o = _three_species_oracle()
    rng = np.random.default_rng(11)
    fired = 0
    for _ in range(4000):
        Yc = rng.dirichlet([0.5, 0.5, 0.5])
        Y = Yc + rng.normal(0.0, 0.3, 3) * rng.choice([1e-3, 1e-1, 1.0])
        out, act = o.y_limiter(Y, Yc)
        Yp = np.maximum(Y, 0.0)
        if abs(Yp.sum() - 1.0) <= 3e-15:
            continue
        assert act
        fired += 1
        assert abs(out.sum() - 1.0) <= 8e-16
        lo, hi = np.minimum(Yp, Yc), np.maximum(Yp, Yc)
        assert np.all(out >= lo - 4e-16) and np.all(out <= hi + 4e-16)
        assert np.all(out >= 0.0)
    assert fired > 3000


# ----------------------------------------------------------------------------
# theta_T / theta_P (reading C10)
# ----------------------------------------------------------------------------
# On the five cells i-2..i+2 this pattern makes WENO5-Z's value at the right
# face of cell i about -0.198 of the amplitude: every candidate stencil is
# rough, the indicators of the outer two are equal (tau5 = 0) and the
# weights fall back to the linear ones, whose five-cell formula has negative
# coefficients on cells i-1 and i+2.
_UNDERSHOOT = np.array([0.0, 1.0, 0.001, 0.0, 1.0, 0.0])
# A pattern (found by a seeded search) that undershoots on the left side of
# the face only: about -0.038 there and +0.019 on the right side.
_ONE_SIDED = np.array([0.022, 0.622, 0.178, 0.0, 1.0, 0.533])


def test_undershoot_patterns():
    o = _three_species_oracle()
    assert o.reconstruct(W.RECON_WENO5Z, _UNDERSHOOT) < -0.19
    assert o.reconstruct(W.RECON_WENO5Z, _UNDERSHOOT[::-1].copy()) < -0.19
    assert o.reconstruct(W.RECON_WENO5Z, _ONE_SIDED) < -0.035
    assert o.reconstruct(W.RECON_WENO5Z, _ONE_SIDED[::-1].copy()) > 0.015


def _line_problem(species, field, values, side, P=1e5, T=300.0):
    """1D periodic line of 16 cells at rest; `field` ('T' or 'P') takes
    `values` on the six stencil cells 5..10 of the face between cells 7 and
    8 (face 8), mirrored when side == 'R' so that the right state is the one
    that undershoots."""
    n = 16
    v = np.asarray(values, dtype=np.float64)
    if side == "R":
        v = v[::-1]
    prim = np.zeros((len(species) + 3, 1, 1, n))
    prim[0] = 1.0
    prim[len(species) + 1] = P
    prim[len(species) + 2] = T
    row = len(species) + (1 if field == "P" else 2)
    prim[row, 0, 0, 5:11] = v
    return W.Problem("theta", 1, (n, 1, 1), 1e-3, species, W.Model(), prim)


@pytest.mark.parametrize("side", ["L", "R"])
def test_theta_T_falls_back_to_the_cell_temperature(side):
    """Ideal gas at uniform P and u with the one-sided pattern in T
    (2 K + 1000 K x pattern): the unlimited face temperature is negative on
    one side; with the limiter that side takes its own cell's T and sets
    THETA_T."""
    T6 = 2.0 + 1000.0 * _ONE_SIDED
    p = _line_problem([W.AIR], "T", T6, side)
    face = (8, 0, 0)
    off = Oracle(p, pos_limiter=0)
    on = Oracle(p)
    U = on.init_state()
    L0, R0, f0, st = off.face_states(U, 0, face)
    assert st == 0 and f0 == 0
    bad, good = (L0, R0) if side == "L" else (R0, L0)
    assert bad["T"] < -30.0 and good["T"] > 10.0
    L1, R1, f1, st = on.face_states(U, 0, face)
    assert st == 0
    Tcell = on.primitives(U)["T"][0, 0]
    cell = 7 if side == "L" else 8
    lim, other = (L1, R1) if side == "L" else (R1, L1)
    bit = 1 << 0 if side == "L" else 1 << 1   # THETA_T_L / THETA_T_R
    assert f1 & 0xF == bit
    assert lim["T"] == Tcell[cell]
    assert lim["T"] == pytest.approx(T6[2], rel=1e-12)
    # nothing else of either side is touched by the T fallback
    assert other["T"] == good["T"]
    for s1, s0 in ((L1, L0), (R1, R0)):
        assert s1["P"] == s0["P"]
        np.testing.assert_array_equal(s1["u"], s0["u"])


@pytest.mark.parametrize("side", ["L", "R"])
def test_theta_P_falls_back_to_the_cell_pressure(side):
    """Stiffened liquid (Pinf 6e8 Pa) at uniform T and u with the one-sided
    pattern in P (1e5 Pa + 2.5e10 Pa x pattern): the unlimited face pressure
    is below -Pinf (v - b < 0) on one side; with the limiter that side takes
    its own cell's P and sets THETA_P."""
    P6 = 1e5 + 2.5e10 * _ONE_SIDED
    p = _line_problem([W.LIQUID_SG], "P", P6, side)
    face = (8, 0, 0)
    off = Oracle(p, pos_limiter=0)
    on = Oracle(p)
    U = on.init_state()
    L0, R0, f0, st = off.face_states(U, 0, face)
    assert st == 0 and f0 == 0
    bad, good = (L0, R0) if side == "L" else (R0, L0)
    assert bad["P"] + W.LIQUID_SG.pinf < -1e8 and good["P"] + W.LIQUID_SG.pinf > 0.0
    L1, R1, f1, st = on.face_states(U, 0, face)
    assert st == 0
    Pcell = on.primitives(U)["P"][0, 0]
    cell = 7 if side == "L" else 8
    lim, other = (L1, R1) if side == "L" else (R1, L1)
    bit = 1 << 2 if side == "L" else 1 << 3   # THETA_P_L / THETA_P_R
    assert f1 & 0xF == bit
    assert lim["P"] == Pcell[cell]
    assert lim["P"] == pytest.approx(P6[2], rel=1e-12)
    assert other["P"] == good["P"]
    for s1, s0 in ((L1, L0), (R1, R0)):
        assert s1["T"] == s0["T"]
        np.testing.assert_array_equal(s1["u"], s0["u"])


def test_theta_P_ignores_an_absent_stiffened_species():
    """Reading C10 tests P + Pinf_k only for species present on that side: a
    face pressure between -Pinf and 0 is admissible in a pure liquid but
    not where gas is present."""
    P6 = 1e5 + 2.0e9 * _UNDERSHOOT       # WENO5-Z value ~ -3.9e8 Pa
    o = _three_species_oracle()
    assert -W.LIQUID_SG.pinf < 1e5 + 2.0e9 * o.reconstruct(0, _UNDERSHOOT) < 0.0
    liq = _line_problem([W.LIQUID_SG], "P", P6, "L")
    on = Oracle(liq)
    U = on.init_state()
    L1, R1, f1, _ = on.face_states(U, 0, (8, 0, 0))
    assert f1 & 0xC == 0 and L1["P"] < 0.0 and R1["P"] < 0.0
    # the same pressures in a liquid-gas mixture of uniform mass fractions
    # (0.999 liquid, 0.001 air): the mass-fraction rows of the
    # characteristic basis are the identity, so the face keeps Y_air = 0.001
    # and P + Pinf_air = P < 0 is refused on both sides
    sp = [W.LIQUID_SG, W.AIR]
    Y = np.array([0.999, 0.001])
    mix = _line_problem(sp, "P", P6, "L")
    P = mix.prim[3, 0, 0]
    v = np.stack([(s.gamma - 1.0) * s.cv * 300.0 / (P + s.pinf) + s.b for s in sp])   # Eq. NASG_EOS
    alpha = Y[:, None] * v / (Y[:, None] * v).sum(0)
    mix.prim[0, 0, 0], mix.prim[1, 0, 0] = alpha[0], alpha[1]
    on2 = Oracle(mix)
    U2 = on2.init_state()
    L2, R2, f2, _ = on2.face_states(U2, 0, (8, 0, 0))
    assert f2 & 0xC == 0xC
    Pc = on2.primitives(U2)["P"][0, 0]
    assert L2["P"] == Pc[7] and R2["P"] == Pc[8]
    np.testing.assert_allclose(L2["Y"], Y, rtol=1e-12)


# ----------------------------------------------------------------------------
# size of the regularization flux
# ----------------------------------------------------------------------------
EPS = 1e-3      # CDI length scale [m]
GAMMA = 10.0    # regularization velocity scale [m/s]
P0, T0 = 1e5, 300.0


def _phase_density_enthalpy(s):
    """rho_p and h_p of a one-species phase at (P0, T0) from Eq. NASG_EOS"""
    v = (s.gamma - 1.0) * s.cv * T0 / (P0 + s.pinf) + s.b
    return 1.0 / v, s.gamma * s.cv * T0 + s.b * P0 + s.q


def _cdi_face_fluxes(w, cells_per_w):
    """Face fluxes of a 1D liquid/gas line at rest with phi_liquid =
    (1 + tanh(x / 2w)) / 2 sampled at cell centres, phi_min = 0, fixed Gamma;
    returns (x of the faces, fluxes [nv, faces])."""
    dx = w / cells_per_w
    n = 40 * cells_per_w                  # the line spans [-20 w, 20 w]
    x = -20.0 * w + (np.arange(n) + 0.5) * dx
    phi = 0.5 * (1.0 + np.tanh(x / (2.0 * w)))
    prim = np.zeros((5, 1, 1, n))
    prim[0, 0, 0], prim[1, 0, 0] = phi, 1.0 - phi
    prim[3], prim[4] = P0, T0
    model = W.Model(cdi=1, phi_min=0.0, cdi_eps=EPS, cdi_gamma=GAMMA, pos_limiter=0)
    p = W.Problem("cdi_tanh", 1, (n, 1, 1), dx, [W.LIQUID_SG, W.GAS_C1], model, prim,
                  bc_lo=(W.BC_ZEROGRAD,) * 3, bc_hi=(W.BC_ZEROGRAD,) * 3)
    o = Oracle(p, nthreads=1)
    U = o.init_state()
    F, st = o.face_fluxes(U, U, (1.0, 0.0, 1.0), 0.0, GAMMA)
    assert st == 0
    xf = -20.0 * w + np.arange(n + 1) * dx
    return xf, F[0][:, 0, 0, :]


def _closed_form(xf, w):
    """continuous fluxes [liquid mass, gas mass, energy] at x = xf"""
    a = GAMMA * (EPS / (4.0 * w) - 0.25) / np.cosh(xf / (2.0 * w)) ** 2
    rl, hl = _phase_density_enthalpy(W.LIQUID_SG)
    rg, hg = _phase_density_enthalpy(W.GAS_C1)
    return np.array([-rl * a, rg * a, -(rl * hl - rg * hg) * a])


@pytest.mark.parametrize("w_over_eps", [2.0, 0.5])
def test_cdi_flux_matches_closed_form_with_second_order(w_over_eps):
    """Profiles twice too thick (sharpened: liquid flux into the liquid) and
    twice too thin (widened): at the faces x = 0 and x = +-w the discrete
    fluxes of both partial densities and of the energy approach the closed
    form at second order."""
    w = w_over_eps * EPS
    errs = []
    for cpw in (4, 8, 16, 32):
        xf, F = _cdi_face_fluxes(w, cpw)
        n0 = 20 * cpw
        sel = [n0 - cpw, n0, n0 + cpw]
        assert np.allclose(xf[sel], [-w, 0.0, w], rtol=0, atol=1e-12 * w)
        exact = np.stack([_closed_form(xf[f], w) for f in sel], axis=1)   # [3, 3]
        got = F[[0, 1, 3]][:, sel]
        scale = np.abs(exact).max(axis=1)
        errs.append((np.abs(got - exact).max(axis=1) / scale).max())
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    print(f"w = {w_over_eps} eps: relative errors {errs}, orders {order}")
    assert errs[-1] < 2e-3
    assert np.all(order > 1.9)


def test_cdi_flux_vanishes_on_the_equilibrium_profile():
    """w = eps: the continuous flux is zero; the discrete one is the
    central difference's truncation error, falling at second order against
    the size Gamma rho_l / 4 of either of its two terms."""
    rl, _ = _phase_density_enthalpy(W.LIQUID_SG)
    ref = GAMMA * rl / 4.0
    errs = []
    for cpw in (4, 8, 16, 32):
        _, F = _cdi_face_fluxes(EPS, cpw)
        errs.append(np.abs(F[0]).max() / ref)
    errs = np.array(errs)
    assert errs[-1] < 1e-3
    assert np.all(np.log2(errs[:-1] / errs[1:]) > 1.9)
