"""Pins of the oracle's thermodynamics (Sec. 2.2-2.3 and Eq. SpeedOfSound)
against textbook special cases, thermodynamic identities and brute force."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W


def _oracle(species, **kw):
    n = 4
    pr = np.zeros((len(species) + 3, 1, 1, n))
    pr[0] = 1.0
    pr[-2] = 1e5
    pr[-1] = 300.0
    p = W.Problem("pt", 1, (n, 1, 1), 1e-3, list(species), W.Model(), pr)
    return Oracle(p, **kw)


def test_ideal_gas_pressure_is_gamma_minus_one_rho_e():
    """Pure ideal gas: P = (gamma - 1) rho e, T = e / cv (textbook)."""
    o = _oracle([W.AIR])
    rng = np.random.default_rng(0)
    for _ in range(50):
        rho, e = rng.uniform(0.1, 10.0), rng.uniform(1e4, 1e6)
        P, T, st = o.eos_pt([1.0], e, 1.0 / rho)
        assert st == 0
        assert P == pytest.approx((W.AIR.gamma - 1.0) * rho * e, rel=1e-14)
        assert T == pytest.approx(e / W.AIR.cv, rel=1e-14)


def test_stiffened_gas_pressure():
    """Pure stiffened gas: P = (gamma - 1) rho (e - q) - gamma Pinf (textbook);
    negative pressures (tension) are returned as they are."""
    liq = W.LIQUID_SG
    o = _oracle([liq])
    rng = np.random.default_rng(1)
    for _ in range(50):
        rho = rng.uniform(900.0, 1100.0)
        e = rng.uniform(1.5e6, 2.5e6)
        P, T, st = o.eos_pt([1.0], e, 1.0 / rho)
        Pref = (liq.gamma - 1.0) * rho * e - liq.gamma * liq.pinf
        assert P == pytest.approx(Pref, abs=1e-12 * liq.gamma * liq.pinf)


def _forward(o, Y, P, T):
    f = o.eos_forward(np.asarray(Y, float), P, T)
    return f["e"], 1.0 / f["rho"]


@pytest.mark.parametrize("species", [[W.LIQUID_SG, W.GAS_C1], [W.AIR, W.HELIUM, W.LIQUID_SG],
                                     [W.WATER_NASG, W.AIR_TABLE]])
def test_closed_form_round_trip(species):
    """(P, T, Y) -> (e, v) -> (P, T): the inversion of Eq. NASG_P recovers the
    state; error measured against P + Pinf (the conditioning of the liquid)."""
    o = _oracle(species)
    rng = np.random.default_rng(2)
    pinf = max(s.pinf for s in species)
    for _ in range(200):
        Y = rng.dirichlet(np.ones(len(species)))
        P, T = rng.uniform(2e4, 5e6), rng.uniform(200.0, 900.0)
        e, v = _forward(o, Y, P, T)
        P2, T2, st = o.eos_pt(Y, e, v)
        assert st == 0
        assert abs(P2 - P) <= 2e-13 * (abs(P) + pinf)
        assert T2 == pytest.approx(T, rel=1e-11)


def test_iterative_equals_closed_form():
    """The bisection on the common-pressure residual reproduces the closed
    form wherever the latter applies (one stiffened component)."""
    sp = [W.AIR, W.HELIUM, W.LIQUID_SG]
    oc, oi = _oracle(sp), _oracle(sp, eos_iterative=1)
    rng = np.random.default_rng(3)
    for _ in range(200):
        Y = rng.dirichlet(np.ones(3))
        e, v = _forward(oc, Y, rng.uniform(5e4, 1e6), rng.uniform(250.0, 600.0))
        Pc, Tc, _ = oc.eos_pt(Y, e, v)
        Pi, Ti, st = oi.eos_pt(Y, e, v)
        assert st == 0
        assert abs(Pc - Pi) <= 1e-12 * (abs(Pc) + W.LIQUID_SG.pinf)
        assert Ti == pytest.approx(Tc, rel=1e-11)


def test_several_liquids_unique_root_brute_force():
    """Two stiffened liquids with distinct Pinf plus two gases: the residual
    has exactly one sign change on the admissible interval (dense scan) and
    the solver lands on it; the state round-trips."""
    sp = [W.LIQUID_SG, W.LIQUID_B, W.AIR, W.HELIUM]
    o = _oracle(sp)
    rng = np.random.default_rng(4)
    Rk = np.array([(s.gamma - 1) * s.cv for s in sp])
    pinf = np.array([s.pinf for s in sp])
    cv = np.array([s.cv for s in sp])
    q = np.array([s.q for s in sp])
    b = np.array([s.b for s in sp])
    for trial in range(60):
        Y = rng.dirichlet(np.ones(4))
        if trial % 3 == 0:
            Y[2:] = 0.0   # liquids only: tension admissible
            Y /= Y.sum()
        P, T = rng.uniform(2e4, 5e6), rng.uniform(250.0, 700.0)
        e, v = _forward(o, Y, P, T)
        P2, T2, st = o.eos_pt(Y, e, v)
        assert st == 0
        assert abs(P2 - P) <= 1e-12 * (abs(P) + pinf.max())
        assert T2 == pytest.approx(T, rel=1e-10)
        # brute-force scan of the residual written from NASG_T1 = NASG_T2
        Ep = (e - Y @ q) / (v - Y @ b)
        lo = -min(pinf[Y > 0])
        grid = lo + np.geomspace(1e-6, 1e12, 20001)
        f = ((Y * Rk)[None, :] * (Ep - pinf)[None, :] / (grid[:, None] + pinf[None, :])).sum(1) - Y @ cv
        changes = np.nonzero(np.diff(np.sign(f)) != 0)[0]
        assert len(changes) == 1
        assert grid[changes[0]] <= P2 <= grid[changes[0] + 1]


@pytest.mark.parametrize("sp,Pinf", [([W.AIR], 0.0), ([W.LIQUID_SG], W.LIQUID_SG.pinf)])
def test_sound_speed_special_cases(sp, Pinf):
    """a^2 = gamma (P + Pinf) / rho for a pure (stiffened) gas."""
    o = _oracle(sp)
    g = sp[0].gamma
    for P, T in [(1e5, 300.0), (3e6, 500.0), (2e4, 250.0)]:
        f = o.eos_forward([1.0], P, T)
        assert f["a"] ** 2 == pytest.approx(g * (P + Pinf) / f["rho"], rel=1e-13)


def test_mixture_sound_speed_from_isentropic_derivative():
    """Eq. SpeedOfSound against the identity a^2 = (dP/drho)_e + P/rho^2 (dP/de)_rho,
    both derivatives taken by central differences of the oracle's inversion
    at fixed mass fractions."""
    for sp in ([W.AIR, W.HELIUM, W.LIQUID_SG], [W.WATER_NASG, W.AIR_TABLE],
               [W.LIQUID_SG, W.LIQUID_B, W.AIR]):
        o = _oracle(sp)
        rng = np.random.default_rng(5)
        for _ in range(20):
            Y = rng.dirichlet(np.ones(len(sp)))
            P, T = rng.uniform(5e4, 2e6), rng.uniform(250.0, 600.0)
            f = o.eos_forward(Y, P, T)
            rho, e = f["rho"], f["e"]
            hr, he = rho * 1e-6, abs(e) * 1e-6
            dPdr = (o.eos_pt(Y, e, 1 / (rho + hr))[0] - o.eos_pt(Y, e, 1 / (rho - hr))[0]) / (2 * hr)
            dPde = (o.eos_pt(Y, e + he, 1 / rho)[0] - o.eos_pt(Y, e - he, 1 / rho)[0]) / (2 * he)
            a2 = dPdr + P / rho ** 2 * dPde
            assert f["a"] ** 2 == pytest.approx(a2, rel=2e-5)
