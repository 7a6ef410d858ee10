"""Characteristic (NSCBC-type) boundaries on the GPU (Sec. 3.5; the reading
in the oracle: per boundary cell, the characteristic fields of Appendix A
that leave the domain keep the cell's values, those that enter take the
far-field state's), through the C ABI:
  * the stage right-hand side against the oracle, element by element, on an
    acoustic pulse reaching each boundary, a subsonic channel with an
    inflow of another composition (2D, periodic in y) and a supersonic
    inflow; the bound and the flag comparison of test_gpu_parity;
  * 100 SSP-RK3 steps against the oracle (state-scaled L1 <= 1e-10, or
    within ten times the oracle's own divergence from a perturbed start);
  * the pulse leaves the domain on the FP64 and the mixed path with the
    oracle's reflection;
  * the adjoint entries refuse the boundary (not differentiated)."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W
from tests.test_gpu_parity import NTH, _steps_parity, rhs_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_2504_14063_gb300 import binding
    return binding


CASES = {
    "pulse_right": lambda: W.acoustic_tube(n=120, amplitude=2e-2, direction=1, x0=0.85),
    "pulse_left": lambda: W.acoustic_tube(n=120, amplitude=2e-2, direction=-1, x0=0.15),
    "channel_2d": lambda: W.acoustic_tube(n=60, amplitude=1e-2, u0=80.0, he=0.1, he_far=0.3, ny=10, x0=0.1),
    "supersonic_inflow": lambda: W.acoustic_tube(n=80, amplitude=1e-3, u0=600.0, he=0.2, he_far=0.05,
                                                 bc_hi=W.BC_ZEROGRAD),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_rhs_parity_characteristic_boundaries(mp, case):
    rhs_parity(mp, CASES[case](), pre_steps=4)


@pytest.mark.parametrize("case, conditioned", [("pulse_right", True), ("channel_2d", False)])
def test_100_steps_characteristic_boundaries(mp, case, conditioned):
    """The 2D channel's 100-step map moves by 1e-12 from a 1e-14 start in the
    oracle itself: there the GPU stays within ten times that divergence."""
    _steps_parity(mp, CASES[case](), 100, conditioned=conditioned)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pulse_leaves_the_domain(mp, precision):
    """The right-running pulse of the oracle pin (amplitude 1e-3, 200 cells)
    after it has left: what remains is the reflection, the oracle's 2.1e-4
    of the amplitude on the FP64 path; the mixed path's FP32 fluxes add
    their rounding (2^-24 of the pressure ~ 6e-3 of this amplitude)."""
    p = W.acoustic_tube(n=200, amplitude=1e-3, direction=1)
    o = Oracle(p, nthreads=NTH)
    t_end = (0.5 + 4 * 0.05) / p.a0
    Uo, _, _, st = o.run(o.init_state(), 10 ** 6, t_end=t_end)
    assert st == 0
    ref = np.abs(o.primitives(Uo)["P"] - 1e5).max() / 1e2
    ctx = mp.Context(p, precision=mp.FP64 if precision == "fp64" else mp.MIXED)
    U = ctx.init_state(torch.from_numpy(p.prim))
    ctx.step_n(U, 10 ** 4, t_end=t_end)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    res = np.abs(o.primitives(U.cpu().numpy())["P"] - 1e5).max() / 1e2
    print(f"{precision}: reflected / incident amplitude {res:.3e} (oracle {ref:.3e})")
    if precision == "fp64":
        assert res == pytest.approx(ref, rel=1e-6)
    else:
        assert res < ref + 1e-2


def test_adjoint_refuses_characteristic_boundaries(mp):
    p = W.acoustic_tube(n=32, amplitude=1e-3)
    ctx = mp.Context(p)
    U = ctx.init_state(torch.from_numpy(p.prim))
    with pytest.raises(mp.MpmcError) as e:
        ctx.rhs_adjoint(U, None, None, torch.ones_like(U))
    assert e.value.code == mp.INVALID_ARG
