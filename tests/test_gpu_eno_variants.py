"""Sec. 4.1's other ENO-type interpolations (WENO5-JS, TENO5, TENO6) on the
FP64 GPU path, through the C ABI, against the oracle: the right-hand side of
one stage on 1D / 2D / 3D configurations (same bound as the WENO5-Z parity
tests), 100 SSP-RK3 steps, one step of the benchmarked workload at full
size, and Table DropAdvectionIECResults after one flow-through; the mixed
path's FP32 versions within the mixed-precision bound; the discrete adjoint
of each (dot products against the oracle's forward-mode tangent)."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W
from tests.test_gpu_adjoint import _dot_check
from tests.test_gpu_parity import L1_TOL, NTH, _cuda, _gross, _steps_parity, rhs_parity, scaled_l1
from tests.test_oracle_jvp import _modulated, _state_and_dir

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
KINDS = {"WENO5JS": W.RECON_WENO5JS, "TENO5": W.RECON_TENO5, "TENO6": W.RECON_TENO6}


@pytest.fixture(scope="module")
def mp():
    from paper_2504_14063_gb300 import binding
    return binding


def _with(p, name):
    p.model.recon = KINDS[name]
    return p


CASES = {
    "slab_1d_cdi": (lambda: W.interface_advection_1d(n=400, cdi=1), 3),
    "shock_bubble_2d": (lambda: W.shock_bubble_2d(nx=100, ny=52, seed=1), 60),
    "periodic_cdi_diffusion_2d": (lambda: W.random_smooth_2d(41, 35, seed=5, cdi=1, diffusion=1), 2),
    "droplet_field_3d": (lambda: W.droplet_field_3d(n=22, ndrops=4, seed=2, rmin=3.0, rmax=5.0), 2),
    "shock_droplet_3d": (lambda: W.shock_droplet_3d(n=24, seed=4), 2),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("name", list(KINDS))
def test_rhs_parity(mp, name, case):
    make, pre = CASES[case]
    rhs_parity(mp, _with(make(), name), pre_steps=pre)


@pytest.mark.parametrize("name", list(KINDS))
def test_100_steps_shock_bubble_2d_cdi(mp, name):
    _steps_parity(mp, _with(W.shock_bubble_2d(nx=72, ny=40, seed=0, liquid_cols=24), name), 100,
                  conditioned=False)


@pytest.mark.parametrize("name", list(KINDS))
def test_full_size_shock_bubble_step(mp, name):
    """The benchmarked workload (1024 x 512, CDI on) with this interpolation:
    one SSP-RK3 step against the oracle."""
    p = _with(W.shock_bubble_2d(nx=1024, ny=512, seed=0), name)
    o = Oracle(p, nthreads=NTH)
    U0 = o.init_state()
    Uo, dt, st = o.rk_step(U0)
    assert st == 0
    ctx = mp.Context(p)
    Ug = _cuda(U0)
    ctx.rk_step(Ug)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    err = scaled_l1(Ug.cpu().numpy(), Uo, p.ns, p.dim)
    print(f"full-size shock_bubble_2d, {name}, one step: scaled L1 err {np.array2string(err, precision=2)}")
    assert err.max() <= L1_TOL, err


@pytest.mark.parametrize("name", list(KINDS))
def test_paper_droplet_advection_golden_on_gpu(mp, name):
    """Table DropAdvectionIECResults, rows WENO5JS / TENO5 / TENO6: one
    flow-through of the 100-cell droplet (end time enforced on the device);
    WENO5-JS and TENO5 within 5x of the printed errors, TENO6 below its
    printed round-off pile-up."""
    g = json.load(open(os.path.join(HERE, "golden", "drop_advection_iec_eno_variants.json")))
    ref = g["max_rel_err"][name]
    p = _with(W.paper_droplet_advection(n=100, cdi=1), name)
    ctx = mp.Context(p)
    U = ctx.init_state(torch.from_numpy(p.prim))
    nmax = 120000
    hist = torch.zeros(nmax, dtype=torch.float64, device="cuda")
    ctx.step_n(U, nmax, dt_out=hist, t_end=p.t_end)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert float(hist.sum()) == pytest.approx(p.t_end, rel=1e-12)
    o = Oracle(p)
    Uh = U.cpu().numpy()
    pr = o.primitives(Uh)
    u = Uh[p.ns] / Uh[:p.ns].sum(0)
    errs = {"P": np.abs(pr["P"] / 101325.0 - 1).max(), "T": np.abs(pr["T"] / 297.0 - 1).max(),
            "u": np.abs(u / 5.0 - 1).max()}
    print(f"GPU droplet advection {name}: P {errs['P']:.2e} (paper {ref['P']:.2e}) T {errs['T']:.2e} "
          f"(paper {ref['T']:.2e}) u {errs['u']:.2e} (paper {ref['u']:.2e})")
    for k in ("P", "T", "u"):
        assert errs[k] <= 5 * ref[k]


@pytest.mark.parametrize("case", ["slab_1d_cdi", "shock_bubble_2d", "shock_droplet_3d"])
@pytest.mark.parametrize("name", list(KINDS))
def test_mixed_rhs_close_to_oracle(mp, name, case):
    """The mixed path's FP32 interpolation: the stage right-hand side within
    the mixed-precision bound of tests/test_gpu_mixed.py (1e-4 of the
    oracle's L1 + 1e-7 of the gross flux + 10 x the oracle's own change
    under a 2^-24 perturbation of its input)."""
    make, pre = CASES[case]
    p = _with(make(), name)
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
    print(f"mixed {name} rhs {case}: rel err {np.array2string(num / ref, precision=2)}, err/bound "
          f"{np.array2string(num / bound, precision=2)}")
    assert np.all(num <= bound)


ADJ_CASES = {
    "smooth_2d_cdi_diff": lambda: W.random_smooth_2d(24, 20, seed=3, cdi=1, diffusion=1),
    "shock_bubble_2d": lambda: _modulated(W.shock_bubble_2d(nx=48, ny=28, seed=1)),
    "droplet_3d": lambda: _modulated(W.droplet_field_3d(n=14, ndrops=2, seed=2, rmin=2.5, rmax=3.5)),
}


@pytest.mark.parametrize("case", list(ADJ_CASES))
@pytest.mark.parametrize("name", list(KINDS))
def test_rhs_adjoint_dot_product(mp, name, case):
    """<lam, J dU> from the oracle's forward-mode tangent (TENO's candidate
    selection held at the point, WENO5-JS differentiated through its weights)
    = <J^T lam, dU> from the GPU adjoint, within 1e-9 of the gross sum."""
    p = _with(ADJ_CASES[case](), name)
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
    _dot_check((lam * dL).sum(), (lamU * dU).sum(), np.abs(lam * dL).sum(), f"rhs {name} {case}")


@pytest.mark.parametrize("name", list(KINDS))
def test_rk_step_adjoint_dot_product(mp, name):
    p = _with(_modulated(W.shock_bubble_2d(nx=48, ny=28, seed=1)), name)
    o = Oracle(p, nthreads=NTH)
    U, dU = _state_and_dir(o, p, np.random.default_rng(6))
    ctx = mp.Context(p)
    dt, G = (float(x) for x in ctx.dt_gamma(_cuda(U)).cpu())
    _, dU1, st = o.rk_step_jvp(U, dU, dt, G)
    assert st == 0
    lam = np.random.default_rng(10).standard_normal(U.shape)
    lam_n = ctx.rk_step_adjoint(_cuda(U), _cuda(lam), dt=dt).cpu().numpy()
    assert ctx.status() == 0
    _dot_check((lam * dU1).sum(), (lam_n * dU).sum(), np.abs(lam * dU1).sum(), f"rk step {name}")
