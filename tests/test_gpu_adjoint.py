"""Discrete adjoint on the GPU (through the C ABI) against the oracle's
forward-mode tangents (the CPU reference gradient):
  * dot-product tests <lam, J dU> (oracle tangent) = <J^T lam, dU> (GPU
    adjoint) for the stage right-hand side, one SSP-RK3 step, the
    initialisation and the primitive recovery, with dt and Gamma frozen;
  * on tiny grids the whole J^T lam element by element, J assembled column
    by column from oracle tangents;
  * determinism: tape replay, recorded stage states and repeated calls give
    bit-identical adjoints (no atomic accumulation anywhere).
Tolerance: the two sides differentiate the same discrete map in different
operation orders; their agreement is bounded by rounding in the gross sum
sum_i |lam_i (J dU)_i| (the products before they cancel), relative 1e-9."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W
from tests.test_oracle_jvp import _modulated, _state_and_dir

pytestmark = pytest.mark.gpu
RTOL = 1e-9


@pytest.fixture(scope="module")
def mp():
    from paper_2504_14063_gb300 import binding
    return binding


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _cases():
    return [
        ("smooth_2d_cdi_diff", lambda: W.random_smooth_2d(24, 20, seed=3, cdi=1, diffusion=1)),
        ("slab_1d_cdi", lambda: _modulated(W.interface_advection_1d(n=47, cdi=1))),
        ("shock_bubble_2d", lambda: _modulated(W.shock_bubble_2d(nx=48, ny=28, seed=1))),
        ("droplet_3d", lambda: _modulated(W.droplet_field_3d(n=14, ndrops=2, seed=2, rmin=2.5, rmax=3.5))),
    ]


def _dot_check(a, b, gross, what):
    err = abs(a - b) / gross
    print(f"{what}: <lam, J dU> {a:.12e}  <J^T lam, dU> {b:.12e}  rel to gross {err:.2e}")
    assert err < RTOL


@pytest.mark.parametrize("name,make", _cases())
@pytest.mark.parametrize("rk", [(1.0, 0.0, 1.0), (0.75, 0.25, 0.25)])
def test_rhs_adjoint_dot_product(mp, name, make, rk):
    p = make()
    o = Oracle(p, nthreads=8)
    U, dU = _state_and_dir(o, p, np.random.default_rng(5))
    dt, G, _ = o.dt_gamma(U)
    # U_n: a nearby state, so that the flux limiter sees U_n != U^(k)
    Un = U if rk[1] == 0.0 else o.rk_step(U, 0.3 * dt)[0]
    _, dL, st = o.stage_jvp(Un, U, dU, rk, dt, G)
    assert st == 0
    lam = np.random.default_rng(9).standard_normal(U.shape)
    ctx = mp.Context(p)
    stage = dict(U_n=_cuda(Un), rk=rk, dt=dt, Gamma=G)
    lamU = ctx.rhs_adjoint(_cuda(U), stage, None, _cuda(lam)).cpu().numpy()
    assert ctx.status() == 0
    _dot_check((lam * dL).sum(), (lamU * dU).sum(), np.abs(lam * dL).sum(), f"rhs {name} rk={rk}")


@pytest.mark.parametrize("name,make", _cases()[:3])
def test_rk_step_adjoint_dot_product(mp, name, make):
    p = make()
    o = Oracle(p, nthreads=8)
    U, dU = _state_and_dir(o, p, np.random.default_rng(6))
    ctx = mp.Context(p)
    # the GPU's own CFL step (it may differ from the oracle's in the last
    # bits, which may move a limiter decision)
    dt, G = (float(x) for x in ctx.dt_gamma(_cuda(U)).cpu())
    _, dU1, st = o.rk_step_jvp(U, dU, dt, G)
    assert st == 0
    lam = np.random.default_rng(10).standard_normal(U.shape)
    lam_n = ctx.rk_step_adjoint(_cuda(U), _cuda(lam), dt=dt).cpu().numpy()
    assert ctx.status() == 0
    _dot_check((lam * dU1).sum(), (lam_n * dU).sum(), np.abs(lam * dU1).sum(), f"rk step {name}")
    # the CFL step recomputed on the device, and the stage states and flags
    # recorded by the forward step, give the same adjoint bit for bit
    lam_c = ctx.rk_step_adjoint(_cuda(U), _cuda(lam), dt=0.0).cpu().numpy()
    assert np.array_equal(lam_c, lam_n)
    Ug = _cuda(U)
    tape = torch.empty(3 * ctx.nfaces_total, dtype=torch.int32, device="cuda")
    stages = ctx.rk_step_record(Ug.clone(), dt, tape)
    lam_r = ctx.rk_step_adjoint(Ug, _cuda(lam), dt=dt, tape=tape, stages=stages).cpu().numpy()
    assert np.array_equal(lam_r, lam_n)
    lam_s = ctx.rk_step_adjoint(Ug, _cuda(lam), dt=dt, stages=stages).cpu().numpy()
    assert np.array_equal(lam_s, lam_n)
    # the primitive caches kept by the recording step stand in for their
    # recomputation, bit for bit
    wst = torch.empty(3 * ctx.cache_doubles, dtype=torch.float64, device="cuda")
    stages_w = ctx.rk_step_record(Ug.clone(), dt, tape, wstages=wst)
    assert torch.equal(stages_w, stages)
    lam_w = ctx.rk_step_adjoint(Ug, _cuda(lam), dt=dt, tape=tape, stages=stages_w, wstages=wst).cpu().numpy()
    assert np.array_equal(lam_w, lam_n)
    with pytest.raises(mp.MpmcError):
        ctx.rk_step_adjoint(Ug, _cuda(lam), dt=dt, tape=tape, wstages=wst)
    # in place
    L = _cuda(lam)
    ctx.rk_step_adjoint(Ug, L, dt=dt, lam_n=L)
    assert np.array_equal(L.cpu().numpy(), lam_n)


def test_init_and_primitives_adjoint_dot_product(mp):
    p = _modulated(W.shock_bubble_2d(nx=48, ny=28, seed=2))
    o = Oracle(p, nthreads=8)
    rng = np.random.default_rng(3)
    prim = p.prim
    dprim = prim * rng.standard_normal(prim.shape)
    U, dU, _ = o.init_state_jvp(prim, dprim)
    lamU = rng.standard_normal(U.shape)
    ctx = mp.Context(p)
    lprim = ctx.init_state_adjoint(_cuda(prim), _cuda(lamU)).cpu().numpy()
    _dot_check((lamU * dU).sum(), (lprim * dprim).sum(), np.abs(lamU * dU).sum(), "init")
    # primitive recovery: [T, P, rho, a] rows against the oracle's tangents
    _, dV = _state_and_dir(o, p, rng)
    out, dout, _ = o.primitives_jvp(U, dV)
    Wg = ctx.primitives(_cuda(U)).cpu().numpy()
    for row, key in enumerate(("T", "P", "rho", "a")):
        assert np.allclose(Wg[row], out[key], rtol=1e-12, atol=0)
    lamW = np.zeros(Wg.shape)
    lamW[:4] = rng.standard_normal((4,) + Wg.shape[1:])
    lamV = ctx.primitives_adjoint(_cuda(U), _cuda(lamW)).cpu().numpy()
    lhs = sum((lamW[r] * dout[k]).sum() for r, k in enumerate(("T", "P", "rho", "a")))
    gross = sum(np.abs(lamW[r] * dout[k]).sum() for r, k in enumerate(("T", "P", "rho", "a")))
    _dot_check(lhs, (lamV * dV).sum(), gross, "primitives")


@pytest.mark.parametrize("name,make", [
    ("slab_1d_cdi_24", lambda: _modulated(W.interface_advection_1d(n=24, cdi=1))),
    ("smooth_2d_8x6", lambda: W.random_smooth_2d(8, 6, seed=4, cdi=1, diffusion=1)),
])
def test_rhs_adjoint_full_transpose(mp, name, make):
    """J assembled from one oracle tangent per unit direction; J^T lam from
    the GPU element by element."""
    p = make()
    o = Oracle(p, nthreads=8)
    U = o.init_state()
    dt, G, _ = o.dt_gamma(U)
    rk = (1.0, 0.0, 1.0)
    n = U.size
    J = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        J[:, i] = o.stage_jvp(U, U, e.reshape(U.shape), rk, dt, G)[1].ravel()
    lam = np.random.default_rng(1).standard_normal(n)
    ref = J.T @ lam
    ctx = mp.Context(p)
    got = ctx.rhs_adjoint(_cuda(U), dict(U_n=None, rk=rk, dt=dt, Gamma=G), None,
                          _cuda(lam.reshape(U.shape))).cpu().numpy().ravel()
    gross = np.abs(J.T) @ np.abs(lam)
    err = np.abs(got - ref) / np.maximum(gross, 1e-300)
    print(f"J^T lam {name}: max elementwise error rel to gross {err.max():.2e}")
    assert err.max() < RTOL


def test_tape_replay_equals_recomputed_decisions(mp):
    p = W.shock_bubble_2d(nx=64, ny=32, seed=0)
    ctx = mp.Context(p)
    U = ctx.init_state(torch.from_numpy(p.prim))
    ctx.step_n(U, 40)
    dtG = ctx.dt_gamma(U).cpu().numpy()
    stage = dict(U_n=U, rk=(1.0, 0.0, 1.0), dt=float(dtG[0]), Gamma=float(dtG[1]))
    flags = torch.zeros(ctx.nfaces_total, dtype=torch.int32, device="cuda")
    ctx.rhs(U, stage=stage, flags=flags)
    assert int((flags != 0).sum()) > 0
    lam = torch.randn_like(U)
    a = ctx.rhs_adjoint(U, stage, flags, lam)
    b = ctx.rhs_adjoint(U, stage, None, lam)
    c = ctx.rhs_adjoint(U, stage, flags, lam)
    assert torch.equal(a, b) and torch.equal(a, c)


def test_adjoint_needs_fp64_context(mp):
    p = W.random_smooth_2d(16, 12, seed=1)
    ctx = mp.Context(p, precision=mp.MIXED)
    U = ctx.init_state(torch.from_numpy(p.prim))
    with pytest.raises(mp.MpmcError):
        ctx.rk_step_adjoint(U, torch.zeros_like(U), dt=1e-9)
