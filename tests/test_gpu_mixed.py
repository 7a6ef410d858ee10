"""Mixed-precision path (FP32 reconstruction and fluxes; FP64 p-T inversion,
positivity bounds and RK accumulation) against the FP64 oracle, through the
C ABI.  Tolerances are FP32-level and each test prints the per-field L1 and
Linf errors it measures:
  * one RHS evaluation: ||L_mixed - L_oracle||_1 <= 1e-4 ||L_oracle||_1
    + 1e-7 G_v + 10 T32_v, with G_v the gross flux (as in the FP64 parity
    tests) and T32_v = ||L(U (1 + 2^-24 xi)) - L(U)||_1 the oracle's own
    change when its input is rounded at FP32 level (trace species and the
    far-field regularization balance have no FP32 relative precision);
  * n SSP-RK3 steps: state-scaled L1 error <= n * 10 * 2^-24 * max(1, A),
    A = the oracle's amplification of a 1e-14 perturbation over the n steps
    (FP32 rounding injected every step, amplified by the problem itself);
  * interface equilibrium: T and u within 1e-5; P within 2^-24 gamma Pinf / P
    (a stiff liquid's pressure is a difference of energies ~ gamma Pinf);
  * conservation: exact up to FP64 round-off (fluxes are shared by both
    neighbours and differenced in FP64).
"""
import os

import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W
from tests.test_gpu_parity import _gross, scaled_l1

pytestmark = pytest.mark.gpu
NTH = os.cpu_count() or 4


@pytest.fixture(scope="module")
def mp():
    from paper_2504_14063_gb300 import binding
    return binding


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _linf(a, b, ns, D):
    rho = np.abs(b[:ns].sum(0)).max()
    out = []
    for v in range(b.shape[0]):
        s = rho if v < ns else (rho * 1000.0 if v < ns + D else np.abs(b[v]).max())
        out.append(np.abs(a[v] - b[v]).max() / s)
    return np.array(out)


@pytest.mark.parametrize("name,make,pre", [
    ("slab", lambda: W.interface_advection_1d(n=400, cdi=1), 3),
    ("shock_bubble", lambda: W.shock_bubble_2d(nx=100, ny=52, seed=1), 60),
    ("droplet_3d", lambda: W.droplet_field_3d(n=22, ndrops=4, seed=2, rmin=3.0, rmax=5.0), 2),
    ("shock_droplet_3d", lambda: W.shock_droplet_3d(n=24, seed=4), 2),
])
def test_mixed_rhs_close_to_oracle(mp, name, make, pre):
    p = make()
    o = Oracle(p, nthreads=NTH)
    Un = o.run(o.init_state(), pre)[0]
    dt, G, _ = o.dt_gamma(Un)
    Uk = o.stage(Un, Un, (1.0, 0.0, 1.0), dt, G)[0]
    rk = (0.75, 0.25, 0.25)
    _, Lo, _, st = o.stage(Un, Uk, rk, dt, G)
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
    print(f"mixed rhs {name}: rel err {np.array2string(num / ref, precision=2)}, err/bound "
          f"{np.array2string(num / bound, precision=2)}")
    assert np.all(num <= bound)


@pytest.mark.parametrize("name,make", [
    ("shock_bubble_lc24", lambda: W.shock_bubble_2d(nx=72, ny=40, seed=0, liquid_cols=24)),
    ("droplet_3d", lambda: W.droplet_field_3d(n=24, ndrops=3, seed=2, rmin=4.0, rmax=6.0, urms=20.0)),
    ("shock_droplet_3d", lambda: W.shock_droplet_3d(n=24, seed=4)),
])
def test_mixed_100_steps_error(mp, name, make):
    n = 100
    p = make()
    o = Oracle(p, nthreads=NTH)
    U0 = o.init_state()
    Uo, _, k, st = o.run(U0, n)
    assert st == 0
    rng = np.random.default_rng(0)
    twin = scaled_l1(o.run(U0 * (1.0 + 1e-14 * rng.standard_normal(U0.shape)), n)[0], Uo, p.ns, p.dim)
    amp = max(1.0, twin.max() / 1e-14)
    ctx = mp.Context(p, precision=mp.MIXED)
    Ug = _cuda(U0)
    ctx.step_n(Ug, n)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    Ugh = Ug.cpu().numpy()
    l1 = scaled_l1(Ugh, Uo, p.ns, p.dim)
    li = _linf(Ugh, Uo, p.ns, p.dim)
    bound = n * 10.0 * 2.0 ** -24 * amp
    print(f"mixed {n} steps {name}: scaled L1 {np.array2string(l1, precision=2)}, scaled Linf "
          f"{np.array2string(li, precision=2)}, amplification {amp:.1f}, bound {bound:.2e}")
    assert l1.max() <= bound


def test_mixed_interface_equilibrium(mp):
    p = W.interface_advection_1d(n=400, cdi=1)
    o = Oracle(p)
    ctx = mp.Context(p, precision=mp.MIXED)
    U = ctx.init_state(torch.from_numpy(p.prim))
    ctx.step_n(U, 300)
    Uh = U.cpu().numpy()
    pr = o.primitives(Uh)
    u = Uh[2] / Uh[:2].sum(0)
    errs = (np.abs(pr["P"] / 1e5 - 1).max(), np.abs(pr["T"] / 300 - 1).max(), np.abs(u / 100 - 1).max())
    # a stiff liquid's pressure is a difference of energies ~ gamma Pinf:
    # one FP32 rounding of an energy flux moves P by ~2^-24 gamma Pinf / P
    kappa = max(s.gamma * s.pinf for s in p.species) / 1e5
    print(f"mixed IEC after 300 steps: P {errs[0]:.2e} (conditioning bound {2 ** -24 * kappa:.2e}) "
          f"T {errs[1]:.2e} u {errs[2]:.2e}")
    assert errs[0] < 2 ** -24 * kappa
    assert errs[1] < 1e-5 and errs[2] < 1e-5


def test_mixed_conservation(mp):
    p = W.random_smooth_2d(64, 48, seed=7, cdi=1, diffusion=1)
    ctx = mp.Context(p, precision=mp.MIXED)
    U = ctx.init_state(torch.from_numpy(p.prim))
    U0 = U.cpu().numpy()
    ctx.step_n(U, 10)
    U1 = U.cpu().numpy()
    for v in range(ctx.nv):
        assert abs(U1[v].sum() - U0[v].sum()) <= 1e-13 * np.abs(U0[v]).sum()


def test_mixed_full_size_shock_bubble_stays_admissible(mp):
    p = W.shock_bubble_2d(nx=1024, ny=512, seed=0)
    ctx = mp.Context(p, precision=mp.MIXED)
    U = ctx.init_state(torch.from_numpy(p.prim))
    ctx.step_n(U, 200)
    torch.cuda.synchronize()
    assert ctx.status() == 0


def test_precision_study_small_3d(mp):
    """bench.py's mixed-vs-FP64 study (the 3D configurations' report) on a
    small droplet field: both paths in lockstep with the FP64 path's step
    size, the study's per-field L1 against an independent host computation
    of the same norm, and the n-step mixed-precision bound above."""
    import bench
    p = W.droplet_field_3d(n=24, ndrops=4, seed=2, rmin=3.0, rmax=5.0)
    out = bench.precision_study(mp, torch, "droplet_field_3d_24", p, 6, n_timed=2, every=3, twin=True)
    assert out["status"] == {"fp64": 0, "mixed": 0, "fp64_twin": 0}
    tw = out["error_vs_fp64"]["twin"]
    assert 0.0 < max(tw["l1"].values()) < 1e-5
    assert all("twin_l1_max" in h for h in out["error_vs_fp64"]["history"])
    assert out["fp64"]["status"] == 0 and out["mixed"]["status"] == 0
    assert [h["step"] for h in out["error_vs_fp64"]["history"]] == [3, 6]
    # the same lockstep on the host side of the check
    c64, cmx = mp.Context(p), mp.Context(p, precision=mp.MIXED)
    A, B = c64.init_state(torch.from_numpy(p.prim)), cmx.init_state(torch.from_numpy(p.prim))
    t = 0.0
    for _ in range(6):
        dt = float(c64.dt_gamma(A)[0])
        c64.rk_step(A, dt)
        cmx.rk_step(B, dt)
        t += dt
    assert t == pytest.approx(out["error_vs_fp64"]["t_end"], rel=1e-15)
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    err = scaled_l1(Bh, Ah, p.ns, p.dim)
    got = np.array(list(out["error_vs_fp64"]["l1"].values()))
    print(f"study 24^3, 6 steps: L1 {np.array2string(got, precision=2)}")
    assert np.allclose(got, err, rtol=1e-6, atol=0)
    assert got.max() <= 6 * 10 * 2 ** -24 * 20
