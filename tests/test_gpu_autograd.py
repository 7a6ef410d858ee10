"""torch.autograd front end of the discrete adjoint: checkpointed rollouts
against the step-by-step chain, and the gradient of a time-integrated
pressure probe with respect to the interface's Fourier amplitudes (the
shock-interface sensitivity workload, reduced in size) against central
differences of the GPU forward and against the oracle's forward-mode
derivative along random directions."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    from paper_2504_14063_gb300 import autograd
    return autograd


@pytest.fixture(scope="module")
def mp():
    from paper_2504_14063_gb300 import binding
    return binding


def _probe(p, col):
    """Unit-weight pressure probe on one column of cells (all rows)."""
    w = np.zeros(p.prim.shape[1:])
    w[..., col] = 1.0 / w[..., col].size
    return torch.from_numpy(w).cuda()


def test_rollout_checkpointing_equals_stepwise_chain(mp, ag):
    p = W.shock_interface_2d(n=64, seed=3)
    ctx = mp.Context(p)
    probe = _probe(p, 30)
    prim = torch.from_numpy(p.prim).cuda().requires_grad_(True)
    U0 = ag.init_state(ctx, prim)
    UN, J, dts = ag.rollout(ctx, U0, 23, every=5, probe=probe)
    g1, = torch.autograd.grad(J + (UN * 1e-9).sum(), prim)
    # the same functional through the plain chain of autograd steps
    prim2 = torch.from_numpy(p.prim).cuda().requires_grad_(True)
    U = ag.init_state(ctx, prim2)
    J2 = torch.zeros((), dtype=torch.float64, device="cuda")
    for k in range(23):
        U = ag.rk_step(ctx, U, float(dts[k]))
        J2 = J2 + float(dts[k]) * (ag.primitives(ctx, U)[1] * probe).sum()
    assert torch.allclose(U.detach(), UN, rtol=0, atol=0)
    assert float(abs(J2 - J)) <= 1e-15 * float(abs(J))
    g2, = torch.autograd.grad(J2 + (U * 1e-9).sum(), prim2)
    # the same rollout differentiated again
    prim3 = torch.from_numpy(p.prim).cuda().requires_grad_(True)
    UN3, J3, _ = ag.rollout(ctx, ag.init_state(ctx, prim3), 23, every=5, probe=probe)
    g3, = torch.autograd.grad(J3 + (UN3 * 1e-9).sum(), prim3)
    scale = g2.abs().max()
    rel = float((g1 - g2).abs().max() / scale)
    rep = float((g1 - g3).abs().max() / scale)
    per = [float((g1[q] - g2[q]).abs().max() / g2[q].abs().max()) for q in range(g2.shape[0])]
    print(f"checkpointed vs stepwise gradient: max rel difference {rel:.2e}; rerun {rep:.2e}; "
          f"per field {np.array2string(np.array(per), precision=2)}")
    # the same operations in the same order: bit for bit
    assert torch.equal(g1, g2) and torch.equal(g1, g3)


def _amplitude_problem(n, G):
    p = W.shock_interface_2d(n=n, seed=3)
    p.model.cdi_gamma = G       # Gamma frozen for the differences
    return p


def _J_of_amps(mp, ag, ctx, p, amps, nsteps, probe, dts=None):
    phi_l = torch.from_numpy(p.prim[2, 0]).cuda()
    a0, a1 = W.interface_fractions(p.n[0], amps, phi_l, xp=torch)
    prim = torch.from_numpy(p.prim).cuda().clone()
    prim = torch.cat([a0[None, None], a1[None, None], prim[2:]], 0)
    U0 = ag.init_state(ctx, prim)
    if dts is None:
        return ag.rollout(ctx, U0, nsteps, every=20, probe=probe)
    U = U0.detach().clone()
    J = 0.0
    for k in range(nsteps):
        ctx.rk_step(U, dts[k])
        J += dts[k] * float((ctx.primitives(U)[1] * probe).sum())
    return U, J


def test_fourier_amplitude_gradient_vs_central_differences(mp, ag):
    """Central differences away from switching points.  The discrete map has
    jumps where a limiter decision flips (of order 1e-10 of J here, e.g. the
    mass-fraction limiter's rounding-level threshold); a flip inside the
    interval [-h, h] of one component moves that component's difference
    quotient by jump / 2h, at one step size and not at the others (measured:
    6e-4 of the gradient at h = 1e-6, 1e-5 at h = 3e-6 and 1e-5).  So each
    component is differenced at h = 1e-5, 3e-6 and 1e-6, and the adjoint is
    compared with the median of the three (a flip spoils at most the one
    whose interval holds it); every step size must still agree with the
    adjoint on all but at most two components."""
    n, nsteps, G = 64, 60, 400.0
    p = _amplitude_problem(n, G)
    ctx = mp.Context(p)
    probe = _probe(p, 24)
    amps0 = W.seeded_fourier_amplitudes(3, 8, 1.0)
    amps = torch.from_numpy(amps0).cuda().requires_grad_(True)
    _, J, dts = _J_of_amps(mp, ag, ctx, p, amps, nsteps, probe)
    grad, = torch.autograd.grad(J, amps)
    grad = grad.cpu().numpy()
    dts = dts.cpu().tolist()
    hs = (1e-5, 3e-6, 1e-6)
    fd = np.zeros((len(hs),) + amps0.shape)
    for q, h in enumerate(hs):
        for m in range(8):
            for c in range(2):
                e = np.zeros_like(amps0)
                e[m, c] = h
                Jp = _J_of_amps(mp, ag, ctx, p, torch.from_numpy(amps0 + e).cuda(), nsteps, probe, dts)[1]
                Jm = _J_of_amps(mp, ag, ctx, p, torch.from_numpy(amps0 - e).cuda(), nsteps, probe, dts)[1]
                fd[q, m, c] = (Jp - Jm) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    med = np.median(fd, axis=0)
    err = np.abs(grad - med).max() / scale
    per_h = np.abs(grad[None] - fd) / scale
    print(f"dJ/d(amplitudes): max |adjoint - median central difference| / max |gradient| = {err:.2e}")
    for q, h in enumerate(hs):
        print(f"  h = {h:.0e}: max {per_h[q].max():.2e}, components above 1e-4: {int((per_h[q] > 1e-4).sum())}")
    print("adjoint", np.array2string(grad.ravel(), precision=4))
    print("fd     ", np.array2string(med.ravel(), precision=4))
    assert err < 1e-4
    for q in range(len(hs)):
        assert (per_h[q] > 1e-4).sum() <= 2


def test_fourier_amplitude_gradient_vs_oracle_tangent(mp, ag):
    """<grad J, da> (GPU adjoint) = dJ along da (oracle Dual through init,
    every RK step with the GPU's dt and the frozen Gamma, and the probe)."""
    n, nsteps, G = 48, 30, 400.0
    p = _amplitude_problem(n, G)
    ctx = mp.Context(p)
    probe = _probe(p, 18)
    amps0 = W.seeded_fourier_amplitudes(3, 8, 1.0)
    amps = torch.from_numpy(amps0).cuda().requires_grad_(True)
    _, J, dts = _J_of_amps(mp, ag, ctx, p, amps, nsteps, probe)
    grad, = torch.autograd.grad(J, amps)
    grad = grad.cpu().numpy()
    dts = dts.cpu().tolist()
    o = Oracle(p, nthreads=8)
    pw = probe.cpu().numpy()
    rng = np.random.default_rng(0)
    for trial in range(2):
        da = rng.standard_normal(amps0.shape)
        # tangent of the primitive fields along da (the geometry map only)
        phi_l = torch.from_numpy(p.prim[2, 0])
        f = lambda a: torch.stack(W.interface_fractions(n, a, phi_l, xp=torch))
        _, dfr = torch.func.jvp(f, (torch.from_numpy(amps0),), (torch.from_numpy(da),))
        prim = p.prim.copy()
        fr = f(torch.from_numpy(amps0)).numpy()
        prim[0, 0], prim[1, 0] = fr[0], fr[1]
        dprim = np.zeros_like(prim)
        dprim[0, 0], dprim[1, 0] = dfr[0].numpy(), dfr[1].numpy()
        U, dU, _ = o.init_state_jvp(prim, dprim)
        dJ = 0.0
        for k in range(nsteps):
            U, dU, st = o.rk_step_jvp(U, dU, dts[k], G)
            assert st == 0
            _, dout, _ = o.primitives_jvp(U, dU)
            dJ += dts[k] * (pw * dout["P"]).sum()
        adj = (grad * da).sum()
        rel = abs(adj - dJ) / abs(dJ)
        print(f"direction {trial}: adjoint {adj:.10e}  oracle tangent {dJ:.10e}  rel {rel:.2e}")
        assert rel < 1e-6


def _J_fixed_dt(mp, ag, ctx, p, amps, nsteps, probe, dt):
    """J of the rollout with every step of length dt, accumulated on the
    device (no host round trip per step)"""
    phi_l = torch.from_numpy(p.prim[2, 0]).cuda()
    a0, a1 = W.interface_fractions(p.n[0], amps, phi_l, xp=torch)
    prim = torch.from_numpy(p.prim).cuda().clone()
    prim = torch.cat([a0[None, None], a1[None, None], prim[2:]], 0)
    U = ctx.init_state(prim)
    J = torch.zeros((), dtype=torch.float64, device="cuda")
    for _ in range(nsteps):
        ctx.rk_step(U, dt)
        J += dt * (ctx.primitives(U)[1] * probe).sum()
    return float(J)


def test_gradient_vs_oracle_tangent_128(mp, ag):
    """The sensitivity workload reduced to 128 x 128 and 50 steps: <grad J,
    da> from the GPU adjoint against dJ along da from the oracle's
    forward-mode derivative (init, every SSP-RK3 step with the GPU's step
    lengths and frozen Gamma, the probe), two random directions."""
    n, nsteps, G = 128, 50, 400.0
    p = _amplitude_problem(n, G)
    ctx = mp.Context(p)
    probe = _probe(p, 35)
    amps0 = W.seeded_fourier_amplitudes(3, 8, 1.0)
    amps = torch.from_numpy(amps0).cuda().requires_grad_(True)
    _, J, dts = _J_of_amps(mp, ag, ctx, p, amps, nsteps, probe)
    grad, = torch.autograd.grad(J, amps)
    grad = grad.cpu().numpy()
    dts = dts.cpu().tolist()
    o = Oracle(p, nthreads=0)
    pw = probe.cpu().numpy()
    rng = np.random.default_rng(1)
    phi_l = torch.from_numpy(p.prim[2, 0])
    f = lambda a: torch.stack(W.interface_fractions(n, a, phi_l, xp=torch))
    for trial in range(2):
        da = rng.standard_normal(amps0.shape)
        _, dfr = torch.func.jvp(f, (torch.from_numpy(amps0),), (torch.from_numpy(da),))
        prim = p.prim.copy()
        fr = f(torch.from_numpy(amps0)).numpy()
        prim[0, 0], prim[1, 0] = fr[0], fr[1]
        dprim = np.zeros_like(prim)
        dprim[0, 0], dprim[1, 0] = dfr[0].numpy(), dfr[1].numpy()
        U, dU, _ = o.init_state_jvp(prim, dprim)
        dJ = 0.0
        for k in range(nsteps):
            U, dU, st = o.rk_step_jvp(U, dU, dts[k], G)
            assert st == 0
            _, dout, _ = o.primitives_jvp(U, dU)
            dJ += dts[k] * (pw * dout["P"]).sum()
        adj = (grad * da).sum()
        rel = abs(adj - dJ) / abs(dJ)
        print(f"128^2 x {nsteps}, direction {trial}: adjoint {adj:.10e}  oracle tangent {dJ:.10e}  rel {rel:.2e}")
        assert rel < 1e-6
