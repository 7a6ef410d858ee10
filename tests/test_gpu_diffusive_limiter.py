"""The diffusive flux (species diffusion with its enthalpy flux, viscous
stress and heat conduction) through the flux limiter that Sec. 3.3.2 applies
to the regularization flux: added to the admissible flux when both
pseudo-updates stay admissible, else not added at that face (flag
MPMC_F_DIFF_DROPPED).  On the GPU, through the C ABI:
  * FP64 stage right-hand side against the oracle on a two-phase field with
    viscosity x 100 and a forward-Euler stage three times the CFL step
    (about 200 faces drop their diffusive flux), flags compared;
  * the mixed path on the same case within the mixed-precision bound, away
    from faces whose FP32 decision differs;
  * the discrete adjoint replaying the decision (dot products against the
    oracle's forward-mode tangent);
  * the 64^3 droplet field (two liquids, trace gas inside the droplets, CDI
    and diffusion) for 120 SSP-RK3 steps on both paths: without the limit
    on the diffusive flux the oracle itself leaves the admissible set at
    step 53 (trace helium inside a droplet turns negative)."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W
from tests.test_gpu_adjoint import _dot_check
from tests.test_gpu_parity import NTH, _cuda, _face_mask_to_cells, _gross, _split_flags, rhs_parity
from tests.test_oracle_jvp import _state_and_dir

pytestmark = pytest.mark.gpu
RK1 = (1.0, 0.0, 1.0)


@pytest.fixture(scope="module")
def mp():
    from paper_2504_14063_gb300 import binding
    return binding


def _strong_diffusion(viscous=0):
    p = W.random_smooth_2d(24, 20, seed=3, cdi=1, diffusion=1)
    for s in p.species:
        s.mu *= 100.0
    p.model.mu_liquid *= 100.0
    if viscous:
        p.model.viscous = 1
        p.model.lambda_liquid *= 100.0
    return p


@pytest.mark.parametrize("viscous", [0, 1])
def test_rhs_parity_with_dropped_diffusive_flux(mp, viscous):
    rep = {}
    rhs_parity(mp, _strong_diffusion(viscous), pre_steps=0, rk=RK1, report=rep, dt_scale=3.0)
    print(f"diffusive flux dropped: oracle {rep['diff_dropped']}, GPU {rep['diff_dropped_gpu']} faces")
    assert rep["diff_dropped"] > 100
    assert abs(rep["diff_dropped_gpu"] - rep["diff_dropped"]) <= rep["ties"]


def test_mixed_rhs_with_dropped_diffusive_flux(mp):
    p = _strong_diffusion()
    o = Oracle(p, nthreads=NTH)
    U = o.init_state()
    dt, G, _ = o.dt_gamma(U)
    dt *= 3.0
    _, Lo, flo, st = o.stage(U, U, RK1, dt, G, flags=True)
    assert st == 0
    F, _ = o.face_fluxes(U, U, RK1, dt, G)
    ctx = mp.Context(p, precision=mp.MIXED)
    flg = torch.zeros(ctx.nfaces_total, dtype=torch.int32, device="cuda")
    Lg = ctx.rhs(_cuda(U), stage=dict(U_n=_cuda(U), rk=RK1, dt=dt, Gamma=G), flags=flg).cpu().numpy()
    assert ctx.status() == 0
    flg = flg.cpu().numpy().view(np.uint32)
    drop_o, drop_g = (flo & 256) != 0, (flg & 256) != 0
    differ = _split_flags(p, (flg & np.uint32(0x13F)) != (flo & np.uint32(0x13F)))
    nd = int(sum(x.sum() for x in differ))
    keep = ~_face_mask_to_cells(p, differ) if nd else np.ones(Lo.shape[1:], dtype=bool)
    rng = np.random.default_rng(1)
    jit = lambda A: A * (1.0 + 2.0 ** -24 * rng.standard_normal(A.shape))
    Lt = o.stage(jit(U), jit(U), RK1, dt, G)[1]
    T32 = np.array([np.abs(Lt[v] - Lo[v])[keep].sum() for v in range(p.ns + p.dim + 1)])
    num = np.array([np.abs(Lg[v] - Lo[v])[keep].sum() for v in range(p.ns + p.dim + 1)])
    ref = np.array([np.abs(Lo[v])[keep].sum() for v in range(p.ns + p.dim + 1)])
    bound = 1e-4 * ref + 1e-7 * _gross(p, F) + 10.0 * T32
    print(f"mixed: dropped oracle {int(drop_o.sum())}, GPU {int(drop_g.sum())}; faces with another decision "
          f"{nd}; rel err {np.array2string(num / ref, precision=2)}")
    assert drop_o.sum() > 100
    assert nd <= 0.05 * drop_o.sum()
    assert np.all(num <= bound)


@pytest.mark.parametrize("viscous", [0, 1])
def test_rhs_adjoint_with_dropped_diffusive_flux(mp, viscous):
    """<lam, J dU> from the oracle's tangent (the drop decision held at the
    point) = <J^T lam, dU> from the GPU adjoint (the decision replayed from
    the forward flags)."""
    p = _strong_diffusion(viscous)
    o = Oracle(p, nthreads=NTH)
    U, dU = _state_and_dir(o, p, np.random.default_rng(5))
    dt, G, _ = o.dt_gamma(U)
    dt *= 3.0
    _, _, flo, _ = o.stage(U, U, RK1, dt, G, flags=True)
    assert ((flo & 256) != 0).sum() > 100
    _, dL, st = o.stage_jvp(U, U, dU, RK1, dt, G)
    assert st == 0
    lam = np.random.default_rng(9).standard_normal(U.shape)
    ctx = mp.Context(p)
    lamU = ctx.rhs_adjoint(_cuda(U), dict(U_n=_cuda(U), rk=RK1, dt=dt, Gamma=G), None, _cuda(lam)).cpu().numpy()
    assert ctx.status() == 0
    _dot_check((lam * dL).sum(), (lamU * dU).sum(), np.abs(lam * dL).sum(),
               f"rhs with dropped diffusive flux, viscous={viscous}")


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_droplet_field_64_stays_admissible(mp, precision):
    p = W.droplet_field_3d(n=64)
    ctx = mp.Context(p, precision=getattr(mp, precision))
    U = ctx.init_state(torch.from_numpy(p.prim))
    ctx.stats(reset=True)
    ctx.step_n(U, 120)
    torch.cuda.synchronize()
    st = ctx.status()
    s = ctx.stats(reset=True)
    rho = U[:p.ns].sum(0)
    ymin = float((U[:p.ns] / rho).min())
    print(f"64^3 droplet field, {precision}, 120 steps: status {st}, min rhoY/rho {ymin:.3e}, "
          f"diffusive flux dropped at {s['diff_dropped']} of {s['faces']} faces")
    assert st == 0
    assert ymin >= -1e-14
    assert s["diff_dropped"] > 0
