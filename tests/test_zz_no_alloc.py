"""mpmc_rhs_noalloc, the right-hand side for callers that cannot allocate
device memory (its scratch is one fixed device array inside the library),
against mpmc_rhs through the C ABI: same inputs, bit-identical result (both
run the same FP64 kernels in the same order), on two calls in a row so that
the contents the first call leaves in the shared array cannot leak into the
second, with an explicit RK stage and with no stage (a forward-Euler stage
whose CFL step and Gamma come from U on the device).  Collected last on
purpose."""
import ctypes

import pytest
import torch

from paper_2504_14063_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    from paper_2504_14063_gb300 import binding
    f = binding.lib.mpmc_rhs_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(binding.Grid), ctypes.POINTER(binding.Eos), ctypes.POINTER(binding.ModelC),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(binding.StageC),
                  ctypes.POINTER(ctypes.c_size_t)]
    return binding


def _noalloc(mp, p, U, stage):
    g, e, m = mp.structs_from_problem(p)
    sc = None
    if stage is not None:
        sc = mp.StageC()
        sc.U_n = stage["U_n"].data_ptr()
        sc.rk0, sc.rk1, sc.rk2 = stage["rk"]
        sc.dt, sc.Gamma = stage["dt"], stage["Gamma"]
    out = torch.full_like(U, float("nan"))
    need = ctypes.c_size_t(0)
    rc = mp.lib.mpmc_rhs_noalloc(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                 ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.byref(sc) if sc is not None else None, ctypes.byref(need))
    assert rc == mp.OK, rc
    assert 0 < need.value <= 32 * 2 ** 20
    return out


def _same(a, b):
    assert bool(torch.isfinite(a).all())
    assert torch.equal(a, b), float((a - b).abs().max())


def test_noalloc_rhs_matches_rhs_on_two_calls(mp):
    p = W.shock_bubble_2d(nx=96, ny=40, seed=1)          # inflow, walls, CDI
    q = W.random_smooth_2d(40, 36, seed=2, cdi=1, diffusion=1)  # periodic, diffusion
    for prob in (p, q):
        ctx = mp.Context(prob)
        Un = ctx.init_state(torch.from_numpy(prob.prim))
        dtG = ctx.dt_gamma(Un).cpu().numpy()
        stage = dict(U_n=Un, rk=(0.75, 0.25, 0.25), dt=float(dtG[0]), Gamma=float(dtG[1]))
        Uk = Un.clone()
        ctx.rk_step(Uk, float(dtG[0]))
        for call in range(2):
            ref = ctx.rhs(Uk, stage=stage)
            got = _noalloc(mp, prob, Uk, stage)
            torch.cuda.synchronize()
            _same(got, ref)
            # no stage: forward Euler from Uk with its own CFL step and Gamma
            ref0 = ctx.rhs(Uk)
            got0 = _noalloc(mp, prob, Uk, None)
            torch.cuda.synchronize()
            _same(got0, ref0)
            assert not torch.equal(got0, got)
            ctx.rk_step(Uk, float(dtG[0]))   # a different input for the second call


def test_noalloc_rejects_grids_beyond_its_scratch(mp):
    p = W.shock_bubble_2d(nx=1024, ny=512, seed=0)
    g, e, m = mp.structs_from_problem(p)
    need = ctypes.c_size_t(0)
    rc = mp.lib.mpmc_rhs_noalloc(ctypes.byref(g), ctypes.byref(e), ctypes.byref(m), None, None, None, None,
                                 ctypes.byref(need))
    assert rc == mp.INVALID_ARG
    assert need.value > 32 * 2 ** 20
