"""Host-side helpers of bench.py on the CPU: the state-scaled per-field
error norms that the mixed-vs-FP64 comparisons report."""
import os
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2504_14063_gb300 import workloads as W  # noqa: E402


def test_field_errors_scaling():
    p = W.random_smooth_2d(8, 6, seed=0)
    ns, D = p.ns, p.dim
    g = torch.Generator().manual_seed(0)
    A = torch.rand((ns + D + 1,) + tuple(p.n[::-1]), generator=g, dtype=torch.float64) + 0.5
    rho = A[:ns].sum(0)
    B = A.clone()
    # one perturbation per kind of field, each at its own cell
    B[1, 0, 2, 3] += 1e-3
    B[ns + 1, 0, 4, 1] -= 2e-2
    B[ns + D, 0, 0, 0] += 5e-4
    B[ns + D, 0, 1, 0] -= 1e-4
    l1, li = bench.field_errors(A, B, p)
    names = [f"rhoY_{s.name}" for s in p.species] + ["m_x", "m_y", "E"]
    assert list(l1) == names and list(li) == names
    sp = names[1]
    assert l1[sp] == pytest.approx(1e-3 / float(rho.sum()), rel=1e-9)
    assert li[sp] == pytest.approx(1e-3 / float(rho.max()), rel=1e-9)
    assert l1["m_y"] == pytest.approx(2e-2 / (1000.0 * float(rho.sum())), rel=1e-9)
    assert li["m_y"] == pytest.approx(2e-2 / (1000.0 * float(rho.max())), rel=1e-9)
    assert l1["E"] == pytest.approx(6e-4 / float(A[ns + D].sum()), rel=1e-9)
    assert li["E"] == pytest.approx(5e-4 / float(A[ns + D].max()), rel=1e-9)
    for k in (names[0], names[2], "m_x"):
        assert l1[k] == 0.0 and li[k] == 0.0


def test_studies_are_the_configurations():
    """The 1D interface advection runs one period (its step count follows
    from the initial CFL step), the 2D shock-bubble 2000 steps, the 3D
    fields 500 and 200; the 1D one reports the interface-equilibrium
    deviation of its uniform (P, T, u)."""
    assert bench.STUDIES["interface_advection_1d"][1] is None
    assert bench.STUDIES["shock_bubble_2d"][1] == 2000
    assert bench.STUDIES["droplet_field_3d"][1] == 500
    assert bench.STUDIES["shock_droplet_3d"][1] == 200
    p = bench.STUDIES["interface_advection_1d"][0](W)
    assert p.n[0] == 400 and p.t_end == pytest.approx(1.0 / 100.0)
    assert bench.IEC_STATE["interface_advection_1d"] == (1e5, 300.0, 100.0)
    q = bench.STUDIES["shock_bubble_2d"][0](W)
    assert tuple(q.n[:2]) == (1024, 512) and q.ns == 3


def test_update_flops_of_the_droplet_field():
    """The FP64 operation count behind the update's roofline: per variable
    2D - 1 for the flux differences, 1 for the scaling and 2 per RK FMA (one
    in stage 1, two after), plus the admissibility test (covolumes and
    reference energies of the NASG liquids present)."""
    p = W.droplet_field_3d(n=16)
    nv, D, ns = 8, 3, 4
    has_b = any(sp.b != 0.0 for sp in p.species)
    has_q = any(sp.q != 0.0 for sp in p.species)
    adm = (ns - 1) + 2 * ns * has_b + 2 * ns * has_q + 1 + (2 * D - 1) + 2 + 2 * has_q
    assert bench.update_flops(p, 1) == nv * (2 * D - 1 + 1 + 2) + adm
    assert bench.update_flops(p, 2) == nv * (2 * D - 1 + 1 + 4) + adm


def test_traffic_is_reported_only_for_the_captured_grid_and_sources():
    """The DRAM bytes of the ncu capture belong to the 256^3 launches of the
    kernels as captured: another grid, or changed sources, report None."""
    assert bench.traffic_of("k_face", 128) is None
    assert bench.traffic_of("no_such_kernel", bench.TRAFFIC_GRID) is None
    if bench.TRAFFIC_SHA256 is not None and bench.sources_sha256() == bench.TRAFFIC_SHA256:
        assert bench.traffic_of("k_face", bench.TRAFFIC_GRID) == bench.TRAFFIC["k_face"]
    else:
        assert bench.traffic_of("k_face", bench.TRAFFIC_GRID) is None


def test_flops_per_face_of_the_benchmark_workload():
    """The algorithmic count behind roofline.achieved: 1592 FP64 operations
    per face for 3 species in 2D with CDI and the positivity limiter; with
    diffusion on, the flux itself and its pseudo-update test add to it."""
    assert bench.flops_per_face(3, 2, 1, 0) == 1592
    nv = 3 + 2 + 1
    extra_flux = 3 + 3 * 10 + 6 * 3 + 2
    extra_test = 2 * (3 * nv) + 2 * (4 * 3 + 2 * 2 + 6)
    assert bench.flops_per_face(3, 2, 1, 1) == 1592 + extra_flux + extra_test
    assert bench.flops_per_face(3, 2, 1, 1, pos_limiter=False) < bench.flops_per_face(3, 2, 1, 1)


def test_update_and_cache_bytes_of_the_droplet_field():
    """The byte counts behind the HBM rooflines: the 256^3 droplet field keeps
    27 FP64 cache fields per cell (T, P, rho, a, 4 Y, 3 u; CDI 2 + 4 + 2;
    diffusion 8); the update moves U^n (+ U^(k) after the first stage),
    every face flux once and U^(k+1)."""
    p = W.droplet_field_3d(n=16)
    assert bench.cache_fields(p) == 27
    N, nv = 16 ** 3, 8
    faces = 3 * 17 * 16 * 16
    assert bench.update_bytes(p, 1) == 8 * nv * (2 * N + faces)
    assert bench.update_bytes(p, 2) == 8 * nv * (3 * N + faces)
    assert bench.prim_bytes(p, 27, 4) == N * (8 * nv + 4 * 27)


def test_slab_sample_keeps_the_field_and_zero_gradient_z():
    p = W.droplet_field_3d(n=16)
    q = bench.slab_of(p, 4)
    assert q.n == (16, 16, 4) and q.dx == p.dx and q.ns == p.ns
    assert q.bc_lo[2] == W.BC_ZEROGRAD and q.bc_hi[2] == W.BC_ZEROGRAD
    assert q.bc_lo[:2] == p.bc_lo[:2]
    assert (q.prim == p.prim[:, :4]).all()
