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


def test_studies_are_the_3d_configurations():
    assert bench.STUDIES["droplet_field_3d"][1] == 500
    assert bench.STUDIES["shock_droplet_3d"][1] == 200


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
