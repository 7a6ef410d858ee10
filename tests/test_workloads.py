"""The input generators: seeded, and problems own their parameters."""
import numpy as np

from paper_2504_14063_gb300 import workloads as W


def test_problem_parameters_are_private_copies():
    p = W.random_smooth_2d(8, 8)
    mu0 = W.AIR.mu
    for s in p.species:
        s.mu *= 1e3
    p.model.cfl = 0.1
    q = W.random_smooth_2d(8, 8)
    assert W.AIR.mu == mu0 and q.species[0].mu == mu0 and q.model.cfl == 0.5


def test_generators_are_seeded_and_volume_fractions_sum_to_one():
    for gen in (lambda: W.shock_bubble_2d(64, 32, seed=3), lambda: W.droplet_field_3d(16, ndrops=2, seed=1),
                lambda: W.shock_droplet_3d(16, seed=2)):
        a, b = gen(), gen()
        assert np.array_equal(a.prim, b.prim)
        s = a.prim[:a.ns].sum(0)
        assert np.abs(s - 1.0).max() < 1e-12
        assert a.prim[:a.ns].min() >= 0.0


def test_solenoidal_velocity_is_divergence_free_spectrally():
    rng = np.random.default_rng(0)
    u = W.solenoidal_velocity(rng, (16, 16, 16), 3, 10.0)
    # spectral divergence of the discrete field vanishes to round-off
    k = np.fft.fftfreq(16) * 16
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    div = KX * np.fft.fftn(u[0]) + KY * np.fft.fftn(u[1]) + KZ * np.fft.fftn(u[2])
    assert np.abs(div).max() < 1e-9 * np.abs(np.fft.fftn(u[0])).max()
    assert abs(np.sqrt((u ** 2).sum(0).mean()) - 10.0) < 1e-9
