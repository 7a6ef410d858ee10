"""Seeded synthetic inputs shaped like the paper's test cases.

This module holds no arithmetic of the method itself (no equation of state,
no reconstruction, no flux).  It builds *primitive* initial fields --
species volume fractions alpha_k, velocity, pressure and temperature -- plus
the material and model parameters, so that the GPU library and the CPU
oracle can each convert them to conserved variables with their own EOS.

Geometry and values follow the paper's cases:
  * isothermal interface advection: Sec. 4.3.2 (inviscid droplet advection,
    Table DropAdvectionSetup), here as a liquid slab in gas;
  * 2D shock-bubble / shock-interface: Sec. 4.2.1 and 4.3.3 (Tables
    ShockBubble-AirHeliumSetup, ShockDroplet-AirWaterSetup);
  * 3D droplet fields and shock-droplet: the 3D analogues, with the
    viscosities and Schmidt numbers of Tables ShockBubble-AirHeliumSetup and
    ShockDroplet-AirWaterSetup;
  * single-phase Sod tube for the exact-Riemann pin.
The inflow state behind a shock comes from the textbook normal-shock
relations of an ideal gas (gas dynamics, not the paper's method).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

R_UNIVERSAL = 8.314462618

BC_PERIODIC, BC_WALL, BC_ZEROGRAD, BC_INFLOW, BC_CHAR = 0, 1, 2, 3, 4
LIQUID, GAS = 0, 1


@dataclasses.dataclass
class Species:
    name: str
    phase: int            # 0 liquid, 1 gas
    cv: float             # J/(kg K)
    gamma: float
    q: float = 0.0        # J/kg
    b: float = 0.0        # m^3/kg
    pinf: float = 0.0     # Pa
    W: float = 0.029      # kg/mol
    mu: float = 1.8e-5    # Pa s
    Sc: float = 1.0


def ideal_gas(name, gamma, W, mu=1.8e-5, Sc=1.0):
    return Species(name, GAS, cv=R_UNIVERSAL / W / (gamma - 1.0), gamma=gamma, W=W, mu=mu, Sc=Sc)


# Materials.  LIQUID_SG: the stiffened-gas liquid of the 1D interface case
# (gamma 4.4, Pinf 6e8 Pa, cv 1.8e3); its molar mass (water's) is a choice.
LIQUID_SG = Species("liquid", LIQUID, cv=1.8e3, gamma=4.4, pinf=6e8, W=0.018, mu=8.9e-4, Sc=1.0)
# second liquid for the several-stiffened-component equilibrium (choice)
LIQUID_B = Species("liquid_b", LIQUID, cv=1.077e3, gamma=2.35, pinf=4e8, W=0.170, mu=8.9e-4, Sc=1.0)
GAS_C1 = Species("gas", GAS, cv=7.2e2, gamma=1.4, W=0.029, mu=1.81e-5, Sc=1.0)
AIR = ideal_gas("air", 1.4, 0.029, mu=1.81e-5, Sc=1.0)
HELIUM = ideal_gas("helium", 1.67, 0.004, mu=1.96e-5, Sc=0.7)
# Table NASGMaterialParamters: water (NASG), air
WATER_NASG = Species("water", LIQUID, cv=4.185e3 / 1.0123, gamma=1.0123, q=-1.143e6, b=9.203e-4,
                     pinf=1.835e8, W=0.018, mu=8.9e-4, Sc=1.0)
AIR_TABLE = Species("air", GAS, cv=1.011e3 / 1.4, gamma=1.4, W=0.029, mu=1.81e-5, Sc=1.0)


# ENO-type interpolations (Sec. 4.1 runs all four; WENO5-Z is the default)
RECON_WENO5Z, RECON_WENO5JS, RECON_TENO5, RECON_TENO6 = 0, 1, 2, 3


@dataclasses.dataclass
class Model:
    weno_eps: float = 1e-40
    cdi: int = 0
    diffusion: int = 0
    pos_limiter: int = 1
    cdi_eps: float = 0.0          # <= 0: one cell
    cdi_gamma: float = 0.0        # <= 0: Gamma = max |u_d| each step
    phi_min: float = 1e-8
    psi_delta: float = 1e-100
    cfl: float = 0.5
    mu_liquid: float = 8.9e-4
    recon: int = RECON_WENO5Z
    viscous: int = 0              # viscous stress and heat conduction
    prandtl: float = 0.72         # gas-phase Prandtl number
    lambda_liquid: float = 0.6    # liquid heat conductivity [W/(m K)]


@dataclasses.dataclass
class Problem:
    name: str
    dim: int
    n: tuple                      # (nx, ny, nz), inactive = 1
    dx: float
    species: List[Species]
    model: Model
    prim: np.ndarray              # [ns + dim + 2, nz, ny, nx] float64
    bc_lo: tuple = (BC_PERIODIC,) * 3
    bc_hi: tuple = (BC_PERIODIC,) * 3
    inflow: Optional[np.ndarray] = None   # [ns + dim + 2]
    t_end: float = 0.0
    nsteps: int = 0

    @property
    def ns(self):
        return len(self.species)

    @property
    def ncells(self):
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def nvars(self):
        return self.ns + self.dim + 1

    def __post_init__(self):
        # private copies: callers may tune a problem's species or model
        # without touching the module's material table
        self.species = [dataclasses.replace(s) for s in self.species]
        self.model = dataclasses.replace(self.model)
        if self.model.cdi_eps <= 0.0:
            self.model.cdi_eps = self.dx
        self.prim = np.ascontiguousarray(self.prim, dtype=np.float64)


# --------------------------------------------------------------------------
# helpers (geometry and random fields only)
# --------------------------------------------------------------------------
def tanh_profile(dist, dx):
    """0.5 (1 + tanh(d / (2 dx))), d > 0 inside (Table DropAdvectionSetup)."""
    return 0.5 * (1.0 + np.tanh(dist / (2.0 * dx)))


def floored(phi, floor):
    """Phase volume fraction kept within [floor, 1 - floor].  With floor =
    phi_min the far field starts at the equilibrium of the regularization
    term (Eq. MPMC_ACDI), which relaxes phase fractions towards phi_min."""
    return np.clip(phi, floor, 1.0 - floor) if floor > 0.0 else phi


def normal_shock(mach, gamma, W, P1, T1):
    """Post-shock (P, T, u) of a shock of Mach `mach` moving into gas at rest."""
    Rg = R_UNIVERSAL / W
    m2 = mach * mach
    p_ratio = 1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0)
    r_ratio = (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    T2 = T1 * p_ratio / r_ratio
    a1 = math.sqrt(gamma * Rg * T1)
    u2 = mach * a1 * (1.0 - 1.0 / r_ratio)
    return P1 * p_ratio, T2, u2


def _prim(ns, dim, shape):
    return np.zeros((ns + dim + 2,) + tuple(shape), dtype=np.float64)


def fourier_radius(theta, R, amps):
    """R + sum_m (a_m cos m theta + b_m sin m theta), amps = [(a_m, b_m)]."""
    r = np.full_like(theta, R, dtype=np.float64)
    for m, (a, b) in enumerate(amps, start=1):
        r = r + a * np.cos(m * theta) + b * np.sin(m * theta)
    return r


def seeded_fourier_amplitudes(seed, nmodes=8, max_amp=1.0):
    """Gaussian mode amplitudes scaled so that the perturbation peaks at max_amp."""
    rng = np.random.default_rng(seed)
    ab = rng.standard_normal((nmodes, 2))
    th = np.linspace(0.0, 2.0 * np.pi, 4096, endpoint=False)
    pert = fourier_radius(th, 0.0, ab)
    return ab * (max_amp / np.abs(pert).max())


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def interface_advection_1d(n=400, cdi=0, u=100.0, P=1e5, T=300.0, periods=1.0,
                           species=None, width_cells=2.0):
    """Isothermal liquid slab 0.3 < x < 0.7 in gas on periodic [0, 1]."""
    species = species or [LIQUID_SG, GAS_C1]
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    phi = 0.5 * (np.tanh((x - 0.3) / (width_cells * dx)) - np.tanh((x - 0.7) / (width_cells * dx)))
    phi = np.clip(phi, 0.0, 1.0)
    pr = _prim(2, 1, (1, 1, n))
    pr[0, 0, 0] = phi
    pr[1, 0, 0] = 1.0 - phi
    pr[2] = u
    pr[3] = P
    pr[4] = T
    return Problem("interface_advection_1d", 1, (n, 1, 1), dx, list(species),
                   Model(cdi=cdi), pr, t_end=periods * 1.0 / abs(u))


def paper_droplet_advection(n=100, cdi=1):
    """Water (NASG) droplet in air, 100 cells, u = 5 m/s, P = 101325, T = 297
    (Table DropAdvectionSetup); the droplet is |x - 0.5| < 0.25."""
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    phi = tanh_profile(0.25 - np.abs(x - 0.5), dx)
    pr = _prim(2, 1, (1, 1, n))
    pr[0, 0, 0] = phi
    pr[1, 0, 0] = 1.0 - phi
    pr[2] = 5.0
    pr[3] = 101325.0
    pr[4] = 297.0
    return Problem("paper_droplet_advection", 1, (n, 1, 1), dx, [WATER_NASG, AIR_TABLE],
                   Model(cdi=cdi), pr, t_end=1.0 / 5.0)


def sod(n=200, gamma=1.4, W=0.029):
    """Single-phase Sod tube on [0, 1], zero-gradient ends; (rho, u, P) =
    (1, 0, 1) | (0.125, 0, 0.1) expressed through T = P W / (rho R)."""
    gas = ideal_gas("gas", gamma, W)
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    Rg = R_UNIVERSAL / W
    P = np.where(x < 0.5, 1.0, 0.1)
    rho = np.where(x < 0.5, 1.0, 0.125)
    pr = _prim(1, 1, (1, 1, n))
    pr[0] = 1.0
    pr[1] = 0.0
    pr[2, 0, 0] = P
    pr[3, 0, 0] = P / (rho * Rg)
    return Problem("sod", 1, (n, 1, 1), dx, [gas], Model(), pr,
                   bc_lo=(BC_ZEROGRAD,) * 3, bc_hi=(BC_ZEROGRAD,) * 3, t_end=0.2)


def shock_bubble_2d(nx=1024, ny=512, seed=0, mach=1.5, bubble_radius=None, liquid_cols=None,
                    shock_col=None, bubble_center=None, cdi=1, diffusion=0, nsteps=2000, phase_floor=1e-8):
    """Mach 1.5 planar shock in air moving +x into a helium bubble whose
    interface carries 8 seeded Fourier modes (peak amplitude one cell), with a
    stiffened liquid layer against a reflecting wall at x = Lx.  Inflow at
    x-, slip walls in y.  Species [air, helium, liquid]."""
    sp = [AIR, HELIUM, LIQUID_SG]
    dx = 1e-4 * (1024.0 / nx)
    s = nx / 1024.0
    R = bubble_radius if bubble_radius is not None else 64.0 * s
    lc = liquid_cols if liquid_cols is not None else int(round(96 * s))
    sc = shock_col if shock_col is not None else int(round(128 * s))
    cx, cy = bubble_center if bubble_center is not None else (256.0 * s, ny / 2.0)
    amps = seeded_fourier_amplitudes(seed, 8, 1.0)
    i = np.arange(nx) + 0.5
    j = np.arange(ny) + 0.5
    X, Y = np.meshgrid(i, j)                      # [ny, nx], cell units
    th = np.arctan2(Y - cy, X - cx)
    d_bub = fourier_radius(th, R, amps) - np.hypot(X - cx, Y - cy)
    phi_b = tanh_profile(d_bub, 1.0)
    phi_l = floored(tanh_profile(X - (nx - lc), 1.0), phase_floor)
    P1, T1 = 1e5, 300.0
    P2, T2, u2 = normal_shock(mach, AIR.gamma, AIR.W, P1, T1)
    post = X < sc
    pr = _prim(3, 2, (1, ny, nx))
    pr[0, 0] = (1.0 - phi_l) * (1.0 - phi_b)
    pr[1, 0] = (1.0 - phi_l) * phi_b
    pr[2, 0] = phi_l
    pr[3, 0] = np.where(post, u2, 0.0)
    pr[4, 0] = 0.0
    pr[5, 0] = np.where(post, P2, P1)
    pr[6, 0] = np.where(post, T2, T1)
    inflow = np.array([1.0 - phase_floor, 0.0, phase_floor, u2, 0.0, P2, T2])
    m = Model(cdi=cdi, diffusion=diffusion)
    return Problem("shock_bubble_2d", 2, (nx, ny, 1), dx, sp, m, pr,
                   bc_lo=(BC_INFLOW, BC_WALL, BC_PERIODIC), bc_hi=(BC_WALL, BC_WALL, BC_PERIODIC),
                   inflow=inflow, nsteps=nsteps)


def shock_interface_2d(n=512, seed=3, amps=None, nsteps=200):
    """512x512 form of the shock-bubble case (bubble radius 64 at (160, 256),
    liquid in the last 64 columns, wall at x = Lx); `amps` (8 x 2) are the
    interface Fourier amplitudes in cells."""
    s = n / 512.0
    p = shock_bubble_2d(nx=n, ny=n, seed=seed, bubble_radius=64.0 * s, liquid_cols=int(round(64 * s)),
                        shock_col=int(round(96 * s)), bubble_center=(160.0 * s, n / 2.0), nsteps=nsteps)
    if amps is not None:
        p = _with_amplitudes(p, n, s, np.asarray(amps, dtype=np.float64))
    p.name = "shock_interface_2d"
    return p


def interface_fractions(n, amps, phi_l, xp=np):
    """Air and helium volume fractions of the n x n shock-interface case for
    interface amplitudes `amps` (8 x 2, cells), with the liquid fraction
    phi_l [n, n] given.  xp: numpy, or torch for a differentiable map from
    the amplitudes (float64 tensors)."""
    s = n / 512.0
    R, cx, cy = 64.0 * s, 160.0 * s, n / 2.0
    if xp is np:
        i = np.arange(n) + 0.5
        X, Y = np.meshgrid(i, i)
    else:
        i = xp.arange(n, dtype=amps.dtype, device=amps.device) + 0.5
        Y, X = xp.meshgrid(i, i, indexing="ij")
    th = xp.arctan2(Y - cy, X - cx) if xp is np else xp.atan2(Y - cy, X - cx)
    r = R + 0.0 * th
    for m in range(amps.shape[0]):
        r = r + amps[m, 0] * xp.cos((m + 1) * th) + amps[m, 1] * xp.sin((m + 1) * th)
    d = r - xp.hypot(X - cx, Y - cy)
    phi_b = 0.5 * (1.0 + xp.tanh(d / 2.0))   # tanh_profile with dx = 1 cell
    return (1.0 - phi_l) * (1.0 - phi_b), (1.0 - phi_l) * phi_b


def _with_amplitudes(p, n, s, amps):
    a0, a1 = interface_fractions(n, amps, p.prim[2, 0])
    p.prim[0, 0] = a0
    p.prim[1, 0] = a1
    return p


def _wavenumbers(shape):
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.rfftfreq(nx) * nx
    return np.meshgrid(kz, ky, kx, indexing="ij")   # each [nz, ny, nx//2+1]


def _smooth_random_field(rng, shape, kmax, ncomp=1):
    """Periodic random fields made of the Fourier modes with |k| <= kmax
    (integer wavenumbers), seeded Gaussian amplitudes, synthesised by FFT."""
    KZ, KY, KX = _wavenumbers(shape)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    mask = (k2 > 0) & (k2 <= kmax * kmax)
    out = np.zeros((ncomp,) + tuple(shape))
    for q in range(ncomp):
        A = (rng.standard_normal(KX.shape) + 1j * rng.standard_normal(KX.shape)) * mask
        out[q] = np.fft.irfftn(A, s=shape, axes=(0, 1, 2))
    return out, int(mask.sum())


def solenoidal_velocity(rng, shape, kmax, urms):
    """Seeded divergence-free random field: Gaussian mode amplitudes with
    |k| <= kmax, projected normal to their wavevector, synthesised by FFT and
    scaled to the requested rms speed.  Component order (u_x, u_y, u_z)."""
    KZ, KY, KX = _wavenumbers(shape)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    mask = (k2 > 0) & (k2 <= kmax * kmax)
    A = [(rng.standard_normal(KX.shape) + 1j * rng.standard_normal(KX.shape)) * mask for _ in range(3)]
    kv = (KX, KY, KZ)
    dot = sum(kv[q] * A[q] for q in range(3))
    inv = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    u = np.stack([np.fft.irfftn(A[q] - kv[q] * dot * inv, s=shape, axes=(0, 1, 2)) for q in range(3)])
    rms = np.sqrt((u ** 2).sum(axis=0).mean())
    return u * (urms / rms)


def droplet_field_3d(n=256, ndrops=32, seed=2, rmin=8.0, rmax=20.0, urms=50.0, nsteps=500,
                     cdi=1, diffusion=1, phase_floor=1e-8):
    """Periodic box with seed-placed droplets of a two-liquid mixture
    (composition by volume U[0.2, 0.8] per droplet) in an air/helium gas whose
    helium fraction is 0.1 +- 0.05 (smooth random); solenoidal random
    velocity with u_rms = 50 m/s; P = 1e5, T = 300.  Species
    [liquid A, liquid B, air, helium].  Radii in cells scale with n/256."""
    rng = np.random.default_rng(seed)
    s = n / 256.0
    dx = 1e-5 * (256.0 / n)
    centers, radii = [], []
    tries = 0
    while len(centers) < ndrops and tries < 100000:
        tries += 1
        r = rng.uniform(rmin, rmax) * s
        c = rng.uniform(0, n, 3)
        ok = True
        for c2, r2 in zip(centers, radii):
            dd = np.abs(c - c2)
            dd = np.minimum(dd, n - dd)
            if np.linalg.norm(dd) < r + r2 + 4.0 * s:
                ok = False
                break
        if ok:
            centers.append(c)
            radii.append(r)
    comp = rng.uniform(0.2, 0.8, len(centers))
    g = np.arange(n) + 0.5
    Z, Yg, X = np.meshgrid(g, g, g, indexing="ij")
    # each cell takes the profile and the liquid composition of the droplet
    # whose surface is nearest, so that trace liquid in the gas carries a
    # continuous composition
    best = np.full((n, n, n), np.inf)
    fa = np.zeros((n, n, n))
    for c, r, ca in zip(centers, radii, comp):
        dxv = np.abs(X - c[0]); dxv = np.minimum(dxv, n - dxv)
        dyv = np.abs(Yg - c[1]); dyv = np.minimum(dyv, n - dyv)
        dzv = np.abs(Z - c[2]); dzv = np.minimum(dzv, n - dzv)
        dist = np.sqrt(dxv ** 2 + dyv ** 2 + dzv ** 2) - r
        take = dist < best
        best = np.where(take, dist, best)
        fa = np.where(take, ca, fa)
    phi = tanh_profile(-best, 1.0)
    he, _ = _smooth_random_field(rng, (n, n, n), 2)
    he = he[0]
    he = 0.1 + 0.05 * he / np.abs(he).max()
    u = solenoidal_velocity(rng, (n, n, n), 4 if n >= 16 else 1, urms)
    phi = floored(phi, phase_floor)
    pr = _prim(4, 3, (n, n, n))
    pr[0] = phi * fa
    pr[1] = phi * (1.0 - fa)
    pr[2] = (1.0 - phi) * (1.0 - he)
    pr[3] = (1.0 - phi) * he
    pr[4:7] = u
    pr[7] = 1e5
    pr[8] = 300.0
    sp = [LIQUID_SG, LIQUID_B, AIR, HELIUM]
    return Problem("droplet_field_3d", 3, (n, n, n), dx, sp, Model(cdi=cdi, diffusion=diffusion), pr,
                   nsteps=nsteps)


def shock_droplet_3d(n=512, seed=4, mach=2.0, nsteps=200, cdi=1, diffusion=1, phase_floor=1e-8):
    """Mach 2 shock in air onto a stiffened-liquid droplet (radius 48 cells at
    (160, 256, 256) for n = 512) whose surface carries a seeded perturbation
    spanning the spherical harmonics of degree <= 4 (peak one cell); a
    helium-enriched gas sphere (helium half of the gas volume, radius 32)
    downstream.  Inflow x-, zero-gradient x+, periodic y/z.  Species
    [air, helium, liquid]."""
    rng = np.random.default_rng(seed)
    s = n / 512.0
    dx = 1e-5 * (512.0 / n)
    g = np.arange(n) + 0.5
    X, Yg, Z = g[None, None, :], g[None, :, None], g[:, None, None]   # broadcast [z, y, x]
    c = np.array([160.0, 256.0, 256.0]) * s
    r = np.sqrt((X - c[0]) ** 2 + (Yg - c[1]) ** 2 + (Z - c[2]) ** 2) + 1e-30
    # all monomials of the direction cosines up to degree 4 span Y_lm, l <= 4
    mons = [(a, b, cc) for a in range(5) for b in range(5) for cc in range(5) if 0 < a + b + cc <= 4]
    coef = rng.standard_normal(len(mons))
    R0 = 48.0 * s
    # the perturbation (peak one cell) matters only near the surface: beyond
    # 21 cells the floored profile is phase_floor or 1 - phase_floor whatever
    # its value.  Its normalization uses the unit sphere of directions, which
    # the shell covers.
    shell = np.abs(r - R0) < 21.0
    idx = np.nonzero(shell)
    rs = r[idx]
    nx_ = (X[0, 0, idx[2]] - c[0]) / rs
    ny_ = (Yg[0, idx[1], 0] - c[1]) / rs
    nz_ = (Z[idx[0], 0, 0] - c[2]) / rs
    pert_s = sum(cf * nx_ ** a * ny_ ** b * nz_ ** cc for cf, (a, b, cc) in zip(coef, mons))
    pert_s = pert_s / np.abs(pert_s).max()
    d = R0 - r
    d[idx] += pert_s
    phi_l = floored(tanh_profile(d, 1.0), phase_floor)
    del d, r
    cg = np.array([320.0, 256.0, 256.0]) * s
    rg = np.sqrt((X - cg[0]) ** 2 + (Yg - cg[1]) ** 2 + (Z - cg[2]) ** 2)
    he = 0.5 * tanh_profile(32.0 * s - rg, 1.0)
    del rg
    P1, T1 = 1e5, 300.0
    P2, T2, u2 = normal_shock(mach, AIR.gamma, AIR.W, P1, T1)
    post = np.broadcast_to(X < 64.0 * s, (n, n, n))
    pr = _prim(3, 3, (n, n, n))
    pr[0] = (1.0 - phi_l) * (1.0 - he)
    pr[1] = (1.0 - phi_l) * he
    pr[2] = phi_l
    pr[3] = np.where(post, u2, 0.0)
    pr[6] = np.where(post, P2, P1)
    pr[7] = np.where(post, T2, T1)
    inflow = np.array([1.0 - phase_floor, 0.0, phase_floor, u2, 0.0, 0.0, P2, T2])
    return Problem("shock_droplet_3d", 3, (n, n, n), dx, [AIR, HELIUM, LIQUID_SG],
                   Model(cdi=cdi, diffusion=diffusion), pr,
                   bc_lo=(BC_INFLOW, BC_PERIODIC, BC_PERIODIC), bc_hi=(BC_ZEROGRAD, BC_PERIODIC, BC_PERIODIC),
                   inflow=inflow, nsteps=nsteps)


def acoustic_tube(n=200, amplitude=1e-3, u0=0.0, direction=1, bc_lo=BC_CHAR, bc_hi=BC_CHAR, ny=1,
                  x0=0.5, width=0.05, he=0.0, he_far=None, P0=1e5, T0=300.0):
    """Air (optionally with a helium mass fraction `he`) in the tube [0, 1],
    at P0, T0 and mean velocity u0, with a Gaussian acoustic pulse of
    relative amplitude `amplitude` centred at x0 running in `direction`
    (+1 / -1): the textbook linear simple wave of an ideal gas, dP =
    amplitude P0 exp(-((x - x0)/width)^2), du = direction dP/(rho0 a0),
    isentropic dT = T0 (gamma - 1)/gamma dP/P0, with the mixture's gamma and
    gas constant.  dim 1, or 2 with `ny` rows periodic in y.  The inflow
    (far-field) state is the undisturbed one, with helium fraction `he_far`
    (default `he`)."""
    he_far = he if he_far is None else he_far
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    sp = [AIR, HELIUM]
    def mix(y_he):
        Y = np.array([1.0 - y_he, y_he])
        R = sum(Y[k] * (s.gamma - 1.0) * s.cv for k, s in enumerate(sp))
        cv = sum(Y[k] * s.cv for k, s in enumerate(sp))
        return Y, R, (R + cv) / cv
    Y, R, g = mix(he)
    rho0 = P0 / (R * T0)
    a0 = math.sqrt(g * P0 / rho0)
    dP = amplitude * P0 * np.exp(-((x - x0) / width) ** 2)
    P = P0 + dP
    u = u0 + direction * dP / (rho0 * a0)
    T = T0 * (1.0 + (g - 1.0) / g * dP / P0)
    dim = 1 if ny == 1 else 2
    shape = (1, ny, n)
    pr = _prim(2, dim, shape)
    # volume fractions of an ideal-gas mixture at common P, T: the mole
    # fractions, Y_k / W_k normalized
    mol = np.array([Y[k] / s.W for k, s in enumerate(sp)])
    vol = mol / mol.sum()
    pr[0], pr[1] = vol[0], vol[1]
    pr[2] = u[None, None, :]
    if dim == 2:
        pr[3] = 0.0
    pr[2 + dim] = P[None, None, :]
    pr[3 + dim] = T[None, None, :]
    Yf, _, _ = mix(he_far)
    molf = np.array([Yf[k] / s.W for k, s in enumerate(sp)])
    volf = molf / molf.sum()
    inflow = np.array([volf[0], volf[1], u0] + ([0.0] if dim == 2 else []) + [P0, T0])
    p = Problem("acoustic_tube", dim, (n, ny, 1), dx, sp, Model(), pr,
                bc_lo=(bc_lo, BC_PERIODIC, BC_PERIODIC), bc_hi=(bc_hi, BC_PERIODIC, BC_PERIODIC), inflow=inflow)
    p.a0, p.rho0 = a0, rho0
    return p


def random_smooth_2d(nx=40, ny=32, seed=0, cdi=1, diffusion=1, bc=BC_PERIODIC, u0=30.0):
    """Small periodic two-phase three-species field with smooth random
    velocity, pressure and temperature perturbations and a blob of liquid:
    a generic state for conservation and parity checks."""
    rng = np.random.default_rng(seed)
    dx = 1e-4
    i = np.arange(nx) + 0.5
    j = np.arange(ny) + 0.5
    X, Y = np.meshgrid(i, j)
    cx, cy, R = nx * 0.45, ny * 0.55, min(nx, ny) * 0.25
    phi_l = tanh_profile(R - np.hypot(X - cx, Y - cy), 1.0)
    f, _ = _smooth_random_field(rng, (1, ny, nx), 2, ncomp=5)
    f = f[:, 0] / np.abs(f).max()
    he = 0.5 + 0.3 * f[0]
    pr = _prim(3, 2, (1, ny, nx))
    pr[0, 0] = (1.0 - phi_l) * (1.0 - he)
    pr[1, 0] = (1.0 - phi_l) * he
    pr[2, 0] = phi_l
    pr[3, 0] = u0 * (1.0 + 0.3 * f[1])
    pr[4, 0] = 0.5 * u0 * f[2]
    pr[5, 0] = 1e5 * (1.0 + 0.05 * f[3])
    pr[6, 0] = 300.0 * (1.0 + 0.05 * f[4])
    return Problem("random_smooth_2d", 2, (nx, ny, 1), dx, [AIR, HELIUM, LIQUID_SG],
                   Model(cdi=cdi, diffusion=diffusion), pr, bc_lo=(bc,) * 3, bc_hi=(bc,) * 3)


def scaled(problem_fn, **kw):
    return problem_fn(**kw)
