"""The 3D workloads at their full sizes on the GPU:
  * 256^3 droplet field (4 species, two stiffened liquids -> the iterative
    p-T equilibrium, CDI and diffusion, periodic);
  * 512^3 shock-droplet (134 M cells; inflow / zero gradient in x, periodic
    y and z; CDI and diffusion).
The FP64 right-hand side of the whole domain is checked against the oracle
on sub-boxes cut out of it: the right-hand side at a cell depends only on
cells within four along each axis (three for the WENO5-Z stencils, one more
for the tangential psi neighbours of the interface normal), so the oracle on
a box with a four-cell rim reproduces the box's interior whatever boundary
it uses.  Bound element by element as in test_gpu_parity: per cell and
field, 1e-12 of |L_oracle| within a local round-off floor (1e-13 of the
cell's gross flux, 1e-14 of the rounding scale of its face fluxes at the
signal speed, 10 x the method's own rounding noise there: the oracle against
its FMA-compiled twin, largest over the cell's neighbours), with the
per-field L1 form (1e-12 of the oracle's L1 + 1e-15 of the gross flux + 10 x the
oracle's own one-ulp conditioning) beside it; cells next to a face whose discrete decision differs (a tie) are
left out.  The mixed path's step is compared with the FP64 step over the
whole domain."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2504_14063_gb300 import workloads as W
from tests.test_gpu_parity import (DECISIVE, YLIM, _gross_cells, _neighbourhood_max, cellwise_parity,
                                   jitter_sensitivity, flux_scale_cells)

pytestmark = pytest.mark.gpu
RIM, HALF = 4, 8                     # 16^3 interior, 24^3 box


@pytest.fixture(scope="module")
def mp():
    from paper_2504_14063_gb300 import binding
    return binding


def _box_index(c, n, periodic):
    idx = np.arange(c - HALF - RIM, c + HALF + RIM)
    if periodic:
        return idx % n
    assert idx[0] >= 0 and idx[-1] < n
    return idx


def _sub(T, zi, yi, xi):
    """rows [:, zi, yi, xi] of a device tensor as a host array"""
    dev = T.device
    a = T.index_select(1, torch.from_numpy(zi).to(dev))
    a = a.index_select(2, torch.from_numpy(yi).to(dev))
    a = a.index_select(3, torch.from_numpy(xi).to(dev))
    return a.cpu().numpy()


def _box_parity(mp, p, ctx, U, L, flags, centers, dt, G):
    periodic = [p.bc_lo[d] == W.BC_PERIODIC for d in range(3)]
    sub = W.Problem("box", 3, (2 * (HALF + RIM),) * 3, p.dx, p.species, p.model,
                    np.zeros((p.ns + 5,) + (2 * (HALF + RIM),) * 3),
                    bc_lo=(W.BC_ZEROGRAD,) * 3, bc_hi=(W.BC_ZEROGRAD,) * 3)
    o = Oracle(sub, nthreads=8)
    twin = Oracle(sub, nthreads=8, fma=True)
    inner = (slice(None),) + (slice(RIM, RIM + 2 * HALF),) * 3
    worst = np.zeros(p.nvars)
    for c in centers:
        xi = _box_index(c[0], p.n[0], periodic[0])
        yi = _box_index(c[1], p.n[1], periodic[1])
        zi = _box_index(c[2], p.n[2], periodic[2])
        Ub = _sub(U, zi, yi, xi)
        Lg = _sub(L, zi, yi, xi)[inner]
        _, Lfull, flo, st = o.stage(Ub, Ub, (1.0, 0.0, 1.0), dt, G, flags=True)
        assert st == 0
        _, Ltw, ftw, st = twin.stage(Ub, Ub, (1.0, 0.0, 1.0), dt, G, flags=True)
        assert st == 0
        Lo = Lfull[inner]
        # decisions on the faces of the interior cells, GPU vs oracle
        bad = np.zeros(Lo.shape[1:], dtype=bool)
        off, nties, nylim = 0, 0, 0
        for d in range(3):
            nb = [2 * (HALF + RIM)] * 3
            nb[d] += 1
            fo = flo[off:off + nb[0] * nb[1] * nb[2]].reshape(nb[2], nb[1], nb[0])
            off += nb[0] * nb[1] * nb[2]
            ng = list(p.n)
            ng[d] += 1
            # global face index of box face j along d: start + j (wrapped)
            ax_idx = [xi, yi, zi]
            fidx = [a.copy() for a in ax_idx]
            st_d = c[d] - HALF - RIM
            fidx[d] = np.arange(st_d, st_d + nb[d])
            fidx[d] = fidx[d] % p.n[d] if periodic[d] else fidx[d]
            fg = flags[d][np.ix_(fidx[2], fidx[1], fidx[0])]
            ft = ftw[off - nb[0] * nb[1] * nb[2]:off].reshape(nb[2], nb[1], nb[0])
            diff = (((fg ^ fo) & DECISIVE) != 0) | (((ft ^ fo) & DECISIVE) != 0)
            ydiff = ((fg ^ fo) & YLIM) != 0
            # faces touching interior cells: box faces RIM .. RIM + 2 HALF along d
            sl = [slice(RIM, RIM + 2 * HALF)] * 3
            for s in (0, 1):
                sl_d = list(sl)
                sl_d[2 - d] = slice(RIM + s, RIM + s + 2 * HALF)
                bad |= diff[tuple(sl_d)]
            sl_f = list(sl)
            sl_f[2 - d] = slice(RIM, RIM + 2 * HALF + 1)
            nties += int(diff[tuple(sl_f)].sum())
            nylim += int(ydiff[tuple(sl_f)].sum())
        keep = ~bad
        F, _ = o.face_fluxes(Ub, Ub, (1.0, 0.0, 1.0), dt, G)
        Gv = np.array([g[tuple(s for s in inner[1:])][keep].sum() for g in _gross_cells(sub, F)])
        Tc = jitter_sensitivity(o, (Ub, Ub, (1.0, 0.0, 1.0), dt, G), Lfull)[inner]
        Tv = np.array([Tc[v][keep].sum() for v in range(p.nvars)])
        num = np.array([np.abs(Lg[v] - Lo[v])[keep].sum() for v in range(p.nvars)])
        ref = np.array([np.abs(Lo[v])[keep].sum() for v in range(p.nvars)])
        bound = 1e-12 * ref + 1e-15 * Gv + 10.0 * Tv
        print(f"{p.name} {p.n} box at {tuple(c)}: rel err {np.array2string(num / ref, precision=2)}, "
              f"err/bound {np.array2string(num / bound, precision=2)}, ties {nties}, "
              f"Y-limiter bits differing {nylim}")
        gc = _gross_cells(sub, F)[inner]
        noise = _neighbourhood_max(np.abs(Ltw - Lfull))[inner]
        sc = flux_scale_cells(o, sub, Ub)[inner]
        cellwise_parity(Lg, Lo, gc, sc, noise, keep, f"{p.name} {p.n} box at {tuple(c)} element-wise")
        assert nties <= 8
        assert nylim <= 0.01 * 3 * Lo[0].size
        assert np.all(num <= bound), (num, bound)
        worst = np.maximum(worst, num / ref)
    return worst


def _interface_center(p, n):
    """a cell on a liquid interface (phase fraction between 0.2 and 0.8)"""
    liq = sum(p.prim[k] for k in range(p.ns) if p.species[k].phase == W.LIQUID)
    z, y, x = np.nonzero((liq > 0.2) & (liq < 0.8))
    i = len(z) // 2
    return (int(x[i]), int(y[i]), int(z[i]))


@pytest.mark.parametrize("name", ["droplet_field_3d_256", "shock_droplet_3d_512"])
def test_full_size_3d_rhs_sampled_parity(mp, name):
    if name.startswith("droplet"):
        p = W.droplet_field_3d(n=256)
    else:
        p = W.shock_droplet_3d(n=512)
    n = p.n[0]
    if name.startswith("droplet"):
        # the whole periodic box is active (random velocity): an interface
        # cell and two seeded positions
        rng = np.random.default_rng(5)
        centers = [_interface_center(p, n)] + [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(2)]
    else:
        # the features of the shock-droplet: the droplet's interface, the
        # shock front (column 64 at the start) and the helium sphere's edge
        s = n / 512.0
        centers = [_interface_center(p, n), (int(round(66 * s)), int(round(200 * s)), int(round(300 * s))),
                   (int(round(289 * s)), int(round(256 * s)), int(round(250 * s)))]
    ctx = mp.Context(p)
    U = ctx.init_state(torch.from_numpy(p.prim))
    ctx.step_n(U, 2)
    dt, G = (float(v) for v in ctx.dt_gamma(U).cpu())
    flags = torch.zeros(ctx.nfaces_total, dtype=torch.int32, device="cuda")
    L = ctx.rhs(U, stage=dict(U_n=None, rk=(1.0, 0.0, 1.0), dt=dt, Gamma=G), flags=flags)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    fl = flags.cpu().numpy().view(np.uint32)
    fsplit, off = [], 0
    for d in range(3):
        ng = list(p.n)
        ng[d] += 1
        sz = ng[0] * ng[1] * ng[2]
        fsplit.append(fl[off:off + sz].reshape(ng[2], ng[1], ng[0]))
        off += sz
    _box_parity(mp, p, ctx, U, L, fsplit, centers, dt, G)
    del L, flags, fl, fsplit
    # one SSP-RK3 step of the mixed path against the FP64 step, same dt
    ctxm = mp.Context(p, precision=mp.MIXED)
    Um = U.clone()
    ctx.rk_step(U, dt)
    ctxm.rk_step(Um, dt)
    torch.cuda.synchronize()
    assert ctx.status() == 0 and ctxm.status() == 0
    ns, D = p.ns, p.dim
    rho = U[:ns].sum(0).abs().sum()
    errs = []
    for v in range(p.nvars):
        s = rho if v < ns else (rho * 1000.0 if v < ns + D else U[v].abs().sum())
        errs.append(float((Um[v] - U[v]).abs().sum() / s))
    bound = 200 * 2.0 ** -24
    print(f"{name}: mixed vs FP64 after one step, state-scaled L1 {np.array2string(np.array(errs), precision=2)} "
          f"(bound {bound:.2e})")
    # FP32 rounding of the fluxes (2^-24), amplified by the cancellation in
    # their differences: a few hundred FP32 ulps of the state at most
    assert max(errs) < bound
