#!/usr/bin/env python
"""Benchmark of the MPMC hot path: SSP-RK3 steps (three right-hand-side
stages with the update fused in) of the 3D droplet field, 256^3 periodic
cells, 4 species (two stiffened liquids, air, helium) in 2 phases, CDI and
non-dilute diffusion on, on one GB300 per rank; the FP64 path and the mixed
path (FP32 bulk, FP64 EOS inversion / positivity bounds / RK accumulation).

One JSON line on rank 0:
  * `value`: device-timed cell-updates/s of the FP64 path (inputs resident
    in HBM; the state, 1.07 GB per copy, is larger than L2, so no flush);
    `mixed`: the same for the mixed path, its speedup and its per-field
    L1 / Linf error against the FP64 path after a stated number of steps
    from the initial state.  The timed steps follow those steps, from the
    developed state;
  * `e2e`: the same metric through the host-buffer C-ABI entry, copies
    included;
  * `roofline`: the FP64 face-flux kernel (the dominant one) against the
    measured FP64 FMA rate; `rooflines`: every kernel family of both paths
    against its binding pipe or HBM;
  * `cpu_baseline`: the CPU oracle on the host cores, on a 16-plane slab of
    the same field.
`--impl reference` times the CPU oracle itself on that slab (there is no
other implementation of the paper's method to install).
With N ranks (torchrun) every rank runs an independent replica (the path is
built for one GPU; the whole-job value sums the replicas).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s (FP64 vs mixed at stated L1 error); adjoint/forward time ratio"
UNIT = "cell-updates/s"
FP64_PEAK_NOMINAL = 1.25e12   # GB300 FP64, nominal (the recipe's table)
GRID_N = 256                  # the droplet field's cells per direction
CPU_SLAB_PLANES = 16          # z-planes of the field in the CPU oracle's sample
L2_BYTES = 129 * 2 ** 20

# dram__bytes_read.sum + dram__bytes_write.sum per launch of each kernel on
# the 256^3 droplet field, in bytes: an ncu capture of the same field at
# 128^3 (every launch of one SSP-RK3 step of each path: nine face launches,
# three of each other kernel, averaged) scaled by the faces (cells) of a
# 256^3 launch, 7.969 (8); the counters take more than one ncu pass, which
# the full-size workload is not captured with.  Reported only on that grid
# and while the kernels' sources hash to the captured version (None
# otherwise).
TRAFFIC_GRID = 256
TRAFFIC = {"k_face": 6.279e9, "mx::k_face": 3.762e9, "k_prim": 4.207e9, "mx::k_prim": 3.110e9,
           "k_update": 5.961e9, "mx::k_update": 5.958e9}
TRAFFIC_SOURCES = ("paper_2504_14063_gb300/csrc/mpmc_kernels.cuh", "paper_2504_14063_gb300/csrc/mpmc_device.cuh",
                   "paper_2504_14063_gb300/csrc/mpmc_kernels_d3.cu", "paper_2504_14063_gb300/csrc/mpmc_mixed.cuh",
                   "paper_2504_14063_gb300/csrc/mpmc_mixed_d3.cu", "paper_2504_14063_gb300/csrc/mpmc_update.cuh")
TRAFFIC_SHA256 = "2fe30e2cc812f9f9efc25d643d0188eb8434e4643e20d8be13770ab9422f1c4d"


def sources_sha256():
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_of(kernel, grid):
    if TRAFFIC_SHA256 is None or kernel not in TRAFFIC or grid != TRAFFIC_GRID:
        return None
    return TRAFFIC[kernel] if sources_sha256() == TRAFFIC_SHA256 else None


def flops_per_face(ns, D, cdi, diffusion, pos_limiter=True):
    """Algorithmic FP64 operations of one face (every +, -, *, /, sqrt,
    transcendental counted once; an FMA counts two), itemized in the order of
    the Godunov approach:"""
    nv = ns + D + 1
    eos_inv = 4 + 6 * ns + 10 + 5 + 2 + 4 + 3 + 7 * ns       # mixture sums, quadratic root, NASG_T1
    eos_fwd = 13 * ns + 10                                     # v, e, alpha, beta, a at (P, T, Y)
    f = 0
    f += 2 * nv + 3 * ns + 2 * D + 6                           # face average of U, decode
    f += eos_inv + eos_fwd + 8                                 # its EOS, X, rho a
    f += 6 * 8                                                 # projection of 6 cells (w1, w5, w6)
    f += 63 * 2 * (3 + ns + (D - 1))                           # WENO5-Z, both sides
    f += 2 * 8                                                 # back-projection
    if pos_limiter:
        f += 2 * (3 * ns + 6) + 2 * (ns + 1)                   # Y limiter, theta_T, theta_P
    f += 2 * (eos_fwd + 3 * ns + 2 * D + 6)                    # face states from the EOS
    f += 22 + 8 * ns + 14 * D + 20                             # HLLC
    if pos_limiter:
        f += 2 * (3 * nv) + 2 * (4 * ns + 2 * D + 6)           # pseudo-updates + admissibility
    if cdi:
        f += 2 + 1 + 6 * (D - 1) + 2 * D + 2 + 1 + 12 + 4 * ns + 8 + 3 * D + 3 + nv
        if pos_limiter:
            f += 2 * (3 * nv) + 2 * (4 * ns + 2 * D + 6)
    if diffusion:
        f += 3 + ns * 10 + 6 * ns + 2
        if pos_limiter:
            f += 2 * (3 * nv) + 2 * (4 * ns + 2 * D + 6)       # the diffusive flux's pseudo-updates
    return f


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload(n=GRID_N):
    from paper_2504_14063_gb300 import workloads as W
    return W.droplet_field_3d(n=n)


def config_of(p):
    """The workload, identical in both arms."""
    return {"workload": "droplet_field_3d", "grid": list(p.n[:p.dim]), "cells": p.ncells, "species": p.ns,
            "phases": 2, "droplets": 32, "cdi": bool(p.model.cdi), "diffusion": bool(p.model.diffusion),
            "integrator": "SSP-RK3", "cfl": p.model.cfl,
            "l2": f"inputs larger than L2 (state {p.nvars * p.ncells * 8 / 1e9:.2f} GB per copy), no flush"}


def slab_of(p, planes=CPU_SLAB_PLANES):
    """The CPU oracle's bounded sample of the workload: its first `planes`
    z-planes, periodic in x and y, zero-gradient in z."""
    from paper_2504_14063_gb300 import workloads as W
    prim = np.ascontiguousarray(p.prim[:, :planes])
    return W.Problem(p.name + "_slab", 3, (p.n[0], p.n[1], planes), p.dx, p.species, p.model, prim,
                     bc_lo=(p.bc_lo[0], p.bc_lo[1], W.BC_ZEROGRAD), bc_hi=(p.bc_hi[0], p.bc_hi[1], W.BC_ZEROGRAD))


def slab_text(q):
    return (f"SSP-RK3 steps of the oracle on a {q.n[0]}x{q.n[1]}x{q.n[2]} slab of the {q.n[0]}^3 field "
            f"(its first {q.n[2]} z-planes, zero-gradient in z), {q.ncells} cells per step")


def cpu_baseline(p, seconds=12.0, planes=CPU_SLAB_PLANES):
    """The CPU oracle, as it stands, on the host cores: SSP-RK3 steps of the
    slab sample until about `seconds` have passed."""
    from oracle import Oracle
    cores = os.cpu_count() or 1
    q = slab_of(p, planes)
    o = Oracle(q, nthreads=cores)
    U = o.init_state()
    t0 = time.perf_counter()
    n = 0
    while True:
        U = o.rk_step(U)[0]
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return {"value": q.ncells * n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} {slab_text(q)} ({el:.1f} s, OpenMP threads = {cores})"}


def field_errors(A, B, p):
    """Per-field L1 and Linf of B - A (device states), scaled by the state:
    partial densities by |rho|, momenta by |rho| x 1000 m/s, energy by |E|
    (sums for L1, maxima for Linf)."""
    ns, D = p.ns, p.dim
    rho = A[:ns].sum(0).abs()
    rho1, rhoi = float(rho.sum()), float(rho.max())
    names = [f"rhoY_{s.name}" for s in p.species] + [f"m_{'xyz'[d]}" for d in range(D)] + ["E"]
    l1, li = {}, {}
    for v in range(A.shape[0]):
        s1 = rho1 if v < ns else (rho1 * 1000.0 if v < ns + D else float(A[v].abs().sum()))
        si = rhoi if v < ns else (rhoi * 1000.0 if v < ns + D else float(A[v].abs().max()))
        d = (B[v] - A[v]).abs()
        l1[names[v]] = float(d.sum()) / s1
        li[names[v]] = float(d.max()) / si
    return l1, li


STUDIES = {
    # name: (workload, the configuration's step count; None: one period of
    # the workload's end time at its initial CFL step)
    "interface_advection_1d": (lambda W: W.interface_advection_1d(n=400), None),
    "shock_bubble_2d": (lambda W: W.shock_bubble_2d(nx=1024, ny=512), 2000),
    "droplet_field_3d": (lambda W: W.droplet_field_3d(n=256), 500),
    "shock_droplet_3d": (lambda W: W.shock_droplet_3d(n=512), 200),
}
# the uniform (P, T, u) of the interface-equilibrium workload, whose
# deviation after the run each path reports
IEC_STATE = {"interface_advection_1d": (1e5, 300.0, 100.0)}


def iec_errors(ctx, U, p, ref):
    """max |P/P0 - 1|, |T/T0 - 1|, |u/u0 - 1| over the cells (Appendix C's
    interface-equilibrium invariant)."""
    W = ctx.primitives(U)
    P0, T0, u0 = ref
    return {"P": float((W[1] / P0 - 1).abs().max()), "T": float((W[0] / T0 - 1).abs().max()),
            "u": float((W[4 + p.ns] / u0 - 1).abs().max())}


def precision_study(mp, torch, name, p, steps, n_timed=5, every=50, t_build=None, twin=False):
    """The mixed path against the FP64 path on a 3D workload at full size:
    both advanced in lockstep from the same initial state with a common
    step size (the FP64 path's CFL step, so that both reach the same
    physical times), per-field L1/Linf of the difference every `every`
    steps; throughput of each path timed separately with CUDA events over
    `n_timed` steps (CFL step on the device, after 3 warm-up steps;
    library profiling off), per-kernel times from as many further steps.
    The states exceed L2 many times over, so no flush is needed.
    twin: a third context, FP64, started from the initial state with a
    relative perturbation 2^-24 xi (xi standard normal, seed 7) and
    advanced with the same steps: its distance to the FP64 path is the
    problem's own response to rounding at FP32 level, the scale against
    which the mixed path's error is read."""
    steps = max(int(steps), 1)
    every = max(every, steps // 10)
    prim = torch.from_numpy(p.prim)
    out = {"study": name, "metric": "mixed vs FP64: per-field L1/Linf of the state difference; cell-updates/s",
           "unit": UNIT, "grid": list(p.n[:p.dim]), "cells": p.ncells, "species": p.ns,
           "cdi": bool(p.model.cdi), "diffusion": bool(p.model.diffusion), "steps": steps,
           "workload_build_s": t_build}
    perf = {}
    for label, prec in (("fp64", mp.FP64), ("mixed", mp.MIXED)):
        ctx = mp.Context(p, precision=prec)
        U = ctx.init_state(prim)
        for _ in range(3):
            ctx.rk_step(U)
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        ts = sum(timed_steps(torch, ctx, U, n_timed)) / 1e3
        clk = clocks.stop()
        kp = kernel_pass(torch, ctx, U, n_timed)
        perf[label] = {"value": p.ncells * n_timed / ts, "ms_per_step": 1e3 * ts / n_timed,
                       "kernel_ms_per_step": {k: v[0] * v[1] for k, v in kp.items()},
                       "timed_steps": n_timed, "clocks": clk, "status": ctx.status()}
        del ctx, U
        torch.cuda.empty_cache()
    perf["mixed"]["speedup_vs_fp64"] = perf["mixed"]["value"] / perf["fp64"]["value"]
    out.update(perf)

    c64, cmx = mp.Context(p), mp.Context(p, precision=mp.MIXED)
    A, B = c64.init_state(prim), cmx.init_state(prim)
    if twin:
        ctw = mp.Context(p)
        g = torch.Generator(device=A.device).manual_seed(7)
        C = A * (1.0 + 2.0 ** -24 * torch.randn(A.shape, generator=g, device=A.device, dtype=A.dtype))
    hist, t_phys = [], 0.0
    t0 = time.perf_counter()
    for n in range(1, steps + 1):
        dt = float(c64.dt_gamma(A)[0])
        c64.rk_step(A, dt)
        cmx.rk_step(B, dt)
        if twin:
            ctw.rk_step(C, dt)
        t_phys += dt
        if n % every == 0 or n == steps:
            l1, li = field_errors(A, B, p)
            hist.append({"step": n, "t": t_phys, "l1_max": max(l1.values()), "linf_max": max(li.values())})
            if twin:
                t1, ti = field_errors(A, C, p)
                hist[-1].update(twin_l1_max=max(t1.values()), twin_linf_max=max(ti.values()))
            print(json.dumps({"study": name, **hist[-1], "elapsed_s": time.perf_counter() - t0}),
                  file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    out["lockstep_s"] = time.perf_counter() - t0
    out["error_vs_fp64"] = {"steps": steps, "t_end": t_phys, "dt": "common: the FP64 path's CFL step each step",
                            "norm": "state-scaled (partial densities by rho, momenta by rho*1000 m/s, energy by E)",
                            "l1": l1, "linf": li, "history": hist}
    out["status"] = {"fp64": c64.status(), "mixed": cmx.status()}
    if name in IEC_STATE:
        # (both states are FP64 vectors; the FP64 context decodes either)
        out["iec"] = {"fp64": iec_errors(c64, A, p, IEC_STATE[name]),
                      "mixed": iec_errors(c64, B, p, IEC_STATE[name]),
                      "note": "max relative deviation of P, T, u from the uniform initial values"}
    if twin:
        out["error_vs_fp64"]["twin"] = {"perturbation": "U0 (1 + 2^-24 xi), xi standard normal, seed 7",
                                        "l1": t1, "linf": ti}
        out["status"]["fp64_twin"] = ctw.status()
    return out


def max_over_ranks(x, device):
    """The largest x over the ranks of the initialised process group (the
    slowest replica's time); x itself on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, cells, steps, seconds):
    """cell-updates/s of all ranks together: each rank advances its own replica
    of `cells` cells by `steps` steps, the job takes the slowest rank's time"""
    return world * cells * steps / seconds


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    p = workload(args.grid)
    q = slab_of(p, min(CPU_SLAB_PLANES, p.n[2]))
    from oracle import Oracle
    cores = os.cpu_count() or 1
    o = Oracle(q, nthreads=cores)
    U = o.init_state()
    for _ in range(args.warmup):
        U = o.rk_step(U)[0]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = o.rk_step(U)[0]
    el = time.perf_counter() - t0
    v = q.ncells * args.steps / el
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": config_of(p),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed {slab_text(q)}, after {args.warmup} warm-up steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def adjoint_section(mp, torch, nsteps=200, every=20, n=512):
    """Reverse mode over `nsteps` SSP-RK3 steps of the 512 x 512 shock-interface
    workload with a checkpoint every `every` steps: gradient of a
    time-integrated pressure probe (one column of cells, x = 140 n/512) with
    respect to the 16 Fourier amplitudes of the initial interface.  Forward
    and backward are timed with CUDA events; the ratio is backward/forward."""
    from paper_2504_14063_gb300 import autograd as ag
    from paper_2504_14063_gb300 import workloads as W
    p = W.shock_interface_2d(n=n, seed=3)
    ctx = mp.Context(p)
    col = int(round(140 * n / 512))
    w = np.zeros(p.prim.shape[1:])
    w[..., col] = 1.0 / w[..., col].size
    probe = torch.from_numpy(w).cuda()
    phi_l = torch.from_numpy(p.prim[2, 0]).cuda()
    rest = torch.from_numpy(p.prim[2:]).cuda()
    amps0 = torch.from_numpy(W.seeded_fourier_amplitudes(3, 8, 1.0)).cuda()

    # fixed step: the CFL step of the initial state
    dt_ic = float(ctx.dt_gamma(ctx.init_state(torch.from_numpy(p.prim)))[0])

    def forward(amps, steps):
        a0, a1 = W.interface_fractions(n, amps, phi_l, xp=torch)
        prim = torch.cat([a0[None, None], a1[None, None], rest], 0)
        U0 = ag.init_state(ctx, prim)
        return ag.rollout(ctx, U0, steps, every=every, probe=probe, dt=dt_ic)

    # warm-up (graph capture, adjoint scratch)
    a = amps0.clone().requires_grad_(True)
    _, J, _ = forward(a, 3)
    torch.autograd.grad(J, a)
    torch.cuda.synchronize()

    # one reverse step with a dense random adjoint (every face active), from
    # a developed state, stage states and flags recorded: the per-step cost
    # once the adjoint covers the whole domain
    Ud = ctx.init_state(torch.from_numpy(p.prim))
    ctx.step_n(Ud, 20)
    dt = float(ctx.dt_gamma(Ud)[0])
    tape = torch.empty(3 * ctx.nfaces_total, dtype=torch.int32, device="cuda")
    stages = ctx.rk_step_record(Ud.clone(), dt, tape)
    lam = torch.randn(Ud.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    lam_n = torch.empty_like(lam)
    Uf = Ud.clone()
    reps = 5
    ef = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    ea = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for r in range(reps):
        Uf.copy_(Ud)
        ef[r][0].record()
        ctx.rk_step(Uf, dt)
        ef[r][1].record()
    for r in range(reps):
        ea[r][0].record()
        ctx.rk_step_adjoint(Ud, lam, dt=dt, tape=tape, lam_n=lam_n, stages=stages)
        ea[r][1].record()
    torch.cuda.synchronize()
    dense_f = float(np.median([x.elapsed_time(y) for x, y in ef]))
    dense_a = float(np.median([x.elapsed_time(y) for x, y in ea]))
    del Ud, Uf, stages, tape, lam, lam_n
    # forward and backward timed alike, the library's per-launch events off
    a = amps0.clone().requires_grad_(True)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    UN, J, dts = forward(a, nsteps)
    e[1].record()
    grad, = torch.autograd.grad(J, a)
    e[2].record()
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    # the backward's per-family kernel times from a second rollout with them on
    a2 = amps0.clone().requires_grad_(True)
    _, J2, _ = forward(a2, nsteps)
    torch.cuda.synchronize()
    ctx.profile(reset=True)
    ctx.set_profiling(True)
    torch.autograd.grad(J2, a2)
    torch.cuda.synchronize()
    ctx.set_profiling(False)
    prof = ctx.profile(reset=True)
    del a2, J2
    state_mb = ctx.nv * ctx.ncells * 8 / 2 ** 20
    return {"workload": f"shock_interface_2d {n}x{n}, {nsteps} SSP-RK3 steps of fixed length (the initial CFL "
                        f"step, {dt_ic:.4e} s), checkpoint every {every} steps",
            "functional": f"sum_k dt_k mean_y P(x={col}, y, t_k); gradient w.r.t. 16 interface Fourier amplitudes",
            "forward_ms": fwd_ms, "backward_ms": bwd_ms, "ratio": bwd_ms / fwd_ms,
            "dense_step": {"forward_ms": dense_f, "adjoint_ms": dense_a, "ratio": dense_a / dense_f,
                           "note": "one SSP-RK3 step vs its reverse (stage states and flags recorded) "
                                   "with a dense random adjoint, median of 5"},
            "backward_kernel_ms": {k: v[0] for k, v in prof.items() if v[1]},
            "timing": "forward and backward each bracketed by CUDA events with the library's per-launch "
                      "events off; backward_kernel_ms from a second rollout with them on",
            "memory_mb": {"state": state_mb, "checkpoints": state_mb * len(range(0, nsteps, every)),
                          "segment_states": state_mb * (every + 1)},
            "J": float(J.detach()), "grad_norm": float(grad.detach().norm()), "status": ctx.status(),
            "note": "backward = per segment one forward replay step per step (stage states and flags "
                    "recorded) + per step the reverse of SSP-RK3"}


def timed_steps(torch, ctx, U, steps):
    """`steps` SSP-RK3 steps of ctx on U, each bracketed by CUDA events on
    torch's current stream (the context's stream is the legacy default
    stream, which synchronizes with it); library profiling off.  Returns the
    per-step times in ms."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        ev[k][0].record()
        ctx.rk_step(U)
        ev[k][1].record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def kernel_pass(torch, ctx, U, steps):
    """`steps` more steps with the library's per-launch CUDA events on its
    stream: per kernel family, (ms per launch, launches per step)."""
    ctx.profile(reset=True)
    ctx.set_profiling(True)
    for _ in range(steps):
        ctx.rk_step(U)
    torch.cuda.synchronize()
    ctx.set_profiling(False)
    prof = ctx.profile(reset=True)
    return {k: (ms / n if n else 0.0, n / steps) for k, (ms, n) in prof.items()}


def fma_peaks(mp, torch, reps=5):
    """Measured FMA rates of the FP64 and FP32 pipes (mpmc_fma_probe, eight
    independent chains per thread, 4 blocks of 256 threads per SM): the best
    of `reps` launches, CUDA events on torch's current stream, with the SM
    clock sampled over a second of repeated launches."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = 4 * sms
    out = {}
    for label, fp64, iters in (("fp64", True, 4096), ("fp32", False, 131072)):
        buf = torch.empty(blocks * 256, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
        mp.fma_probe(fp64, blocks, iters, buf)
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            flops = mp.fma_probe(fp64, blocks, iters, buf)
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3
            best = t if best is None or t < best else best
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 1.0:
            mp.fma_probe(fp64, blocks, iters, buf)
            torch.cuda.synchronize()
        clk = clocks.stop()
        out[label] = {"tflops": flops / best / 1e12, "launch_ms": best * 1e3, "flops_per_launch": flops,
                      "blocks": blocks, "threads": 256, "iters": iters, "clocks": clk}
    return out


def update_bytes(p, stage):
    """Bytes the divergence + RK update kernel moves as designed for one
    launch: U^n (and U^(k) when distinct, stages 2 and 3), each face flux of
    every direction once, and U^(k+1)."""
    nv, D, N = p.nvars, p.dim, p.ncells
    faces = sum(N // p.n[d] * (p.n[d] + 1) for d in range(D))
    states = 2 if stage == 1 else 3
    return 8 * nv * (states * N) + 8 * nv * faces


def update_flops(p, stage):
    """FP64 arithmetic of the divergence + RK update per cell as the method
    states it (comparisons not counted): per variable the D flux
    differences summed (2D - 1), the scaling by rk2 dt / dx (1) and the RK
    combination (one FMA in stage 1, two in stages 2 and 3, 2 flops each);
    the admissibility test of Eqs. PositivityReqs1/2: the density sum
    (NS - 1), the covolume and reference-energy sums (2 NS each when
    present), -YTOL rho (1), |m|^2 (2D - 1) and rho E - |m|^2/2 (2), minus
    rho sum rhoY_k q_k (2 when present)."""
    nv, D, ns = p.nvars, p.dim, p.ns
    has_b = any(getattr(sp, "b", 0.0) != 0.0 for sp in p.species)
    has_q = any(getattr(sp, "q", 0.0) != 0.0 for sp in p.species)
    per_var = (2 * D - 1) + 1 + 2 * (1 if stage == 1 else 2)
    adm = (ns - 1) + 2 * ns * has_b + 2 * ns * has_q + 1 + (2 * D - 1) + 2 + 2 * has_q
    return nv * per_var + adm


def cache_fields(p):
    """Fields of the primitive cache a context keeps per cell: T, P, rho, a,
    Y_k, u_d; with CDI phi_0, psi, (Y^c/Y_p) rho_p, h_p rho_p of both
    phases; with diffusion X^c/X_p and W^c D^c_p / W_p; with viscous terms
    mu and lambda (the layout of the library's cache)."""
    m = p.model
    return (4 + p.ns + p.dim + (4 + p.ns if m.cdi else 0) + (2 * p.ns if m.diffusion else 0)
            + (2 if m.viscous else 0))


def prim_bytes(p, n_w, wbytes):
    """Bytes of one primitive-recovery launch: U read, n_w cache fields written."""
    return p.ncells * (8 * p.nvars + wbytes * n_w)


def lockstep_error(mp, torch, p, c64, cmx, A, B, steps, every=25):
    """FP64 (A) and mixed (B) advanced in lockstep with a common step (the
    FP64 path's CFL step each step) from the same state; per-field L1/Linf
    of the difference after `steps` steps and every `every` steps."""
    hist, t_phys = [], 0.0
    l1 = li = None
    for n in range(1, steps + 1):
        dt = float(c64.dt_gamma(A)[0])
        c64.rk_step(A, dt)
        cmx.rk_step(B, dt)
        t_phys += dt
        if n % every == 0 or n == steps:
            l1, li = field_errors(A, B, p)
            hist.append({"step": n, "l1_max": max(l1.values()), "linf_max": max(li.values())})
    torch.cuda.synchronize()
    return {"steps": steps, "t_end": t_phys, "dt": "common: the FP64 path's CFL step each step",
            "norm": "state-scaled (partial densities by rho, momenta by rho*1000 m/s, energy by E)",
            "l1": l1, "linf": li, "history": hist}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=GRID_N,
                    help="cells per direction of the droplet field (256 is the benchmarked configuration)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare-steps", type=int, default=100,
                    help="steps of the FP64-vs-mixed lockstep from the initial state, before the timed steps")
    ap.add_argument("--kernel-steps", type=int, default=3)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-recon", action="store_true")
    ap.add_argument("--recon-steps", type=int, default=3)
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--study", choices=sorted(STUDIES), action="append",
                    help="instead of the benchmark line: the mixed-vs-FP64 precision study of a 3D workload "
                         "(one JSON line each)")
    ap.add_argument("--study-steps", type=int, default=None)
    ap.add_argument("--twin", action="store_true",
                    help="with --study: also an FP64 run from a 2^-24-perturbed initial state")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if args.study:
        if rank != 0:
            return 0
        from paper_2504_14063_gb300 import binding as mp
        from paper_2504_14063_gb300 import workloads as W
        for name in args.study:
            make, nsteps = STUDIES[name]
            t0 = time.perf_counter()
            p = make(W)
            t_build = time.perf_counter() - t0
            if nsteps is None:
                c = mp.Context(p)
                dt0 = float(c.dt_gamma(c.init_state(torch.from_numpy(p.prim)))[0])
                nsteps = int(np.ceil(p.t_end / dt0))
                del c
            line = precision_study(mp, torch, name, p, args.study_steps or nsteps, t_build=t_build,
                                   twin=args.twin)
            print(json.dumps(line), flush=True)
            del p
        return 0
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2504_14063_gb300 import binding as mp
    t0 = time.perf_counter()
    p = workload(args.grid)
    t_build = time.perf_counter() - t0
    prim = torch.from_numpy(p.prim)
    ctx = mp.Context(p)
    ctxm = mp.Context(p, precision=mp.MIXED)

    # ---- mixed vs FP64 from the initial state; the timed steps follow ------
    U = ctx.init_state(prim)
    Um = ctxm.init_state(prim)
    err = lockstep_error(mp, torch, p, ctx, ctxm, U, Um, args.compare_steps)

    # ---- device-timed region: FP64, then mixed ------------------------------
    for _ in range(args.warmup):
        ctx.rk_step(U)
        ctxm.rk_step(Um)
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms = timed_steps(torch, ctx, U, args.steps)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    status = ctx.status()
    stats = ctx.stats(reset=True)
    total_s = max_over_ranks(sum(step_ms) / 1e3, "cuda")
    value = whole_job_value(world, p.ncells, args.steps, total_s)

    clocks_m = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks_m.start()
    step_ms_m = timed_steps(torch, ctxm, Um, args.steps)
    if world > 1:
        dist.barrier()
    clk_m = clocks_m.stop()
    tm = max_over_ranks(sum(step_ms_m) / 1e3, "cuda")
    vm = whole_job_value(world, p.ncells, args.steps, tm)
    mstat = ctxm.status()

    # ---- per-kernel times: a separate pass with the library's events -------
    kp = kernel_pass(torch, ctx, U, args.kernel_steps)
    kpm = kernel_pass(torch, ctxm, Um, args.kernel_steps)
    launches_per_step = sum(n for _, n in kp.values())
    peaks = fma_peaks(mp, torch)
    fp64_peak = peaks["fp64"]["tflops"]
    fp32_peak = peaks["fp32"]["tflops"]
    hbm_peak, hbm_src = None, "MEASURED_PEAKS.json hbm_gbs (driver-measured copy)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        hbm_peak, hbm_src = 6800.0, "recipe fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"

    faces_per_launch = ctx.nfaces_total / p.dim
    fpf = flops_per_face(p.ns, p.dim, p.model.cdi, p.model.diffusion, p.model.pos_limiter)

    def alu(kernel, ms, peak, pipe):
        ach = fpf * faces_per_launch / (ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic_of(kernel, p.n[0]), "kernel": kernel, "pipe": pipe, "flops_per_face": fpf,
                "faces_per_launch": faces_per_launch, "avg_launch_ms": ms}

    def hbm(kernel, ms, nbytes, note):
        ach = nbytes / (ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                "traffic": traffic_of(kernel, p.n[0]), "kernel": kernel, "bytes_per_launch": nbytes,
                "avg_launch_ms": ms, "note": note}

    n_w64 = cache_fields(p)
    upd_b = (update_bytes(p, 1) + 2 * update_bytes(p, 2)) / 3.0
    upd_f = p.ncells * (update_flops(p, 1) + 2 * update_flops(p, 2)) / 3.0

    def update_roof(kernel, ms, note):
        """The update against both roofs; `bound` names the one whose time
        at its peak is the longer (the FP64 pipe on GB300)."""
        mem = hbm(kernel, ms, upd_b, note)
        ach = upd_f / (ms / 1e3) / 1e12
        fp64 = {"achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                "flops_per_launch": upd_f, "pipe": "FP64"}
        if upd_f / (fp64_peak * 1e12) > upd_b / (hbm_peak * 1e9):
            out = dict(mem, bound="alu", achieved=ach, peak=fp64_peak, unit="TFLOP/s", frac=ach / fp64_peak,
                       flops_per_launch=upd_f, pipe="FP64")
            out["hbm"] = {k: mem[k] for k in ("achieved", "peak", "unit", "frac", "bytes_per_launch")}
            return out
        return dict(mem, fp64=fp64)
    peak_note = (f"measured: mpmc_fma_probe, FP64 FMA chains, {peaks['fp64']['blocks']} blocks x 256 threads, "
                 f"best of 5 (SM clock {peaks['fp64']['clocks'].get('sm_mhz')} MHz)")
    roofline = alu("k_face", kp["face"][0], fp64_peak, "FP64")
    roofline["peak_source"] = peak_note
    rooflines = {
        "k_face": roofline,
        "mx::k_face": dict(alu("mx::k_face", kpm["face"][0], fp32_peak, "FP32"),
                           peak_source="measured: mpmc_fma_probe, FP32 FMA chains (the same algorithmic "
                                       "operation count, executed in FP32 but for the FP64 limiter re-checks)"),
        "k_update": update_roof("k_update", kp["update"][0],
                                "FP64 flux differences and RK combination; bytes and flops averaged over "
                                "the three stages"),
        "mx::k_update": update_roof("mx::k_update", kpm["update"][0], "the same body on the FP64 fluxes"),
    }
    prim_note = ("bound by the FP64 pipe, not HBM: an ncu capture of the 128^3 case shows the FP64 pipe "
                 "82-88 % active and DRAM at 2-4 % of peak; the iterative p-T solve has no fixed flop "
                 "count, so the HBM fraction of the bytes it moves is what is reported")
    rooflines["k_prim"] = hbm("k_prim", kp["prim"][0], prim_bytes(p, n_w64, 8), "FP64 p-T inversion; " + prim_note)
    rooflines["mx::k_prim"] = hbm("mx::k_prim", kpm["prim"][0], prim_bytes(p, n_w64, 4),
                                  "FP64 p-T inversion, FP32 cache; " + prim_note)
    mixed = {"value": vm, "unit": UNIT, "ms_per_step": 1e3 * tm / args.steps, "speedup_vs_fp64": vm / value,
             "clocks": clk_m, "kernel_ms_per_step": {k: v[0] * v[1] for k, v in kpm.items()},
             "error_vs_fp64": err, "status": mstat}
    del ctxm, Um
    torch.cuda.empty_cache()

    # ---- Sec. 4.1's other ENO-type interpolations and the viscous terms ----
    recon = None
    if not args.no_recon:
        import dataclasses
        from paper_2504_14063_gb300 import workloads as W
        recon = {"note": "the FP64 SSP-RK3 step of the same workload from the same developed state with each "
                         "other interpolation (WENO5-JS, TENO5, TENO6) and with viscous stress and heat "
                         "conduction on, CUDA events per step after one warm-up step"}
        variants = (("WENO5JS", dict(recon=W.RECON_WENO5JS)), ("TENO5", dict(recon=W.RECON_TENO5)),
                    ("TENO6", dict(recon=W.RECON_TENO6)), ("viscous", dict(viscous=1)))
        for rname, fields in variants:
            pr_ = dataclasses.replace(p, model=dataclasses.replace(p.model, **fields))
            ctxr = mp.Context(pr_)
            Ur = U.clone()
            ctxr.rk_step(Ur)
            torch.cuda.synchronize()
            ms_r = timed_steps(torch, ctxr, Ur, args.recon_steps)
            kr = kernel_pass(torch, ctxr, Ur, 1)
            tr = max_over_ranks(sum(ms_r) / 1e3, "cuda")
            vr = whole_job_value(world, pr_.ncells, args.recon_steps, tr)
            recon[rname] = {"value": vr, "unit": UNIT, "ms_per_step": 1e3 * tr / args.recon_steps,
                            "vs_base_step": vr / value, "steps": args.recon_steps,
                            "face_ms_per_step": kr["face"][0] * kr["face"][1], "status": ctxr.status()}
            del ctxr, Ur
            torch.cuda.empty_cache()

    adjoint = None
    if not args.no_adjoint and rank == 0:
        adjoint = adjoint_section(mp, torch, nsteps=args.adjoint_steps)

    # ---- end to end through the host-buffer entry --------------------------
    H = U.cpu().pin_memory()
    ctx.step_n_host(H, 1)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.step_n_host(H, 1)
    e2e_s = max_over_ranks(time.perf_counter() - t0, "cuda")
    nbytes = ctx.nv * ctx.ncells * 8

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(p),
            "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU",
            "timed_window": f"steps {args.compare_steps + args.warmup + 1}-"
                            f"{args.compare_steps + args.warmup + args.steps} of the field (after the "
                            f"{args.compare_steps}-step FP64-vs-mixed comparison and {args.warmup} warm-up steps)",
            "clocks": clk,
            "e2e": {"value": whole_job_value(world, p.ncells, args.steps, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "rhs_cell_evaluations_per_s": 3 * value,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "roofline": roofline,
            "rooflines": rooflines,
            "peaks": {"fp64_fma": peaks["fp64"], "fp32_fma": peaks["fp32"], "hbm_gbs": hbm_peak,
                      "hbm_source": hbm_src, "fp64_nominal_tflops": FP64_PEAK_NOMINAL / 1e12},
            "kernel_ms_per_step": {k: v[0] * v[1] for k, v in kp.items()},
            "limiter_activity": {k: stats[k] / max(stats["faces"], 1) for k in
                                 ("hllc_fallback", "cdi_dropped", "theta_p", "theta_t", "ylim", "diff_dropped")},
            "mixed": mixed,
            "status": status,
            "workload_build_s": t_build,
        }
        if recon is not None:
            line["variants"] = recon
        if adjoint is not None:
            line["adjoint"] = adjoint
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds, min(CPU_SLAB_PLANES, p.n[2]))
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
