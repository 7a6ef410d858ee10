"""torch.autograd front end of the discrete adjoint (FP64 contexts).

Every backward pass runs the library's hand-written reverse kernels through
the C ABI (mpmc_rk_step_adjoint, mpmc_init_state_adjoint,
mpmc_primitives_adjoint); torch only holds the tensors and chains the calls.
The adjoint is that of the discrete map: the limiter decisions of the forward
pass are replayed and each step's dt and Gamma are frozen (Sec. 3.3, 3.4).

  init_state(ctx, prim)             U = conserved state of primitive fields
  rk_step(ctx, U, dt=0.0)           one SSP-RK3 step (out of place)
  primitives(ctx, U)                [T, P, rho, a, Y_k, u_d] per cell
  RKStep.apply(ctx, U, dt)          the same step as an autograd Function
  step_n_checkpointed(ctx, U0, n, every=20)   U_n of a checkpointed rollout
  rollout(ctx, U0, n, every=20, probe=None, dt=0.0)
        n steps (of fixed length dt > 0, or each the CFL step of its own
        state) with a checkpoint every `every` steps; returns (U_n, J, dts)
        with J = sum_{k=1..n} dt_k sum_c probe_c P_c(U^k) (zero without a
        probe).  The backward pass replays each segment from its checkpoint
        (one forward step per step, keeping each step's input, stage states
        and limiter flags) and sweeps it in reverse, so memory holds the
        checkpoints plus one segment of inputs, stage states and flags.
"""
import torch

from . import binding as _b


class _InitState(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, prim):
        prim = prim.detach().contiguous()
        fctx.ctx = ctx
        fctx.save_for_backward(prim)
        return ctx.init_state(prim)

    @staticmethod
    def backward(fctx, gU):
        (prim,) = fctx.saved_tensors
        return None, fctx.ctx.init_state_adjoint(prim, gU.contiguous())


class _RKStep(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, U, dt):
        U = U.detach().contiguous()
        out = U.clone()
        ctx.rk_step(out, dt)
        fctx.ctx = ctx
        fctx.dt = dt
        fctx.save_for_backward(U)
        return out

    @staticmethod
    def backward(fctx, g):
        (U,) = fctx.saved_tensors
        return None, fctx.ctx.rk_step_adjoint(U, g.contiguous(), dt=fctx.dt), None


class _Primitives(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, U):
        U = U.detach().contiguous()
        fctx.ctx = ctx
        fctx.save_for_backward(U)
        return ctx.primitives(U)

    @staticmethod
    def backward(fctx, gW):
        (U,) = fctx.saved_tensors
        return None, fctx.ctx.primitives_adjoint(U, gW.contiguous())


def _stage_caches(ctx, m, device, share=0.5):
    """Buffers for the primitive caches of a segment's m steps (3 stages
    each), which spare the reverse steps their recomputation, when they fit
    in `share` of the device's free memory; else None (recomputed)."""
    nbytes = m * 3 * ctx.cache_doubles * 8
    free, _ = torch.cuda.mem_get_info(device)
    if nbytes > share * free:
        return None
    return torch.empty((m, 3 * ctx.cache_doubles), dtype=torch.float64, device=device)


def _probe_term(ctx, U, probe):
    """sum_c probe_c P_c(U)"""
    return (ctx.primitives(U)[1] * probe).sum()


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, U0, n, every, probe, dt):
        U = U0.detach().contiguous().clone()
        ckpts = []
        dts = torch.empty(n, dtype=torch.float64, device=U.device)
        slot = torch.empty(1, dtype=torch.float64, device=U.device)
        J = torch.zeros((), dtype=torch.float64, device=U.device)
        for k in range(n):
            if k % every == 0:
                ckpts.append(U.clone())
            if dt > 0.0:
                ctx.rk_step(U, dt)              # fixed step
                dts[k] = dt
            else:
                ctx.step_n(U, 1, slot)          # CFL step of U^k, recorded
                dts[k] = slot[0]
            if probe is not None:
                J += dts[k] * _probe_term(ctx, U, probe)
        fctx.ctx, fctx.n, fctx.every, fctx.probe = ctx, n, every, probe
        fctx.ckpts, fctx.dts = ckpts, dts
        fctx.mark_non_differentiable(dts)
        return U, J, dts

    @staticmethod
    def backward(fctx, gU, gJ, _gdts):
        ctx, n, every, probe, dts = fctx.ctx, fctx.n, fctx.every, fctx.probe, fctx.dts
        lam = gU.contiguous().clone() if gU is not None else torch.zeros_like(fctx.ckpts[0])
        gJ = float(gJ) if gJ is not None else 0.0
        dt_host = dts.cpu().tolist()
        lamW = None
        if probe is not None and gJ != 0.0:
            lamW = torch.zeros((len(ctx.prim_fields),) + tuple(lam.shape[1:]), dtype=torch.float64,
                               device=lam.device)
        nf = ctx.nfaces_total
        for seg in reversed(range(len(fctx.ckpts))):
            k0, k1 = seg * every, min(n, (seg + 1) * every)
            m = k1 - k0
            # replay the segment, keeping every step's input, stage states and flags
            states = torch.empty((m + 1,) + tuple(lam.shape), dtype=lam.dtype, device=lam.device)
            stages = torch.empty((m, 2) + tuple(lam.shape), dtype=lam.dtype, device=lam.device)
            tapes = torch.empty((m, 3 * nf), dtype=torch.int32, device=lam.device)
            wst = _stage_caches(ctx, m, lam.device)
            states[0].copy_(fctx.ckpts[seg])
            for q in range(m):
                states[q + 1].copy_(states[q])
                ctx.rk_step_record(states[q + 1], dt_host[k0 + q], tapes[q], stages[q],
                                   wst[q] if wst is not None else None)
            for q in reversed(range(m)):
                k = k0 + q
                if lamW is not None:
                    # dJ/dU^{k+1} = gJ dt_k (dP/dU)^T probe
                    lamW[1] = (gJ * dt_host[k]) * probe
                    ctx.primitives_adjoint(states[q + 1], lamW, lam)
                ctx.rk_step_adjoint(states[q], lam, dt=dt_host[k], tape=tapes[q], lam_n=lam, stages=stages[q],
                                    wstages=wst[q] if wst is not None else None)
        return None, lam, None, None, None, None


def init_state(ctx, prim):
    return _InitState.apply(ctx, prim)


def rk_step(ctx, U, dt=0.0):
    return _RKStep.apply(ctx, U, float(dt))


def primitives(ctx, U):
    return _Primitives.apply(ctx, U)


def rollout(ctx, U0, n, every=20, probe=None, dt=0.0):
    """dt > 0: every step has that length; otherwise each step takes the CFL
    step of its own U^k (recorded, and frozen in the backward pass)."""
    if ctx.precision != _b.FP64:
        raise ValueError("the discrete adjoint needs an FP64 context")
    return _Rollout.apply(ctx, U0, int(n), int(every), probe, float(dt))


# the autograd Function of one step, for callers that chain steps themselves
RKStep = _RKStep


def step_n_checkpointed(ctx, U0, n, every=20):
    """n CFL steps from U0 with a checkpoint every `every` steps; returns U_n
    (differentiable with respect to U0)."""
    return rollout(ctx, U0, n, every)[0]
