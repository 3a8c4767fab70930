"""Differentiable rollouts of the particle operator (torch.autograd.Function).

The loss of a rollout of `steps` collision steps followed by a projection,
L = 0.5 * ||P(S_steps(x0, v0), q) - T||^2, is differentiated with each step's pair
set held fixed: the forward pass lets pc_collide choose the pairs and advances the
state with pc_collide_replay in id order (bit-identical); it keeps the pair set
of every step and the state every `checkpoint_every` steps. The backward pass
applies pc_project_adjoint, then for each segment (last first) replays the states
from its checkpoint and applies pc_collide_adjoint step by step. All arithmetic
runs in the CUDA library; this module only moves tensors.

Rollout32 is the FP32 variant on the mixed-precision path: the state is quantised
to FP32 cell-relative storage, pc_collide_f32 chooses each step's pairs and
pc_collide_replay_f32 advances the state in id order (bit-identical), the field is
the tensor-core projection, and the backward pass runs the FP32 adjoints
(pc_project_adjoint_f32, pc_collide_adjoint_f32). Its gradients are returned as
float64 tensors, the quantisation taken as the identity.

Both require ids 0..n-1 with the arrays in id order (partners are looked up by id).
"""
import torch

from . import pc


def _state(x, v, r, m, ids, q):
    return pc.State(x.contiguous(), v.contiguous(), r, m, ids, q)


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x0, v0, q, r, m, ids, target, ctx, dt, steps, checkpoint_every=10):
        n = x0.shape[1]
        cur = _state(x0.detach().clone(), v0.detach().clone(), r, m, ids, q.detach().contiguous())
        tmp = pc.State.empty(n, with_q=False)
        partners, checkpoints = [], []
        for s in range(steps):
            if s % checkpoint_every == 0:
                checkpoints.append((cur.x.clone(), cur.v.clone()))
            ctx.collide(pc.State(cur.x, cur.v, r, m, ids, None), tmp, dt)
            partner = ctx.partner_by_id(n)
            nxt = pc.State(torch.empty_like(cur.x), torch.empty_like(cur.v), r, m, ids, cur.q)
            ctx.collide_replay(cur, nxt, partner, dt)
            partners.append(partner)
            cur = nxt
        field = ctx.new_field()
        ctx.project(cur, field)
        ctx.sync()
        diff = field - target
        loss = 0.5 * (diff * diff).sum()
        fctx.pc = (ctx, dt, steps, checkpoint_every, partners, checkpoints)
        fctx.save_for_backward(cur.x, cur.v, cur.q, r, m, ids, diff)
        return loss

    @staticmethod
    def backward(fctx, gloss):
        ctx, dt, steps, every, partners, checkpoints = fctx.pc
        xS, vS, q, r, m, ids, diff = fctx.saved_tensors
        n = xS.shape[1]
        G = (diff * gloss).contiguous()
        gq = torch.empty(4, n, dtype=torch.float64, device="cuda")
        gx = torch.empty(3, n, dtype=torch.float64, device="cuda")
        ctx.project_adjoint(pc.State(xS, vS, r, m, ids, q), G, gq, gx)
        gv = torch.zeros(3, n, dtype=torch.float64, device="cuda")
        gx2, gv2 = torch.empty_like(gx), torch.empty_like(gv)
        for seg in reversed(range(len(checkpoints))):
            s0 = seg * every
            s1 = min(steps, s0 + every)
            xs, vs = checkpoints[seg]
            states = [(xs, vs)]
            for s in range(s0, s1 - 1):
                a = pc.State(states[-1][0], states[-1][1], r, m, ids, None)
                b = pc.State(torch.empty_like(xs), torch.empty_like(vs), r, m, ids, None)
                ctx.collide_replay(a, b, partners[s], dt)
                states.append((b.x, b.v))
            for s in reversed(range(s0, s1)):
                pre = pc.State(states[s - s0][0], states[s - s0][1], r, m, ids, None)
                ctx.collide_adjoint(pre, partners[s], dt, gx, gv, gx2, gv2)
                gx, gx2 = gx2, gx
                gv, gv2 = gv2, gv
        ctx.sync()
        return gx, gv, gq, None, None, None, None, None, None, None, None


class Rollout32(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x0, v0, q, r, m, ids, target, ctx, dt, steps, checkpoint_every=10, tc="f16"):
        n = x0.shape[1]
        cur = pc.StateF32.empty(n)
        ctx.quantize(pc.State(x0.detach().contiguous(), v0.detach().contiguous(), r, m, ids, q.detach().contiguous()),
                     cur)
        tmp = pc.StateF32.empty(n, with_q=False)
        partners, checkpoints = [], []
        for s in range(steps):
            if s % checkpoint_every == 0:
                checkpoints.append((cur.cell.clone(), cur.o.clone(), cur.v.clone()))
            ctx.collide_f32(pc.StateF32(cur.id, cur.cell, cur.o, cur.v, cur.r, cur.m, None), tmp, dt)
            partner = ctx.partner_by_id(n)
            nxt = pc.StateF32(cur.id, torch.empty_like(cur.cell), torch.empty_like(cur.o), torch.empty_like(cur.v),
                              cur.r, cur.m, cur.q)
            ctx.collide_replay_f32(cur, nxt, partner, dt)
            partners.append(partner)
            cur = nxt
        field = ctx.new_field_f32()
        ctx.project_f32(cur, field, tc)
        ctx.sync()
        diff = field - target
        loss = 0.5 * (diff.double() * diff.double()).sum()
        fctx.pc = (ctx, dt, steps, checkpoint_every, partners, checkpoints, cur)
        fctx.save_for_backward(diff)
        return loss

    @staticmethod
    def backward(fctx, gloss):
        ctx, dt, steps, every, partners, checkpoints, last = fctx.pc
        (diff,) = fctx.saved_tensors
        n = last.n
        G = (diff * gloss.float()).contiguous()
        f32 = dict(dtype=torch.float32, device="cuda")
        gq = torch.empty(4, n, **f32)
        gx = torch.empty(3, n, **f32)
        ctx.project_adjoint_f32(last, G, gq, gx)
        gv = torch.zeros(3, n, **f32)
        gx2, gv2 = torch.empty_like(gx), torch.empty_like(gv)
        for seg in reversed(range(len(checkpoints))):
            s0 = seg * every
            s1 = min(steps, s0 + every)
            cs, os_, vs = checkpoints[seg]
            states = [pc.StateF32(last.id, cs, os_, vs, last.r, last.m, None)]
            for s in range(s0, s1 - 1):
                b = pc.StateF32(last.id, torch.empty_like(cs), torch.empty_like(os_), torch.empty_like(vs), last.r,
                                last.m, None)
                ctx.collide_replay_f32(states[-1], b, partners[s], dt)
                states.append(b)
            for s in reversed(range(s0, s1)):
                ctx.collide_adjoint_f32(states[s - s0], partners[s], dt, gx, gv, gx2, gv2)
                gx, gx2 = gx2, gx
                gv, gv2 = gv2, gv
        ctx.sync()
        return gx.double(), gv.double(), gq.double(), None, None, None, None, None, None, None, None, None


def rollout_loss(x0, v0, q, r, m, ids, target, ctx, dt, steps, checkpoint_every=10):
    """L = 0.5 ||P(S_steps(x0, v0), q) - T||^2 with the gradient of Rollout."""
    return Rollout.apply(x0, v0, q, r, m, ids, target, ctx, dt, steps, checkpoint_every)


def rollout_loss_f32(x0, v0, q, r, m, ids, target, ctx, dt, steps, checkpoint_every=10, tc="f16"):
    """The FP32 rollout loss (Rollout32); target is an FP32 field."""
    return Rollout32.apply(x0, v0, q, r, m, ids, target, ctx, dt, steps, checkpoint_every, tc)
