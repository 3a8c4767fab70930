"""FP32 rollouts on the mixed-precision path through the C ABI: the fixed-pair replay is
bit-identical to pc_collide_f32, and the FP32 adjoints of one step, of the projection
and of a 20-step rollout (checkpoints every 10 steps) agree with the FP64 oracle's
adjoints evaluated at the dequantised states of the same trajectory.

Tolerance: normwise per component, max |g32 - g64| / max |g64| <= 1e-4. FP32 rounding
(2^-24) of sums over ~1500 support nodes per particle and of the contact-time
derivative, whose 1 / (s . dv) grows near grazing, stays orders of magnitude below it."""
import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs
from tests.gpu_helpers import by_id

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_05340_gb300 import autograd, pc  # noqa: E402

T = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)
F32 = torch.float32
GRAD_TOL = 1e-4


def _norm_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max(axis=-1) / np.maximum(np.abs(b).max(axis=-1), 1e-300)


def _setup(n, seed, dtmul, name="dense_1m"):
    w = inputs.draw(name, seed=seed, n=n)
    wl = w["workload"]
    dt = dtmul * w["dt"]
    ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], dt) * 1.5)
    s32 = pc.StateF32.empty(n)
    ctx.quantize(pc.State.from_arrays(w), s32)
    return w, wl, dt, ctx, s32


def _x64(ctx, d):
    return oracle.dequantize(d["cell"], d["o"], ctx.cells_per_side)


def test_replay_f32_bit_identical_to_collide_f32():
    w, wl, dt, ctx, a = _setup(30000, 0, 10)
    b = pc.StateF32.empty(a.n)
    ctx.collide_f32(a, b, dt)
    partner = ctx.partner_by_id(a.n)
    c = pc.StateF32(a.id, torch.empty_like(a.cell), torch.empty_like(a.o), torch.empty_like(a.v), a.r, a.m, a.q)
    ctx.collide_replay_f32(a, c, partner, dt)
    ctx.sync()
    g = by_id(b.numpy())
    assert (partner >= 0).sum().item() > 100
    for k in ("cell", "o", "v"):
        assert np.array_equal(getattr(c, k).cpu().numpy(), g[k]), k


@pytest.mark.parametrize("name,n", [("dense_1m", 20000), ("small_8192", 3000)])
def test_project_adjoint_f32_matches_oracle(name, n):
    w, wl, dt, ctx, s32 = _setup(n, 1, 1, name)
    d = s32.numpy()
    rng = np.random.default_rng(2)
    G = rng.normal(size=(wl.ne ** 3, 4, (wl.degree + 1) ** 3)).astype(np.float32)
    gq, gx = torch.empty(4, n, dtype=F32, device="cuda"), torch.empty(3, n, dtype=F32, device="cuda")
    ctx.project_adjoint_f32(s32, T(G, F32), gq, gx)
    ctx.sync()
    oq, ox = oracle.project_adjoint(_x64(ctx, d), d["q"].astype(np.float64), G.astype(np.float64), wl.ne,
                                    wl.degree, wl.sigma)
    eq, ex = _norm_err(gq.cpu().numpy(), oq), _norm_err(gx.cpu().numpy(), ox)
    print("project adjoint f32 normwise errors: gq", eq, "gx", ex)
    assert np.all(eq <= GRAD_TOL) and np.all(ex <= GRAD_TOL)


def test_collide_adjoint_f32_matches_oracle():
    w, wl, dt, ctx, a = _setup(30000, 0, 10)
    b = pc.StateF32.empty(a.n)
    ctx.collide_f32(a, b, dt)
    partner = ctx.partner_by_id(a.n)
    rng = np.random.default_rng(0)
    gxo, gvo = rng.normal(size=(3, a.n)).astype(np.float32), rng.normal(size=(3, a.n)).astype(np.float32)
    gx, gv = torch.empty(3, a.n, dtype=F32, device="cuda"), torch.empty(3, a.n, dtype=F32, device="cuda")
    ctx.collide_adjoint_f32(a, partner, dt, T(gxo, F32), T(gvo, F32), gx, gv)
    ctx.sync()
    d = a.numpy()
    p = partner.cpu().numpy().astype(np.int64)
    assert (p >= 0).sum() > 100
    ox, ov = oracle.collide_adjoint(_x64(ctx, d), d["v"].astype(np.float64), d["r"].astype(np.float64),
                                    d["m"].astype(np.float64), p, w["e"], dt, gxo.astype(np.float64),
                                    gvo.astype(np.float64))
    ex, ev = _norm_err(gx.cpu().numpy(), ox), _norm_err(gv.cpu().numpy(), ov)
    print("collide adjoint f32 normwise errors: gx", ex, "gv", ev)
    assert np.all(ex <= GRAD_TOL) and np.all(ev <= GRAD_TOL)


def test_rollout32_gradient_matches_fp64_reference():
    """20,000 spheres of the dense workload, 20 mixed steps (checkpoints every 10), loss
    against the FP32 projection of a 1 % perturbed copy. Reference: the FP64 oracle's
    projection and step adjoints chained backwards through the dequantised states and
    pair sets of the same (deterministic) trajectory."""
    w, wl, dt, ctx, _ = _setup(20000, 3, 5)
    n = w["x"].shape[1]
    rng = np.random.default_rng(7)
    xp = w["x"] + 0.01 * wl.sigma * rng.normal(size=w["x"].shape)
    xp -= np.floor(xp)
    pert = pc.StateF32.empty(n)
    ctx.quantize(pc.State.from_arrays(dict(w, x=xp, v=w["v"] * (1 + 0.01 * rng.normal(size=w["v"].shape)),
                                           q=w["q"] * (1 + 0.01 * rng.normal(size=w["q"].shape)))), pert)
    target = ctx.new_field_f32()
    ctx.project_f32(pert, target)
    x0, v0, q = (T(w[k]).requires_grad_(True) for k in ("x", "v", "q"))
    r, m, ids = T(w["r"]), T(w["m"]), T(w["id"], torch.int32)
    steps = 20
    loss = autograd.rollout_loss_f32(x0, v0, q, r, m, ids, target, ctx, dt, steps, 10)
    loss.backward()
    # the same trajectory again: states and pair sets
    cur = pc.StateF32.empty(n)
    ctx.quantize(pc.State.from_arrays(w), cur)
    tmp = pc.StateF32.empty(n, with_q=False)
    states, partners = [], []
    for s in range(steps):
        states.append(cur.numpy())
        ctx.collide_f32(pc.StateF32(cur.id, cur.cell, cur.o, cur.v, cur.r, cur.m, None), tmp, dt)
        p = ctx.partner_by_id(n)
        nxt = pc.StateF32(cur.id, torch.empty_like(cur.cell), torch.empty_like(cur.o), torch.empty_like(cur.v),
                          cur.r, cur.m, cur.q)
        ctx.collide_replay_f32(cur, nxt, p, dt)
        partners.append(p.cpu().numpy().astype(np.int64))
        cur = nxt
    field = ctx.new_field_f32()
    ctx.project_f32(cur, field)
    ctx.sync()
    assert sum(int((p >= 0).sum()) for p in partners) > 200
    G = (field - target).double().cpu().numpy()
    dS = cur.numpy()
    L = 0.5 * float((G * G).sum())
    assert abs(L - float(loss.detach())) <= 1e-12 * abs(L)
    gq_ref, gx_ref = oracle.project_adjoint(_x64(ctx, dS), dS["q"].astype(np.float64), G, wl.ne, wl.degree,
                                            wl.sigma)
    gv_ref = np.zeros_like(gx_ref)
    r64, m64 = dS["r"].astype(np.float64), dS["m"].astype(np.float64)
    for s in reversed(range(steps)):
        d = states[s]
        gx_ref, gv_ref = oracle.collide_adjoint(_x64(ctx, d), d["v"].astype(np.float64), r64, m64, partners[s],
                                                w["e"], dt, gx_ref, gv_ref)
    errs = {k: _norm_err(a.grad.cpu().numpy(), ref) for k, a, ref in
            (("x", x0, gx_ref), ("v", v0, gv_ref), ("q", q, gq_ref))}
    print("rollout32 normwise gradient errors", errs)
    for k, e in errs.items():
        assert np.all(e <= GRAD_TOL), (k, e)
