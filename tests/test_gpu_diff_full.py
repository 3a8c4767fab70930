"""Differentiation at its full size: 1,048,576 spheres of the dense workload on the 32^3
degree-5 mesh, 50 steps with the recorded pair sets and checkpoints every 10 steps,
loss 0.5 ||P(S_50(x, v), q) - T||^2 with T the projection of a copy perturbed by 1 %
Gaussian noise (positions by 0.01 sigma, v and q relatively).

FP64: the gradient of autograd.Rollout against central finite differences on 64 random
directions, each a random unit vector over the 10 state components (x, v, q) of one
random particle. Over 50 steps a perturbation reaches ~100 particles through the
recorded collisions and grows ~100-fold, so at h = 1e-6 the O(h^2) term of a central
difference is still 1e-6..1e-3 of the derivative for most directions (measured: the
error falls 4x per halving of h down to a 1e-8 rounding floor). Each direction
therefore starts at h = 1e-6 and halves h (at most 5 times) until two successive
Richardson estimates (4 FD(h/2) - FD(h)) / 3 agree within 2e-7; the adjoint must match
that value within 1e-6. A direction is redrawn, and counted by cause, when a perturbed
rollout loses a recorded pair (no root any more) or changes the cutoff support of the
final state at every h, or when the estimates do not settle.

FP32: the gradient of autograd.Rollout32 (mixed forward, FP32 adjoints) against the
FP64 adjoints (pc_project_adjoint, pc_collide_adjoint, pinned against the oracle at
small sizes) chained backwards through the dequantised states and the pair sets of the
same FP32 trajectory, normwise per component within 1e-4."""
import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_05340_gb300 import autograd, pc  # noqa: E402

T = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)
STEPS, EVERY, NDIR = 50, 10, 64


@pytest.fixture(scope="module")
def problem():
    w = inputs.draw("dense_1m", seed=0)
    wl = w["workload"]
    dt = w["dt"]
    n = w["x"].shape[1]
    ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], dt) * 1.5)
    rng = np.random.default_rng(11)
    xp = w["x"] + 0.01 * wl.sigma * rng.normal(size=w["x"].shape)
    xp -= np.floor(xp)
    pert = dict(w, x=xp, v=w["v"] * (1 + 0.01 * rng.normal(size=w["v"].shape)),
                q=w["q"] * (1 + 0.01 * rng.normal(size=w["q"].shape)))
    return w, wl, dt, n, ctx, pert


def _nodes(wl):
    eta, _ = np.polynomial.legendre.leggauss(wl.degree + 1)
    X = np.sort(((np.arange(wl.ne)[:, None] + 0.5 * (eta[None, :] + 1.0)) / wl.ne).ravel())
    return T(np.concatenate([X - 1.0, X, X + 1.0]))


def _support(x, Xe, rc):
    """Per particle and axis: the number of 1-D nodes within the box cutoff (device)."""
    return (torch.searchsorted(Xe, (x + rc).contiguous(), right=True) -
            torch.searchsorted(Xe, (x - rc).contiguous(), right=False))


def _fixed_pair_field(ctx, x0, v0, q, r, m, ids, partners, dt):
    cur = pc.State(x0.contiguous(), v0.contiguous(), r, m, ids, None)
    for p in partners:
        nxt = pc.State(torch.empty_like(cur.x), torch.empty_like(cur.v), r, m, ids, None)
        ctx.collide_replay(cur, nxt, p, dt)
        cur = nxt
    f = ctx.new_field()
    ctx.project(pc.State(cur.x, cur.v, r, m, ids, q.contiguous()), f)
    try:
        ctx.sync()
    except pc.PcError as err:
        if err.status == pc.PC_EREPLAY:
            return None, None
        raise
    return f, cur.x


def test_fp64_rollout_gradient_full_size(problem):
    w, wl, dt, n, ctx, pert = problem
    target = ctx.new_field()
    ctx.project(pc.State.from_arrays(pert), target)
    x0, v0, q = (T(w[k]).requires_grad_(True) for k in ("x", "v", "q"))
    r, m, ids = T(w["r"]), T(w["m"]), T(w["id"], torch.int32)
    loss = autograd.rollout_loss(x0, v0, q, r, m, ids, target, ctx, dt, STEPS, EVERY)
    loss.backward()
    gx, gv, gq = x0.grad, v0.grad, q.grad
    # the pair sets of the base trajectory, recorded again
    partners = []
    cur = pc.State(T(w["x"]), T(w["v"]), r, m, ids, None)
    tmp = pc.State.empty(n, with_q=False)
    for s in range(STEPS):
        ctx.collide(cur, tmp, dt)
        p = ctx.partner_by_id(n).clone()
        nxt = pc.State(torch.empty_like(cur.x), torch.empty_like(cur.v), r, m, ids, None)
        ctx.collide_replay(cur, nxt, p, dt)
        partners.append(p)
        cur = nxt
    npairs = sum(int((p >= 0).sum()) // 2 for p in partners)
    print("pairs over %d steps: %d" % (STEPS, npairs))
    assert npairs > 100000
    F0, xS = _fixed_pair_field(ctx, T(w["x"]), T(w["v"]), T(w["q"]), r, m, ids, partners, dt)
    L0 = 0.5 * float(((F0 - target) ** 2).sum())
    assert abs(L0 - float(loss.detach())) <= 1e-12 * abs(L0)
    Xe, rc = _nodes(wl), wl.cutoff_sigmas * wl.sigma
    sig0 = _support(xS, Xe, rc)
    rng = np.random.default_rng(5)
    h = 1e-6
    accepted, worst, fd_h0 = 0, 0.0, 0.0
    why = {"pair lost": 0, "support": 0, "not settled": 0}
    while accepted < NDIR and sum(why.values()) < 6 * NDIR:
        k = int(rng.integers(n))
        u = rng.normal(size=10)
        u /= np.linalg.norm(u)
        ux, uv, uq = (torch.zeros(c, n, dtype=torch.float64, device="cuda") for c in (3, 3, 4))
        ux[:, k], uv[:, k], uq[:, k] = T(u[:3]), T(u[3:6]), T(u[6:])

        def central(hh):
            fields = []
            for sgn in (1, -1):
                xs = T(w["x"]) + sgn * hh * ux
                xs -= torch.floor(xs)
                F, xSs = _fixed_pair_field(ctx, xs, T(w["v"]) + sgn * hh * uv, T(w["q"]) + sgn * hh * uq, r, m, ids,
                                           partners, dt)
                if F is None:
                    return "pair lost"
                if not torch.equal(_support(xSs, Xe, rc), sig0):
                    return "support"
                fields.append(F)
            # L(+) - L(-) = 1/2 sum (F+ - F-)(F+ + F- - 2T): nodes the perturbation does not
            # reach contribute exactly zero instead of rounding noise of the whole loss
            dF = fields[0] - fields[1]
            return 0.5 * float((dF * (fields[0] + fields[1] - 2 * target)).sum()) / (2 * hh)

        ad = float((gx * ux).sum() + (gv * uv).sum() + (gq * uq).sum())
        fds, rich, settled, last_fail = [], [], None, None
        for lvl in range(6):
            f = central(1e-6 / 2 ** lvl)
            if isinstance(f, str):
                last_fail = f
                fds, rich = [], []
                continue
            fds.append(f)
            if len(fds) >= 2:
                rich.append((4 * fds[-1] - fds[-2]) / 3)
            if len(rich) >= 2 and abs(rich[-1] - rich[-2]) <= 2e-7 * abs(rich[-1]):
                settled = rich[-1]
                break
        if settled is None:
            why[last_fail if last_fail and len(fds) < 3 else "not settled"] += 1
            continue
        err = abs(settled - ad) / abs(ad)
        assert err <= 1e-6, (fds, rich, ad)
        worst = max(worst, err)
        if lvl == 2:
            fd_h0 = max(fd_h0, abs(fds[0] - ad) / abs(ad))
        accepted += 1
    print("FP64 full size: %d directions accepted (worst |Richardson - adjoint| / |adjoint| %.3e; directions "
          "settled from h = 1e-6: worst |FD(1e-6) - adjoint| / |adjoint| %.3e), redrawn %s" % (accepted, worst,
                                                                                             fd_h0, why))
    assert accepted == NDIR


def test_fp32_rollout_gradient_full_size(problem):
    w, wl, dt, n, ctx, pert = problem
    p32 = pc.StateF32.empty(n)
    ctx.quantize(pc.State.from_arrays(pert), p32)
    target = ctx.new_field_f32()
    ctx.project_f32(p32, target)
    x0, v0, q = (T(w[k]).requires_grad_(True) for k in ("x", "v", "q"))
    r, m, ids = T(w["r"]), T(w["m"]), T(w["id"], torch.int32)
    loss = autograd.rollout_loss_f32(x0, v0, q, r, m, ids, target, ctx, dt, STEPS, EVERY)
    loss.backward()
    # the FP32 trajectory again: dequantised states and pair sets
    nc = ctx.cells_per_side
    cur = pc.StateF32.empty(n)
    ctx.quantize(pc.State.from_arrays(w), cur)
    tmp = pc.StateF32.empty(n, with_q=False)
    xs64, vs64, partners = [], [], []
    deq = lambda s: T(oracle.dequantize(s.cell.cpu().numpy(), s.o.cpu().numpy(), nc))
    for s in range(STEPS):
        xs64.append(deq(cur))
        vs64.append(cur.v.double())
        ctx.collide_f32(pc.StateF32(cur.id, cur.cell, cur.o, cur.v, cur.r, cur.m, None), tmp, dt)
        p = ctx.partner_by_id(n)
        nxt = pc.StateF32(cur.id, torch.empty_like(cur.cell), torch.empty_like(cur.o), torch.empty_like(cur.v),
                          cur.r, cur.m, cur.q)
        ctx.collide_replay_f32(cur, nxt, p, dt)
        partners.append(p)
        cur = nxt
    field = ctx.new_field_f32()
    ctx.project_f32(cur, field)
    ctx.sync()
    G = (field - target).double().contiguous()
    r64, m64, q64 = cur.r.double(), cur.m.double(), cur.q.double().contiguous()
    gq_ref = torch.empty(4, n, dtype=torch.float64, device="cuda")
    gx_ref = torch.empty(3, n, dtype=torch.float64, device="cuda")
    ctx.project_adjoint(pc.State(deq(cur), cur.v.double(), r64, m64, ids, q64), G, gq_ref, gx_ref)
    gv_ref = torch.zeros(3, n, dtype=torch.float64, device="cuda")
    gx2, gv2 = torch.empty_like(gx_ref), torch.empty_like(gv_ref)
    for s in reversed(range(STEPS)):
        ctx.collide_adjoint(pc.State(xs64[s], vs64[s], r64, m64, ids, None), partners[s], dt, gx_ref, gv_ref, gx2,
                            gv2)
        gx_ref, gx2 = gx2, gx_ref
        gv_ref, gv2 = gv2, gv_ref
    ctx.sync()

    def err(a, b):
        return ((a - b).abs().amax(dim=1) / b.abs().amax(dim=1)).cpu().numpy()

    errs = {"x": err(x0.grad, gx_ref), "v": err(v0.grad, gv_ref), "q": err(q.grad, gq_ref)}
    print("FP32 full size: normwise gradient errors against the FP64 adjoints", errs)
    for k, e in errs.items():
        assert np.all(e <= 1e-4), (k, e)
