"""Differentiation through the C ABI: replay with a fixed pair set, the adjoints of
one step and of the projection against the oracle's adjoints (themselves pinned by
a torch float64 restatement), and the gradient of a rollout against central
finite differences (h = 1e-6) with the pair sets held fixed."""
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


def _setup(n=20000, seed=0, dtmul=5):
    w = inputs.draw("dense_1m", seed=seed, n=n)
    wl = w["workload"]
    dt = dtmul * w["dt"]
    ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], dt) * 1.5)
    return w, wl, dt, ctx


def test_replay_bit_identical_to_collide():
    w, wl, dt, ctx = _setup(n=30000, dtmul=10)
    a = pc.State.from_arrays(w)
    b = pc.State.empty(a.n)
    ctx.collide(a, b, dt)
    partner = ctx.partner_by_id(a.n)
    c = pc.State(torch.empty_like(a.x), torch.empty_like(a.v), a.r, a.m, a.id, None)
    ctx.collide_replay(pc.State(a.x, a.v, a.r, a.m, a.id, None), c, partner, dt)
    ctx.sync()
    g = by_id(b.numpy())
    assert (partner >= 0).sum().item() > 100
    assert np.array_equal(c.x.cpu().numpy(), g["x"]) and np.array_equal(c.v.cpu().numpy(), g["v"])
    p = partner.cpu().numpy().astype(np.int64)
    x2, v2 = oracle.collide_replay(w["x"], w["v"], w["r"], w["m"], p, w["e"], dt)
    assert np.array_equal(c.x.cpu().numpy(), x2) and np.array_equal(c.v.cpu().numpy(), v2)


def test_collide_adjoint_matches_oracle():
    w, wl, dt, ctx = _setup(n=30000, dtmul=10)
    a = pc.State.from_arrays(w, with_q=False)
    b = pc.State.empty(a.n, with_q=False)
    ctx.collide(a, b, dt)
    partner = ctx.partner_by_id(a.n)
    rng = np.random.default_rng(0)
    gxo, gvo = rng.normal(size=(3, a.n)), rng.normal(size=(3, a.n))
    gx, gv = torch.empty(3, a.n, dtype=torch.float64, device="cuda"), torch.empty(3, a.n, dtype=torch.float64,
                                                                                   device="cuda")
    ctx.collide_adjoint(a, partner, dt, T(gxo), T(gvo), gx, gv)
    ctx.sync()
    p = partner.cpu().numpy().astype(np.int64)
    ox, ov = oracle.collide_adjoint(w["x"], w["v"], w["r"], w["m"], p, w["e"], dt, gxo, gvo)
    assert np.allclose(gx.cpu().numpy(), ox, rtol=1e-12, atol=1e-12 * np.abs(ox).max())
    assert np.allclose(gv.cpu().numpy(), ov, rtol=1e-12, atol=1e-12 * np.abs(ov).max())


@pytest.mark.parametrize("name,n", [("small_8192", 3000), ("dense_1m", 20000)])
def test_project_adjoint_matches_oracle(name, n):
    w = inputs.draw(name, seed=1, n=n)
    wl = w["workload"]
    ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], 0.05)
    rng = np.random.default_rng(1)
    G = rng.normal(size=(wl.ne ** 3, 4, (wl.degree + 1) ** 3))
    a = pc.State.from_arrays(w)
    gq, gx = torch.empty(4, n, dtype=torch.float64, device="cuda"), torch.empty(3, n, dtype=torch.float64,
                                                                                 device="cuda")
    ctx.project_adjoint(a, T(G), gq, gx)
    ctx.sync()
    oq, ox = oracle.project_adjoint(w["x"], w["q"], G, wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
    assert np.max(np.abs(gq.cpu().numpy() - oq)) <= 1e-12 * np.abs(oq).max()
    assert np.max(np.abs(gx.cpu().numpy() - ox)) <= 1e-12 * np.abs(ox).max()


def _fixed_pair_field(ctx, x0, v0, q, r, m, ids, partners, dt):
    """Field of the rollout with the recorded pair sets (replay only); None if a pair lost its root."""
    n = x0.shape[1]
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


def _support_signature(x, wl):
    eta, _ = np.polynomial.legendre.leggauss(wl.degree + 1)
    X = np.sort(((np.arange(wl.ne)[:, None] + 0.5 * (eta[None, :] + 1.0)) / wl.ne).ravel())
    Xe = np.concatenate([X - 1.0, X, X + 1.0])
    rc = wl.cutoff_sigmas * wl.sigma
    return np.stack([np.searchsorted(Xe, x[a] + rc, side="right") - np.searchsorted(Xe, x[a] - rc, side="left")
                     for a in range(3)])


def test_rollout_gradient_matches_finite_differences():
    """20,000 spheres of the dense workload, 20 steps (checkpoints every 10), loss against
    the projection of a 1 % perturbed copy; 8 random directions (each on 50 random
    particles) accepted at h = 1e-6, a direction that changes a pair or the cutoff
    support between the two evaluations being redrawn."""
    w, wl, dt, ctx = _setup(n=20000, seed=3, dtmul=5)
    n = w["x"].shape[1]
    rng = np.random.default_rng(7)
    xp = w["x"] + 0.01 * wl.sigma * rng.normal(size=w["x"].shape)
    xp -= np.floor(xp)
    pert = pc.State.from_arrays(dict(w, x=xp, v=w["v"] * (1 + 0.01 * rng.normal(size=w["v"].shape)),
                                     q=w["q"] * (1 + 0.01 * rng.normal(size=w["q"].shape))))
    target = ctx.new_field()
    ctx.project(pert, target)
    x0 = T(w["x"]).requires_grad_(True)
    v0 = T(w["v"]).requires_grad_(True)
    q = T(w["q"]).requires_grad_(True)
    r, m, ids = T(w["r"]), T(w["m"]), T(w["id"], torch.int32)
    steps = 20
    loss = autograd.rollout_loss(x0, v0, q, r, m, ids, target, ctx, dt, steps, 10)
    loss.backward()
    gx, gv, gq = x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), q.grad.cpu().numpy()
    # the pair sets of the base trajectory, recorded again
    partners = []
    cur = pc.State(T(w["x"]), T(w["v"]), r, m, ids, None)
    tmp = pc.State.empty(n, with_q=False)
    for s in range(steps):
        ctx.collide(cur, tmp, dt)
        p = ctx.partner_by_id(n).clone()
        nxt = pc.State(torch.empty_like(cur.x), torch.empty_like(cur.v), r, m, ids, None)
        ctx.collide_replay(cur, nxt, p, dt)
        partners.append(p)
        cur = nxt
    assert sum(int((p >= 0).sum()) for p in partners) > 200
    F0, xS = _fixed_pair_field(ctx, T(w["x"]), T(w["v"]), T(w["q"]), r, m, ids, partners, dt)
    L0 = 0.5 * float(((F0 - target) ** 2).sum())
    assert abs(L0 - float(loss.detach())) <= 1e-12 * abs(L0)
    sig0 = _support_signature(xS.cpu().numpy(), wl)
    h = 1e-6
    accepted, replaced, curved = 0, 0, 0
    while accepted < 8 and replaced < 60:
        # random direction on 50 random particles: a dense direction moves some particle
        # across a node's cutoff (a jump of the loss) for almost every draw
        sub = rng.choice(n, 50, replace=False)
        ux, uv, uq = np.zeros((3, n)), np.zeros((3, n)), np.zeros((4, n))
        ux[:, sub], uv[:, sub], uq[:, sub] = rng.normal(size=(3, 50)), rng.normal(size=(3, 50)), rng.normal(size=(4, 50))
        def central(hh):
            fields = []
            for sgn in (1, -1):
                xs = w["x"] + sgn * hh * ux
                xs -= np.floor(xs)
                F, xSs = _fixed_pair_field(ctx, T(xs), T(w["v"] + sgn * hh * uv), T(w["q"] + sgn * hh * uq), r, m,
                                           ids, partners, dt)
                if F is None or not np.array_equal(_support_signature(xSs.cpu().numpy(), wl), sig0):
                    return None
                fields.append(F)
            # L(+) - L(-) = 1/2 sum (F+ - F-)(F+ + F- - 2T): nodes the perturbation does not
            # reach contribute exactly zero instead of rounding noise of the whole loss
            dF = fields[0] - fields[1]
            return 0.5 * float((dF * (fields[0] + fields[1] - 2 * target)).sum()) / (2 * hh)

        fd = central(h)
        fd2 = central(h / 2) if fd is not None else None
        if fd is None or fd2 is None:
            replaced += 1
            continue
        ad = (gx * ux).sum() + (gv * uv).sum() + (gq * uq).sum()
        # central differences carry an O(h^2) truncation error that is large when a
        # perturbed particle is in a nearly grazing pair (t ~ sqrt of the discriminant):
        # such a direction is as unusable as one that crosses a cutoff, and is redrawn
        if abs(fd - fd2) > 1e-5 * abs(fd):
            curved += 1
            replaced += 1
            continue
        # in the asymptotic regime the O(h^2) term cancels in (4 FD(h/2) - FD(h)) / 3
        rich = (4 * fd2 - fd) / 3
        print("direction %d: FD(h) %.12e Richardson %.12e adjoint %.12e" % (accepted, fd, rich, ad))
        assert abs(fd - ad) <= 2e-5 * abs(ad), (fd, fd2, ad)
        assert abs(rich - ad) <= 1e-7 * abs(ad), (fd, fd2, rich, ad)
        accepted += 1
    print("directions replaced: %d (%d strongly curved)" % (replaced, curved))
    assert accepted == 8, "directions replaced: %d" % replaced
