"""Parity of the collision step with Coulomb friction and rotation (pc_collide_rot, through
the C ABI) with the oracle: pairs, contact times, positions, velocities and angular
velocities bit-identical (FP64 in the same operation order on both sides)."""
import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs
from tests.gpu_helpers import oracle_pairs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_05340_gb300 import pc  # noqa: E402

T = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", torch.float64)


def _ctx(w, n, dt):
    wl = w["workload"]
    return pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], dt),
                      cutoff_sigmas=wl.cutoff_sigmas)


def _step(ctx, cur, w_id, mu, dt, e):
    """One GPU step from the state `cur` and spins `w_id` (same order), against one oracle
    step; both sides are compared in id order. Returns the oracle's next state and spins
    (in the order of `cur`) and the pair count."""
    src = pc.State.from_arrays(cur)
    dst = pc.State.empty(src.n)
    w_in = T(w_id)
    w_out = torch.empty_like(w_in)
    ctx.collide_rot(src, dst, w_in, w_out, mu, dt)
    ctx.sync()
    gids, gt = ctx.pairs()
    x1, v1, w1, partner, tc, k = oracle.collide_step_rot(cur["x"], cur["v"], w_id, cur["r"], cur["m"], cur["id"], e,
                                                         mu, dt)
    oids, ot = oracle_pairs(partner, tc, cur["id"])
    assert np.array_equal(gids, oids), "pair sets differ"
    assert np.array_equal(gt, ot), "contact times differ"
    g = dst.numpy()
    o = np.argsort(g["id"], kind="stable")
    oc = np.argsort(cur["id"], kind="stable")
    gw = w_out.cpu().numpy()[:, o]
    assert np.array_equal(g["id"][o], cur["id"][oc])
    assert np.array_equal(g["x"][:, o], x1[:, oc]), "positions differ"
    assert np.array_equal(g["v"][:, o], v1[:, oc]), "velocities differ"
    assert np.array_equal(gw, w1[:, oc]), "angular velocities differ"
    nxt = dict(cur)
    nxt["x"], nxt["v"] = x1, v1
    return nxt, w1, k


@pytest.mark.parametrize("mu", [0.0, 0.05, 0.3, 10.0])
def test_small_rollout_bit_identical(mu):
    """8192 spheres, e = 0.9, spins N(0, 30^2): 15 steps, every step bit-identical; mu
    from frictionless through sliding to always sticking."""
    w = inputs.draw("small_8192", seed=0)
    dt, e = w["dt"], w["e"]
    ctx = _ctx(w, 8192, dt)
    cur = {k: w[k] for k in ("x", "v", "r", "m", "id")}
    spins = 30.0 * np.random.default_rng(1).normal(size=(3, 8192))
    total = 0
    for _ in range(15):
        cur, spins, k = _step(ctx, cur, spins, mu, dt, e)
        total += k
    assert total > 200


def test_rollout_with_permuted_ids():
    """Ids a random permutation of the indices, the state kept in index order: the two
    rotational terms of the contact-point velocity are added in id order, so order by id
    and order by index must not be confused. 8 steps of 4000 spheres at 10x the time step,
    mu = 0.3, every step bit-identical."""
    w = inputs.draw("small_8192", seed=6, n=4000)
    dt = 10 * w["dt"]
    ctx = _ctx(w, 4000, dt)
    cur = {"x": w["x"], "v": w["v"], "r": w["r"], "m": w["m"],
           "id": np.random.default_rng(6).permutation(4000).astype(np.int32)}
    spins = 30.0 * np.random.default_rng(7).normal(size=(3, 4000))
    total = 0
    for _ in range(8):
        cur, spins, k = _step(ctx, cur, spins, 0.3, dt, w["e"])
        total += k
    assert total > 100


def test_head_on_without_spin_has_no_tangential_impulse():
    """A head-on pair of non-spinning spheres with mu = 0.3: the tangential contact
    velocity is exactly zero, so there is no tangential impulse (no 0/0 direction); bit-
    identical to the oracle, finite, and the spins stay zero."""
    w = dict(x=np.array([[0.5, 0.504], [0.5, 0.5], [0.5, 0.5]]), v=np.array([[1.0, -1.0], [0.0, 0.0], [0.0, 0.0]]),
             r=np.full(2, 0.001), m=np.array([1.0, 3.0]), id=np.arange(2, dtype=np.int32), e=0.9)
    ctx = pc.Context(2, 8, 3, 0.02, 0.9, pc.reach_of(w["r"], w["v"], 0.01))
    cur = {k: w[k] for k in ("x", "v", "r", "m", "id")}
    nxt, spins, k = _step(ctx, cur, np.zeros((3, 2)), 0.3, 0.01, 0.9)
    assert k == 1 and np.all(np.isfinite(nxt["v"])) and not spins.any()


def test_dense_full_size_step_bit_identical():
    """1,048,576 spheres of the dense workload, mu = 0.2, one step: every pair and bit."""
    w = inputs.draw("dense_1m", seed=2)
    n = w["x"].shape[1]
    ctx = _ctx(w, n, w["dt"])
    spins = 50.0 * np.random.default_rng(2).normal(size=(3, n))
    cur = {k: w[k] for k in ("x", "v", "r", "m", "id")}
    _, _, k = _step(ctx, cur, spins, 0.2, w["dt"], w["e"])
    assert k > 10000


def test_zero_friction_matches_pc_collide_and_keeps_spin():
    w = inputs.draw("dense_1m", seed=3, n=40000)
    dt = 5 * w["dt"]
    ctx = _ctx(w, 40000, dt)
    src = pc.State.from_arrays(w)
    a, b = pc.State.empty(40000), pc.State.empty(40000)
    ctx.collide(src, a, dt)
    spins = T(np.random.default_rng(3).normal(size=(3, 40000)))
    w_out = torch.empty_like(spins)
    ctx.collide_rot(src, b, spins, w_out, 0.0, dt)
    ctx.sync()
    for key in ("x", "v", "id"):
        assert torch.equal(getattr(a, key), getattr(b, key)), key
    perm = b.id.long()
    assert torch.equal(w_out, spins[:, perm])


def test_argument_checks():
    w = inputs.draw("small_8192", seed=4, n=100)
    ctx = _ctx(w, 100, w["dt"])
    src, dst = pc.State.from_arrays(w), pc.State.empty(100)
    s = T(np.zeros((3, 100)))
    for args in ((s, s, 0.1), (s, torch.empty_like(s), -0.1), (s, torch.empty_like(s), float("inf"))):
        with pytest.raises(pc.PcError) as ei:
            ctx.collide_rot(src, dst, args[0], args[1], args[2], w["dt"])
        assert ei.value.status == pc.PC_EINVAL
