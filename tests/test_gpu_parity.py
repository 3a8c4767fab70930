"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Collisions: pair sets, contact times, positions and velocities bit-identical.
Projection: fields within 1e-12 normwise per component (max |F - F_ref| / max |F_ref|).
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs
from tests.gpu_helpers import by_id, field_err, oracle_pairs, quad_weights

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_05340_gb300 import pc  # noqa: E402

FIELD_TOL = 1e-12


def make_ctx(w, n, dt, **kw):
    wl = w["workload"]
    reach = pc.reach_of(w["r"], w["v"], dt)
    return pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], reach, cutoff_sigmas=wl.cutoff_sigmas, **kw)


def compare_collide_step(ctx, src, dst, cur, dt, e):
    """One GPU step src->dst against one oracle step on cur (id order). Returns the new oracle state."""
    ctx.collide(src, dst, dt)
    ctx.sync()
    gids, gt = ctx.pairs()
    x1, v1, partner, tc, k = oracle.collide_step(cur["x"], cur["v"], cur["r"], cur["m"], cur["id"], e, dt)
    oids, ot = oracle_pairs(partner, tc, cur["id"])
    assert np.array_equal(gids, oids), "pair sets differ"
    assert np.array_equal(gt, ot), "contact times differ"
    g = by_id(dst.numpy())
    assert np.array_equal(g["id"], cur["id"])
    assert np.array_equal(g["v"], v1), "velocities differ"
    assert np.array_equal(g["x"], x1), "positions differ"
    assert np.array_equal(g["r"], cur["r"]) and np.array_equal(g["m"], cur["m"])
    if "q" in cur:
        assert np.array_equal(g["q"], cur["q"])
    nxt = dict(cur)
    nxt["x"], nxt["v"] = x1, v1
    return nxt, k


def test_small_rollout_bit_identical():
    """8192 spheres d=0.02, e=0.9, dt=2e-3: 100 steps, every step bit-identical."""
    w = inputs.draw("small_8192", seed=0)
    dt, e = w["dt"], w["e"]
    a = pc.State.from_arrays(w)
    b = pc.State.empty(a.n)
    ctx = make_ctx(w, a.n, dt)
    cur = {k: w[k] for k in ("x", "v", "r", "m", "id", "q")}
    total = 0
    for s in range(100):
        cur, k = compare_collide_step(ctx, a, b, cur, dt, e)
        total += k
        a, b = b, a
    assert total > 1000


@pytest.mark.parametrize("e", [0.0, 1.0])
def test_restitution_limits_rollout(e):
    """Perfectly inelastic (e = 0: the pair leaves with equal normal velocities) and
    elastic (e = 1) collisions: 20 steps of 4000 spheres at 5x the time step, every step
    bit-identical."""
    w = dict(inputs.draw("small_8192", seed=8, n=4000))
    w["e"] = e
    dt = 5 * w["dt"]
    a = pc.State.from_arrays(w)
    b = pc.State.empty(a.n)
    ctx = make_ctx(w, a.n, dt)
    cur = {k: w[k] for k in ("x", "v", "r", "m", "id", "q")}
    total = 0
    for _ in range(20):
        cur, k = compare_collide_step(ctx, a, b, cur, dt, e)
        total += k
        a, b = b, a
    assert total > 100


def test_dense_full_size_steps_bit_identical():
    """1,048,576 spheres (phi ~0.19) at the full size: 3 steps, every pair and bit."""
    w = inputs.draw("dense_1m", seed=1)
    dt, e = w["dt"], w["e"]
    a = pc.State.from_arrays(w)
    b = pc.State.empty(a.n)
    ctx = make_ctx(w, a.n, dt)
    cur = {k: w[k] for k in ("x", "v", "r", "m", "id", "q")}
    for s in range(3):
        cur, k = compare_collide_step(ctx, a, b, cur, dt, e)
        assert k > 20000
        st = ctx.stats()
        assert st["status"] == 0 and st["stencil"] == 1
        a, b = b, a


@pytest.mark.parametrize("n", [1, 2, 31, 33, 1007])
def test_ragged_sizes(n):
    w = inputs.draw("dense_1m", seed=3, n=n)
    dt = 30 * w["dt"]
    a = pc.State.from_arrays(w)
    b = pc.State.empty(n)
    ctx = make_ctx(w, n, dt)
    cur = {k: w[k] for k in ("x", "v", "r", "m", "id", "q")}
    for s in range(3):
        cur, _ = compare_collide_step(ctx, a, b, cur, dt, w["e"])
        a, b = b, a


def test_empty_input():
    w = inputs.draw("small_8192", n=16)
    ctx = make_ctx(w, 16, w["dt"])
    a, b = pc.State.empty(0), pc.State.empty(0)
    ctx.collide(a, b, 1e-3)
    f = ctx.new_field()
    ctx.project(a, f)
    ctx.sync()
    assert float(f.abs().max()) == 0.0


def test_pair_across_periodic_corner():
    """Two spheres approaching through the corner of the periodic cube."""
    x = np.array([[0.999, 0.001], [0.999, 0.001], [0.999, 0.001]])
    v = np.array([[1.0, -1.0], [1.0, -1.0], [1.0, -1.0]])
    d = dict(x=x, v=v, r=np.array([0.001, 0.001]), m=np.array([1.0, 2.0]), id=np.array([7, 3], np.int32),
             q=np.ones((4, 2)))
    a = pc.State.from_arrays(d)
    b = pc.State.empty(2)
    ctx = pc.Context(2, 8, 3, 0.02, 0.7, 0.01)
    cur = dict(d)
    cur = by_id(cur)
    nxt, k = compare_collide_step(ctx, a, b, cur, 1e-3, 0.7)
    assert k == 1


def test_free_flight_wraps_tiny_negative_positions_to_zero():
    """Free flight across x = 0 by less than half an ulp of 1: y - floor(y) rounds to 1.0,
    which the wrap maps to 0.0 (as in the oracle), so every coordinate stays in [0, 1);
    one ordinary wrap across x = 1 beside it."""
    x = np.array([[0.0, 0.9995, 1e-17], [0.2, 0.5, 0.7], [0.3, 0.5, 0.1]])
    v = np.array([[-1e-20, 0.002, -1e-16], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    d = dict(x=x, v=v, r=np.full(3, 1e-3), m=np.ones(3), id=np.array([2, 0, 1], np.int32), q=np.ones((4, 3)))
    a, b = pc.State.from_arrays(d), pc.State.empty(3)
    ctx = pc.Context(3, 8, 3, 0.02, 0.9, pc.reach_of(d["r"], v, 0.5))
    nxt, k = compare_collide_step(ctx, a, b, by_id(dict(d)), 0.5, 0.9)
    g = b.numpy()
    assert k == 0 and np.all((g["x"] >= 0.0) & (g["x"] < 1.0))
    assert nxt["x"][0, 1] == 0.0 and nxt["x"][0, 2] == 0.0  # ids 1 and 2


def test_get_pairs_copies_a_prefix_and_reports_the_count():
    """pc_get_pairs with a capacity below the pair count writes the first pairs of the
    sorted list and still reports the full count."""
    w = inputs.draw("small_8192", seed=9, n=3000)
    dt = 10 * w["dt"]
    ctx = make_ctx(w, 3000, dt)
    a, b = pc.State.from_arrays(w), pc.State.empty(3000)
    ctx.collide(a, b, dt)
    ctx.sync()
    ids, t = ctx.pairs()
    assert len(ids) > 10
    part_ids, part_t, cnt = np.zeros(10, np.int32), np.zeros(5), ctypes.c_int64()
    st = pc.library().pc_get_pairs(ctx._h, part_ids.ctypes.data_as(ctypes.c_void_p),
                                   part_t.ctypes.data_as(ctypes.c_void_p), 5, ctypes.byref(cnt))
    assert st == pc.PC_OK and cnt.value == len(ids)
    assert np.array_equal(part_ids.reshape(5, 2), ids[:5]) and np.array_equal(part_t, t[:5])


def test_grazing_double_root_is_not_a_collision():
    """A sphere passing another at exactly R while approaching (binary-exact values, so
    b^2 - a c is exactly 0): a double root, no collision; beside it a head-on pair that
    does collide. Pairs, times, x and v bit-identical to the oracle."""
    x = np.array([[0.375, 0.5, 0.125, 0.1875], [0.5625, 0.5, 0.125, 0.125], [0.5, 0.5, 0.875, 0.875]])
    v = np.array([[1.0, 0.0, 0.5, -0.5], [0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0]])
    d = dict(x=x, v=v, r=np.array([0.03125, 0.03125, 0.0078125, 0.0078125]), m=np.array([1.0, 2.0, 1.0, 1.5]),
             id=np.arange(4, dtype=np.int32), q=np.ones((4, 4)))
    a, b = pc.State.from_arrays(d), pc.State.empty(4)
    ctx = pc.Context(4, 8, 3, 0.02, 0.9, pc.reach_of(d["r"], v, 0.2))
    _, k = compare_collide_step(ctx, a, b, by_id(dict(d)), 0.2, 0.9)
    assert k == 1
    ids, t = ctx.pairs()
    assert ids.tolist() == [[2, 3]] and t[0] == 0.046875


def test_chain_matched_one_pair_per_round():
    """Six spheres in a row, each faster to the right than its right neighbour, with gaps
    growing along the row: contact times grow along the chain, so the matching rounds
    commit one pair per round ((0,1), then (2,3), then (4,5)); bit-identical to the oracle."""
    gaps = [0.010, 0.012, 0.014, 0.016, 0.018]
    r0 = 0.01
    xs = [0.2]
    for g in gaps:
        xs.append(xs[-1] + 2 * r0 + g)
    n = 6
    x = np.array([xs, [0.5] * n, [0.5] * n])
    v = np.array([[-0.5 * i for i in range(n)], [0.0] * n, [0.0] * n])
    d = dict(x=x, v=v, r=np.full(n, r0), m=np.ones(n), id=np.arange(n, dtype=np.int32), q=np.ones((4, n)))
    a, b = pc.State.from_arrays(d), pc.State.empty(n)
    ctx = pc.Context(n, 8, 3, 0.02, 0.9, pc.reach_of(d["r"], v, 0.05))
    _, k = compare_collide_step(ctx, a, b, by_id(dict(d)), 0.05, 0.9)
    assert k == 3
    assert ctx.pairs()[0].tolist() == [[0, 1], [2, 3], [4, 5]]


@pytest.mark.parametrize("target_reach", [0.45, 0.49])
def test_reach_spanning_the_box(target_reach):
    """A step whose reach exceeds a third of the box (but stays below half of it, where the
    minimum image is the only image that can collide): the grid keeps 3 cells per side and
    the stencil covers every cell once; pairs, times, x and v bit-identical to the oracle."""
    rng = np.random.default_rng(int(target_reach * 100))
    n = 500
    d = dict(x=rng.random((3, n)), v=rng.normal(size=(3, n)), r=np.full(n, 0.015), m=rng.uniform(0.5, 2.0, n),
             id=np.arange(n, dtype=np.int32), q=rng.normal(size=(4, n)))
    vmax = float(np.sqrt((d["v"] ** 2).sum(0)).max())
    dt = (target_reach - 0.03) / (2 * vmax)
    a, b = pc.State.from_arrays(d), pc.State.empty(n)
    ctx = pc.Context(n, 8, 3, 0.02, 0.9, pc.reach_of(d["r"], d["v"], dt, margin=1.0))
    assert ctx.cells_per_side == 3
    _, k = compare_collide_step(ctx, a, b, by_id(dict(d)), dt, 0.9)
    assert k > 5


def test_reach_above_the_hint():
    """A step whose actual reach (0.1) is 2.5 times the hint (0.04): 24 cells per side and a
    stencil of 3 cells on each side (7 of 24 per axis), whose rows wrap at the faces; pairs,
    times, x and v bit-identical to the oracle."""
    rng = np.random.default_rng(11)
    n = 3000
    d = dict(x=rng.random((3, n)), v=rng.normal(size=(3, n)), r=np.full(n, 0.008), m=rng.uniform(0.5, 2.0, n),
             id=np.arange(n, dtype=np.int32), q=rng.normal(size=(4, n)))
    vmax = float(np.sqrt((d["v"] ** 2).sum(0)).max())
    dt = (0.1 - 0.016) / (2 * vmax)
    a, b = pc.State.from_arrays(d), pc.State.empty(n)
    ctx = pc.Context(n, 8, 3, 0.02, 0.9, 0.04)
    assert ctx.cells_per_side == 24
    _, k = compare_collide_step(ctx, a, b, by_id(dict(d)), dt, 0.9)
    st = ctx.stats()
    assert k > 5 and st["status"] == 0 and st["stencil"] == 3


def test_reach_of_half_the_box_is_refused():
    """A reach of half the box or more: pc_init refuses such a hint on the host, and a step
    whose actual reach reaches 0.5 under a smaller hint is refused on the GPU (PC_EINVAL
    from pc_sync), since another periodic image than the minimum one could then collide."""
    with pytest.raises(pc.PcError, match="PC_EINVAL"):
        pc.Context(10, 8, 3, 0.02, 0.9, 0.5)
    rng = np.random.default_rng(80)
    n = 500
    d = dict(x=rng.random((3, n)), v=rng.normal(size=(3, n)), r=np.full(n, 0.015), m=rng.uniform(0.5, 2.0, n),
             id=np.arange(n, dtype=np.int32), q=rng.normal(size=(4, n)))
    vmax = float(np.sqrt((d["v"] ** 2).sum(0)).max())
    dt = (0.8 - 0.03) / (2 * vmax)
    a, b = pc.State.from_arrays(d), pc.State.empty(n)
    ctx = pc.Context(n, 8, 3, 0.02, 0.9, 0.3)
    ctx.collide(a, b, dt)
    with pytest.raises(pc.PcError, match="PC_EINVAL"):
        ctx.sync()
    ctx.sync()  # the status is cleared once reported


def test_clustered_cells():
    """Many particles in few cells (high occupancy, many candidates per particle)."""
    w = inputs.draw("dense_1m", seed=5, n=3000)
    w["x"] = w["x"] * 0.25  # compress into 1/64 of the box: overlapping pairs are ignored (c <= 0)
    dt = 3 * w["dt"]
    a = pc.State.from_arrays(w)
    b = pc.State.empty(a.n)
    ctx = make_ctx(w, a.n, dt, cand_cap=32)
    cur = {k: w[k] for k in ("x", "v", "r", "m", "id", "q")}
    for s in range(3):
        cur, k = compare_collide_step(ctx, a, b, cur, dt, w["e"])
        a, b = b, a


def test_candidate_overflow_is_reported():
    # particle 0 has two approaching partners; with cand_cap=1 the list overflows
    x = np.array([[0.5, 0.503, 0.497], [0.5, 0.5, 0.5], [0.5, 0.5, 0.5]])
    v = np.array([[0.0, -1.0, 1.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    d = dict(x=x, v=v, r=np.full(3, 0.001), m=np.ones(3), id=np.arange(3, dtype=np.int32))
    a = pc.State.from_arrays(d, with_q=False)
    b = pc.State.empty(3, with_q=False)
    ctx = pc.Context(3, 8, 3, 0.02, 0.9, 0.01, cand_cap=1)
    ctx.collide(a, b, 1e-2)
    with pytest.raises(pc.PcError) as ei:
        ctx.sync()
    assert ei.value.status == pc.PC_ECAPACITY


def test_invalid_positions_are_reported():
    d = dict(x=np.array([[0.5, 1.5], [0.5, 0.5], [0.5, 0.5]]), v=np.zeros((3, 2)), r=np.full(2, 0.001),
             m=np.ones(2), id=np.arange(2, dtype=np.int32))
    a = pc.State.from_arrays(d, with_q=False)
    b = pc.State.empty(2, with_q=False)
    ctx = pc.Context(2, 8, 3, 0.02, 0.9, 0.01)
    ctx.collide(a, b, 1e-3)
    with pytest.raises(pc.PcError) as ei:
        ctx.sync()
    assert ei.value.status == pc.PC_EINVAL


def test_determinism_bitwise():
    w = inputs.draw("small_8192", seed=2)
    outs = []
    for rep in range(2):
        a = pc.State.from_arrays(w)
        b = pc.State.empty(a.n)
        ctx = make_ctx(w, a.n, w["dt"])
        f = ctx.new_field()
        for s in range(10):
            ctx.collide(a, b, w["dt"])
            a, b = b, a
        ctx.project(a, f)
        ctx.sync()
        outs.append((a.numpy(), f.cpu().numpy()))
    for k in ("x", "v", "id"):
        assert np.array_equal(outs[0][0][k], outs[1][0][k])
    assert np.array_equal(outs[0][1], outs[1][1])


# ----------------------------------------------------------------- projection

def test_project_small_full_field():
    w = inputs.draw("small_8192", seed=0)
    wl = w["workload"]
    a = pc.State.from_arrays(w)
    ctx = make_ctx(w, a.n, w["dt"])
    f = ctx.new_field()
    ctx.project(a, f)
    ctx.sync()
    F = f.cpu().numpy()
    R, Z = oracle.project(w["x"], w["q"], wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
    err = field_err(F, R)
    assert np.all(err <= FIELD_TOL), err
    tot = np.einsum("ecg,g->c", F, quad_weights(wl.ne, wl.degree))
    assert np.all(np.abs(tot - w["q"].sum(axis=1)) <= 1e-12 * np.abs(w["q"]).sum(axis=1))


def test_project_after_rollout_matches_oracle():
    """collide+project steps: the field of the GPU state equals the oracle's field of the oracle state."""
    w = inputs.draw("small_8192", seed=4)
    wl = w["workload"]
    a = pc.State.from_arrays(w)
    b = pc.State.empty(a.n)
    ctx = make_ctx(w, a.n, w["dt"])
    f = ctx.new_field()
    cur = {k: w[k] for k in ("x", "v", "r", "m", "id", "q")}
    for s in range(5):
        cur, _ = compare_collide_step(ctx, a, b, cur, w["dt"], w["e"])
        ctx.project(b, f)
        a, b = b, a
    ctx.sync()
    R, _ = oracle.project(cur["x"], cur["q"], wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
    assert np.all(field_err(f.cpu().numpy(), R) <= FIELD_TOL)


def _neighbourhood_particles(x, elems, ne, rho):
    e = np.minimum((x * ne).astype(np.int64), ne - 1)
    keep = np.zeros(x.shape[1], bool)
    for el in elems:
        ex, ey, ez = el % ne, (el // ne) % ne, el // (ne * ne)
        d = [((e[0] - ex + ne // 2) % ne) - ne // 2, ((e[1] - ey + ne // 2) % ne) - ne // 2,
             ((e[2] - ez + ne // 2) % ne) - ne // 2]
        keep |= (np.abs(d[0]) <= rho) & (np.abs(d[1]) <= rho) & (np.abs(d[2]) <= rho)
    return keep


@pytest.mark.parametrize("name,n", [("dense_1m", None), ("dense_1m", 50000)])
def test_project_dense_sampled_elements(name, n):
    """Full-size dense field: conservation everywhere, and sampled elements against the
    oracle run on the particles that can reach them."""
    w = inputs.draw(name, seed=6, n=n)
    wl = w["workload"]
    a = pc.State.from_arrays(w)
    ctx = make_ctx(w, a.n, w["dt"])
    f = ctx.new_field()
    ctx.project(a, f)
    ctx.sync()
    F = f.cpu().numpy()
    tot = np.einsum("ecg,g->c", F, quad_weights(wl.ne, wl.degree))
    assert np.all(np.abs(tot - w["q"].sum(axis=1)) <= 1e-11 * np.abs(w["q"]).sum(axis=1))
    rng = np.random.default_rng(0)
    elems = rng.choice(wl.ne ** 3, 6, replace=False)
    keep = _neighbourhood_particles(w["x"], elems, wl.ne, 1)
    R, _ = oracle.project(w["x"][:, keep], w["q"][:, keep], wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
    scale = np.abs(F).max(axis=(0, 2))
    err = np.abs(F[elems] - R[elems]).max(axis=(0, 2)) / scale
    assert np.all(err <= FIELD_TOL), err


@pytest.mark.parametrize("degree,ne,sigma", [(0, 6, 0.03), (1, 6, 0.03), (2, 6, 0.03), (3, 6, 0.03), (4, 6, 0.03),
                                               (5, 6, 0.03), (6, 6, 0.03), (7, 6, 0.03), (5, 8, 0.05), (7, 8, 0.05)])
def test_project_every_degree(degree, ne, sigma):
    """Full field against the oracle for N + 1 = 1..8 Gauss nodes per axis (every shape of
    the tensor-core deposit), and with a support spanning 2 elements on each side
    (sigma 0.05 on 8 elements per side)."""
    w = inputs.draw("small_8192", seed=12 + degree, n=2500)
    a = pc.State.from_arrays(w)
    ctx = pc.Context(a.n, ne, degree, sigma, w["e"], 0.05)
    f = ctx.new_field()
    ctx.project(a, f)
    ctx.sync()
    R, _ = oracle.project(w["x"], w["q"], ne, degree, sigma, 3.0)
    assert np.all(field_err(f.cpu().numpy(), R) <= FIELD_TOL)


@pytest.mark.parametrize("degree", [3, 7])
def test_project_crowded_element_in_segments(degree):
    """6000 particles inside one element's neighbourhood (an element keeps more of them
    than one accumulation segment holds, 1024 for degree 3 and 512 for degree 7, so its
    deposit is accumulated in several segments) and a few far away: the full field
    against the oracle, and conservation."""
    rng = np.random.default_rng(21)
    n = 6000
    x = 0.5 + 0.05 * (rng.random((3, n)) - 0.5)
    x[:, :40] = rng.random((3, 40))
    d = dict(x=x, v=np.zeros((3, n)), r=np.full(n, 1e-4), m=np.ones(n), id=np.arange(n, dtype=np.int32),
             q=rng.normal(size=(4, n)))
    a = pc.State.from_arrays(d)
    ctx = pc.Context(n, 8, degree, 0.02, 0.9, 0.05)
    f = ctx.new_field()
    ctx.project(a, f)
    ctx.sync()
    F = f.cpu().numpy()
    R, _ = oracle.project(x, d["q"], 8, degree, 0.02, 3.0)
    assert np.all(field_err(F, R) <= FIELD_TOL)
    tot = np.einsum("ecg,g->c", F, quad_weights(8, degree))
    assert np.all(np.abs(tot - d["q"].sum(axis=1)) <= 1e-12 * np.abs(d["q"]).sum(axis=1))


@pytest.mark.parametrize("cs", [1.0, 6.0])
def test_project_other_cutoffs(cs):
    """Cutoff 1 sigma (most nodes near the edge) and 6 sigma (exp down to -18)."""
    w = inputs.draw("small_8192", seed=7, n=3000)
    wl = w["workload"]
    a = pc.State.from_arrays(w)
    ctx = pc.Context(a.n, wl.ne, wl.degree, wl.sigma, w["e"], 0.05, cutoff_sigmas=cs)
    f = ctx.new_field()
    ctx.project(a, f)
    ctx.sync()
    R, _ = oracle.project(w["x"], w["q"], wl.ne, wl.degree, wl.sigma, cs)
    assert np.all(field_err(f.cpu().numpy(), R) <= FIELD_TOL)


def test_project_dirac_limit_on_node():
    """sigma far below the node spacing with the particle on a node: F = q / W at that node."""
    ne, n1 = 8, 4
    eta, om = np.polynomial.legendre.leggauss(n1)
    h = 1 / ne
    xp = np.array([[(3 + 0.5 * (eta[1] + 1)) * h], [(5 + 0.5 * (eta[2] + 1)) * h], [(6 + 0.5 * (eta[0] + 1)) * h]])
    d = dict(x=xp, v=np.zeros((3, 1)), r=np.full(1, 1e-3), m=np.ones(1), id=np.zeros(1, np.int32),
             q=np.array([[1.0], [2.0], [-3.0], [4.0]]))
    a = pc.State.from_arrays(d)
    ctx = pc.Context(1, ne, n1 - 1, 1e-4, 0.9, 0.05)
    f = ctx.new_field()
    ctx.project(a, f)
    ctx.sync()
    R, _ = oracle.project(xp, d["q"], ne, n1 - 1, 1e-4, 3.0)
    F = f.cpu().numpy()
    assert np.all(field_err(F, R) <= FIELD_TOL)
    e = (6 * ne + 5) * ne + 3
    g = (0 * n1 + 2) * n1 + 1
    W = om[1] * om[2] * om[0] * (h / 2) ** 3
    assert np.allclose(F[e, :, g], d["q"][:, 0] / W, rtol=1e-12)
