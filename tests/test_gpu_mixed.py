"""Mixed-precision path (FP32 cell-relative storage, tensor-core projection) through
the C ABI, against the oracle.

Collisions: pairs, cells, offsets and velocities bit-identical to the oracle's
cell-relative step. Projection: FP16 split within 1e-5 normwise per component of
the FP64 oracle field of the stored (dequantized) state; BF16 within 1e-4.
"""
import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs
from tests.gpu_helpers import by_id, field_err, oracle_pairs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_05340_gb300 import pc  # noqa: E402

F16_TOL = 1e-5
BF16_TOL = 1e-4


def mixed_state(w, ctx):
    """FP64 workload -> GPU FP32 cell-relative state via pc_quantize."""
    s64 = pc.State.from_arrays(w)
    s32 = pc.StateF32.empty(s64.n)
    ctx.quantize(s64, s32)
    ctx.sync()
    return s32


def test_quantize_matches_oracle_rule():
    w = inputs.draw("mixed_16m", seed=0, n=20000)
    ctx = pc.Context(w["x"].shape[1], 64, 7, 4e-3, w["e"], pc.reach_of(w["r"], w["v"], w["dt"]))
    s32 = mixed_state(w, ctx)
    g = s32.numpy()
    cell, o = oracle.quantize(w["x"], ctx.cells_per_side)
    assert np.array_equal(g["cell"], cell) and np.array_equal(g["o"], o)
    assert np.array_equal(g["v"], w["v"].astype(np.float32))
    assert np.all((g["o"] >= 0) & (g["o"] < 1))


@pytest.mark.parametrize("name,n,dtmul", [("mixed_16m", 3000, 60), ("dense_1m", 2500, 25), ("small_8192", 2000, 1)])
def test_collide_f32_bit_identical(name, n, dtmul):
    w = inputs.draw(name, seed=1, n=n)
    dt = dtmul * w["dt"]
    ctx = pc.Context(n, w["workload"].ne, w["workload"].degree, w["workload"].sigma, w["e"],
                     pc.reach_of(w["r"], w["v"], dt))
    nc = ctx.cells_per_side
    a = mixed_state(w, ctx)
    b = pc.StateF32.empty(n)
    cur = by_id(a.numpy())
    total = 0
    for step in range(5):
        ctx.collide_f32(a, b, dt)
        ctx.sync()
        gids, gt = ctx.pairs()
        cell, o, v, partner, tc, k = oracle.collide_step_cellrel(cur["cell"], cur["o"], cur["v"], cur["r"], cur["m"],
                                                                 cur["id"], nc, w["e"], dt)
        oids, ot = oracle_pairs(partner, tc, cur["id"])
        assert np.array_equal(gids, oids) and np.array_equal(gt, ot)
        g = by_id(b.numpy())
        assert np.array_equal(g["cell"], cell), "cells differ"
        assert np.array_equal(g["o"], o), "offsets differ"
        assert np.array_equal(g["v"], v), "velocities differ"
        assert np.array_equal(g["q"], cur["q"]) and np.array_equal(g["m"], cur["m"])
        cur = dict(cur)
        cur["cell"], cur["o"], cur["v"] = cell, o, v
        total += k
        a, b = b, a
    assert total > 0


def test_collide_f32_permuted_ids():
    """Ids a random permutation of the indices, the state kept in index order (order by
    id and by index differ inside every cell): 4 steps of 3000 spheres of the mixed law,
    pairs, times, cells, offsets and velocities bit-identical, compared by id."""
    w = inputs.draw("mixed_16m", seed=4, n=3000)
    w["id"] = np.random.default_rng(4).permutation(3000).astype(np.int32)
    dt = 60 * w["dt"]
    ctx = pc.Context(3000, w["workload"].ne, w["workload"].degree, w["workload"].sigma, w["e"],
                     pc.reach_of(w["r"], w["v"], dt))
    nc = ctx.cells_per_side
    a = mixed_state(w, ctx)
    b = pc.StateF32.empty(3000)
    cur = a.numpy()
    total = 0
    for _ in range(4):
        ctx.collide_f32(a, b, dt)
        ctx.sync()
        gids, gt = ctx.pairs()
        cell, o, v, partner, tc, k = oracle.collide_step_cellrel(cur["cell"], cur["o"], cur["v"], cur["r"], cur["m"],
                                                                 cur["id"], nc, w["e"], dt)
        oids, ot = oracle_pairs(partner, tc, cur["id"])
        assert np.array_equal(gids, oids) and np.array_equal(gt, ot)
        g, ref = by_id(b.numpy()), by_id(dict(cell=cell, o=o, v=v, id=cur["id"]))
        for key in ("cell", "o", "v"):
            assert np.array_equal(g[key], ref[key]), key
        cur = dict(cur)
        cur["cell"], cur["o"], cur["v"] = cell, o, v
        total += k
        a, b = b, a
    assert total > 0


@pytest.mark.parametrize("target_reach", [0.45, 0.49])
def test_collide_f32_reach_spanning_the_box(target_reach):
    """Mixed path with a reach above a third of the box (below half of it): 3 cells per
    side, the stencil covers every cell once; pairs, times, cells, offsets and velocities
    bit-identical."""
    rng = np.random.default_rng(int(target_reach * 100) + 1)
    n = 500
    w = dict(x=rng.random((3, n)), v=rng.normal(size=(3, n)), r=np.full(n, 0.015), m=rng.uniform(0.5, 2.0, n),
             id=np.arange(n, dtype=np.int32), q=rng.normal(size=(4, n)))
    vmax = float(np.sqrt((w["v"] ** 2).sum(0)).max())
    dt = (target_reach - 0.03) / (2 * vmax)
    ctx = pc.Context(n, 8, 3, 0.02, 0.9, pc.reach_of(w["r"], w["v"], dt, margin=1.0))
    assert ctx.cells_per_side == 3
    a = mixed_state(w, ctx)
    b = pc.StateF32.empty(n)
    cur = by_id(a.numpy())
    ctx.collide_f32(a, b, dt)
    ctx.sync()
    gids, gt = ctx.pairs()
    cell, o, v, partner, tc, k = oracle.collide_step_cellrel(cur["cell"], cur["o"], cur["v"], cur["r"], cur["m"],
                                                             cur["id"], 3, 0.9, dt)
    oids, ot = oracle_pairs(partner, tc, cur["id"])
    assert k > 5 and np.array_equal(gids, oids) and np.array_equal(gt, ot)
    g = by_id(b.numpy())
    for key, ref in (("cell", cell), ("o", o), ("v", v)):
        assert np.array_equal(g[key], ref), key


def test_collide_f32_reach_above_the_hint():
    """Mixed path, actual reach 0.076 under a hint of 0.04: 24 cells per side and a stencil
    of 2 cells on each side (5 of 24 per axis) whose rows wrap at the faces; the largest
    move, 0.03, stays within a cell (1/24); pairs, times, cells, offsets and velocities
    bit-identical."""
    rng = np.random.default_rng(12)
    n = 3000
    w = dict(x=rng.random((3, n)), v=rng.normal(size=(3, n)), r=np.full(n, 0.008), m=rng.uniform(0.5, 2.0, n),
             id=np.arange(n, dtype=np.int32), q=rng.normal(size=(4, n)))
    vmax = float(np.sqrt((w["v"] ** 2).sum(0)).max())
    dt = (0.076 - 0.016) / (2 * vmax)
    ctx = pc.Context(n, 8, 3, 0.02, 0.9, 0.04)
    assert ctx.cells_per_side == 24
    a = mixed_state(w, ctx)
    b = pc.StateF32.empty(n)
    cur = by_id(a.numpy())
    ctx.collide_f32(a, b, dt)
    ctx.sync()
    st = ctx.stats()
    assert st["status"] == 0 and st["stencil"] == 2
    gids, gt = ctx.pairs()
    cell, o, v, partner, tc, k = oracle.collide_step_cellrel(cur["cell"], cur["o"], cur["v"], cur["r"], cur["m"],
                                                             cur["id"], 24, 0.9, dt)
    oids, ot = oracle_pairs(partner, tc, cur["id"])
    assert k > 5 and np.array_equal(gids, oids) and np.array_equal(gt, ot)
    g = by_id(b.numpy())
    for key, ref in (("cell", cell), ("o", o), ("v", v)):
        assert np.array_equal(g[key], ref), key


def test_collide_f32_reach_of_half_the_box_is_refused():
    """A mixed step whose actual reach is 0.8 box lengths under a hint of 0.3: refused on
    the GPU (PC_EINVAL from pc_sync), as the FP64 path refuses it."""
    rng = np.random.default_rng(81)
    n = 500
    w = dict(x=rng.random((3, n)), v=rng.normal(size=(3, n)), r=np.full(n, 0.015), m=rng.uniform(0.5, 2.0, n),
             id=np.arange(n, dtype=np.int32), q=rng.normal(size=(4, n)))
    vmax = float(np.sqrt((w["v"] ** 2).sum(0)).max())
    dt = (0.8 - 0.03) / (2 * vmax)
    ctx = pc.Context(n, 8, 3, 0.02, 0.9, 0.3)
    a = mixed_state(w, ctx)
    b = pc.StateF32.empty(n)
    ctx.collide_f32(a, b, dt)
    with pytest.raises(pc.PcError, match="PC_EINVAL"):
        ctx.sync()
    ctx.sync()


def _ctx_10_cells(n):
    """A context whose collision grid has 10 cells per side (reach hint 0.095)."""
    ctx = pc.Context(n, 8, 3, 0.02, 1.0, 0.095)
    assert ctx.cells_per_side == 10
    return ctx


def test_collide_f32_tiny_negative_offset_stays_in_the_cell():
    """Free flight to an offset of -2^-30 cells (dt nc = 1, v = -2^-29): adding one cell
    rounds to 1.0 in FP32, so the offset becomes 0 in the same cell, as in the oracle."""
    ctx = _ctx_10_cells(4)
    d = dict(id=np.arange(4, dtype=np.int32), cell=np.array([3 + 10 * (4 + 10 * 5), 1, 222, 777], np.int32),
             o=np.full((3, 4), 0.5, np.float32), v=np.zeros((3, 4), np.float32), r=np.full(4, 1e-3, np.float32),
             m=np.ones(4, np.float32), q=np.zeros((4, 4), np.float32))
    d["o"][0, 0] = 2.0 ** -30
    d["v"][0, 0] = -(2.0 ** -29)
    a, b = pc.StateF32.from_arrays(d), pc.StateF32.empty(4)
    ctx.collide_f32(a, b, 0.1)
    ctx.sync()
    c1, o1, v1, partner, tc, k = oracle.collide_step_cellrel(d["cell"], d["o"], d["v"], d["r"], d["m"], d["id"], 10,
                                                             1.0, 0.1)
    g = by_id(b.numpy())
    assert k == 0 and c1[0] == d["cell"][0] and o1[0, 0] == 0.0
    assert np.array_equal(g["cell"], c1) and np.array_equal(g["o"], o1) and np.array_equal(g["v"], v1)


def test_collide_f32_pair_wraps_through_the_lower_face():
    """A pair colliding near x = 0 (e = 1, equal masses): the struck sphere leaves through
    the lower face and wraps to cell 9 of 10; pair, cells, offsets and velocities
    bit-identical to the oracle's cell-relative step."""
    ctx = _ctx_10_cells(2)
    w = dict(x=np.array([[0.03, 0.045], [0.5, 0.5], [0.5, 0.5]]), v=np.array([[0.0, -2.0], [0.0, 0.0], [0.0, 0.0]]),
             r=np.full(2, 0.002), m=np.ones(2), id=np.arange(2, dtype=np.int32), q=np.zeros((4, 2)))
    a = mixed_state(w, ctx)
    b = pc.StateF32.empty(2)
    cur = by_id(a.numpy())
    ctx.collide_f32(a, b, 0.03)
    ctx.sync()
    gids, gt = ctx.pairs()
    c1, o1, v1, partner, tc, k = oracle.collide_step_cellrel(cur["cell"], cur["o"], cur["v"], cur["r"], cur["m"],
                                                             cur["id"], 10, 1.0, 0.03)
    oids, ot = oracle_pairs(partner, tc, cur["id"])
    assert k == 1 and c1[0] % 10 == 9
    assert np.array_equal(gids, oids) and np.array_equal(gt, ot)
    g = by_id(b.numpy())
    for key, ref in (("cell", c1), ("o", o1), ("v", v1)):
        assert np.array_equal(g[key], ref), key


def test_collide_f32_collided_offset_that_rounds_to_one_is_carried():
    """A head-on pair (e = 1) with dt chosen so that the struck sphere ends 1e-9 cells below
    the face x = 4 cells: its FP32 offset rounds to 1.0 and is stored as offset 0 of cell 4;
    pair, cells, offsets and velocities bit-identical to the oracle."""
    ctx = _ctx_10_cells(2)
    w = dict(x=np.array([[0.30, 0.36], [0.55, 0.55], [0.45, 0.45]]), v=np.array([[1.0, -1.0], [0.0, 0.0], [0.0, 0.0]]),
             r=np.full(2, 0.01), m=np.ones(2), id=np.arange(2, dtype=np.int32), q=np.zeros((4, 2)))
    a = mixed_state(w, ctx)
    cur = by_id(a.numpy())
    xd = oracle.dequantize(cur["cell"], cur["o"], 10) * 10
    R = (float(cur["r"][0]) + float(cur["r"][1])) * 10
    t = (xd[0, 1] - xd[0, 0] - R) / 20.0
    dt = t + (4.0 - 1e-9 - (xd[0, 1] - t * 10)) / 10
    b = pc.StateF32.empty(2)
    ctx.collide_f32(a, b, dt)
    ctx.sync()
    gids, gt = ctx.pairs()
    c1, o1, v1, partner, tc, k = oracle.collide_step_cellrel(cur["cell"], cur["o"], cur["v"], cur["r"], cur["m"],
                                                             cur["id"], 10, 1.0, dt)
    oids, ot = oracle_pairs(partner, tc, cur["id"])
    assert k == 1 and c1[1] % 10 == 4 and o1[0, 1] == 0.0
    assert np.array_equal(gids, oids) and np.array_equal(gt, ot)
    g = by_id(b.numpy())
    for key, ref in (("cell", c1), ("o", o1), ("v", v1)):
        assert np.array_equal(g[key], ref), key


def _oracle_field_of(s32np, nc, wl, ne=None):
    x = oracle.dequantize(s32np["cell"], s32np["o"], nc)
    return oracle.project(x, s32np["q"].astype(np.float64), ne or wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)[0]


@pytest.mark.parametrize("tc,tol", [("f16", F16_TOL), ("bf16", BF16_TOL)])
def test_project_f32_reduced_mesh(tc, tol):
    """16^3 mesh, degree 7, sigma = 0.016 (3 sigma < h), 20000 particles."""
    w = inputs.draw("mixed_16m", seed=2, n=20000)
    ctx = pc.Context(w["x"].shape[1], 16, 7, 0.016, w["e"], pc.reach_of(w["r"], w["v"], w["dt"]))
    s32 = mixed_state(w, ctx)
    f = ctx.new_field_f32()
    ctx.project_f32(s32, f, tc)
    ctx.sync()
    F = f.cpu().numpy().astype(np.float64)
    g = s32.numpy()
    x = oracle.dequantize(g["cell"], g["o"], ctx.cells_per_side)
    R, _ = oracle.project(x, g["q"].astype(np.float64), 16, 7, 0.016, 3.0)
    err = field_err(F, R)
    print("normwise error per component (%s):" % tc, err)
    assert np.all(err <= tol), err


@pytest.mark.parametrize("degree", range(8))
@pytest.mark.parametrize("tc,tol", [("f16", F16_TOL), ("bf16", BF16_TOL)])
def test_project_f32_every_degree(degree, tc, tol):
    """Every compiled degree of the tensor-core deposit (n1 = 1..8) on a 6^3 mesh with
    3 sigma = 0.9 h and about 14 particles per element (several 32-particle chunks per
    element, the last one partial), against the FP64 oracle."""
    n, ne, sigma = 3000, 6, 0.05
    w = inputs.draw("mixed_16m", seed=10 + degree, n=n)
    ctx = pc.Context(n, ne, degree, sigma, w["e"], pc.reach_of(w["r"], w["v"], w["dt"]))
    s32 = mixed_state(w, ctx)
    f = ctx.new_field_f32()
    ctx.project_f32(s32, f, tc)
    ctx.sync()
    g = s32.numpy()
    x = oracle.dequantize(g["cell"], g["o"], ctx.cells_per_side)
    R, _ = oracle.project(x, g["q"].astype(np.float64), ne, degree, sigma, 3.0)
    err = field_err(f.cpu().numpy().astype(np.float64), R)
    assert np.all(err <= tol), (degree, tc, err)


def test_project_f32_crowded_elements():
    """About 470 particles per element of a 4^3 mesh (degree 2): elements of many full
    chunks plus a partial one, and more kept particles than the worker's ring holds."""
    n, ne, degree, sigma = 30000, 4, 2, 0.06
    w = inputs.draw("mixed_16m", seed=21, n=n)
    ctx = pc.Context(n, ne, degree, sigma, w["e"], pc.reach_of(w["r"], w["v"], w["dt"]))
    s32 = mixed_state(w, ctx)
    f = ctx.new_field_f32()
    ctx.project_f32(s32, f, "f16")
    ctx.sync()
    g = s32.numpy()
    x = oracle.dequantize(g["cell"], g["o"], ctx.cells_per_side)
    R, _ = oracle.project(x, g["q"].astype(np.float64), ne, degree, sigma, 3.0)
    assert np.all(field_err(f.cpu().numpy().astype(np.float64), R) <= F16_TOL)


@pytest.mark.parametrize("n", [1, 17, 300])
def test_project_f32_small_counts(n):
    w = inputs.draw("small_8192", seed=3, n=n)
    wl = w["workload"]
    ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], w["dt"]))
    s32 = mixed_state(w, ctx)
    f = ctx.new_field_f32()
    ctx.project_f32(s32, f, "f16")
    ctx.sync()
    g = s32.numpy()
    x = oracle.dequantize(g["cell"], g["o"], ctx.cells_per_side)
    R, _ = oracle.project(x, g["q"].astype(np.float64), wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
    assert np.all(field_err(f.cpu().numpy().astype(np.float64), R) <= F16_TOL)


def test_project_f32_deterministic():
    w = inputs.draw("mixed_16m", seed=4, n=20000)
    ctx = pc.Context(w["x"].shape[1], 16, 7, 0.016, w["e"], pc.reach_of(w["r"], w["v"], w["dt"]))
    s32 = mixed_state(w, ctx)
    f1, f2 = ctx.new_field_f32(), ctx.new_field_f32()
    ctx.project_f32(s32, f1)
    ctx.project_f32(s32, f2)
    ctx.sync()
    assert torch.equal(f1, f2)


@pytest.fixture(scope="module")
def full16():
    """The mixed workload at its full size (16,777,216 spheres), quantised on the GPU."""
    w = inputs.draw("mixed_16m", seed=5)
    wl = w["workload"]
    n = w["x"].shape[1]
    ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], w["dt"]))
    return w, ctx, mixed_state(w, ctx)


def test_collide_f32_full_size_sampled(full16):
    """One step at 16,777,216 spheres. For 8 random sub-cubes of half-side 0.06 the oracle
    runs the mixed-storage step (brute-force candidates) on the ~29,000 particles of the
    cube; every particle in the cube's core (half-side 0.03) must have the same partner
    and the same new cell, offsets and velocity. The 0.03 margin is ~7 collision reaches:
    a difference caused by the cube's boundary would need a chain of 7 blocking
    collisions to reach the core."""
    w, ctx, s32 = full16
    n, dt, nc = w["x"].shape[1], w["dt"], ctx.cells_per_side
    b = pc.StateF32.empty(n)
    ctx.collide_f32(s32, b, dt)
    ctx.sync()
    gids, _ = ctx.pairs()
    gpart = np.full(n, -1, np.int64)
    gpart[gids[:, 0]], gpart[gids[:, 1]] = gids[:, 1], gids[:, 0]
    a = s32.numpy()  # quantised in id order
    g = by_id(b.numpy())
    x = oracle.dequantize(a["cell"], a["o"], nc)
    rng = np.random.default_rng(3)
    compared = pairs = 0
    for _ in range(8):
        c = rng.random(3)
        d = np.abs((x - c[:, None] + 0.5) % 1.0 - 0.5)
        sub = np.nonzero((d <= 0.06).all(axis=0))[0]
        core = (d[:, sub] <= 0.03).all(axis=0)
        cell, o, v, partner, tc, k = oracle.collide_step_cellrel(a["cell"][sub], a["o"][:, sub], a["v"][:, sub],
                                                                 a["r"][sub], a["m"][sub], a["id"][sub], nc, w["e"], dt)
        opart = np.where(partner >= 0, sub[np.maximum(partner, 0)], -1)
        ids = sub[core]
        assert np.array_equal(gpart[ids], opart[core])
        assert np.array_equal(g["cell"][ids], cell[core])
        assert np.array_equal(g["o"][:, ids], o[:, core]) and np.array_equal(g["v"][:, ids], v[:, core])
        compared += len(ids)
        pairs += int((opart[core] >= 0).sum())
    print("full-size collide: %d core particles compared, %d of them in pairs" % (compared, pairs))
    assert pairs > 100


def test_project_f32_full_size_sampled(full16):
    """16,777,216 spheres on the 64^3 degree-7 mesh: conservation, and sampled elements
    against the oracle run on the particles that can reach them."""
    w, ctx, s32 = full16
    wl = w["workload"]
    n = w["x"].shape[1]
    f = ctx.new_field_f32()
    ctx.project_f32(s32, f, "f16")
    ctx.sync()
    nc = ctx.cells_per_side
    cell = s32.cell.cpu().numpy()
    o = s32.o.cpu().numpy()
    q = s32.q.cpu().numpy().astype(np.float64)
    x = oracle.dequantize(cell, o, nc)
    eta, om = np.polynomial.legendre.leggauss(wl.degree + 1)
    W = (np.einsum("k,j,i->kji", om, om, om) * (0.5 / wl.ne) ** 3).ravel()
    tot = (f.double().sum(dim=0) * torch.as_tensor(W, device="cuda")).sum(dim=1).cpu().numpy()
    assert np.all(np.abs(tot - q.sum(axis=1)) <= 1e-5 * np.abs(q).sum(axis=1))
    rng = np.random.default_rng(1)
    elems = rng.choice(wl.ne ** 3, 4, replace=False)
    e_of = np.minimum((x * wl.ne).astype(np.int64), wl.ne - 1)
    keep = np.zeros(n, bool)
    for el in elems:
        c = [el % wl.ne, (el // wl.ne) % wl.ne, el // wl.ne ** 2]
        near = np.ones(n, bool)
        for a in range(3):
            d = (e_of[a] - c[a] + wl.ne // 2) % wl.ne - wl.ne // 2
            near &= np.abs(d) <= 1
        keep |= near
    R, _ = oracle.project(x[:, keep], q[:, keep], wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
    F = f[torch.as_tensor(elems, device="cuda")].cpu().numpy().astype(np.float64)
    scale = f.abs().amax(dim=(0, 2)).cpu().numpy()
    err = np.abs(F - R[elems]).max(axis=(0, 2)) / scale
    print("sampled normwise error", err)
    assert np.all(err <= F16_TOL), err
