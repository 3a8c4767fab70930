"""Slab decomposition of the collision step (Sec. 4.1, 4.3: halo, one collision per
particle) on CPU ranks (gloo): ghost import within the reach, matching rounds with the
neighbour exchange of picks and matched flags and an "any left" allreduce, migration.
The local operations are the oracle's; after a few steps the positions, velocities and
each step's pair set equal the single-domain oracle's bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")

STEPS = 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _best_free(cand, free, ids):
    """Earliest free candidate partner of every local particle, ties to the smaller id."""
    ci, cj, ct = cand
    n = len(free)
    best = np.full(n, -1, np.int64)
    ok = free[ci] & free[cj]
    a = np.concatenate([ci[ok], cj[ok]])
    b = np.concatenate([cj[ok], ci[ok]])
    t = np.concatenate([ct[ok], ct[ok]])
    if len(a):
        order = np.lexsort((ids[b], t, a))  # by particle, then time, then partner id
        a, b = a[order], b[order]
        first = np.ones(len(a), bool)
        first[1:] = a[1:] != a[:-1]
        best[a[first]] = b[first]
    return best


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    from paper_2501_05340_gb300 import inputs, slabs

    dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=__import__("datetime").timedelta(seconds=120))
    try:
        w = inputs.draw("small_8192", seed=3)
        dt = 4 * w["dt"]
        mine = slabs.slab_of(w["x"][0], ws) == rank
        own = {k: np.ascontiguousarray(w[k][..., mine]) for k in slabs.FIELDS}
        ops = slabs.LocalOps(candidates=lambda x, v, r, dt_: oracle.candidates(x, v, r, dt_),
                             best_free=_best_free,
                             respond=lambda x, v, m, p, tc, e, dt_: oracle.respond_advance(x, v, m, p, tc, e, dt_))
        sl = slabs.Slabs(dist)
        all_pairs = []
        for _ in range(STEPS):
            own, pairs = sl.collide_step(own, w["e"], dt, ops)
            all_pairs.append(pairs)
        gathered = [None] * ws
        dist.all_gather_object(gathered, (own, all_pairs))
        if rank == 0:
            q.put(gathered)
        dist.barrier()
    except Exception as exc:  # report at once instead of leaving the parent waiting
        q.put("rank %d: %r" % (rank, exc))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_slab_rollout_equals_single_domain_oracle(ws):
    import oracle
    from paper_2501_05340_gb300 import inputs

    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
    assert not isinstance(gathered, str), gathered
    for p in procs:
        assert p.exitcode == 0
    # distributed result in id order
    x = np.concatenate([g[0]["x"] for g in gathered], axis=1)
    v = np.concatenate([g[0]["v"] for g in gathered], axis=1)
    ids = np.concatenate([g[0]["id"] for g in gathered])
    o = np.argsort(ids)
    assert np.array_equal(ids[o], np.arange(len(ids)))
    x, v = x[:, o], v[:, o]
    # single-domain oracle
    w = inputs.draw("small_8192", seed=3)
    dt = 4 * w["dt"]
    xs, vs = w["x"], w["v"]
    from paper_2501_05340_gb300 import slabs
    cross = total = 0
    for s in range(STEPS):
        sl0 = slabs.slab_of(xs[0], ws)
        xs, vs, partner, tc, k = oracle.collide_step(xs, vs, w["r"], w["m"], w["id"], w["e"], dt)
        ref = sorted((int(i), int(partner[i]), float(tc[i])) for i in range(len(partner))
                     if partner[i] >= 0 and i < partner[i])
        got = sorted(p for g in gathered for p in g[1][s])
        assert got == ref, "pairs of step %d" % s
        total += len(ref)
        cross += sum(1 for i, j, _ in ref if sl0[i] != sl0[j])
    assert np.array_equal(x, xs) and np.array_equal(v, vs)
    assert total > 40 and cross > 0, (total, cross)  # pairs across slab faces occurred
