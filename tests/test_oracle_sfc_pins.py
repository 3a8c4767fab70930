"""Pins of the oracle's first-found pair selection (Sec. 4.3) against its defining
properties, checked with independent code (the Morton codes are recomputed here by
arithmetic, not bit loops): every committed pair is a candidate (a valid collision within
the step); the matching is maximal; and it is the first-found one: when a particle was
visited, every candidate ranked before its partner was already taken by a pair that began
earlier on the curve. Plus a hand-built chain where first-found and earliest-contact
differ."""
import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs


def _morton(c):
    """Interleave (cx, cy, cz) < 1024 into x bits 0, 3, 6, ..., y bits 1, 4, ..., z bits 2, 5, ..."""
    code = np.zeros(c.shape[1], dtype=np.int64)
    for b in range(10):
        for a in range(3):
            code += ((c[a] // 2 ** b) % 2).astype(np.int64) * 2 ** (3 * b + a)
    return code


def _ranks(x, ids, ncell):
    c = np.clip(np.floor(x * ncell).astype(np.int64), 0, ncell - 1)
    key = _morton(c) * 2 ** 32 + ids.astype(np.int64)
    order = np.argsort(key, kind="stable")
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    return rank


@pytest.mark.parametrize("seed,ncell,mult,shuffle", [(0, 12, 10, False), (1, 7, 20, False), (2, 20, 10, False),
                                                  (3, 7, 20, True)])
def test_first_found_characterisation(seed, ncell, mult, shuffle):
    """shuffle: ids are a random permutation of the indices, so that order by id and
    order by index differ inside a cell."""
    d = inputs.draw("small_8192", seed=seed, n=3000)
    dt = mult * d["dt"]
    x, v, r, m, ids = d["x"], d["v"], d["r"], d["m"], d["id"]
    if shuffle:
        ids = np.random.default_rng(seed).permutation(len(ids)).astype(np.int32)
    x1, v1, partner, tc, k = oracle.collide_step_sfc(x, v, r, m, ids, 0.9, dt, ncell)
    ci, cj, ct = oracle.candidates(x, v, r, dt)
    assert k > 30 and len(ci) > k
    cand = {}
    for a, b, t in zip(ci, cj, ct):
        cand.setdefault(a, {})[b] = t
        cand.setdefault(b, {})[a] = t
    rank = _ranks(x, ids, ncell)
    # committed pairs are candidates, with their contact time
    for i in np.nonzero(partner >= 0)[0]:
        j = partner[i]
        assert partner[j] == i and tc[i] == cand[i][j]
    # maximal: no candidate pair with both ends free
    for a, b in zip(ci, cj):
        assert partner[a] >= 0 or partner[b] >= 0
    # the pair of a matched particle begins at the smaller rank of its two ends
    start = np.full(len(partner), np.iinfo(np.int64).max)
    mt = partner >= 0
    start[mt] = np.minimum(rank[mt], rank[partner[mt]])
    for i in np.nonzero(mt)[0]:
        j = partner[i]
        if rank[i] > rank[j]:
            continue  # i is the later end; it was taken when j was visited
        for kk in cand[i]:
            if rank[kk] < rank[j]:
                # an earlier-ranked candidate must have been taken before i was visited
                assert start[kk] < rank[i], (i, j, kk)
    # momentum
    assert np.allclose((m * v1).sum(1), (m * v).sum(1), rtol=0, atol=1e-12)


def test_chain_first_found_differs_from_earliest_contact():
    """Three spheres on a line: B between A and C, B meets C first but A comes first on
    the curve. First-found pairs (A, B); earliest contact pairs (B, C)."""
    r = np.full(3, 0.01)
    m = np.ones(3)
    ids = np.arange(3, dtype=np.int32)
    # A in cell 0, B and C in cell 1 (ncell = 2 along x); B-C gap smaller than A-B gap
    x = np.array([[0.45, 0.52, 0.545], [0.25, 0.25, 0.25], [0.25, 0.25, 0.25]])
    v = np.array([[1.0, 0.0, -1.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    dt = 0.06
    _, _, p_sfc, _, k1 = oracle.collide_step_sfc(x, v, r, m, ids, 1.0, dt, 2)
    _, _, p_t, _, k2 = oracle.collide_step(x, v, r, m, ids, 1.0, dt)
    assert k1 == 1 and k2 == 1
    assert p_sfc[0] == 1 and p_sfc[1] == 0 and p_sfc[2] == -1
    assert p_t[1] == 2 and p_t[2] == 1 and p_t[0] == -1
