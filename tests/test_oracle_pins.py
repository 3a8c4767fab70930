"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what it pins: closed forms, library routines for special cases,
invariants of the physics, brute force on tiny inputs, and an independent
(closest-approach) formulation of the collision predicate.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Gauss tables

@pytest.mark.parametrize("n1", [1, 2, 3, 4, 6, 8, 12])
def test_gauss_legendre_matches_numpy_and_is_exact(n1):
    """Sec. 3.1 Legendre-Gauss rule: numpy's leggauss, sum w = 2, exact to degree 2N+1."""
    eta, w = oracle.gauss_legendre(n1)
    ref_x, ref_w = np.polynomial.legendre.leggauss(n1)
    assert np.allclose(eta, ref_x, rtol=0, atol=1e-15)
    assert np.allclose(w, ref_w, rtol=1e-14, atol=0)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * n1):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs((w * eta ** k).sum() - exact) < 1e-14
    assert np.allclose(eta, -eta[::-1], atol=1e-16)
    assert np.all(np.diff(eta) > 0)


# ----------------------------------------------------------------- contact time

def test_contact_time_head_on_closed_form():
    """Head-on pair on a line: t = (separation - R) / closing speed, exact in binary."""
    t = oracle.contact_time([0.25, 0.5, 0.5], [0.375, 0.5, 0.5], [1, 0, 0], [-1, 0, 0], 0.03125, 0.03125, 1.0)
    assert t == 0.03125


def test_contact_time_inclusive_dt_and_rejections():
    xi, xj, vi, vj = [0.25, 0.5, 0.5], [0.375, 0.5, 0.5], [1, 0, 0], [-1, 0, 0]
    assert oracle.contact_time(xi, xj, vi, vj, 0.03125, 0.03125, 0.03125) == 0.03125  # t == dt counts
    assert math.isinf(oracle.contact_time(xi, xj, vi, vj, 0.03125, 0.03125, 0.03))    # t > dt
    assert math.isinf(oracle.contact_time(xi, xj, [-1, 0, 0], [1, 0, 0], 0.03125, 0.03125, 1.0))  # receding
    assert math.isinf(oracle.contact_time(xi, xj, vi, vj, 0.0625, 0.0625, 1.0))       # overlapping at t=0
    assert math.isinf(oracle.contact_time(xi, xj, [0, 1, 0], [0, 1, 0], 0.03125, 0.03125, 1.0))  # no relative motion
    # grazing: the closest approach is exactly R -> double root, no collision
    assert math.isinf(oracle.contact_time([0.5, 0.5, 0.5], [0.5, 0.75, 0.5], [0, 0, 0], [1, 0, 0], 0.125, 0.125, 10.0))
    # grazing while approaching (b < 0): offset exactly R across the line of motion, binary-exact
    # values, so b^2 - a c is exactly 0: a double root, no collision
    assert math.isinf(oracle.contact_time([0.375, 0.5625, 0.5], [0.5, 0.5, 0.5], [1, 0, 0], [0, 0, 0], 0.03125,
                                          0.03125, 1.0))


def test_contact_time_across_periodic_face():
    """Minimum image: a pair straddling x=0 approaches through the face."""
    t = oracle.contact_time([0.96875, 0.5, 0.5], [0.03125, 0.5, 0.5], [1, 0, 0], [-1, 0, 0], 0.0078125, 0.0078125, 1.0)
    assert t == (0.0625 - 0.015625) / 2.0


def test_contact_time_symmetric_bitwise():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        xi, xj = rng.random(3), rng.random(3)
        xj = xi + rng.normal(0, 0.02, 3)
        xj -= np.floor(xj)
        vi, vj = rng.normal(size=3), rng.normal(size=3)
        a = oracle.contact_time(xi, xj, vi, vj, 0.004, 0.005, 0.01)
        b = oracle.contact_time(xj, xi, vj, vi, 0.005, 0.004, 0.01)
        assert a == b or (math.isinf(a) and math.isinf(b))


def test_contact_time_against_high_precision_root():
    """The FP64 root agrees with a 50-digit root of the same quadratic (mpmath)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(2)
    checked = 0
    while checked < 300:
        xi = rng.random(3) * 0.5 + 0.25
        xj = xi + rng.normal(0, 0.01, 3)
        vi, vj = rng.normal(size=3), rng.normal(size=3)
        R = 0.006
        t = oracle.contact_time(xi, xj, vi, vj, R / 2, R / 2, 0.01)
        dx = [mpmath.mpf(float(a)) - mpmath.mpf(float(b)) for a, b in zip(xi, xj)]
        dv = [mpmath.mpf(float(a)) - mpmath.mpf(float(b)) for a, b in zip(vi, vj)]
        a = sum(u * u for u in dv)
        b = sum(u * w for u, w in zip(dx, dv))
        c = sum(u * u for u in dx) - mpmath.mpf(R) ** 2
        disc = b * b - a * c
        if math.isinf(t):
            if b < 0 and c > 0 and disc > 0:
                assert (-b - mpmath.sqrt(disc)) / a > mpmath.mpf("0.01") * (1 - mpmath.mpf("1e-12"))
            continue
        ref = (-b - mpmath.sqrt(disc)) / a
        # conditioning: relative error bound grows like |b| / sqrt(disc)
        cond = float(abs(b) / mpmath.sqrt(disc))
        assert abs(float(ref) - t) <= 1e-14 * max(1.0, cond) * abs(t) + 1e-18
        checked += 1


def _closest_approach_hits(dx, dv, R, dt):
    """Independent predicate: the distance along [0, dt] drops below R while approaching."""
    a = dv @ dv
    if a == 0:
        return False
    ts = min(max(-(dx @ dv) / a, 0.0), dt)
    dmin = np.linalg.norm(dx + ts * dv)
    return np.linalg.norm(dx) > R and (dx @ dv) < 0 and dmin < R


def test_candidate_predicate_matches_closest_approach():
    rng = np.random.default_rng(3)
    agree = 0
    for _ in range(20000):
        xi = rng.random(3) * 0.5 + 0.25
        xj = xi + rng.normal(0, 0.008, 3)
        vi, vj = rng.normal(size=3), rng.normal(size=3)
        R, dt = 0.007, 2e-3
        t = oracle.contact_time(xi, xj, vi, vj, R / 2, R / 2, dt)
        dx, dv = xi - xj, vi - vj
        hit = _closest_approach_hits(dx, dv, R, dt)
        if not math.isinf(t):
            assert hit or abs(np.linalg.norm(dx + dt * dv) - R) < 1e-12
            assert abs(np.linalg.norm(dx + t * dv) - R) < 1e-12
            agree += 1
        else:
            if hit:
                # only a root within rounding of dt or of a grazing touch may be missed
                ts = min(max(-(dx @ dv) / (dv @ dv), 0.0), dt)
                assert R - np.linalg.norm(dx + ts * dv) < 1e-12
    assert agree > 100


def test_two_particle_paper_geometry_ballistic():
    """Sec. 5.2 geometry in the unit cube (lengths / 2.2): the ballistic pair meets its
    periodic image at t = (1.2 - sqrt(0.04^2 - 0.037^2)) / 30. The paper's own value
    9.96237e-2 includes drag (parity unpinned)."""
    g = json.load(open(os.path.join(GOLDEN, "two_particle_sec5_2.json")))
    L = g["box"][1] - g["box"][0]
    x = np.array([[(a - g["box"][0]) / L for a in g["x1"]], [(a - g["box"][0]) / L for a in g["x2"]]]).T.copy()
    v = np.array([[a / L for a in g["v1"]], [a / L for a in g["v2"]]]).T.copy()
    r = np.full(2, g["diameter"] / 2 / L)
    m = np.ones(2)
    ids = np.arange(2, dtype=np.int32)
    dt = 1e-3
    t_hit = None
    for s in range(60):
        x, v, partner, tc, k = oracle.collide_step(x, v, r, m, ids, 1.0, dt, method="bruteforce")
        if k:
            t_hit = s * dt + tc[0]
            break
    exact = (1.2 - math.sqrt(0.04 ** 2 - 0.037 ** 2)) / 30.0
    assert t_hit is not None
    assert abs(t_hit - exact) <= 1e-13 * exact
    assert abs(exact - 0.0394934) < 1e-7


# ----------------------------------------------------------------- candidates

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cell_list_equals_bruteforce_random(seed):
    w = inputs.draw("dense_1m", seed=seed, n=1500)
    # a larger dt produces many candidates
    for dt in (w["dt"], 20 * w["dt"]):
        a = oracle.candidates(w["x"], w["v"], w["r"], dt, "cells")
        b = oracle.candidates(w["x"], w["v"], w["r"], dt, "bruteforce")
        for u, z in zip(a, b):
            assert np.array_equal(u, z)


def test_cell_list_equals_bruteforce_adversarial():
    """Pairs across the periodic faces, edges and the corner, and on cell boundaries."""
    rng = np.random.default_rng(7)
    pts = []
    for _ in range(400):
        base = rng.choice([0.0, 1.0 - 1e-12, 0.5, 1.0 / 3.0], size=3)
        pts.append(base + rng.normal(0, 0.004, 3))
    x = np.array(pts).T.copy()
    x -= np.floor(x)
    x[x >= 1.0] = 0.0
    n = x.shape[1]
    v = rng.normal(size=(3, n))
    r = np.full(n, 0.0015)
    for dt in (1e-3, 3e-3):
        a = oracle.candidates(x, v, r, dt, "cells")
        b = oracle.candidates(x, v, r, dt, "bruteforce")
        assert len(a[0]) > 10
        for u, z in zip(a, b):
            assert np.array_equal(u, z)


def test_cell_list_reaches_fast_head_on_pairs():
    """Sec. 4.3 reach: two spheres can meet within dt from up to 2 r_max + 2 v_max dt apart.
    Small spheres (the velocity term dominates the reach) in head-on pairs at the
    fastest speed, their centres 0.17-0.19 apart along x, y, z and diagonals, with dt = 0.1
    (reach 0.202), among slow background spheres: the cell list finds what brute force
    finds, every fast pair included. Cells sized with half the velocity term miss pairs."""
    rng = np.random.default_rng(11)
    r0, vmax, dt = 1e-3, 1.0, 0.1
    nb = 300
    xs, vs, fast = [rng.random((3, nb))], [rng.normal(0, 0.01, (3, nb))], []
    dirs = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 1), (0, 1, -1)]
    for k in range(24):
        u = np.array(dirs[k % len(dirs)], float)
        u /= np.linalg.norm(u)
        d = rng.uniform(0.17, 0.19)
        c = rng.random(3)
        a, b = c - 0.5 * d * u, c + 0.5 * d * u
        xs.append(np.stack([a, b], 1))
        vs.append(np.stack([vmax * u, -vmax * u], 1))
        fast.append((nb + 2 * k, nb + 2 * k + 1))
    x = np.concatenate(xs, 1)
    x -= np.floor(x)
    x[x >= 1.0] = 0.0
    v = np.concatenate(vs, 1)
    n = x.shape[1]
    r = np.full(n, r0)
    a = oracle.candidates(x, v, r, dt, "cells")
    b = oracle.candidates(x, v, r, dt, "bruteforce")
    for u_, z in zip(a, b):
        assert np.array_equal(u_, z)
    found = set(zip(a[0].tolist(), a[1].tolist()))
    assert all(p in found for p in fast), [p for p in fast if p not in found]


def test_cell_list_at_the_reach_limit():
    """A head-on pair 0.20005 apart with reach 2 r + 2 v dt = 0.20008 (dt = 0.09904): the
    grid has 4 cells per side (1 / reach = 4.998); the pair meets within the step and the
    cell list finds it, as brute force does. A grid sized from a reach only 0.1 % smaller
    has 5 cells per side and puts the two spheres 2 cells apart."""
    x = np.array([[0.19995, 0.40], [0.5, 0.5], [0.5, 0.5]])
    v = np.array([[1.0, -1.0], [0.0, 0.0], [0.0, 0.0]])
    r, dt = np.full(2, 1e-3), 0.09904
    reach = 2 * 1e-3 + 2 * 1.0 * dt
    assert int(1.0 / reach) == 4 and int(1.0 / (0.999 * reach)) == 5
    a = oracle.candidates(x, v, r, dt, "cells")
    b = oracle.candidates(x, v, r, dt, "bruteforce")
    assert len(a[0]) == 1 and (a[0][0], a[1][0]) == (0, 1)
    for u, z in zip(a, b):
        assert np.array_equal(u, z)


@pytest.mark.parametrize("target_reach", [0.45, 0.8])
def test_cell_list_with_fewer_than_three_cells(target_reach):
    """A reach above 1/3 leaves fewer than 3 cells per side, where the 27-cell stencil
    would visit a cell more than once: the candidates still equal brute force, each pair
    once."""
    rng = np.random.default_rng(int(target_reach * 100))
    n = 500
    x = rng.random((3, n))
    v = rng.normal(size=(3, n))
    r = np.full(n, 0.015)
    vmax = float(np.sqrt((v * v).sum(0)).max())
    dt = (target_reach - 0.03) / (2 * vmax)
    a = oracle.candidates(x, v, r, dt, "cells")
    b = oracle.candidates(x, v, r, dt, "bruteforce")
    assert len(a[0]) > 5
    for u, z in zip(a, b):
        assert np.array_equal(u, z)


# ----------------------------------------------------------------- matching

def _is_greedy(n, ids, ci, cj, ct, partner):
    """Characterisation of the greedy matching under the strict order (t, lo id, hi id):
    it is a matching, and every unmatched edge has an endpoint matched by a smaller edge."""
    key = {}
    for a, b, t in zip(ci, cj, ct):
        key[(a, b)] = key[(b, a)] = (t, min(ids[a], ids[b]), max(ids[a], ids[b]))
    for i in range(n):
        j = partner[i]
        if j >= 0:
            assert partner[j] == i and (i, j) in key
    for a, b, t in zip(ci, cj, ct):
        if partner[a] == b:
            continue
        k = key[(a, b)]
        blocked = (partner[a] >= 0 and key[(a, partner[a])] < k) or (partner[b] >= 0 and key[(b, partner[b])] < k)
        assert blocked
    return True


@pytest.mark.parametrize("seed", range(6))
def test_matching_greedy_equals_rounds_random_graphs(seed):
    rng = np.random.default_rng(seed)
    n = 300
    m = 600
    ci = rng.integers(0, n, m)
    cj = rng.integers(0, n, m)
    keep = ci != cj
    ci, cj = np.minimum(ci, cj)[keep], np.maximum(ci, cj)[keep]
    pairs = sorted(set(zip(ci.tolist(), cj.tolist())))
    ci = np.array([p[0] for p in pairs])
    cj = np.array([p[1] for p in pairs])
    ct = rng.integers(0, 20, len(ci)).astype(float) * 1e-4  # many ties in t
    ids = rng.permutation(n).astype(np.int32)
    pg, tg, kg = oracle.match(ids, ci, cj, ct, n, "greedy")
    pr, tr, kr, rounds = oracle.match(ids, ci, cj, ct, n, "rounds")
    assert np.array_equal(pg, pr) and kg == kr
    assert _is_greedy(n, ids, ci, cj, ct, pg)


def test_matching_chains():
    ids = np.arange(4, dtype=np.int32)
    # A-B-C with t_AB < t_BC: AB collide, C stays free
    p, t, k = oracle.match(ids[:3], [0, 1], [1, 2], [1e-3, 2e-3], 3)
    assert list(p) == [1, 0, -1] and k == 1
    # A-B-C-D with t_BC smallest: BC collide, A and D stay free
    p, t, k = oracle.match(ids, [0, 1, 2], [1, 2, 3], [2e-3, 1e-3, 2e-3], 4)
    assert list(p) == [-1, 2, 1, -1]
    # A-B-C-D with t_AB = t_CD < t_BC: both outer pairs
    p, t, k = oracle.match(ids, [0, 1, 2], [1, 2, 3], [1e-3, 2e-3, 1e-3], 4)
    assert list(p) == [1, 0, 3, 2]
    # tie between B's partners at equal t: the smaller id wins
    p, t, k = oracle.match(ids[:3], [0, 1], [1, 2], [1e-3, 1e-3], 3)
    assert list(p) == [1, 0, -1]
    p, t, k = oracle.match(np.array([5, 1, 0], np.int32), [0, 1], [1, 2], [1e-3, 1e-3], 3)
    assert list(p) == [-1, 2, 1]


def test_matching_rounds_one_pair_per_round():
    """A path 0-1-2-3-4-5 whose contact times grow along it: each round of mutual earliest
    picks commits exactly one pair ((0,1), then (2,3), then (4,5)), and the rounds must go
    on until no free particle has a free candidate; the result equals the greedy matching."""
    ids = np.arange(6, dtype=np.int32)
    ci, cj, ct = [0, 1, 2, 3, 4], [1, 2, 3, 4, 5], [1e-3, 2e-3, 3e-3, 4e-3, 5e-3]
    pg, tg, kg = oracle.match(ids, ci, cj, ct, 6)
    pr, tr, kr, rounds = oracle.match(ids, ci, cj, ct, 6, method="rounds")
    assert list(pg) == [1, 0, 3, 2, 5, 4] and kg == 3
    assert np.array_equal(pr, pg) and np.array_equal(tr, tg) and kr == 3 and rounds == 3


@pytest.mark.parametrize("method", ["cells", "bruteforce"])
def test_step_with_more_candidates_than_the_first_buffer(method):
    """40 spheres contracting towards one point: all 780 pairs are candidates, more than the
    4 n entries the step first allocates, so it must grow its candidate buffers and use every
    candidate: its pairs are the greedy matching of the full brute-force candidate list, and
    the first-found step's pairs form a maximal matching of the same list."""
    rng = np.random.default_rng(23)
    n = 40
    c = np.array([0.5, 0.5, 0.5])
    x = c[:, None] + rng.uniform(-0.05, 0.05, (3, n))
    v = -(x - c[:, None]) / 0.1
    r, m, ids, dt = np.full(n, 0.002), rng.uniform(0.5, 2.0, n), np.arange(n, dtype=np.int32), 0.1
    ci, cj, ct = oracle.candidates(x, v, r, dt, "bruteforce")
    assert len(ci) > 4 * n
    pg, tg, kg = oracle.match(ids, ci, cj, ct, n)
    _, _, p, t, k = oracle.collide_step(x, v, r, m, ids, 0.9, dt, method)
    assert k == kg == n // 2 and np.array_equal(p, pg) and np.array_equal(t, tg)
    _, _, ps, ts, ks = oracle.collide_step_sfc(x, v, r, m, ids, 0.9, dt, 4)
    assert ks == n // 2 and all(ps[ps[i]] == i for i in range(n))
    for a, b in zip(ci, cj):
        assert ps[a] >= 0 or ps[b] >= 0


# ----------------------------------------------------------------- response

def _pair_state(rng, e_same_mass=True):
    x = np.array([[0.5, 0.5 + 0.004], [0.5, 0.501], [0.5, 0.4995]])
    v = np.array([[1.0, -1.0], [0.3, -0.2], [0.1, 0.05]])
    m = np.array([1.0, 1.0]) if e_same_mass else np.array([1.0, 2.5])
    r = np.array([0.002, 0.002])
    return x, v, m, r


@pytest.mark.parametrize("e", [1.0, 0.9, 0.5, 0.0])
@pytest.mark.parametrize("same", [True, False])
def test_response_laws(e, same):
    """Sec. 2.4: momentum conserved, (v1'-v2').n = -e (v1-v2).n, tangential parts kept,
    KE loss = 1/2 m_r (1-e^2) (v_r.n)^2; the pair touches at the contact time."""
    x, v, m, r = _pair_state(None, same)
    ids = np.arange(2, dtype=np.int32)
    dt = 5e-3
    ci, cj, ct = oracle.candidates(x, v, r, dt, "bruteforce")
    assert len(ci) == 1
    t = ct[0]
    x1, v1, partner, tc, k = oracle.collide_step(x, v, r, m, ids, e, dt, "bruteforce")
    assert k == 1 and tc[0] == t
    xc = x + t * v
    nvec = (xc[:, 1] - xc[:, 0])
    assert abs(np.linalg.norm(nvec) - 0.004) < 1e-13
    nvec /= np.linalg.norm(nvec)
    p0, p1 = (m * v).sum(axis=1), (m * v1).sum(axis=1)
    assert np.allclose(p0, p1, rtol=0, atol=1e-15)
    vr0, vr1 = v[:, 0] - v[:, 1], v1[:, 0] - v1[:, 1]
    assert abs(vr1 @ nvec + e * (vr0 @ nvec)) < 1e-14
    assert np.allclose(vr1 - (vr1 @ nvec) * nvec, vr0 - (vr0 @ nvec) * nvec, atol=1e-14)
    mr = m[0] * m[1] / (m[0] + m[1])
    ke0, ke1 = 0.5 * (m * (v * v).sum(axis=0)).sum(), 0.5 * (m * (v1 * v1).sum(axis=0)).sum()
    assert abs((ke0 - ke1) - 0.5 * mr * (1 - e * e) * (vr0 @ nvec) ** 2) < 1e-14
    if same and e == 1.0:
        # equal masses, elastic: normal components exchanged
        assert np.allclose(v1[:, 0] @ nvec, v[:, 1] @ nvec, atol=1e-15)
        assert np.allclose(v1[:, 1] @ nvec, v[:, 0] @ nvec, atol=1e-15)
    # position: contact point with old velocity, then new velocity for dt - t
    assert np.allclose(x1, (xc + (dt - t) * v1) % 1.0, atol=1e-15)


def test_free_flight_and_wrap():
    x = np.array([[0.999], [1e-17], [0.5]])
    v = np.array([[1.0], [-1.0], [0.0]])
    x1, v1 = oracle.respond_advance(x, v, np.ones(1), np.array([-1]), np.array([np.inf]), 0.9, 0.01)
    assert np.array_equal(v1, v)
    assert abs(x1[0, 0] - 0.009) < 1e-15 and abs(x1[1, 0] - 0.99) < 1e-15 and x1[2, 0] == 0.5
    x = np.array([[-1e-20 + 0.0], [0.2], [0.3]])
    x1, _ = oracle.respond_advance(np.array([[0.0], [0.2], [0.3]]), np.array([[-1e-20], [0.0], [0.0]]),
                                   np.ones(1), np.array([-1]), np.array([np.inf]), 0.9, 1.0)
    assert 0.0 <= x1[0, 0] < 1.0


def test_step_conserves_momentum_dense():
    w = inputs.draw("dense_1m", n=20000, seed=4)
    x1, v1, partner, tc, k = oracle.collide_step(w["x"], w["v"], w["r"], w["m"], w["id"], w["e"], 20 * w["dt"])
    assert k > 100
    p0 = (w["m"] * w["v"]).sum(axis=1)
    p1 = (w["m"] * v1).sum(axis=1)
    scale = (w["m"] * np.abs(w["v"])).sum(axis=1)
    assert np.all(np.abs(p1 - p0) <= 1e-14 * scale)
    assert np.all((x1 >= 0) & (x1 < 1))


@pytest.mark.slow
def test_kinetic_gas_energy_and_maxwell():
    """Sec. 5.3 analogue: e = 1, frictionless, periodic box. Total KE is preserved to
    rounding and the speed distribution relaxes to Maxwell-Boltzmann (KS test)."""
    scipy_stats = pytest.importorskip("scipy.stats")
    g = inputs.gas(5000, 0.01, 0.5, seed=11)
    x, v, r, m, ids = g["x"], g["v"], g["r"], g["m"], g["id"]
    s0 = np.sqrt((v * v).sum(axis=0))
    a0 = math.sqrt((s0 ** 2).mean() / 3)
    assert scipy_stats.kstest(s0, scipy_stats.maxwell(scale=a0).cdf).pvalue < 1e-6
    ke0 = 0.5 * (m * (v * v).sum(axis=0)).sum()
    total = 0
    for step in range(600):
        x, v, partner, tc, k = oracle.collide_step(x, v, r, m, ids, 1.0, 0.02)
        total += k
    ke1 = 0.5 * (m * (v * v).sum(axis=0)).sum()
    assert abs(ke1 - ke0) <= 1e-13 * ke0
    s = np.sqrt((v * v).sum(axis=0))
    a = math.sqrt((s ** 2).mean() / 3)
    assert total > 20000
    assert scipy_stats.kstest(s, scipy_stats.maxwell(scale=a).cdf).pvalue > 1e-3


# ----------------------------------------------------------------- projection

def _nodes_1d(ne, n1):
    eta, _ = np.polynomial.legendre.leggauss(n1)
    h = 1.0 / ne
    return ((np.arange(ne)[:, None] + 0.5 * (eta[None, :] + 1.0)) * h).ravel()


def _separable_reference(xp, qp, ne, degree, sigma, cs):
    """Independent restatement for one particle with the box cutoff: the kernel is a
    product of 1-D Gaussians and Z a product of three 1-D quadrature sums."""
    n1 = degree + 1
    eta, om = np.polynomial.legendre.leggauss(n1)
    h = 1.0 / ne
    X = _nodes_1d(ne, n1)
    W1 = np.tile(om, ne) * h / 2
    fac = []
    for ax in range(3):
        d = X - xp[ax]
        d = d - np.round(d)
        k = np.where(np.abs(d) <= cs * sigma, np.exp(-d * d / (2 * sigma * sigma)), 0.0)
        fac.append((k, (W1 * k).sum()))
    Z = fac[0][1] * fac[1][1] * fac[2][1]
    kx, ky, kz = fac[0][0], fac[1][0], fac[2][0]
    F = np.zeros((ne ** 3, 4, n1 ** 3))
    full = np.einsum("c,k,j,i->ckji", qp, kz, ky, kx) / Z  # [4][z][y][x] global nodes
    full = full.reshape(4, ne, n1, ne, n1, ne, n1)  # c, ez, k, ey, j, ex, i
    F = full.transpose(1, 3, 5, 0, 2, 4, 6).reshape(ne ** 3, 4, n1 ** 3)
    return F, Z


@pytest.mark.parametrize("pos", [(0.5, 0.5, 0.5), (0.01, 0.99, 0.3), (0.126, 0.874, 0.0)])
def test_projection_single_particle_separable(pos):
    xp = np.array(pos)
    q = np.array([1.5, -0.5, 2.0, 0.25])
    F, Z = oracle.project(xp.reshape(3, 1), q.reshape(4, 1), 8, 3, 0.02)
    Fr, Zr = _separable_reference(xp, q, 8, 3, 0.02, 3.0)
    assert abs(Z[0] - Zr) <= 1e-14 * Zr
    assert np.max(np.abs(F - Fr)) <= 1e-13 * np.max(np.abs(Fr))


def test_projection_conservation_many():
    w = inputs.draw("small_8192", n=3000, seed=5)
    F, Z = oracle.project(w["x"], w["q"], 8, 3, 0.02)
    eta, om = np.polynomial.legendre.leggauss(4)
    h = 1 / 8
    Wg = (np.einsum("k,j,i->kji", om, om, om) * (h / 2) ** 3).ravel()
    tot = np.einsum("ecg,g->c", F, Wg)
    ref = w["q"].sum(axis=1)
    assert np.all(np.abs(tot - ref) <= 1e-13 * np.abs(w["q"]).sum(axis=1))


def test_normalisation_converges_to_gaussian_integral():
    """With a wide cutoff Z is a Gauss quadrature of the Gaussian: (sigma sqrt(2 pi))^3."""
    sigma = 0.03
    F, Z = oracle.project(np.array([[0.4], [0.55], [0.61]]), np.ones((4, 1)), 16, 7, sigma, cutoff_sigmas=12.0)
    ref = (sigma * math.sqrt(2 * math.pi)) ** 3
    assert abs(Z[0] - ref) <= 1e-9 * ref


def test_projection_dirac_limit():
    """sigma -> 0 with the particle on a node: the whole source sits on that node, F = q / W."""
    ne, n1 = 4, 3
    eta, om = np.polynomial.legendre.leggauss(n1)
    h = 1 / ne
    ex, ey, ez, i, j, k = 1, 2, 3, 0, 2, 1
    xp = np.array([(ex + 0.5 * (eta[i] + 1)) * h, (ey + 0.5 * (eta[j] + 1)) * h, (ez + 0.5 * (eta[k] + 1)) * h])
    q = np.array([1.0, 2.0, -3.0, 4.0])
    F, Z = oracle.project(xp.reshape(3, 1), q.reshape(4, 1), ne, n1 - 1, 1e-4)
    W = om[i] * om[j] * om[k] * (h / 2) ** 3
    e = (ez * ne + ey) * ne + ex
    g = (k * n1 + j) * n1 + i
    assert np.allclose(F[e, :, g], q / W, rtol=1e-12)
    F[e, :, g] = 0
    assert np.max(np.abs(F)) < 1e-100


def test_projection_translation_by_one_element():
    w = inputs.draw("small_8192", n=400, seed=9)
    F0, _ = oracle.project(w["x"], w["q"], 8, 3, 0.02)
    xs = w["x"].copy()
    xs[0] = (xs[0] + 0.125) % 1.0
    F1, _ = oracle.project(xs, w["q"], 8, 3, 0.02)
    F0r = F0.reshape(8, 8, 8, 4, 64)
    F1r = F1.reshape(8, 8, 8, 4, 64)
    assert np.max(np.abs(np.roll(F0r, 1, axis=2) - F1r)) <= 1e-12 * np.max(np.abs(F0))


def test_curved_map_jacobian_and_volume():
    """det of the analytic Jacobian vs central differences; the map preserves the
    cube's volume, so sum_g W_g over all nodes is 1."""
    rng = np.random.default_rng(12)
    amp = 0.02
    for _ in range(20):
        xi = rng.random(3)
        X, dj = oracle.mesh_map(xi, amp)
        Jfd = np.zeros((3, 3))
        hh = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = hh
            Jfd[:, a] = (oracle.mesh_map(xi + e, amp)[0] - oracle.mesh_map(xi - e, amp)[0]) / (2 * hh)
        assert abs(np.linalg.det(Jfd) - dj) < 1e-8
    ne, n1 = 6, 4
    eta, om = np.polynomial.legendre.leggauss(n1)
    tot = 0.0
    X1 = _nodes_1d(ne, n1)
    W1 = np.tile(om, ne) / ne / 2
    for a in range(ne * n1):
        for b in range(ne * n1):
            for c in range(ne * n1):
                tot += W1[a] * W1[b] * W1[c] * oracle.mesh_map(np.array([X1[a], X1[b], X1[c]]), amp)[1]
    assert abs(tot - 1.0) < 1e-13


def test_curved_projection_affine_limit_and_conservation():
    w = inputs.draw("small_8192", n=300, seed=13)
    Fa, Za = oracle.project(w["x"], w["q"], 8, 3, 0.02, cutoff="sphere", amp=0.0)
    # the sphere cutoff removes box corners: it differs from the box result
    Fb, Zb = oracle.project(w["x"], w["q"], 8, 3, 0.02, cutoff="box")
    assert np.max(np.abs(Fa - Fb)) > 1e-6
    Fc, Zc = oracle.project(w["x"], w["q"], 8, 3, 0.02, cutoff="sphere", amp=0.02)
    eta, om = np.polynomial.legendre.leggauss(4)
    h = 1 / 8
    # weights with the Jacobian at every node
    X1 = _nodes_1d(8, 4)
    W1 = np.tile(om, 8) * h / 2
    Wg = np.zeros((512, 64))
    for ez in range(8):
        for ey in range(8):
            for ex in range(8):
                e = (ez * 8 + ey) * 8 + ex
                for k in range(4):
                    for j in range(4):
                        for i in range(4):
                            xi = np.array([X1[ex * 4 + i], X1[ey * 4 + j], X1[ez * 4 + k]])
                            Wg[e, (k * 4 + j) * 4 + i] = W1[ex * 4 + i] * W1[ey * 4 + j] * W1[ez * 4 + k] * \
                                oracle.mesh_map(xi, 0.02)[1]
    tot = np.einsum("ecg,eg->c", Fc, Wg)
    assert np.all(np.abs(tot - w["q"].sum(axis=1)) <= 1e-12 * np.abs(w["q"]).sum(axis=1))


@pytest.mark.parametrize("cutoff", ["box", "sphere"])
def test_cutoff_is_inclusive_at_exactly_rc(cutoff):
    """Reading: the cutoff is inclusive (<= 3 sigma, box or sphere). A particle on the x
    line of a Gauss node with x - X exactly -r_c in FP64 (and equal y, z): that node takes
    the weight exp(-r_c^2 / (2 sigma^2)) / Z in the forward projection, and in the adjoint a
    unit dL/dfield at that node gives dL/dq_0 = K / Z."""
    ne, degree, sigma, cs = 4, 3, 0.02, 3.0
    n1 = degree + 1
    rc = cs * sigma
    eta, _ = oracle.gauss_legendre(n1)
    h = 1.0 / ne
    i, j, k = 1, 2, 1
    X = [(1 + 0.5 * (eta[a] + 1.0)) * h for a in (i, j, k)]  # node (i, j, k) of element (1, 1, 1)
    xp0 = X[0] - rc
    for step in range(64):
        if X[0] - xp0 == rc:
            break
        xp0 = np.nextafter(xp0, -np.inf if X[0] - xp0 < rc else np.inf)
    assert X[0] - xp0 == rc
    x = np.array([[xp0], [X[1]], [X[2]]])
    q = np.array([[1.0], [2.0], [3.0], [4.0]])
    F, Z = oracle.project(x, q, ne, degree, sigma, cs, cutoff=cutoff)
    e, g = (1 * ne + 1) * ne + 1, (k * n1 + j) * n1 + i
    K = math.exp(-(rc * rc) * (1.0 / (2.0 * sigma * sigma)))
    assert K > 0 and Z[0] > 0
    assert np.allclose(F[e, :, g], q[:, 0] * K / Z[0], rtol=1e-13, atol=0)
    G = np.zeros_like(F)
    G[e, 0, g] = 1.0
    gq, _ = oracle.project_adjoint(x, q, G, ne, degree, sigma, cs, cutoff=cutoff)
    assert gq[0, 0] == pytest.approx(K / Z[0], rel=1e-13)


def test_curved_projection_equals_an_all_node_brute_force():
    """Curved mesh (amp = 0.02, sphere cutoff): the projection equals a brute force over
    every node of the mesh (physical node positions from the mapping, weights with det J,
    Z summed over all nodes), so no node whose physical distance is within r_c is missed
    by the logical-coordinate scan."""
    ne, degree, sigma, cs, amp = 6, 2, 0.02, 3.0, 0.02
    n1 = degree + 1
    rng = np.random.default_rng(17)
    n = 40
    x, q = rng.random((3, n)), rng.normal(size=(4, n))
    F, _ = oracle.project(x, q, ne, degree, sigma, cs, cutoff="sphere", amp=amp)
    eta, om = np.polynomial.legendre.leggauss(n1)
    h = 1.0 / ne
    Xg = np.zeros((ne ** 3, n1 ** 3, 3))
    Wg = np.zeros((ne ** 3, n1 ** 3))
    for ez in range(ne):
        for ey in range(ne):
            for ex in range(ne):
                e = (ez * ne + ey) * ne + ex
                for kk in range(n1):
                    for jj in range(n1):
                        for ii in range(n1):
                            xi = np.array([(ex + 0.5 * (eta[ii] + 1)) * h, (ey + 0.5 * (eta[jj] + 1)) * h,
                                           (ez + 0.5 * (eta[kk] + 1)) * h])
                            Xp, dj = oracle.mesh_map(xi, amp)
                            g = (kk * n1 + jj) * n1 + ii
                            Xg[e, g] = Xp
                            Wg[e, g] = om[ii] * om[jj] * om[kk] * (h / 2) ** 3 * dj
    R = np.zeros_like(F)
    rc = cs * sigma
    for p in range(n):
        d = Xg - x[:, p]
        d -= np.round(d)
        d2 = (d * d).sum(-1)
        K = np.where(d2 <= rc * rc, np.exp(-d2 / (2 * sigma * sigma)), 0.0)
        Zp = (Wg * K).sum()
        if Zp > 0:
            R += q[:, p][None, :, None] * (K / Zp)[:, None, :]
    err = np.abs(F - R).max(axis=(0, 2)) / np.abs(R).max(axis=(0, 2))
    assert np.all(err <= 1e-12), err


def test_curved_map_special_points():
    """x = xi + a (sin 2pi xi_y sin 2pi xi_z, cyclic): at xi = (0, 1/4, 1/4) only the
    first component moves, by a; on the planes xi_k = 0 the map is the identity."""
    X, dj = oracle.mesh_map(np.array([0.0, 0.25, 0.25]), 0.02)
    assert np.allclose(X, [0.02, 0.25, 0.25], atol=1e-17)
    X, dj = oracle.mesh_map(np.array([0.25, 0.0, 0.25]), 0.02)
    assert np.allclose(X, [0.25, 0.02, 0.25], atol=1e-17)
    X, dj = oracle.mesh_map(np.array([0.25, 0.25, 0.0]), 0.02)
    assert np.allclose(X, [0.25, 0.25, 0.02], atol=1e-17)
    X, dj = oracle.mesh_map(np.array([0.3, 0.0, 0.0]), 0.02)
    assert np.allclose(X, [0.3, 0.0, 0.0], atol=1e-17)


# ----------------------------------------------------------------- mixed storage

def test_quantize_carries_an_offset_that_rounds_to_one():
    """Quantisation rule of the FP32 cell-relative storage: an offset s - floor(s) that
    rounds to 1.0 in FP32 is stored as offset 0 in the next cell, wrapping from n_c - 1 to
    0 (on a power-of-two grid s = x n_c is exact, so the offset 1 - 2^-40 reaches the
    cast); dequantising gives a position in [0, 1) within FP32 rounding of one cell of x
    (modulo the periodic wrap)."""
    nc = 8
    x = np.array([[(3 + 1 - 2.0 ** -40) / nc, (nc - 2.0 ** -40) / nc, 0.5625], [0.5] * 3, [0.5] * 3])
    assert list(np.floor(x[0] * nc)) == [3.0, 7.0, 4.0]
    cell, o = oracle.quantize(x, nc)
    assert list(cell % nc) == [4, 0, 4] and list(o[0]) == [0.0, 0.0, 0.5]
    assert np.all((o >= 0.0) & (o < 1.0))
    xd = oracle.dequantize(cell, o, nc)
    assert np.all((xd >= 0.0) & (xd < 1.0))  # in the box itself, not only modulo 1
    d = xd - x
    d -= np.round(d)
    assert np.abs(d).max() * nc <= 2.0 ** -24


def test_cellrel_step_matches_fp64_on_dequantized_state():
    """The cell-relative step equals the FP64 step on the dequantized state up to the
    storage rounding: same pairs, positions within 1e-7 cells, velocities within FP32 rounding."""
    w = inputs.draw("dense_1m", n=3000, seed=21)
    nc = 25
    cell, o = oracle.quantize(w["x"], nc)
    vf, rf, mf = w["v"].astype(np.float32), w["r"].astype(np.float32), w["m"].astype(np.float32)
    dt = 40 * w["dt"]
    c1, o1, v1, p1, tc1, k1 = oracle.collide_step_cellrel(cell, o, vf, rf, mf, w["id"], nc, 0.9, dt)
    xd = oracle.dequantize(cell, o, nc)
    x2, v2, p2, tc2, k2 = oracle.collide_step(xd, vf.astype(np.float64), rf.astype(np.float64),
                                              mf.astype(np.float64), w["id"], 0.9, dt)
    assert k1 == k2 > 5 and np.array_equal(p1, p2)
    assert np.allclose(tc1, tc2, rtol=1e-12, atol=0)
    d = oracle.dequantize(c1, o1, nc) - x2
    d -= np.round(d)
    assert np.max(np.abs(d)) * nc < 1e-6
    assert np.allclose(v1, v2, rtol=1e-6, atol=1e-6)


def test_cellrel_free_flight_carry():
    """Free flight across the upper and lower cell faces and the periodic boundary."""
    nc = 10
    cell = np.array([9, 0 + 10 * 5, 5 + 10 * 3], np.int32)  # x-cells 9, 0, 5 (different y-cells)
    o = np.zeros((3, 3), np.float32)
    o[0] = [0.99, 0.01, 0.5]
    o[1] = 0.5
    o[2] = 0.5
    v = np.zeros((3, 3), np.float32)
    v[0] = [1.0, -1.0, 0.0]
    r = np.full(3, 1e-4, np.float32)
    m = np.ones(3, np.float32)
    c1, o1, v1, p, tc, k = oracle.collide_step_cellrel(cell, o, v, r, m, np.arange(3, dtype=np.int32), nc, 1.0, 0.002)
    assert k == 0
    assert c1[0] % 10 == 0 and abs(o1[0, 0] - np.float32(np.float32(0.99) + np.float32(0.02) - 1)) < 1e-7
    assert c1[1] == 9 + 10 * 5 and abs(o1[0, 1] - (np.float32(0.01) - np.float32(0.02) + 1)) < 1e-6
    assert c1[2] == cell[2] and np.array_equal(o1[:, 2], o[:, 2])


def test_cellrel_tiny_negative_offset_stays_in_the_cell():
    """Free flight to an offset of -2^-30 cells: adding one cell rounds to exactly 1.0 in
    FP32, so the offset is set to 0 in the same cell (an offset of 1.0 would leave [0, 1));
    the stored position is within FP32 rounding of the exact one."""
    nc = 10
    cell = np.array([3 + 10 * (4 + 10 * 5)], np.int32)
    o = np.full((3, 1), 0.5, np.float32)
    o[0, 0] = 2.0 ** -30
    v = np.zeros((3, 1), np.float32)
    v[0, 0] = -(2.0 ** -29)
    c1, o1, v1, p, tc, k = oracle.collide_step_cellrel(cell, o, v, np.full(1, 1e-3, np.float32),
                                                       np.ones(1, np.float32), np.zeros(1, np.int32), nc, 1.0, 0.1)
    assert k == 0 and c1[0] == cell[0] and o1[0, 0] == 0.0
    assert np.all((o1 >= 0.0) & (o1 < 1.0))


def test_cellrel_collision_across_the_lower_face():
    """A pair that collides near x = 0: after the exchange (e = 1, equal masses) the
    struck sphere leaves through the lower face and wraps to cell nc - 1 of the
    periodic box; equal to the FP64 step on the dequantized state."""
    nc = 10
    x = np.array([[0.03, 0.045], [0.5, 0.5], [0.5, 0.5]])
    cell, o = oracle.quantize(x, nc)
    v = np.array([[0.0, -2.0], [0.0, 0.0], [0.0, 0.0]], np.float32)
    r, m, ids, dt = np.full(2, 0.002, np.float32), np.ones(2, np.float32), np.arange(2, dtype=np.int32), 0.03
    c1, o1, v1, p1, tc1, k1 = oracle.collide_step_cellrel(cell, o, v, r, m, ids, nc, 1.0, dt)
    x2, v2, p2, tc2, k2 = oracle.collide_step(oracle.dequantize(cell, o, nc), v.astype(np.float64),
                                              r.astype(np.float64), m.astype(np.float64), ids, 1.0, dt)
    assert k1 == k2 == 1 and np.array_equal(p1, p2)
    assert c1[0] % nc == nc - 1 and abs(x2[0, 0] - 0.981) < 1e-6
    d = oracle.dequantize(c1, o1, nc) - x2
    d -= np.round(d)
    assert np.max(np.abs(d)) * nc < 1e-6


def test_cellrel_collided_offset_that_rounds_to_one_is_carried():
    """A head-on pair (e = 1, equal masses) with dt chosen so that the struck sphere ends
    1e-9 cells below the face x = 4 cells: its offset rounds to 1.0 in FP32 and must be
    stored as offset 0 of cell 4 (every offset stays in [0, 1)); the position equals the
    FP64 step on the dequantized state."""
    nc = 10
    x = np.array([[0.30, 0.36], [0.55, 0.55], [0.45, 0.45]])
    cell, o = oracle.quantize(x, nc)
    v = np.array([[1.0, -1.0], [0.0, 0.0], [0.0, 0.0]], np.float32)
    r, m, ids = np.full(2, 0.01, np.float32), np.ones(2, np.float32), np.arange(2, dtype=np.int32)
    xd = oracle.dequantize(cell, o, nc) * nc                     # cell units
    R = (float(r[0]) + float(r[1])) * nc
    t = (xd[0, 1] - xd[0, 0] - R) / (2.0 * nc)                   # closing speed 2 nc cells per unit time
    dt = t + (4.0 - 1e-9 - (xd[0, 1] - t * nc)) / nc             # sphere 1 leaves at +1 after the exchange
    c1, o1, v1, p, tc, k = oracle.collide_step_cellrel(cell, o, v, r, m, ids, nc, 1.0, dt)
    assert k == 1 and np.all((o1 >= 0.0) & (o1 < 1.0))
    assert c1[1] % nc == 4 and o1[0, 1] == 0.0
    x2, _, _, _, _ = oracle.collide_step(oracle.dequantize(cell, o, nc), v.astype(np.float64), r.astype(np.float64),
                                         m.astype(np.float64), ids, 1.0, dt)
    assert abs(x2[0, 1] * nc - (4.0 - 1e-9)) < 1e-10
    d = oracle.dequantize(c1, o1, nc) - x2
    d -= np.round(d)
    assert np.max(np.abs(d)) * nc < 1e-6


def test_cellrel_momentum_conserved_to_storage_rounding():
    w = inputs.draw("dense_1m", n=2500, seed=22)
    nc = 25
    cell, o = oracle.quantize(w["x"], nc)
    vf, rf, mf = w["v"].astype(np.float32), w["r"].astype(np.float32), w["m"].astype(np.float32)
    c1, o1, v1, p, tc, k = oracle.collide_step_cellrel(cell, o, vf, rf, mf, w["id"], nc, 0.8, 40 * w["dt"])
    assert k > 5
    p0 = (mf.astype(np.float64) * vf).sum(axis=1)
    p1 = (mf.astype(np.float64) * v1).sum(axis=1)
    scale = (mf.astype(np.float64) * np.abs(vf)).sum(axis=1)
    assert np.all(np.abs(p1 - p0) <= 1e-6 * scale)
