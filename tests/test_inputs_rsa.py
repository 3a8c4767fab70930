"""The batched placement of large sphere packings (worker threads test a batch of
candidates against the spheres placed before it, the main thread commits them in
order) gives exactly the packing of the one-by-one random sequential addition:
positions bit for bit, the same count of rejected candidates, the same early exit
when the rejections exceed their bound."""
import numpy as np
import pytest

from paper_2501_05340_gb300 import inputs


def _place(fn, name, n, seed, max_reject, monkeypatch=None, threads=None):
    lib = inputs._load()
    w = inputs.WORKLOADS[name]
    d = np.zeros(n)
    assert lib.pcgen_diameters(n, seed, w.dkind, *[float(a) for a in w.dparams], inputs._p(d)) == 0
    r = 0.5 * d
    x = np.zeros((3, n))
    rej = np.zeros(1, np.int64)
    if threads is not None:
        monkeypatch.setenv("PCGEN_THREADS", str(threads))
    rc = getattr(lib, fn)(n, seed, inputs._p(r), inputs._p(x), int(max_reject), inputs._p(rej))
    return rc, x, int(rej[0])


@pytest.mark.parametrize("name,n,threads", [("dense_1m", 300000, 3), ("mixed_16m", 400000, 8),
                                            ("curved_67m", 600000, 5)])
def test_batched_equals_one_by_one(name, n, threads, monkeypatch):
    a = _place("pcgen_rsa", name, n, 7, 50 * n, monkeypatch, threads)
    b = _place("pcgen_rsa_sequential", name, n, 7, 50 * n)
    assert a[0] == b[0] == 0
    assert a[2] == b[2] and a[2] > 0
    assert np.array_equal(a[1], b[1])


def test_batched_stops_like_one_by_one(monkeypatch):
    """A packing far too dense for the box: both stop after the same number of
    rejections with the same spheres placed."""
    a = _place("pcgen_rsa", "small_8192", 300000, 3, 1000, monkeypatch, 4)
    b = _place("pcgen_rsa_sequential", "small_8192", 300000, 3, 1000)
    assert a[0] == b[0] == 3 and a[2] == b[2] == 1001
    assert np.array_equal(a[1], b[1])


def test_batched_two_grids_equal_one_by_one(monkeypatch):
    """A very wide lognormal size law (median d = 1e-3, log-sigma 1.0, 60,000 spheres):
    the largest sphere sets a coarse grid of a few thousand cells, so the batched
    placement holds the spheres up to 1.5x the mean radius in a fine grid (searched
    several cells deep) and the rest in the coarse one; the packing is still the
    one-by-one packing."""
    lib = inputs._load()
    n = 60000
    d = np.zeros(n)
    assert lib.pcgen_diameters(n, 11, 2, 1e-3, 1.0, 0.0, 0.0, inputs._p(d)) == 0
    r = 0.5 * d
    coarse_cells = np.floor(1.0 / (2 * r.max() * (1 + 1e-9))) ** 3
    assert n >= 8 * coarse_cells  # the two-grid mode of the batched placement
    out = []
    for fn in ("pcgen_rsa", "pcgen_rsa_sequential"):
        if fn == "pcgen_rsa":
            monkeypatch.setenv("PCGEN_THREADS", "6")
            monkeypatch.setenv("PCGEN_MIN_BATCHED", "1000")
        x = np.zeros((3, n))
        rej = np.zeros(1, np.int64)
        rc = getattr(lib, fn)(n, 11, inputs._p(r), inputs._p(x), 50 * n, inputs._p(rej))
        out.append((rc, x, int(rej[0])))
    assert out[0][0] == out[1][0] == 0
    assert out[0][2] == out[1][2]
    assert np.array_equal(out[0][1], out[1][1])


def test_largest_first_placement_is_a_packing_of_the_drawn_sizes():
    """The curved-mesh workload places its spheres largest first (ties by index), each
    keeping its drawn diameter and index: at a reduced count the result holds the same
    diameters as the drawn law, no two spheres overlap in the periodic box, and the
    positions are those of the one-by-one placement of the sorted radii."""
    n = 20000
    w = inputs.draw("curved_67m", seed=5, n=n)
    lib = inputs._load()
    wl = inputs.WORKLOADS["curved_67m"]
    d = np.zeros(n)
    assert lib.pcgen_diameters(n, 5, wl.dkind, *[float(a) for a in wl.dparams], inputs._p(d)) == 0
    assert np.array_equal(w["r"], 0.5 * d)
    order = sorted(range(n), key=lambda i: (-d[i], i))
    rs = np.ascontiguousarray(0.5 * d[order])
    xs = np.zeros((3, n))
    rej = np.zeros(1, np.int64)
    assert lib.pcgen_rsa_sequential(n, 5, inputs._p(rs), inputs._p(xs), 50 * n, inputs._p(rej)) == 0
    assert np.array_equal(w["x"][:, order], xs) and w["rejects"] == int(rej[0])
    # no overlaps: cell list with cells no smaller than the largest diameter
    x, r = w["x"], w["r"]
    nc = int(1.0 / (2 * r.max()))
    c = np.floor(x * nc).astype(np.int64) % nc
    key = (c[2] * nc + c[1]) * nc + c[0]
    cells = {}
    for i, k in enumerate(key):
        cells.setdefault(k, []).append(i)
    worst = np.inf
    for i in range(n):
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    k = (((c[2, i] + dz) % nc) * nc + (c[1, i] + dy) % nc) * nc + (c[0, i] + dx) % nc
                    for j in cells.get(k, ()):
                        if j <= i:
                            continue
                        dd = x[:, j] - x[:, i]
                        dd -= np.round(dd)
                        worst = min(worst, np.sqrt(dd @ dd) - r[i] - r[j])
    assert worst >= 0.0, worst


def _min_gap(x, r):
    """Smallest surface gap over all pairs in the periodic unit cube (cell list, vectorised)."""
    n = x.shape[1]
    nc = max(1, int(1.0 / (2 * r.max() * (1 + 1e-9))))
    c = np.floor(x * nc).astype(np.int64) % nc
    key = (c[2] * nc + c[1]) * nc + c[0]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    starts = np.searchsorted(ks, np.arange(nc ** 3))
    ends = np.searchsorted(ks, np.arange(nc ** 3), side="right")
    worst = np.inf
    for i in range(n):
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    k = (((c[2, i] + dz) % nc) * nc + (c[1, i] + dy) % nc) * nc + (c[0, i] + dx) % nc
                    js = order[starts[k]:ends[k]]
                    js = js[js > i]
                    if len(js):
                        d = x[:, js] - x[:, i:i + 1]
                        d -= np.round(d)
                        gap = np.sqrt((d * d).sum(0)) - r[i] - r[js]
                        worst = min(worst, float(gap.min()))
    return worst


@pytest.mark.parametrize("name,n", [("small_8192", 8192), ("dense_1m", 20000), ("mixed_16m", 20000),
                                    ("curved_67m", 20000)])
def test_every_workload_draw_is_a_valid_state(name, n):
    """Each workload's draw (at a reduced count where the full one is large): positions in
    [0, 1), no two spheres overlapping or touching in the periodic cube, ids 0..n-1,
    m = pi d^3 / 6, the time-step rule, and the reported volume fraction."""
    w = inputs.draw(name, seed=1, n=n)
    x, r = w["x"], w["r"]
    assert x.shape == (3, n) and w["v"].shape == (3, n) and w["q"].shape == (4, n)
    assert np.all((x >= 0.0) & (x < 1.0))
    assert np.array_equal(w["id"], np.arange(n, dtype=np.int32))
    assert np.allclose(w["m"], np.pi / 6 * (2 * r) ** 3, rtol=1e-15, atol=0)
    assert _min_gap(x, r) > 0.0
    assert abs(w["phi"] - float((np.pi / 6 * (2 * r) ** 3).sum())) <= 1e-12
    wl = w["workload"]
    if wl.dt == 0:
        assert w["dt"] == inputs.dt_rule(2 * r, w["v"])
        assert w["dt"] <= 0.99 * 0.25 * (2 * r).min() / np.sqrt((w["v"] ** 2).sum(0)).max()
