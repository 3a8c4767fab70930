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
