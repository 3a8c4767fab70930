"""Pins of the oracle's corner-node (IDW) and nearest-node (Dirac) depositions, Sec. 2.3
and Sec. 4.2, against facts written in physical coordinates: the periodic tent
(hat) function of a corner node, a uniform source that every partition of unity maps
to a constant, brute-force nearest DOF over the whole periodic mesh, conservation,
and translation by one element."""
import numpy as np
import pytest

import oracle


def _nodes_1d(ne, n1):
    """Physical coordinates of the Gauss nodes of each element along one axis [ne][n1]."""
    eta, w = np.polynomial.legendre.leggauss(n1)
    return (np.arange(ne)[:, None] + 0.5 * (eta[None, :] + 1.0)) / ne, w


def _weights(ne, n1):
    """Quadrature weight W_g |J| of each DOF, shaped like one element's [n1^3] block."""
    _, w = np.polynomial.legendre.leggauss(n1)
    W = np.einsum("k,j,i->kji", w, w, w).ravel()
    return W * (0.5 / ne) ** 3


def _total(field, ne, n1):
    return np.einsum("ecg,g->c", field, _weights(ne, n1))


def _tent(d, h):
    """Periodic 1-D hat of half-width h at minimum-image distance d."""
    d = np.abs(d - np.round(d))
    return np.clip(1.0 - d / h, 0.0, None)


def _idw_physical(x, q, ne, n1):
    """IDW field from its physical form: node sums S_n = sum_p q_p tent(x_p - X_n) and
    F(X_g) = sum_n S_n tent(X_g - X_n) / h^3 over every corner node of the periodic mesh."""
    h = 1.0 / ne
    X1, _ = _nodes_1d(ne, n1)
    grid = np.arange(ne) * h
    # per axis: tent of each particle and of each Gauss node against each corner plane
    tp = [_tent(x[a][:, None] - grid[None, :], h) for a in range(3)]  # [n][ne]
    S = np.einsum("cp,pz,py,px->czyx", q, tp[2], tp[1], tp[0])
    tg = _tent(X1.ravel()[:, None] - grid[None, :], h).reshape(ne, n1, ne)  # [element][i][corner plane]
    F = np.einsum("czyx,akz,bjy,dix->abdckji", S, tg, tg, tg, optimize=True) / h ** 3
    return F.reshape(ne ** 3, 4, n1 ** 3)


@pytest.mark.parametrize("ne,degree", [(3, 0), (3, 1), (4, 2), (3, 5)])
def test_idw_matches_physical_tent_form(ne, degree):
    """Random sources: the oracle (reference coordinates, corner signs, quadrature node
    volumes) equals the same deposition written with periodic tents in physical space
    (node volume h^3, which the quadrature reaches exactly for the affine mesh)."""
    rng = np.random.default_rng(ne * 10 + degree)
    n = 50
    x = rng.random((3, n))
    q = rng.normal(size=(4, n))
    F = oracle.project_idw(x, q, ne, degree)
    ref = _idw_physical(x, q, ne, degree + 1)
    assert np.allclose(F, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("degree", [0, 1, 3])
def test_idw_particle_on_corner_node_is_its_hat(degree):
    """A unit source exactly on corner node (2, 1, 3)/ne: the field is that node's hat
    function over its 8 elements, divided by the node volume h^3, zero elsewhere."""
    ne, n1 = 4, degree + 1
    h = 1.0 / ne
    node = np.array([2, 1, 3]) * h
    x = node[:, None].copy()
    q = np.array([[1.0], [0.0], [2.0], [-1.0]])
    F = oracle.project_idw(x, q, ne, degree)
    X1, _ = _nodes_1d(ne, n1)
    hat = [_tent(X1 - node[a], h) for a in range(3)]  # [ne][n1]
    ref = np.einsum("zk,yj,xi->zyxkji", hat[2], hat[1], hat[0]).reshape(ne ** 3, n1 ** 3) / h ** 3
    for c in range(4):
        assert np.allclose(F[:, c], q[c, 0] * ref, rtol=0, atol=1e-12 / h ** 3)
    assert np.count_nonzero(np.abs(F[:, 0]).max(axis=1)) == 8


@pytest.mark.parametrize("degree", [0, 2, 4])
def test_idw_uniform_sources_give_constant_density(degree):
    """One source per element at its centre puts q/8 on each corner 8 times: equal node
    sums, so the density is q / h^3 at every DOF (partition of unity)."""
    ne = 3
    c1 = (np.arange(ne) + 0.5) / ne
    x = np.stack([a.ravel() for a in np.meshgrid(c1, c1, c1, indexing="ij")])
    q = np.tile(np.array([[1.5], [-2.0], [0.25], [3.0]]), x.shape[1])
    F = oracle.project_idw(x, q, ne, degree)
    for c in range(4):
        assert np.allclose(F[:, c], q[c, 0] * ne ** 3, rtol=1e-13, atol=0)


@pytest.mark.parametrize("kind", ["idw", "dirac"])
def test_deposition_conserves_each_source(kind):
    """Sec. 4.2 conservative deposition: sum_g W_g |J| F_gc = sum_p q_pc per component."""
    rng = np.random.default_rng(3)
    ne, degree = 4, 3
    x, q = rng.random((3, 300)), rng.normal(size=(4, 300))
    f = oracle.project_idw if kind == "idw" else oracle.project_dirac
    F = f(x, q, ne, degree)
    assert np.allclose(_total(F, ne, degree + 1), q.sum(axis=1), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", ["idw", "dirac"])
def test_deposition_translates_with_the_mesh(kind):
    """Moving every source by one element along x (periodic) moves the field by one element."""
    rng = np.random.default_rng(4)
    ne, degree = 3, 2
    # quarter-element offsets: x * ne stays exactly representable after the shift
    x = rng.integers(0, 4 * ne, size=(3, 40)) / (4.0 * ne) + 1.0 / (8.0 * ne)
    q = rng.normal(size=(4, 40))
    f = oracle.project_idw if kind == "idw" else oracle.project_dirac
    F = f(x, q, ne, degree).reshape(ne, ne, ne, 4, -1)
    xs = x.copy()
    xs[0] = (xs[0] + 1.0 / ne) % 1.0
    Fs = f(xs, q, ne, degree).reshape(ne, ne, ne, 4, -1)
    assert np.allclose(np.roll(F, 1, axis=2), Fs, rtol=0, atol=1e-12 * np.abs(F).max())


@pytest.mark.parametrize("ne,degree", [(2, 1), (3, 2), (2, 5)])
def test_dirac_is_the_nearest_dof_by_brute_force(ne, degree):
    """Each source lands on the DOF nearest to it in physical space, found by scanning
    every DOF of the periodic mesh with minimum-image distances, as q / (W_g |J|)."""
    n1 = degree + 1
    rng = np.random.default_rng(ne + degree)
    n = 200
    x = rng.random((3, n))
    q = rng.normal(size=(4, n))
    F = oracle.project_dirac(x, q, ne, degree)
    X1, _ = _nodes_1d(ne, n1)
    Xz, Xy, Xx = np.meshgrid(X1.ravel(), X1.ravel(), X1.ravel(), indexing="ij")  # global (z, y, x) order
    W = _weights(ne, n1)
    ref = np.zeros_like(F)
    for p in range(n):
        d2 = sum((np.abs(Xa - x[a, p]) - np.round(np.abs(Xa - x[a, p]))) ** 2 for a, Xa in ((0, Xx), (1, Xy), (2, Xz)))
        gz, gy, gx = np.unravel_index(np.argmin(d2), d2.shape)
        e = ((gz // n1) * ne + gy // n1) * ne + gx // n1
        g = ((gz % n1) * n1 + gy % n1) * n1 + gx % n1
        ref[e, :, g] += q[:, p] / W[g]
    assert np.allclose(F, ref, rtol=1e-13, atol=0)


def test_dirac_source_on_a_gauss_node():
    """A source placed on DOF (e, g) gives q / (W_g |J|) there and nothing elsewhere."""
    ne, degree = 3, 3
    n1 = degree + 1
    X1, _ = _nodes_1d(ne, n1)
    x = np.array([[X1[2, 1]], [X1[0, 3]], [X1[1, 0]]])
    q = np.array([[2.0], [1.0], [-1.0], [0.5]])
    F = oracle.project_dirac(x, q, ne, degree)
    e, g = (1 * ne + 0) * ne + 2, (0 * n1 + 3) * n1 + 1
    W = _weights(ne, n1)
    assert np.allclose(F[e, :, g], q[:, 0] / W[g], rtol=1e-14)
    F[e, :, g] = 0
    assert not F.any()


@pytest.mark.parametrize("degree", [1, 3, 5, 7])
def test_dirac_tie_goes_to_the_lower_node(degree):
    """Reading of the nearest-DOF deposition: a source exactly halfway between two nodes of
    an axis goes to the lower one. With an even node count the element centre (reference
    coordinate exactly 0) is halfway between the two middle nodes on every axis (the rule's
    nodes are symmetric bit for bit, checked first): the whole source lands on node
    (a, a, a), a = n1/2 - 1, of that element, as q / (w_a^3 (h/2)^3), and nowhere else."""
    ne, n1 = 3, degree + 1
    eta, w = oracle.gauss_legendre(n1)
    a = n1 // 2 - 1
    assert eta[a] == -eta[a + 1]
    x = np.full((3, 1), 0.5)  # centre of element (1, 1, 1)
    q = np.array([[2.0], [-1.0], [0.5], [3.0]])
    F = oracle.project_dirac(x, q, ne, degree)
    e = (1 * ne + 1) * ne + 1
    g = (a * n1 + a) * n1 + a
    h = 1.0 / ne
    expect = np.zeros_like(F)
    expect[e, :, g] = q[:, 0] / (w[a] ** 3 * (h / 2) ** 3)
    assert np.allclose(F, expect, rtol=1e-14, atol=0)
