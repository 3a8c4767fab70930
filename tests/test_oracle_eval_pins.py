"""Pins of the oracle's field evaluation at particles (Sec. 3.2) and drag sources (Sec. 2.2,
2.3) against facts that do not come from the oracle: a DG field that samples a polynomial
of degree <= N per axis reproduces it exactly anywhere in the element; scipy's barycentric
Lagrange interpolation on a separable field; values at the nodes; the Stokes limit and
the Schiller-Naumann factor at Re = 1 (1.15) in closed form; sources are minus the force
and minus its power."""
import math

import numpy as np
import pytest

import oracle

interpolate = pytest.importorskip("scipy.interpolate")


def _nodes(ne, n1):
    eta, _ = np.polynomial.legendre.leggauss(n1)
    return (np.arange(ne)[:, None] + 0.5 * (eta[None, :] + 1.0)) / ne  # [element][i]


def _field_from(fun, ne, n1, nvar):
    """Field [ne^3][nvar][n1^3] sampling fun(c, X, Y, Z) at every Gauss node."""
    X1 = _nodes(ne, n1)
    F = np.zeros((ne, ne, ne, nvar, n1, n1, n1))
    for ez in range(ne):
        for ey in range(ne):
            for ex in range(ne):
                Z, Y, X = np.meshgrid(X1[ez], X1[ey], X1[ex], indexing="ij")
                for c in range(nvar):
                    F[ez, ey, ex, c] = fun(c, X, Y, Z)
    return F.reshape(ne ** 3, nvar, n1 ** 3)


@pytest.mark.parametrize("ne,degree", [(3, 0), (3, 2), (2, 5), (4, 7)])
def test_polynomial_of_degree_n_is_reproduced(ne, degree):
    """Inside one element a field sampling a product of per-axis polynomials of degree <=
    N is that polynomial: random coefficients, particles anywhere in the box (each is
    evaluated from its own element's sampling of the same global polynomial)."""
    rng = np.random.default_rng(ne * 10 + degree)
    n1 = degree + 1
    coef = rng.normal(size=(2, 3, n1))
    fun = lambda c, X, Y, Z: (np.polyval(coef[c, 0], X) * np.polyval(coef[c, 1], Y) * np.polyval(coef[c, 2], Z))
    F = _field_from(fun, ne, n1, 2)
    x = rng.random((3, 300))
    out = oracle.eval_field(x, F, ne, degree)
    ref = np.stack([fun(c, x[0], x[1], x[2]) for c in range(2)])
    assert np.allclose(out, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_separable_field_matches_scipy_barycentric():
    """A field that is a product of arbitrary per-axis node values: the evaluation is the
    product of three 1-D Lagrange interpolants (scipy's barycentric formula)."""
    ne, degree = 3, 4
    n1 = degree + 1
    rng = np.random.default_rng(7)
    vals = rng.normal(size=(3, ne, n1))  # per axis, per element, node values
    X1 = _nodes(ne, n1)

    def fun(c, X, Y, Z):
        out = np.ones_like(X)
        for a, A in enumerate((X, Y, Z)):
            e = np.clip(np.floor(A * ne).astype(int), 0, ne - 1)
            i = np.argmin(np.abs(X1[e] - A[..., None]), axis=-1)
            out = out * vals[a, e, i]
        return out

    F = _field_from(fun, ne, n1, 1)
    x = rng.random((3, 200))
    out = oracle.eval_field(x, F, ne, degree)[0]
    ref = np.ones(200)
    for a in range(3):
        e = np.clip(np.floor(x[a] * ne).astype(int), 0, ne - 1)
        for p in range(200):
            ref[p] *= interpolate.BarycentricInterpolator(X1[e[p]], vals[a, e[p]])(x[a, p])
    assert np.allclose(out, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_value_at_a_node_is_the_coefficient():
    ne, degree = 2, 3
    n1 = degree + 1
    rng = np.random.default_rng(8)
    F = rng.normal(size=(ne ** 3, 3, n1 ** 3))
    X1 = _nodes(ne, n1)
    x = np.array([[X1[1, 2]], [X1[0, 0]], [X1[1, 3]]])
    out = oracle.eval_field(x, F, ne, degree)[:, 0]
    e = (1 * ne + 0) * ne + 1
    g = (3 * n1 + 0) * n1 + 2
    assert np.allclose(out, F[e, :, g], rtol=1e-14, atol=1e-15)


def test_drag_stokes_limit_and_schiller_naumann_at_re_one():
    mu_f = 1.8e-5
    r = np.array([1e-4, 2e-4, 5e-5])
    d = 2 * r
    rho = np.array([1.2, 1.2, 1.0])
    v = np.array([[1.0, -0.3, 0.0], [0.2, 0.0, 0.0], [0.0, 0.1, 0.0]])  # [3][n]
    U = v.copy()
    U[0, 0] += mu_f / (rho[0] * d[0])          # particle 0: slip along x with Re = 1
    U[0, 2] += 1e-3 * mu_f / (rho[2] * d[2])   # particle 2: Re = 1e-3 (Stokes regime); particle 1: no slip
    q = oracle.drag_sources(v, r, np.concatenate([rho[None], U]), mu_f)
    rel = U - v
    re = rho * np.sqrt((rel ** 2).sum(0)) * d / mu_f
    assert abs(re[0] - 1.0) < 1e-12 and abs(re[2] - 1e-3) < 1e-15
    assert np.allclose(-q[:3, 0], 3 * math.pi * mu_f * d[0] * 1.15 * rel[:, 0], rtol=1e-13, atol=0)
    assert not q[:, 1].any()
    assert np.allclose(-q[:3, 2], 3 * math.pi * mu_f * d[2] * rel[:, 2], rtol=2e-3, atol=0)
    for p in range(3):
        assert abs(q[3, p] - (q[:3, p] * v[:, p]).sum()) <= 1e-15 * max(1.0, abs(q[3, p]))


@pytest.mark.parametrize("re,cd", [(10, 4.15106594049), (100, 1.09173109109), (800, 0.474258079492)])
def test_drag_coefficient_of_the_schiller_naumann_curve(re, cd):
    """The force in drag-coefficient form, C_D = |F| / (rho |w|^2 / 2 * pi d^2 / 4), w the
    slip, against the correlation's tabulated values C_D = 24/Re (1 + 0.15 Re^0.687)
    (the numbers are written out here, computed to 12 digits in 30-digit arithmetic):
    wrong exponent, coefficient, or d/r/mu/rho placement fails it. The force is along
    the slip, in any direction."""
    rng = np.random.default_rng(re)
    mu_f, rho, r = 1.8e-5, 1.1, 3e-4
    d = 2 * r
    e = rng.normal(size=3)
    e /= np.linalg.norm(e)
    speed = re * mu_f / (rho * d)
    v = rng.normal(size=(3, 1))
    U = v + speed * e[:, None]
    q = oracle.drag_sources(v, np.array([r]), np.concatenate([[[rho]], U]), mu_f)
    F = -q[:3, 0]
    assert abs(np.linalg.norm(F) / (0.5 * rho * speed ** 2 * math.pi * d ** 2 / 4) - cd) <= 1e-9 * cd
    assert np.allclose(F / np.linalg.norm(F), e, rtol=0, atol=1e-14)
