"""Pins of the oracle's response with Coulomb friction and rotation (Sec. 2.4) against facts
that do not come from the oracle: the frictionless response (pinned on its own), the
sticking limit (the tangential contact-point velocity leaves reversed and scaled by e, so
it vanishes at e = 0: the 2/7 law), the sliding law (tangential impulse mu J_n), and the
conservation of linear and angular momentum of every pair about the contact point; total
kinetic energy (translational + rotational) does not grow for e <= 1."""
import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs


def _cross(a, b):
    return np.cross(a, b, axis=0)


def _pair_case(rng, vt_scale=1.0, wscale=1.0):
    """Two spheres about to touch: returns x, v, w, r, m, partner, tc at a chosen contact."""
    r = np.array([0.011, 0.017])
    m = np.array([1.3, 0.6])
    nrm = rng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    t = 0.3e-3
    dt = 1e-3
    # relative velocity: approaching along n plus a tangential part
    tang = rng.normal(size=3)
    tang -= tang.dot(nrm) * nrm
    vr = 2.0 * nrm + vt_scale * tang  # v1 - v2, approaching: (v1 - v2).n > 0
    v2 = rng.normal(size=3)
    v1 = v2 + vr
    xc = np.array([0.5, 0.5, 0.5])
    x1c = xc - r[0] * nrm
    x2c = xc + r[1] * nrm
    x = np.stack([x1c - t * v1, x2c - t * v2], axis=1)
    v = np.stack([v1, v2], axis=1)
    w = wscale * rng.normal(size=(3, 2))
    return x, v, w, r, m, np.array([1, 0]), np.array([t, t]), dt, nrm


def _contact_velocity(v, w, r, nrm):
    return (v[:, 0] - v[:, 1]) + r[0] * np.cross(w[:, 0], nrm) + r[1] * np.cross(w[:, 1], nrm)


def _run(x, v, w, r, m, partner, tc, e, mu, dt):
    ids = np.arange(x.shape[1], dtype=np.int32)
    return oracle.respond_advance_rot(x, v, w, r, m, ids, partner, tc, e, mu, dt)


@pytest.mark.parametrize("e", [0.0, 0.5, 0.9, 1.0])
def test_sticking_reverses_tangential_contact_velocity_by_e(e):
    """Large mu (sticking): J_t = -(2/7)(1+e) m_r |v_rt|, which for solid spheres turns the
    tangential contact-point velocity into -e times itself; at e = 0 it vanishes."""
    rng = np.random.default_rng(1)
    x, v, w, r, m, partner, tc, dt, nrm = _pair_case(rng, vt_scale=0.3)
    _, v1, w1 = _run(x, v, w, r, m, partner, tc, e, 10.0, dt)
    vc0 = _contact_velocity(v, w, r, nrm)
    vc1 = _contact_velocity(v1, w1, r, nrm)
    vt0 = vc0 - vc0.dot(nrm) * nrm
    vt1 = vc1 - vc1.dot(nrm) * nrm
    assert np.allclose(vt1, -e * vt0, rtol=0, atol=1e-12 * np.abs(vt0).max())
    # and the normal relative velocity is reversed by e, as without friction
    vn0 = (v[:, 0] - v[:, 1]).dot(nrm)
    vn1 = (v1[:, 0] - v1[:, 1]).dot(nrm)
    assert abs(vn1 + e * vn0) <= 1e-12 * abs(vn0)


def test_sliding_tangential_impulse_is_mu_jn():
    """Small mu (sliding): the tangential impulse on particle 1 is mu J_n along t."""
    rng = np.random.default_rng(2)
    x, v, w, r, m, partner, tc, dt, nrm = _pair_case(rng, vt_scale=3.0)
    e, mu = 0.8, 0.05
    _, v1, _ = _run(x, v, w, r, m, partner, tc, e, mu, dt)
    mr = m[0] * m[1] / (m[0] + m[1])
    Jn = -mr * (1 + e) * (v[:, 0] - v[:, 1]).dot(nrm)
    vc0 = _contact_velocity(v, w, r, nrm)
    vt0 = vc0 - vc0.dot(nrm) * nrm
    t = vt0 / np.linalg.norm(vt0)
    J = m[0] * (v1[:, 0] - v[:, 0])
    assert np.allclose(J, Jn * nrm + mu * Jn * t, rtol=0, atol=1e-12 * abs(Jn))
    assert np.allclose(m[1] * (v1[:, 1] - v[:, 1]), -J, rtol=0, atol=1e-12 * abs(Jn))


def test_zero_friction_equals_frictionless_response_and_keeps_spin():
    w_ = inputs.draw("small_8192", seed=3, n=3000)
    rng = np.random.default_rng(3)
    w0 = rng.normal(size=(3, 3000)) * 50
    x1, v1, part, tc, k = oracle.collide_step(w_["x"], w_["v"], w_["r"], w_["m"], w_["id"], 0.9, 10 * w_["dt"])
    assert k > 20
    x2, v2, w2 = oracle.respond_advance_rot(w_["x"], w_["v"], w0, w_["r"], w_["m"], w_["id"], part, tc, 0.9, 0.0,
                                            10 * w_["dt"])
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2) and np.array_equal(w0, w2)


@pytest.mark.parametrize("mu", [0.0, 0.1, 0.4, 5.0])
def test_momentum_and_angular_momentum_conserved_energy_not_increased(mu):
    """Every pair: sum m v and sum (m (x_c - X) x v + I w) about any point X are unchanged
    (x_c the positions at contact); E = sum (m v^2 + I w^2)/2 does not grow (e <= 1)."""
    d = inputs.draw("small_8192", seed=4, n=4000)
    rng = np.random.default_rng(4)
    w0 = rng.normal(size=(3, 4000)) * 30
    dt, e = 10 * d["dt"], 0.7
    x, v, r, m = d["x"], d["v"], d["r"], d["m"]
    x1, v1, w1, part, tc, k = oracle.collide_step_rot(x, v, w0, r, m, d["id"], e, mu, dt)
    assert k > 20
    inertia = 0.4 * m * r * r
    i = np.nonzero(part >= 0)[0]
    j = part[i]
    keep = i < j
    i, j = i[keep], j[keep]
    dp = m[i] * (v1[:, i] - v[:, i]) + m[j] * (v1[:, j] - v[:, j])
    assert np.abs(dp).max() <= 1e-13 * np.abs(m[i] * v[:, i]).max()
    # contact positions relative to particle i's contact position (minimum image)
    rel = x[:, j] - x[:, i]
    rel -= np.round(rel)
    rel += tc[i] * (v[:, j] - v[:, i])
    L0 = m[j] * _cross(rel, v[:, j]) + inertia[i] * w0[:, i] + inertia[j] * w0[:, j]
    L1 = m[j] * _cross(rel, v1[:, j]) + inertia[i] * w1[:, i] + inertia[j] * w1[:, j]
    # about particle i's centre at contact, its own orbital term is zero
    scale = np.abs(L0).max()
    assert np.abs(L1 - L0).max() <= 1e-12 * scale
    E0 = 0.5 * (m * (v * v).sum(0) + inertia * (w0 * w0).sum(0))
    E1 = 0.5 * (m * (v1 * v1).sum(0) + inertia * (w1 * w1).sum(0))
    pair_E0 = E0[i] + E0[j]
    pair_E1 = E1[i] + E1[j]
    assert np.all(pair_E1 <= pair_E0 * (1 + 1e-13))


def test_free_particles_keep_spin_and_fly():
    d = inputs.draw("small_8192", seed=5, n=500)
    w0 = np.random.default_rng(5).normal(size=(3, 500))
    part = -np.ones(500, np.int64)
    x1, v1, w1 = oracle.respond_advance_rot(d["x"], d["v"], w0, d["r"], d["m"], d["id"], part, np.zeros(500), 0.9,
                                            0.3, 1e-3)
    assert np.array_equal(w1, w0) and np.array_equal(v1, d["v"])
    ref = d["x"] + 1e-3 * d["v"]
    ref -= np.floor(ref)
    assert np.allclose(x1, ref, rtol=0, atol=1e-15)


def test_head_on_without_spin_has_no_tangential_impulse():
    """A head-on collision of non-spinning spheres: the contact-point velocity is exactly
    normal (|v_rt| = 0), so friction adds no tangential impulse whatever mu: the response
    is the frictionless one bit for bit and the spins stay zero (no 0/0 direction)."""
    x = np.array([[0.5, 0.504], [0.5, 0.5], [0.5, 0.5]])
    v = np.array([[1.0, -1.0], [0.0, 0.0], [0.0, 0.0]])
    r, m, ids = np.full(2, 0.001), np.array([1.0, 3.0]), np.arange(2, dtype=np.int32)
    dt = 0.01
    t = oracle.contact_time(x[:, 0], x[:, 1], v[:, 0], v[:, 1], r[0], r[1], dt)
    assert 0 < t <= dt
    partner, tc = np.array([1, 0]), np.array([t, t])
    x0, v0 = oracle.respond_advance(x, v, m, partner, tc, 0.9, dt)
    x1, v1, w1 = oracle.respond_advance_rot(x, v, np.zeros((3, 2)), r, m, ids, partner, tc, 0.9, 0.3, dt)
    assert np.all(np.isfinite(v1)) and np.array_equal(v1, v0) and np.array_equal(x1, x0)
    assert not w1.any()
