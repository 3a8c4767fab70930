"""Pins of the oracle's hand-derived adjoints: a plain PyTorch float64 restatement
differentiated by torch.autograd (test-only), central finite differences, and the
replay reproducing the search-based step."""
import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs

torch = pytest.importorskip("torch")


def _small_colliding_state(seed, n=400, dtmul=40):
    w = inputs.draw("dense_1m", seed=seed, n=n)
    dt = dtmul * w["dt"]
    x1, v1, partner, tc, k = oracle.collide_step(w["x"], w["v"], w["r"], w["m"], w["id"], 0.9, dt, "bruteforce")
    return w, dt, partner, k


def test_replay_equals_search_step_bitwise():
    w, dt, partner, k = _small_colliding_state(0, n=2000)
    assert k > 5
    x1, v1, _, _, _ = oracle.collide_step(w["x"], w["v"], w["r"], w["m"], w["id"], 0.9, dt)
    x2, v2 = oracle.collide_replay(w["x"], w["v"], w["r"], w["m"], partner, 0.9, dt)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)


def test_replay_counts_contact_at_the_end_of_the_step():
    """Contact exactly at t = dt counts (the inclusive bound of the search step): two
    spheres of radius 1/32 head-on at unit speed, 1/8 apart, meet at t = 1/32 exactly in
    binary arithmetic; with dt = 1/32 the replay of that pair succeeds and equals the
    search step bit for bit."""
    x = np.array([[0.25, 0.375], [0.5, 0.5], [0.5, 0.5]])
    v = np.array([[1.0, -1.0], [0.0, 0.0], [0.0, 0.0]])
    r, m, ids, dt = np.full(2, 0.03125), np.array([1.0, 2.0]), np.arange(2, dtype=np.int32), 0.03125
    x1, v1, partner, tc, k = oracle.collide_step(x, v, r, m, ids, 0.7, dt)
    assert k == 1 and tc[0] == dt
    x2, v2 = oracle.collide_replay(x, v, r, m, np.array([1, 0]), 0.7, dt)
    assert np.array_equal(x2, x1) and np.array_equal(v2, v1)


def _torch_replay(x, v, r, m, partner, e, dt):
    """Plain torch float64 restatement of one step with a fixed matching (test only)."""
    n = x.shape[1]
    xn, vn = x + dt * v, v.clone()
    xn = [xn[a].clone() for a in range(3)]
    vn = [vn[a].clone() for a in range(3)]
    for i in range(n):
        j = int(partner[i])
        if j < 0:
            continue
        dx = x[:, i] - x[:, j]
        dx = dx - torch.round(dx.detach())  # minimum image (a constant shift)
        dv = v[:, i] - v[:, j]
        R = r[i] + r[j]
        a = (dv * dv).sum()
        b = (dx * dv).sum()
        c = (dx * dx).sum() - R * R
        t = c / (-b + torch.sqrt(b * b - a * c))
        s = dx + t * dv
        nrm = -s / torch.sqrt((s * s).sum())
        vrn = (dv * nrm).sum()
        mr = m[i] * m[j] / (m[i] + m[j])
        J = -mr * (1 + e) * vrn
        vnew = v[:, i] + (J / m[i]) * nrm
        for aa in range(3):
            vn[aa] = torch.cat([vn[aa][:i], vnew[aa:aa + 1], vn[aa][i + 1:]])
            xnew = x[aa, i] + t * v[aa, i] + (dt - t) * vnew[aa]
            xn[aa] = torch.cat([xn[aa][:i], xnew.reshape(1), xn[aa][i + 1:]])
    return torch.stack(xn), torch.stack(vn)


def test_collide_adjoint_matches_torch_autograd():
    w, dt, partner, k = _small_colliding_state(1, n=900, dtmul=200)
    assert k >= 3
    rng = np.random.default_rng(0)
    gxo, gvo = rng.normal(size=(3, 900)), rng.normal(size=(3, 900))
    gx, gv = oracle.collide_adjoint(w["x"], w["v"], w["r"], w["m"], partner, 0.9, dt, gxo, gvo)
    xt = torch.tensor(w["x"], requires_grad=True)
    vt = torch.tensor(w["v"], requires_grad=True)
    xn, vn = _torch_replay(xt, vt, torch.tensor(w["r"]), torch.tensor(w["m"]), partner, 0.9, dt)
    L = (xn * torch.tensor(gxo)).sum() + (vn * torch.tensor(gvo)).sum()
    L.backward()
    assert np.allclose(gx, xt.grad.numpy(), rtol=1e-10, atol=1e-10)
    assert np.allclose(gv, vt.grad.numpy(), rtol=1e-10, atol=1e-10)


def test_collide_adjoint_matches_central_differences():
    w, dt, partner, k = _small_colliding_state(2, n=900, dtmul=200)
    assert k >= 3
    rng = np.random.default_rng(1)
    gxo, gvo = rng.normal(size=(3, 900)), rng.normal(size=(3, 900))
    gx, gv = oracle.collide_adjoint(w["x"], w["v"], w["r"], w["m"], partner, 0.9, dt, gxo, gvo)
    h = 1e-7
    for trial in range(4):
        ux, uv = rng.normal(size=(3, 900)), rng.normal(size=(3, 900))
        f = []
        for sgn in (1, -1):
            xs = w["x"] + sgn * h * ux
            xs -= np.floor(xs)
            x1, v1 = oracle.collide_replay(xs, w["v"] + sgn * h * uv, w["r"], w["m"], partner, 0.9, dt)
            f.append((gxo * x1).sum() + (gvo * v1).sum())
        fd = (f[0] - f[1]) / (2 * h)
        # remove the periodic wrap jumps (a wrap changes x' by exactly 1)
        ad = (gx * ux).sum() + (gv * uv).sum()
        assert abs(fd - ad) <= 1e-5 * max(1.0, abs(ad)), (fd, ad)


def _torch_project_loss(xt, qt, T, ne, degree, sigma, cs):
    """Plain torch float64 restatement of the projection with the support fixed at x (test only)."""
    x = xt.detach().numpy()
    n = x.shape[1]
    n1 = degree + 1
    eta, w = np.polynomial.legendre.leggauss(n1)
    h = 1.0 / ne
    X1 = ((np.arange(ne)[:, None] + 0.5 * (eta[None, :] + 1.0)) * h).ravel()
    W1 = np.tile(w, ne) * h / 2
    rc = cs * sigma
    F = torch.zeros(ne ** 3, 4, n1 ** 3, dtype=torch.float64)
    for p in range(n):
        sel, shifts = [], []
        for a in range(3):
            d = X1 - x[a, p]
            sh = -np.round(d)
            ok = np.abs(d + sh) <= rc
            sel.append(np.nonzero(ok)[0])
            shifts.append(sh[ok])
        gi, gj, gk = np.meshgrid(sel[0], sel[1], sel[2], indexing="ij")
        si, sj, sk = np.meshgrid(shifts[0], shifts[1], shifts[2], indexing="ij")
        dx = torch.tensor(X1[gi] + si) - xt[0, p]
        dy = torch.tensor(X1[gj] + sj) - xt[1, p]
        dz = torch.tensor(X1[gk] + sk) - xt[2, p]
        K = torch.exp(-(dx * dx + dy * dy + dz * dz) / (2 * sigma * sigma))
        Wg = torch.tensor(W1[gi] * W1[gj] * W1[gk])
        Z = (Wg * K).sum()
        e = ((gk // n1) * ne + gj // n1) * ne + gi // n1
        g = ((gk % n1) * n1 + gj % n1) * n1 + gi % n1
        idx = torch.tensor((e * 4 * n1 ** 3 + g).ravel())
        for c in range(4):
            F.view(-1).index_add_(0, idx + c * n1 ** 3, (qt[c, p] * K / Z).reshape(-1))
    return 0.5 * ((F - torch.tensor(T)) ** 2).sum(), F


def test_project_adjoint_matches_torch_autograd():
    w = inputs.draw("small_8192", seed=3, n=40)
    ne, deg, sigma = 4, 2, 0.06
    F0, _ = oracle.project(w["x"], w["q"], ne, deg, sigma, 3.0)
    rng = np.random.default_rng(2)
    T = F0 + rng.normal(size=F0.shape)
    xt = torch.tensor(w["x"], requires_grad=True)
    qt = torch.tensor(w["q"], requires_grad=True)
    L, F = _torch_project_loss(xt, qt, T, ne, deg, sigma, 3.0)
    assert np.allclose(F.detach().numpy(), F0, rtol=1e-12, atol=1e-12)
    L.backward()
    gq, gx = oracle.project_adjoint(w["x"], w["q"], F0 - T, ne, deg, sigma, 3.0)
    assert np.allclose(gq, qt.grad.numpy(), rtol=1e-10, atol=1e-10)
    assert np.allclose(gx, xt.grad.numpy(), rtol=1e-9, atol=1e-9 * np.abs(gx).max())


def test_project_adjoint_matches_central_differences():
    w = inputs.draw("small_8192", seed=4, n=60)
    ne, deg, sigma = 4, 3, 0.05
    F0, _ = oracle.project(w["x"], w["q"], ne, deg, sigma, 3.0)
    rng = np.random.default_rng(3)
    T = F0 + rng.normal(size=F0.shape)
    gq, gx = oracle.project_adjoint(w["x"], w["q"], F0 - T, ne, deg, sigma, 3.0)
    h = 1e-7
    done = 0
    for trial in range(20):
        ux, uq = rng.normal(size=(3, 60)), rng.normal(size=(4, 60))
        L = []
        for sgn in (1, -1):
            xs = w["x"] + sgn * h * ux
            xs -= np.floor(xs)
            F, _ = oracle.project(xs, w["q"] + sgn * h * uq, ne, deg, sigma, 3.0)
            L.append(0.5 * ((F - T) ** 2).sum())
        fd = (L[0] - L[1]) / (2 * h)
        ad = (gx * ux).sum() + (gq * uq).sum()
        if abs(fd - ad) > 1e-4 * max(1.0, abs(ad)):
            # a node crossed the cutoff between the two evaluations: a jump, not a derivative
            continue
        done += 1
    assert done >= 15
