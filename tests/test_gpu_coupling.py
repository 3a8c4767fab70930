"""Parity of the fluid -> particle coupling (pc_eval_field, pc_drag_sources, through the C
ABI) with the oracle.

Field evaluation: double-float arithmetic (coefficients kept to 46 bits, products and sums
to about 2^-46, the reference coordinate to 2^-47) against the oracle's compensated FP64
sums. The coordinate's error enters through the basis' derivative, which grows like
(N+1)^2, so for random coefficients the normwise error is about 2^-47 (N+1)^2 times the
ratio of sum |U l| to max |U|: the test asks for 1e-12 normwise per variable for N <= 7
(the workloads' degrees) and 2e-11 above. Drag sources: within 1e-13 of |F| (1 + |v|) per
particle (FP64 on both sides; CUDA's pow and the C library's may differ in the last bit, and
the power F.v may cancel)."""
import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs
from tests.gpu_helpers import field_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_05340_gb300 import pc  # noqa: E402

T = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", torch.float64)


def _state(x, v=None, r=None):
    n = x.shape[1]
    return pc.State.from_arrays(dict(x=x, v=np.zeros((3, n)) if v is None else v,
                                     r=np.full(n, 1e-3) if r is None else r, m=np.ones(n),
                                     id=np.arange(n, dtype=np.int32), q=np.zeros((4, n))))


def _norm_err(a, b):
    return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)


@pytest.mark.parametrize("ne,degree,n,nvar", [(4, 3, 3000, 5), (3, 5, 1029, 4), (5, 0, 777, 1), (3, 7, 129, 3),
                                              (3, 11, 200, 2), (3, 15, 65, 1)])
def test_eval_matches_oracle(ne, degree, n, nvar):
    rng = np.random.default_rng(ne * 100 + degree + n)
    x = rng.random((3, n))
    field = rng.normal(size=(ne ** 3, nvar, (degree + 1) ** 3))
    ctx = pc.Context(n, ne, degree, 0.1 / ne, 0.9, 0.1)
    out = ctx.eval_field(_state(x), T(field))
    ctx.sync()
    ref = oracle.eval_field(x, field, ne, degree)
    err = _norm_err(out.cpu().numpy(), ref)
    assert np.all(err <= (1e-12 if degree <= 7 else 2e-11)), err


def test_eval_clustered_and_on_faces():
    """5000 particles in one element (many chunks) plus positions on element faces and
    corners (reference coordinate exactly -1)."""
    rng = np.random.default_rng(3)
    ne, degree = 4, 4
    x = np.concatenate([(2 + rng.random((3, 5000))) / ne, rng.integers(0, 2 * ne, size=(3, 300)) / (2.0 * ne)], 1)
    field = rng.normal(size=(ne ** 3, 3, (degree + 1) ** 3))
    ctx = pc.Context(x.shape[1], ne, degree, 0.1 / ne, 0.9, 0.1)
    out = ctx.eval_field(_state(x), T(field))
    ctx.sync()
    err = _norm_err(out.cpu().numpy(), oracle.eval_field(x, field, ne, degree))
    assert np.all(err <= 1e-12), err


def test_eval_full_size_and_drag_sources():
    """1,048,576 spheres of the dense workload on the 32^3 degree-5 mesh: a smooth fluid
    state (rho, u) evaluated at every particle, then the drag sources, both against the
    oracle."""
    w = inputs.draw("dense_1m", seed=0)
    wl = w["workload"]
    n = w["x"].shape[1]
    eta, _ = np.polynomial.legendre.leggauss(wl.degree + 1)
    X1 = ((np.arange(wl.ne)[:, None] + 0.5 * (eta[None, :] + 1.0)) / wl.ne)
    # nodal values of rho = 1.2 + 0.1 sin(2 pi x), u = (sin 2 pi y, cos 2 pi z, 0.3 sin 2 pi x)
    E = np.arange(wl.ne)
    ez, ey, ex = np.meshgrid(E, E, E, indexing="ij")
    n1 = wl.degree + 1
    Z = X1[ez.ravel()][:, :, None, None] + 0 * X1[0][None, None, :, None] + 0 * X1[0][None, None, None, :]
    Y = X1[ey.ravel()][:, None, :, None] + 0 * X1[0][None, :, None, None] + 0 * X1[0][None, None, None, :]
    X = X1[ex.ravel()][:, None, None, :] + 0 * X1[0][None, :, None, None] + 0 * X1[0][None, None, :, None]
    tp = 2 * np.pi
    field = np.stack([1.2 + 0.1 * np.sin(tp * X), np.sin(tp * Y), np.cos(tp * Z), 0.3 * np.sin(tp * X)], axis=1)
    field = field.reshape(wl.ne ** 3, 4, n1 ** 3)
    ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], 0.05)
    s = pc.State.from_arrays(w)
    fluid = ctx.eval_field(s, T(field))
    q = ctx.drag_sources(s, fluid, 1.8e-5)
    ctx.sync()
    ref = oracle.eval_field(w["x"], field, wl.ne, wl.degree)
    err = _norm_err(fluid.cpu().numpy(), ref)
    assert np.all(err <= 1e-12), err
    # the interpolant of a smooth field is close to the field itself (sanity of the data)
    assert np.abs(ref[1] - np.sin(tp * w["x"][1])).max() < 1e-3
    qref = oracle.drag_sources(w["v"], w["r"], fluid.cpu().numpy(), 1.8e-5)
    # per particle, relative to |F| (1 + |v|): the power F.v may cancel
    scale = np.sqrt((qref[:3] ** 2).sum(0)) * (1 + np.sqrt((w["v"] ** 2).sum(0)))
    rel = np.abs(q.cpu().numpy() - qref) / np.maximum(scale, 1e-300)
    assert rel.max() <= 1e-13, rel.max()


def test_chain_eval_drag_project_matches_oracle_chain():
    """Two-way source loop on 20,000 particles: pc_eval_field -> pc_drag_sources ->
    pc_project against the same chain in the oracle (field within 1e-12 normwise)."""
    w = inputs.draw("dense_1m", seed=1, n=20000)
    wl = w["workload"]
    n = 20000
    rng = np.random.default_rng(4)
    fl = np.concatenate([1.0 + 0.1 * rng.random((wl.ne ** 3, 1, (wl.degree + 1) ** 3)),
                         rng.normal(size=(wl.ne ** 3, 3, (wl.degree + 1) ** 3))], axis=1)
    ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], 0.05)
    s = pc.State.from_arrays(w)
    fluid = ctx.eval_field(s, T(fl))
    ctx.drag_sources(s, fluid, 1.8e-5, q=s.q)
    F = ctx.new_field()
    ctx.project(s, F)
    ctx.sync()
    fref = oracle.eval_field(w["x"], fl, wl.ne, wl.degree)
    qref = oracle.drag_sources(w["v"], w["r"], fref, 1.8e-5)
    Fref, _ = oracle.project(w["x"], qref, wl.ne, wl.degree, wl.sigma)
    err = field_err(F.cpu().numpy(), Fref)
    assert np.all(err <= 1e-12), err


def test_argument_checks():
    ctx = pc.Context(10, 3, 2, 0.03, 0.9, 0.1)
    s = _state(np.full((3, 10), 0.5))
    f = torch.zeros(27, 17, 27, dtype=torch.float64, device="cuda")
    out = torch.empty(17, 10, dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcError) as ei:
        ctx.eval_field(s, f, out)
    assert ei.value.status == pc.PC_EINVAL
    with pytest.raises(pc.PcError) as ei:
        ctx.drag_sources(s, torch.zeros(4, 10, dtype=torch.float64, device="cuda"), 0.0)
    assert ei.value.status == pc.PC_EINVAL
