"""Parity of the corner-node (IDW) and nearest-DOF (Dirac) depositions (pc_project_idw,
pc_project_dirac, through the C ABI) with the CPU oracle, element by element.

IDW: within 1e-12 normwise per component (FP64 sums of at most a few hundred terms per
node in another order than the oracle's compensated sums). Dirac: the same DOFs are
hit (the nearest-node decision is taken in FP64 on both sides from the same rounded
reference coordinate) and the values agree within 1e-12 normwise."""
import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs
from tests.gpu_helpers import field_err, quad_weights

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_05340_gb300 import pc  # noqa: E402

TOL = 1e-12
KINDS = ("idw", "dirac")


def _state(x, q):
    n = x.shape[1]
    return pc.State.from_arrays(dict(x=x, v=np.zeros((3, n)), r=np.full(n, 1e-3), m=np.ones(n),
                                     id=np.arange(n, dtype=np.int32), q=q))


def _run(kind, x, q, ne, degree, ctx=None):
    n = x.shape[1]
    if ctx is None:
        ctx = pc.Context(max(n, 1), ne, degree, 0.1 / ne, 0.9, 0.1)
    f = torch.full((ne ** 3, 4, (degree + 1) ** 3), np.nan, dtype=torch.float64, device="cuda")
    getattr(ctx, "project_" + kind)(_state(x, q), f)
    ctx.sync()
    return f.cpu().numpy()


def _oracle(kind, x, q, ne, degree):
    return getattr(oracle, "project_" + kind)(x, q, ne, degree)


def _check(kind, F, R):
    assert np.isfinite(F).all()
    if kind == "dirac":
        assert np.array_equal(F != 0, R != 0), "different DOFs hit"
    err = field_err(F, R)
    assert np.all(err <= TOL), err


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("ne,degree,n", [(4, 3, 3000), (3, 5, 1029), (5, 0, 777), (3, 7, 129), (3, 2, 65),
                                         (6, 1, 33), (3, 15, 400)])
def test_matches_oracle(kind, ne, degree, n):
    """Several tiles per element and ragged chunk tails (33, 65, 129 particles), degree 0
    (one node per element), the smallest mesh (3 per side), degree 15."""
    rng = np.random.default_rng(ne * 100 + degree * 7 + n)
    x, q = rng.random((3, n)), rng.normal(size=(4, n))
    _check(kind, _run(kind, x, q, ne, degree), _oracle(kind, x, q, ne, degree))


@pytest.mark.parametrize("kind", KINDS)
def test_clustered_sources(kind):
    """5000 sources inside one element and a few elsewhere: many chunks in one CTA,
    most elements empty."""
    rng = np.random.default_rng(9)
    ne, degree = 4, 4
    x = np.concatenate([(1 + rng.random((3, 5000))) / ne, rng.random((3, 37))], axis=1)
    q = rng.normal(size=(4, x.shape[1]))
    _check(kind, _run(kind, x, q, ne, degree), _oracle(kind, x, q, ne, degree))


@pytest.mark.parametrize("kind", KINDS)
def test_sources_on_element_faces_and_corners(kind):
    """Positions on element faces, edges and corner nodes (x ne an integer), including 0,
    and on element mid-planes (x ne + 1/2 an integer). An odd number of nodes per axis
    keeps the mid-plane on the middle node, not on a tie between two nodes."""
    rng = np.random.default_rng(12)
    ne, degree = 4, 4
    x = rng.integers(0, 2 * ne, size=(3, 500)) / (2.0 * ne)
    q = rng.normal(size=(4, 500))
    _check(kind, _run(kind, x, q, ne, degree), _oracle(kind, x, q, ne, degree))


@pytest.mark.parametrize("kind", KINDS)
def test_empty_input_gives_zero_field(kind):
    F = _run(kind, np.zeros((3, 0)), np.zeros((4, 0)), 3, 2)
    assert not F.any()


@pytest.mark.parametrize("kind", KINDS)
def test_position_outside_the_box_is_rejected(kind):
    x = np.full((3, 4), 0.5)
    x[1, 2] = 1.0
    ctx = pc.Context(4, 3, 2, 0.03, 0.9, 0.1)
    f = torch.empty(27, 4, 27, dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcError) as ei:
        getattr(ctx, "project_" + kind)(_state(x, np.ones((4, 4))), f)
        ctx.sync()
    assert ei.value.status == pc.PC_EINVAL


@pytest.fixture(scope="module")
def dense():
    w = inputs.draw("dense_1m", seed=0)
    wl = w["workload"]
    ctx = pc.Context(w["x"].shape[1], wl.ne, wl.degree, wl.sigma, w["e"], 0.05)
    return w, wl, ctx


@pytest.mark.parametrize("kind", KINDS)
def test_full_size_matches_oracle(dense, kind):
    """1,048,576 spheres of the dense workload on the 32^3 degree-5 mesh: every DOF
    against the oracle, and sum_g W_g F_gc = sum_p q_pc."""
    w, wl, ctx = dense
    F = _run(kind, w["x"], w["q"], wl.ne, wl.degree, ctx)
    R = _oracle(kind, w["x"], w["q"], wl.ne, wl.degree)
    _check(kind, F, R)
    tot = np.einsum("ecg,g->c", F, quad_weights(wl.ne, wl.degree))
    assert np.allclose(tot, w["q"].sum(axis=1), rtol=1e-11, atol=1e-9)


def test_idw_and_dirac_are_deterministic(dense):
    w, wl, ctx = dense
    for kind in KINDS:
        a = _run(kind, w["x"], w["q"], wl.ne, wl.degree, ctx)
        b = _run(kind, w["x"], w["q"], wl.ne, wl.degree, ctx)
        assert np.array_equal(a, b), kind
