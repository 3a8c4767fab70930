"""The curved-mesh workload at full size: 67,108,864 spheres (lognormal d, median 1.6e-3,
log-sigma 0.25, placed largest first) on the 128^3 mesh of degree 3 curved by the sine
map (amplitude 0.02), spherical-cutoff Gaussian sigma = 3e-3 (Sec. 3.2.1 localisation,
Sec. 4.2 deposition). One collision step on the FP32 cell-relative storage, then the
curved projection; sampled elements of the field against the oracle run on the
particles that can reach them (the dequantised stored state), 1e-5 normwise per
component with the whole field's maximum as the scale. Drawing the state takes a few
minutes on the host."""
import numpy as np
import pytest

import oracle
from paper_2501_05340_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_05340_gb300 import pc  # noqa: E402

TOL = 1e-5


def _phi(xi, amp):
    s = np.sin(2 * np.pi * xi)
    return xi + amp * np.stack([s[1] * s[2], s[2] * s[0], s[0] * s[1]])


def test_curved_full_size_sampled():
    w = inputs.draw("curved_67m", seed=0)
    wl = w["workload"]
    n = w["x"].shape[1]
    dt = w["dt"]
    assert n == 1 << 26
    ctx = pc.Context(n, wl.ne, wl.degree, wl.sigma, w["e"], pc.reach_of(w["r"], w["v"], w["dt"]),
                     cutoff="sphere", amp=wl.amp)
    s64 = pc.State.from_arrays(w)
    del w["x"], w["v"]
    a = pc.StateF32.empty(n)
    ctx.quantize(s64, a)
    del s64
    b = pc.StateF32.empty(n)
    ctx.collide_f32(a, b, dt)
    f = ctx.new_field_f32()
    ctx.project_curved_f32(b, f)
    ctx.sync()
    st = ctx.stats()
    assert st["pairs"] > 0
    nc = ctx.cells_per_side
    g = b.numpy()
    x = oracle.dequantize(g["cell"], g["o"], nc)
    q = g["q"].astype(np.float64)
    del g
    rng = np.random.default_rng(5)
    ne = wl.ne
    elems = rng.choice(ne ** 3, 3, replace=False)
    keep = np.zeros(n, bool)
    for el in elems:
        xi = (np.array([el % ne, (el // ne) % ne, el // ne ** 2]) + 0.5) / ne
        c = _phi(xi, wl.amp)
        d = np.abs((x - c[:, None] + 0.5) % 1.0 - 0.5)
        keep |= (d <= 0.03).all(axis=0)
    R, _ = oracle.project(x[:, keep], q[:, keep], ne, wl.degree, wl.sigma, wl.cutoff_sigmas, cutoff="sphere",
                          amp=wl.amp)
    F = f[torch.as_tensor(elems, device="cuda")].cpu().numpy().astype(np.float64)
    scale = f.abs().amax(dim=(0, 2)).cpu().numpy()
    err = np.abs(F - R[elems]).max(axis=(0, 2)) / scale
    print("curved full size: %d particles near the sampled elements, normwise error %s" % (keep.sum(), err))
    assert keep.sum() > 1000
    assert np.all(err <= TOL), err
