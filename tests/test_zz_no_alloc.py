"""pc_project_noalloc, the projection for callers that may not allocate device
memory (its scratch is a fixed array inside the library), against pc_project on
two calls in a row with different inputs, and the smaller case against the
oracle too; free device memory is unchanged across its calls. Collected last on
purpose."""
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

FIELD_TOL = 1e-12


def _reference_field(w, wl):
    a = pc.State.from_arrays(w)
    ctx = pc.Context(a.n, wl.ne, wl.degree, wl.sigma, w["e"], 0.05, cutoff_sigmas=wl.cutoff_sigmas)
    f = ctx.new_field()
    ctx.project(a, f)
    ctx.sync()
    out = f.cpu().numpy()
    ctx.close()
    return a, out


def test_noalloc_matches_project_twice():
    cases = [("small_8192", None, 0), ("dense_1m", 5000, 1)]
    for name, n, seed in cases:
        w = inputs.draw(name, seed=seed, n=n)
        wl = w["workload"]
        a, ref = _reference_field(w, wl)
        f = torch.full((wl.ne ** 3, 4, (wl.degree + 1) ** 3), float("nan"), dtype=torch.float64, device="cuda")
        pc.project_noalloc(a, f, wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
        torch.cuda.synchronize()
        got = f.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.all(field_err(got, ref) <= FIELD_TOL), name
        if name == "small_8192":
            R, _ = oracle.project(w["x"], w["q"], wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
            assert np.all(field_err(got, R) <= FIELD_TOL), "oracle"


def test_noalloc_allocates_nothing():
    """After a first call (which may load the library's kernels onto the device), further
    calls leave the device's free memory unchanged: the scratch is the fixed array."""
    w = inputs.draw("dense_1m", seed=2, n=20000)
    wl = w["workload"]
    a = pc.State.from_arrays(w)
    f = torch.empty((wl.ne ** 3, 4, (wl.degree + 1) ** 3), dtype=torch.float64, device="cuda")
    pc.project_noalloc(a, f, wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        pc.project_noalloc(a, f, wl.ne, wl.degree, wl.sigma, wl.cutoff_sigmas)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_oversized_problem():
    n = 200000  # about 512 bytes per particle on a 32^3 mesh of degree 5: beyond 32 MiB
    a = pc.State.empty(n)
    f = torch.empty(32 ** 3, 4, 6 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcError) as ei:
        pc.project_noalloc(a, f, 32, 5, 0.01, 3.0)
    assert ei.value.status == pc.PC_ECAPACITY
    assert "bytes of scratch" in str(ei.value)
