"""The C-ABI library builds, loads and exports every symbol its headers declare,
and rejects invalid arguments before touching the GPU (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pc_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_declared_symbols():
    from paper_2501_05340_gb300 import build
    lib = ctypes.CDLL(build.build())
    names = _declared()
    assert {"pc_init", "pc_collide", "pc_project", "pc_destroy"} <= names
    for s in sorted(names):
        assert hasattr(lib, s), s


def test_argument_validation_without_gpu():
    from paper_2501_05340_gb300 import pc
    lib = pc.library()
    h = ctypes.c_void_p()
    assert lib.pc_init(ctypes.byref(h), None) == pc.PC_EINVAL
    bad = [dict(n_max=0), dict(ne=2), dict(degree=16), dict(sigma=0.0), dict(restitution=1.5),
           dict(reach_hint=0.0), dict(reach_hint=0.5), dict(reach_hint=0.8), dict(cand_cap=33),
           dict(sigma=0.2)]  # sigma=0.2: cutoff beyond half the box; reach >= 0.5: minimum image not unique
    for b in bad:
        kw = dict(n_max=100, ne=8, degree=3, sigma=0.02, cutoff_sigmas=3.0, cutoff_kind=0, restitution=0.9,
                  reach_hint=0.04, cand_cap=16, stream=None)
        kw.update(b)
        cfg = pc.PcConfig(**kw)
        assert lib.pc_init(ctypes.byref(h), ctypes.byref(cfg)) == pc.PC_EINVAL, b
        assert not h.value
    assert lib.pc_collide(None, None, None, 1e-3) == pc.PC_EINVAL
    assert lib.pc_project(None, None, None) == pc.PC_EINVAL
    lib.pc_destroy(None)


def test_noalloc_rejects_more_than_int32_particles_without_gpu():
    """pc_project_noalloc refuses n >= 2^31 (int32 indices on the device) before it
    sizes its scratch or touches the GPU (the pointers are never dereferenced)."""
    from paper_2501_05340_gb300 import pc
    lib = pc.library()
    cfg = pc.PcConfig(n_max=0, ne=8, degree=3, sigma=0.02, cutoff_sigmas=3.0, cutoff_kind=0, restitution=0.0,
                      reach_hint=0.0, cand_cap=0, stream=None)
    fake = ctypes.c_void_p(256)
    p = pc.PcParticles(1 << 31, fake, fake, fake, fake, fake, fake)
    msg = ctypes.create_string_buffer(128)
    assert lib.pc_project_noalloc(ctypes.byref(cfg), ctypes.byref(p), fake, msg, 128) == pc.PC_EINVAL
    assert b"2^31" in msg.value


def test_binding_rejects_host_and_misshaped_tensors():
    """The binding hands raw device pointers to the library, so it refuses host tensors,
    other dtypes, non-contiguous views and wrong shapes before any call (the library
    cannot tell a host pointer from a device one)."""
    torch = pytest.importorskip("torch")
    from paper_2501_05340_gb300 import pc
    host = torch.zeros(3, 5, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        pc._dev(host, "w_in", torch.float64, (3, 5))
    n = 5
    f64 = lambda *s: torch.zeros(*s, dtype=torch.float64)
    with pytest.raises(ValueError, match="State.x"):
        pc.State(f64(3, n), f64(3, n), f64(n), f64(n), torch.zeros(n, dtype=torch.int32))
    with pytest.raises(ValueError, match="StateF32.id"):
        pc.StateF32(torch.zeros(n, dtype=torch.int32), torch.zeros(n, dtype=torch.int32),
                    torch.zeros(3, n), torch.zeros(3, n), torch.zeros(n), torch.zeros(n))
    # the shape test itself, on a tensor that passes every other check but residence
    t = f64(4, n).t()
    assert not t.is_contiguous()
    for bad, shape in ((f64(4, n), (3, n)), (f64(4, n), (4, n, 1)), (t, (n, 4))):
        with pytest.raises(ValueError):
            pc._dev(bad, "q", torch.float64, shape)


def test_every_entry_point_rejects_a_null_context():
    """Every function the header declares has its argument types set in the binding and
    refuses a NULL context (or configuration) with PC_EINVAL before any CUDA call; the
    three non-status functions return their documented values."""
    from paper_2501_05340_gb300 import pc
    lib = pc.library()
    names = _declared()
    special = {"pc_cells_per_side": 0, "pc_last_error": b"null context", "pc_destroy": None}
    for name in sorted(names):
        f = getattr(lib, name)
        assert f.argtypes is not None, "%s has no argtypes in the binding" % name
        args = [0.0 if t is ctypes.c_double else 0 if t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64) else None
                for t in f.argtypes]
        got = f(*args)
        if name in special:
            assert got == special[name], name
        else:
            assert got == pc.PC_EINVAL, (name, got)
