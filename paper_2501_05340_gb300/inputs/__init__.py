"""Seeded synthetic workloads shaped like the paper's dense particle-laden cases.

This module only draws inputs (``gen.c``): sphere centres by random sequential
addition in the periodic unit cube, diameters, N(0,1) velocities and N(0,1)
sources. It holds none of the collision or projection arithmetic, so both the
CPU oracle and the CUDA library can consume what it writes.

Workloads are named by what they are, with their sizes:

* ``small_8192``   8192 monodisperse spheres d=0.02, 8^3 mesh N=3, sigma=0.02, dt=2e-3, e=0.9
* ``dense_1m``     1,048,576 spheres d~U[0.006,0.008], 32^3 mesh N=5, sigma=0.01, e=0.9
* ``mixed_16m``    16,777,216 spheres d lognormal(2.2e-3, 0.2) clipped [1e-3,4e-3], 64^3 mesh N=7, sigma=4e-3, e=0.85
* ``curved_67m``   67,108,864 spheres d lognormal(1.6e-3, 0.25), 128^3 curved mesh N=3, sigma=3e-3, e=0.9,
                   placed largest first: in drawn order the largest spheres (3-4x the median) come
                   up when the box is already near phi = 0.19 and find almost no free space left

Every workload can be drawn at a reduced particle count (``n=``) with the same
diameter law; the mesh and kernel are kept, the time step follows the same rule.
"""
import ctypes
import dataclasses
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libpcgen.so")
_lib = None


def build(force=False):
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, i64, u64, d, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        lib.pcgen_normal.argtypes = [i64, u64, u64, d, P]
        lib.pcgen_uniform.argtypes = [i64, u64, u64, d, d, P]
        lib.pcgen_fixed_speed.argtypes = [i64, u64, u64, d, P]
        lib.pcgen_diameters.argtypes = [i64, u64, i32, d, d, d, d, P]
        lib.pcgen_rsa.argtypes = [i64, u64, P, P, i64, P]
        lib.pcgen_rsa_sequential.argtypes = [i64, u64, P, P, i64, P]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    dkind: int            # 0 constant, 1 uniform, 2 lognormal
    dparams: tuple        # (p0, p1, p2, p3) of the diameter law
    e: float              # restitution
    steps: int
    ne: int               # elements per side
    degree: int           # DG degree N, n1 = N + 1 nodes per axis
    sigma: float          # Gaussian width
    cutoff_sigmas: float = 3.0
    cutoff: str = "box"   # "box" (separable) or "sphere"
    amp: float = 0.0      # curved-mesh amplitude (0 = affine)
    dt: float = 0.0       # 0: dt = 0.99 * 0.25 * d_min / max|v|, 3 significant figures, rounded down
    place: str = "drawn"  # placement order: "drawn" (index order) or "largest_first" (ties by index)


WORKLOADS = {
    "small_8192": Workload("small_8192", 8192, 0, (0.02, 0, 0, 0), 0.9, 100, 8, 3, 0.02, dt=2e-3),
    "dense_1m": Workload("dense_1m", 1 << 20, 1, (0.006, 0.008, 0, 0), 0.9, 50, 32, 5, 0.01),
    "mixed_16m": Workload("mixed_16m", 1 << 24, 2, (2.2e-3, 0.2, 1e-3, 4e-3), 0.85, 20, 64, 7, 4e-3),
    "curved_67m": Workload("curved_67m", 1 << 26, 2, (1.6e-3, 0.25, 0.0, 0.0), 0.9, 10, 128, 3, 3e-3,
                           cutoff="sphere", amp=0.02, place="largest_first"),
}


def dt_rule(d, v):
    """dt = 0.99 * 0.25 * d_min / max|v|, rounded down to 3 significant figures."""
    vmax = float(np.sqrt((v * v).sum(axis=0)).max())
    raw = 0.99 * 0.25 * float(d.min()) / vmax
    e10 = math.floor(math.log10(raw))
    return math.floor(raw / 10 ** (e10 - 2)) * 10 ** (e10 - 2)


def draw(workload, seed=0, n=None, max_reject=None):
    """Draw one workload. Returns a dict of numpy arrays (SoA, float64):

    x[3][n], v[3][n], r[n], m[n] (rho = 1: m = pi d^3 / 6), id[n] (int32, 0..n-1),
    q[4][n], plus the scalars dt, e and the achieved volume fraction phi.
    """
    w = WORKLOADS[workload] if isinstance(workload, str) else workload
    n = w.n if n is None else int(n)
    lib = _load()
    d = np.zeros(n)
    if lib.pcgen_diameters(n, seed, w.dkind, *[float(a) for a in w.dparams], _p(d)):
        raise ValueError("bad diameter law")
    r = 0.5 * d
    if w.place == "drawn":
        perm = None
    elif w.place == "largest_first":
        perm = np.argsort(-r, kind="stable")
    else:
        raise ValueError("unknown placement order %r" % (w.place,))
    rp = r if perm is None else np.ascontiguousarray(r[perm])
    xp = np.zeros((3, n))
    rej = np.zeros(1, np.int64)
    rc = lib.pcgen_rsa(n, seed, _p(rp), _p(xp), int(max_reject or 50 * n + 1000), _p(rej))
    if rc:
        raise RuntimeError("random sequential addition failed (code %d)" % rc)
    if perm is None:
        x = xp
    else:
        x = np.empty_like(xp)
        x[:, perm] = xp
    v = np.zeros((3, n))
    lib.pcgen_normal(3 * n, seed, 3, 1.0, _p(v))
    q = np.zeros((4, n))
    lib.pcgen_normal(4 * n, seed, 4, 1.0, _p(q))
    m = math.pi / 6.0 * d ** 3
    dt = w.dt if w.dt > 0 else dt_rule(d, v)
    phi = float((math.pi / 6.0 * d ** 3).sum())
    return dict(x=x, v=v, r=r, m=m, id=np.arange(n, dtype=np.int32), q=q, dt=dt, e=w.e, phi=phi,
                workload=w, rejects=int(rej[0]))


def gas(n, d, speed, seed=0):
    """Kinetic-gas set-up: n spheres of diameter d, |v| = speed, random directions."""
    lib = _load()
    r = np.full(n, 0.5 * d)
    x = np.zeros((3, n))
    rej = np.zeros(1, np.int64)
    if lib.pcgen_rsa(n, seed, _p(r), _p(x), 50 * n + 1000, _p(rej)):
        raise RuntimeError("random sequential addition failed")
    v = np.zeros((3, n))
    lib.pcgen_fixed_speed(n, seed, 5, float(speed), _p(v))
    m = np.full(n, math.pi / 6.0 * d ** 3)
    return dict(x=x, v=v, r=r, m=m, id=np.arange(n, dtype=np.int32))


def normal(n, seed, stream, scale=1.0):
    out = np.zeros(n)
    _load().pcgen_normal(n, seed, stream, float(scale), _p(out))
    return out


def uniform(n, seed, stream, lo=0.0, hi=1.0):
    out = np.zeros(n)
    _load().pcgen_uniform(n, seed, stream, float(lo), float(hi), _p(out))
    return out
