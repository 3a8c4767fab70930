"""CPU oracle for the particle collision and projection operator (arXiv 2501.05340).

TEST INFRASTRUCTURE ONLY. Plain FP64 C (``oracle.c``) behind ctypes. Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may load
it; the library under ``paper_2501_05340_gb300`` never does and shares no code
with it. Arrays are numpy, SoA ``[3][n]`` / ``[4][n]``, in the caller's order.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile ``liboracle.so`` next to the source (strict IEEE: no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, d = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.or_gauss_legendre.argtypes = [i32, P, P]
        lib.or_contact_time.argtypes = [P, P, P, P, d, d, d]
        lib.or_contact_time.restype = d
        for f in (lib.or_candidates_bruteforce, lib.or_candidates_cells):
            f.argtypes = [i64, P, P, P, d, i64, P, P, P]
            f.restype = i64
        lib.or_match_greedy.argtypes = [i64, P, i64, P, P, P, P, P]
        lib.or_match_greedy.restype = i64
        lib.or_match_rounds.argtypes = [i64, P, i64, P, P, P, P, P, P]
        lib.or_match_rounds.restype = i64
        lib.or_respond_advance.argtypes = [i64, P, P, P, P, P, d, d]
        lib.or_respond_advance.restype = None
        lib.or_collide_step.argtypes = [i64, P, P, P, P, P, d, d, i32, P, P]
        lib.or_collide_step.restype = i64
        lib.or_collide_step_cellrel.argtypes = [i64, i32, P, P, P, P, P, P, d, d, P, P]
        lib.or_collide_step_cellrel.restype = i64
        lib.or_collide_replay.argtypes = [i64, P, P, P, P, P, d, d]
        lib.or_collide_replay.restype = i32
        lib.or_collide_adjoint.argtypes = [i64, P, P, P, P, P, d, d, P, P, P, P]
        lib.or_collide_adjoint.restype = i32
        lib.or_project_adjoint.argtypes = [i64, P, P, i32, i32, d, d, i32, P, P, P]
        lib.or_project_adjoint.restype = i32
        lib.or_mesh_map.argtypes = [P, d, P, P]
        lib.or_mesh_map.restype = None
        lib.or_project.argtypes = [i64, P, P, i32, i32, d, d, i32, d, P, P]
        lib.or_project.restype = i32
        lib.or_respond_advance_rot.argtypes = [i64, P, P, P, P, P, P, P, P, d, d, d]
        lib.or_respond_advance_rot.restype = None
        lib.or_eval_field.argtypes = [i64, P, P, i32, i32, i32, P]
        lib.or_eval_field.restype = i32
        lib.or_drag_sources.argtypes = [i64, P, P, P, d, P]
        lib.or_drag_sources.restype = None
        lib.or_collide_step_sfc.argtypes = [i64, P, P, P, P, P, d, d, i64, P, P]
        lib.or_collide_step_sfc.restype = i64
        for f in (lib.or_project_idw, lib.or_project_dirac):
            f.argtypes = [i64, P, P, i32, i32, P]
            f.restype = i32
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def gauss_legendre(n1):
    """Legendre-Gauss nodes (ascending) and weights on [-1, 1]."""
    eta, w = np.zeros(n1), np.zeros(n1)
    if _load().or_gauss_legendre(n1, _p(eta), _p(w)):
        raise ValueError("bad n1")
    return eta, w


def contact_time(xi, xj, vi, vj, ri, rj, dt):
    """Smaller positive root of |dx + t dv| = ri + rj if it is a candidate, else inf."""
    a = [_f64(u) for u in (xi, xj, vi, vj)]
    return _load().or_contact_time(*[_p(u) for u in a], float(ri), float(rj), float(dt))


def candidates(x, v, r, dt, method="cells"):
    """Candidate pairs (i<j, input indices) and their contact times, sorted by (i, j)."""
    x, v, r = _f64(x), _f64(v), _f64(r)
    n = r.shape[0]
    f = _load().or_candidates_cells if method == "cells" else _load().or_candidates_bruteforce
    cap = max(64, 4 * n)
    while True:
        ci, cj = np.zeros(cap, np.int64), np.zeros(cap, np.int64)
        ct = np.zeros(cap)
        cnt = f(n, _p(x), _p(v), _p(r), float(dt), cap, _p(ci), _p(cj), _p(ct))
        if cnt < 0:
            raise MemoryError("oracle candidates")
        if cnt <= cap:
            break
        cap = cnt
    ci, cj, ct = ci[:cnt], cj[:cnt], ct[:cnt]
    o = np.lexsort((cj, ci))
    return ci[o], cj[o], ct[o]


def match(ids, ci, cj, ct, n, method="greedy"):
    """Matching of a candidate list: returns (partner, tc, npairs[, rounds])."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    ci, cj = np.ascontiguousarray(ci, np.int64), np.ascontiguousarray(cj, np.int64)
    ct = _f64(ct)
    partner, tc = np.zeros(n, np.int64), np.zeros(n)
    lib = _load()
    if method == "greedy":
        k = lib.or_match_greedy(n, _p(ids), len(ci), _p(ci), _p(cj), _p(ct), _p(partner), _p(tc))
        return partner, tc, k
    rounds = np.zeros(1, np.int64)
    k = lib.or_match_rounds(n, _p(ids), len(ci), _p(ci), _p(cj), _p(ct), _p(partner), _p(tc), _p(rounds))
    return partner, tc, k, int(rounds[0])


def respond_advance(x, v, m, partner, tc, e, dt):
    """Response of committed pairs + free flight + wrap; returns new (x, v)."""
    x, v = _f64(x).copy(), _f64(v).copy()
    m = _f64(m)
    partner = np.ascontiguousarray(partner, np.int64)
    tc = _f64(tc)
    _load().or_respond_advance(m.shape[0], _p(x), _p(v), _p(m), _p(partner), _p(tc), float(e), float(dt))
    return x, v


def respond_advance_rot(x, v, w, r, m, ids, partner, tc, e, mu, dt):
    """Response with friction and rotation + free flight + wrap; returns new (x, v, w)."""
    x, v, w = _f64(x).copy(), _f64(v).copy(), _f64(w).copy()
    r, m = _f64(r), _f64(m)
    ids = np.ascontiguousarray(ids, np.int32)
    partner = np.ascontiguousarray(partner, np.int64)
    tc = _f64(tc)
    _load().or_respond_advance_rot(m.shape[0], _p(x), _p(v), _p(w), _p(r), _p(m), _p(ids), _p(partner), _p(tc),
                                   float(e), float(mu), float(dt))
    return x, v, w


def collide_step_rot(x, v, w, r, m, ids, e, mu, dt, method="cells"):
    """One collision step with friction and rotation: the pairs of collide_step (they do
    not depend on w), then respond_advance_rot. Returns (x', v', w', partner, tc, npairs)."""
    _, _, partner, tc, k = collide_step(x, v, r, m, ids, e, dt, method)
    x1, v1, w1 = respond_advance_rot(x, v, w, r, m, ids, partner, tc, e, mu, dt)
    return x1, v1, w1, partner, tc, k


def collide_step_sfc(x, v, r, m, ids, e, dt, ncell):
    """One collision step with first-found pair selection along the Morton curve over
    ncell^3 cells; returns (x', v', partner, tc, npairs)."""
    x, v = _f64(x).copy(), _f64(v).copy()
    r, m = _f64(r), _f64(m)
    ids = np.ascontiguousarray(ids, np.int32)
    n = r.shape[0]
    partner, tc = np.zeros(n, np.int64), np.zeros(n)
    k = _load().or_collide_step_sfc(n, _p(x), _p(v), _p(r), _p(m), _p(ids), float(e), float(dt), int(ncell),
                                    _p(partner), _p(tc))
    if k < 0:
        raise MemoryError("oracle collide")
    return x, v, partner, tc, k


def collide_step(x, v, r, m, ids, e, dt, method="cells"):
    """One collision step in the input order; returns (x', v', partner, tc, npairs)."""
    x, v = _f64(x).copy(), _f64(v).copy()
    r, m = _f64(r), _f64(m)
    ids = np.ascontiguousarray(ids, np.int32)
    n = r.shape[0]
    partner, tc = np.zeros(n, np.int64), np.zeros(n)
    k = _load().or_collide_step(n, _p(x), _p(v), _p(r), _p(m), _p(ids), float(e), float(dt),
                                1 if method == "bruteforce" else 0, _p(partner), _p(tc))
    if k < 0:
        raise MemoryError("oracle collide")
    return x, v, partner, tc, k


def quantize(x, nc):
    """FP64 positions in [0,1) -> (linear cell, FP32 offsets in cell units) of an nc^3 grid:
    s = x nc, c = floor(s) (clamped), o = float32(s - c), and o == 1 carried into the next cell."""
    x = _f64(x)
    s = x * float(nc)
    c = np.clip(np.floor(s), 0, nc - 1).astype(np.int64)
    o = (s - c).astype(np.float32)
    carry = o >= np.float32(1.0)
    o[carry] = 0.0
    c[carry] = (c[carry] + 1) % nc
    cell = ((c[2] * nc + c[1]) * nc + c[0]).astype(np.int32)
    return cell, np.ascontiguousarray(o)


def dequantize(cell, o, nc):
    """Linear cell + FP32 offsets -> FP64 positions (c + o) / nc in [0,1)."""
    cell = np.asarray(cell, np.int64)
    c = np.stack([cell % nc, (cell // nc) % nc, cell // (nc * nc)]).astype(np.float64)
    return (c + np.asarray(o, np.float64)) / float(nc)


def collide_step_cellrel(cell, o, v, r, m, ids, nc, e, dt):
    """One step of the mixed-storage method; returns (cell', o', v', partner, tc, npairs)."""
    cell = np.ascontiguousarray(cell, np.int32).copy()
    o = np.ascontiguousarray(o, np.float32).copy()
    v = np.ascontiguousarray(v, np.float32).copy()
    r = np.ascontiguousarray(r, np.float32)
    m = np.ascontiguousarray(m, np.float32)
    ids = np.ascontiguousarray(ids, np.int32)
    n = r.shape[0]
    partner, tc = np.zeros(n, np.int64), np.zeros(n)
    k = _load().or_collide_step_cellrel(n, int(nc), _p(cell), _p(o), _p(v), _p(r), _p(m), _p(ids), float(e),
                                        float(dt), _p(partner), _p(tc))
    if k < 0:
        raise MemoryError("oracle collide_step_cellrel")
    return cell, o, v, partner, tc, k


def collide_replay(x, v, r, m, partner, e, dt):
    """One step with a fixed matching; returns (x', v'). Raises if a pair lost its root."""
    x, v = _f64(x).copy(), _f64(v).copy()
    r, m = _f64(r), _f64(m)
    partner = np.ascontiguousarray(partner, np.int64)
    rc = _load().or_collide_replay(r.shape[0], _p(x), _p(v), _p(r), _p(m), _p(partner), float(e), float(dt))
    if rc != 0:
        raise ValueError("replay: a recorded pair has no contact in [0, dt]")
    return x, v


def collide_adjoint(x, v, r, m, partner, e, dt, gx_out, gv_out):
    """Cotangents of the pre-step (x, v) of one replayed step."""
    x, v, r, m = _f64(x), _f64(v), _f64(r), _f64(m)
    partner = np.ascontiguousarray(partner, np.int64)
    gxo, gvo = _f64(gx_out), _f64(gv_out)
    gx, gv = np.zeros_like(x), np.zeros_like(v)
    rc = _load().or_collide_adjoint(r.shape[0], _p(x), _p(v), _p(r), _p(m), _p(partner), float(e), float(dt),
                                    _p(gxo), _p(gvo), _p(gx), _p(gv))
    if rc != 0:
        raise ValueError("adjoint: a recorded pair has no contact in [0, dt]")
    return gx, gv


def project_adjoint(x, q, G, ne, degree, sigma, cutoff_sigmas=3.0, cutoff="box"):
    """(dL/dq [4][n], dL/dx [3][n]) for dL/dfield = G."""
    x, q, G = _f64(x), _f64(q), _f64(G)
    n = x.shape[-1]
    gq, gx = np.zeros((4, n)), np.zeros((3, n))
    rc = _load().or_project_adjoint(n, _p(x), _p(q), ne, degree, float(sigma), float(cutoff_sigmas),
                                    0 if cutoff == "box" else 1, _p(G), _p(gq), _p(gx))
    if rc:
        raise ValueError("or_project_adjoint failed")
    return gq, gx


def project_idw(x, q, ne, degree):
    """Field [ne^3][4][n1^3] of the linear corner-node (IDW) deposition."""
    x, q = _f64(x), _f64(q)
    n = x.shape[-1]
    n1 = degree + 1
    field = np.zeros((ne ** 3, 4, n1 ** 3))
    rc = _load().or_project_idw(n, _p(x), _p(q), ne, degree, _p(field))
    if rc:
        raise ValueError("or_project_idw failed (%d)" % rc)
    return field


def project_dirac(x, q, ne, degree):
    """Field [ne^3][4][n1^3] of the nearest-node (Dirac) deposition."""
    x, q = _f64(x), _f64(q)
    n = x.shape[-1]
    n1 = degree + 1
    field = np.zeros((ne ** 3, 4, n1 ** 3))
    rc = _load().or_project_dirac(n, _p(x), _p(q), ne, degree, _p(field))
    if rc:
        raise ValueError("or_project_dirac failed (%d)" % rc)
    return field


def eval_field(x, field, ne, degree):
    """DG solution at the particles: out [nvar][n] from field [ne^3][nvar][n1^3]."""
    x, field = _f64(x), _f64(field)
    n = x.shape[-1]
    nvar = field.shape[1]
    out = np.zeros((nvar, n))
    rc = _load().or_eval_field(n, _p(x), _p(field), ne, degree, nvar, _p(out))
    if rc:
        raise ValueError("or_eval_field failed (%d)" % rc)
    return out


def drag_sources(v, r, fluid, mu_f):
    """Sources q [4][n] = (-F, -F.v) of the drag force from fluid [4][n] = (rho, u)."""
    v, r, fluid = _f64(v), _f64(r), _f64(fluid)
    q = np.zeros((4, r.shape[0]))
    _load().or_drag_sources(r.shape[0], _p(v), _p(r), _p(fluid), float(mu_f), _p(q))
    return q


def mesh_map(xi, amp):
    """Curved periodic mapping of one logical point: (X, det J)."""
    xi = _f64(xi)
    X, dj = np.zeros(3), np.zeros(1)
    _load().or_mesh_map(_p(xi), float(amp), _p(X), _p(dj))
    return X, float(dj[0])


def project(x, q, ne, degree, sigma, cutoff_sigmas=3.0, cutoff="box", amp=0.0):
    """Field [ne^3][4][n1^3] and normalisation Z[n] of the Gaussian deposition."""
    x, q = _f64(x), _f64(q)
    n = x.shape[-1]
    n1 = degree + 1
    field = np.zeros((ne ** 3, 4, n1 ** 3))
    Z = np.zeros(n)
    rc = _load().or_project(n, _p(x), _p(q), ne, degree, float(sigma), float(cutoff_sigmas),
                            0 if cutoff == "box" else 1, float(amp), _p(field), _p(Z))
    if rc:
        raise ValueError("or_project failed (%d)" % rc)
    return field, Z
