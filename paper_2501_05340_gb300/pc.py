"""Python binding of the pc C ABI (``include/pc.h``): argument marshalling only.

Every step of the operator runs in the CUDA library ``libpc.so``; there is no
CPU fallback. The first call that needs the library builds it if it is missing
or stale (nvcc, sm_103a) and loads it; a failed build or load raises.

Particle state lives in torch CUDA tensors (SoA, float64): ``x[3, n]``,
``v[3, n]``, ``r[n]``, ``m[n]``, ``q[4, n]`` and ``id[n]`` (int32).
"""
import ctypes

import numpy as np
import torch

from . import build as _build

c_i64, c_i32, c_d, c_p = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p

PC_OK, PC_EINVAL, PC_ENOMEM, PC_ECUDA, PC_ENOCONVERGE, PC_ECAPACITY, PC_ETIMEOUT, PC_EREPLAY = range(8)
STATUS_NAMES = {0: "PC_OK", 1: "PC_EINVAL", 2: "PC_ENOMEM", 3: "PC_ECUDA", 4: "PC_ENOCONVERGE", 5: "PC_ECAPACITY",
                6: "PC_ETIMEOUT", 7: "PC_EREPLAY"}
PC_TC_F16, PC_TC_BF16 = 0, 1


class PcConfig(ctypes.Structure):
    _fields_ = [("n_max", c_i64), ("ne", c_i32), ("degree", c_i32), ("sigma", c_d), ("cutoff_sigmas", c_d),
                ("cutoff_kind", c_i32), ("restitution", c_d), ("reach_hint", c_d), ("cand_cap", c_i32),
                ("stream", c_p), ("amp", c_d)]


class PcParticles(ctypes.Structure):
    _fields_ = [("n", c_i64), ("id", c_p), ("x", c_p), ("v", c_p), ("r", c_p), ("m", c_p), ("q", c_p)]


class PcParticlesF32(ctypes.Structure):
    _fields_ = [("n", c_i64), ("id", c_p), ("cell", c_p), ("o", c_p), ("v", c_p), ("r", c_p), ("m", c_p),
                ("q", c_p)]


class PcStats(ctypes.Structure):
    _fields_ = [("pairs", c_i64), ("candidates", c_i64), ("worklist", c_i64), ("rounds", c_i64),
                ("fp64_solves", c_i64), ("max_candidates", c_i64), ("cells_per_side", c_i32), ("stencil", c_i32),
                ("device_status", c_i32), ("kernel_launches", c_i64)]

PHASES = ("bin", "gather", "search", "match", "respond", "pbin", "factors", "deposit")


class PcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def library():
    """The loaded ``libpc.so`` (built on first use)."""
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.pc_init.argtypes = [ctypes.POINTER(c_p), ctypes.POINTER(PcConfig)]
        lib.pc_collide.argtypes = [c_p, ctypes.POINTER(PcParticles), ctypes.POINTER(PcParticles), c_d]
        lib.pc_project.argtypes = [c_p, ctypes.POINTER(PcParticles), c_p]
        lib.pc_collide_rot.argtypes = [c_p, ctypes.POINTER(PcParticles), ctypes.POINTER(PcParticles), c_p, c_p, c_d,
                                       c_d]
        lib.pc_collide_rot.restype = ctypes.c_int
        lib.pc_eval_field.argtypes = [c_p, ctypes.POINTER(PcParticles), c_p, c_i32, c_p]
        lib.pc_eval_field.restype = ctypes.c_int
        lib.pc_drag_sources.argtypes = [c_p, ctypes.POINTER(PcParticles), c_p, c_d, c_p]
        lib.pc_drag_sources.restype = ctypes.c_int
        lib.pc_set_pair_policy.argtypes = [c_p, c_i32]
        lib.pc_set_pair_policy.restype = ctypes.c_int
        for f in (lib.pc_project_idw, lib.pc_project_dirac):
            f.argtypes = [c_p, ctypes.POINTER(PcParticles), c_p]
            f.restype = ctypes.c_int
        lib.pc_get_pairs.argtypes = [c_p, c_p, c_p, c_i64, ctypes.POINTER(c_i64)]
        lib.pc_get_stats.argtypes = [c_p, ctypes.POINTER(PcStats)]
        lib.pc_sync.argtypes = [c_p]
        lib.pc_set_timing.argtypes = [c_p, ctypes.c_int]
        lib.pc_get_timing.argtypes = [c_p, c_p, c_p]
        lib.pc_project_curved_f32.argtypes = [c_p, ctypes.POINTER(PcParticlesF32), c_p]
        lib.pc_project_curved_f32.restype = ctypes.c_int
        lib.pc_pairs_to_partner.argtypes = [c_p, c_p, c_i64]
        lib.pc_collide_replay.argtypes = [c_p, ctypes.POINTER(PcParticles), ctypes.POINTER(PcParticles), c_p, c_d]
        lib.pc_collide_adjoint.argtypes = [c_p, ctypes.POINTER(PcParticles), c_p, c_d, c_p, c_p, c_p, c_p]
        lib.pc_project_adjoint.argtypes = [c_p, ctypes.POINTER(PcParticles), c_p, c_p, c_p]
        for f in ("pc_pairs_to_partner", "pc_collide_replay", "pc_collide_adjoint", "pc_project_adjoint"):
            getattr(lib, f).restype = ctypes.c_int
        lib.pc_cells_per_side.argtypes = [c_p]
        lib.pc_cells_per_side.restype = ctypes.c_int32
        lib.pc_quantize.argtypes = [c_p, ctypes.POINTER(PcParticles), ctypes.POINTER(PcParticlesF32)]
        lib.pc_collide_f32.argtypes = [c_p, ctypes.POINTER(PcParticlesF32), ctypes.POINTER(PcParticlesF32), c_d]
        lib.pc_project_f32.argtypes = [c_p, ctypes.POINTER(PcParticlesF32), c_p, ctypes.c_int32]
        lib.pc_collide_replay_f32.argtypes = [c_p, ctypes.POINTER(PcParticlesF32), ctypes.POINTER(PcParticlesF32),
                                              c_p, c_d]
        lib.pc_collide_adjoint_f32.argtypes = [c_p, ctypes.POINTER(PcParticlesF32), c_p, c_d, c_p, c_p, c_p, c_p]
        lib.pc_project_adjoint_f32.argtypes = [c_p, ctypes.POINTER(PcParticlesF32), c_p, c_p, c_p]
        for f in ("pc_quantize", "pc_collide_f32", "pc_project_f32", "pc_collide_replay_f32", "pc_collide_adjoint_f32",
                  "pc_project_adjoint_f32"):
            getattr(lib, f).restype = ctypes.c_int
        lib.pc_project_noalloc.argtypes = [ctypes.POINTER(PcConfig), ctypes.POINTER(PcParticles), c_p,
                                            ctypes.c_char_p, c_i64]
        lib.pc_project_noalloc.restype = ctypes.c_int
        lib.pc_last_error.argtypes = [c_p]
        lib.pc_last_error.restype = ctypes.c_char_p
        lib.pc_destroy.argtypes = [c_p]
        lib.pc_destroy.restype = None
        for f in ("pc_init", "pc_collide", "pc_project", "pc_get_pairs", "pc_get_stats", "pc_sync", "pc_set_timing",
                  "pc_get_timing"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(t):
    return c_p(t.data_ptr()) if t is not None else c_p(0)


def _dev(t, name, dtype, shape, device=None):
    """Check that t is a contiguous CUDA tensor of dtype and shape (None matches any
    extent) on the given CUDA device index; the library reads and writes it through a
    raw device pointer with that layout. Returns t."""
    ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous() and
          t.dim() == len(shape) and all(want is None or got == want for got, want in zip(t.shape, shape)) and
          (device is None or t.device.index == device))
    if not ok:
        dims = ", ".join("*" if d is None else str(d) for d in shape)
        where = "" if device is None else " on cuda:%d" % device
        raise ValueError("%s must be a contiguous CUDA %s tensor of shape (%s)%s" % (name, dtype, dims, where))
    return t


class State:
    """FP64 device particle state (SoA torch tensors)."""

    def __init__(self, x, v, r, m, id, q=None):
        self.x, self.v, self.r, self.m, self.id, self.q = x, v, r, m, id, q
        n = r.shape[0]
        for name, t, shape, dt in (("x", x, (3, n), torch.float64), ("v", v, (3, n), torch.float64),
                                   ("r", r, (n,), torch.float64), ("m", m, (n,), torch.float64),
                                   ("id", id, (n,), torch.int32)):
            if tuple(t.shape) != shape or t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
                raise ValueError("State.%s must be a contiguous CUDA %s tensor of shape %s" % (name, dt, shape))
        if q is not None:
            _dev(q, "State.q", torch.float64, (4, n))
        if len({t.device for t in (x, v, r, m, id, q) if t is not None}) != 1:
            raise ValueError("State tensors must be on one CUDA device")

    @property
    def n(self):
        return self.r.shape[0]

    @property
    def device(self):
        return self.r.device.index

    @staticmethod
    def empty(n, device="cuda", with_q=True):
        f = dict(dtype=torch.float64, device=device)
        return State(torch.empty(3, n, **f), torch.empty(3, n, **f), torch.empty(n, **f), torch.empty(n, **f),
                     torch.empty(n, dtype=torch.int32, device=device),
                     torch.empty(4, n, **f) if with_q else None)

    @staticmethod
    def from_arrays(d, device="cuda", with_q=True):
        """From a dict of numpy arrays (x[3][n], v, r, m, id, q) as drawn by ``inputs.draw``."""
        t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        return State(t(d["x"]), t(d["v"]), t(d["r"]), t(d["m"]), t(d["id"], torch.int32),
                     t(d["q"]) if with_q and "q" in d else None)

    def copy_(self, other):
        for a in ("x", "v", "r", "m", "id"):
            getattr(self, a).copy_(getattr(other, a))
        if self.q is not None and other.q is not None:
            self.q.copy_(other.q)
        return self

    def struct(self):
        return PcParticles(self.n, _ptr(self.id), _ptr(self.x), _ptr(self.v), _ptr(self.r), _ptr(self.m),
                           _ptr(self.q))

    def numpy(self):
        out = dict(x=self.x.cpu().numpy(), v=self.v.cpu().numpy(), r=self.r.cpu().numpy(), m=self.m.cpu().numpy(),
                   id=self.id.cpu().numpy())
        if self.q is not None:
            out["q"] = self.q.cpu().numpy()
        return out


class StateF32:
    """FP32 cell-relative device particle state of the mixed-precision path."""

    def __init__(self, id, cell, o, v, r, m, q=None):
        self.id, self.cell, self.o, self.v, self.r, self.m, self.q = id, cell, o, v, r, m, q
        n = r.shape[0]
        for name, t, shape, dt in (("id", id, (n,), torch.int32), ("cell", cell, (n,), torch.int32),
                                   ("o", o, (3, n), torch.float32), ("v", v, (3, n), torch.float32),
                                   ("r", r, (n,), torch.float32), ("m", m, (n,), torch.float32)):
            if tuple(t.shape) != shape or t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
                raise ValueError("StateF32.%s must be a contiguous CUDA %s tensor of shape %s" % (name, dt, shape))
        if q is not None:
            _dev(q, "StateF32.q", torch.float32, (4, n))
        if len({t.device for t in (id, cell, o, v, r, m, q) if t is not None}) != 1:
            raise ValueError("StateF32 tensors must be on one CUDA device")

    @property
    def n(self):
        return self.r.shape[0]

    @property
    def device(self):
        return self.r.device.index

    @staticmethod
    def empty(n, device="cuda", with_q=True):
        f = dict(dtype=torch.float32, device=device)
        i = dict(dtype=torch.int32, device=device)
        return StateF32(torch.empty(n, **i), torch.empty(n, **i), torch.empty(3, n, **f), torch.empty(3, n, **f),
                        torch.empty(n, **f), torch.empty(n, **f), torch.empty(4, n, **f) if with_q else None)

    @staticmethod
    def from_arrays(d, device="cuda", with_q=True):
        """From numpy arrays id, cell, o[3][n], v[3][n], r, m, q[4][n]."""
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        return StateF32(t(d["id"], torch.int32), t(d["cell"], torch.int32), t(d["o"], torch.float32),
                        t(d["v"], torch.float32), t(d["r"], torch.float32), t(d["m"], torch.float32),
                        t(d["q"], torch.float32) if with_q and "q" in d else None)

    def struct(self):
        return PcParticlesF32(self.n, _ptr(self.id), _ptr(self.cell), _ptr(self.o), _ptr(self.v), _ptr(self.r),
                              _ptr(self.m), _ptr(self.q))

    def numpy(self):
        out = dict(id=self.id.cpu().numpy(), cell=self.cell.cpu().numpy(), o=self.o.cpu().numpy(),
                   v=self.v.cpu().numpy(), r=self.r.cpu().numpy(), m=self.m.cpu().numpy())
        if self.q is not None:
            out["q"] = self.q.cpu().numpy()
        return out


class Context:
    """One operator instance (pc_init). All calls run on ``stream`` (default: torch's current)."""

    def __init__(self, n_max, ne, degree, sigma, restitution, reach_hint, cutoff_sigmas=3.0, cand_cap=16,
                 stream=None, cutoff="box", amp=0.0):
        lib = library()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.cfg = PcConfig(int(n_max), int(ne), int(degree), float(sigma), float(cutoff_sigmas),
                            0 if cutoff == "box" else 1, float(restitution), float(reach_hint), int(cand_cap),
                            c_p(stream.cuda_stream), float(amp))
        h = c_p()
        st = lib.pc_init(ctypes.byref(h), ctypes.byref(self.cfg))
        if st != PC_OK:
            raise PcError(st, "pc_init failed")
        self._h = h
        self.n1 = degree + 1
        self.ne = ne
        self.device = torch.cuda.current_device()

    def _check(self, st):
        if st != PC_OK:
            raise PcError(st, library().pc_last_error(self._h).decode())

    def _on(self, *states):
        """Structs of the states, after checking that they live on the context's device."""
        for s in states:
            if s.device != self.device:
                raise ValueError("particle state on cuda:%s, context on cuda:%d" % (s.device, self.device))
        return [s.struct() for s in states]

    def _t(self, t, name, dtype, shape):
        return _dev(t, name, dtype, shape, self.device)

    def _field_shape(self, nvar=4):
        return (self.ne ** 3, nvar, self.n1 ** 3)

    def collide(self, src, dst, dt):
        """One collision step src -> dst (distinct states, same n)."""
        a, b = self._on(src, dst)
        self._check(library().pc_collide(self._h, ctypes.byref(a), ctypes.byref(b), float(dt)))

    def project(self, state, field):
        """field[ne^3, 4, n1^3] (float64, CUDA) <- projection of state.q at state.x."""
        self._t(field, "field", torch.float64, self._field_shape())
        (s,) = self._on(state)
        self._check(library().pc_project(self._h, ctypes.byref(s), _ptr(field)))

    def set_pair_policy(self, policy):
        """Pair selection of collide / collide_rot: "earliest" or "sfc_first"."""
        code = {"earliest": 0, "sfc_first": 1}[policy]
        self._check(library().pc_set_pair_policy(self._h, code))

    def collide_rot(self, src, dst, w_in, w_out, mu, dt):
        """One step with Coulomb friction mu and rotation: dst (cell-sorted) and w_out
        (angular velocities [3][n] float64 in dst's order) from src and w_in (src's order)."""
        self._t(w_in, "w_in", torch.float64, (3, src.n))
        self._t(w_out, "w_out", torch.float64, (3, src.n))
        a, b = self._on(src, dst)
        self._check(library().pc_collide_rot(self._h, ctypes.byref(a), ctypes.byref(b), _ptr(w_in), _ptr(w_out),
                                             float(mu), float(dt)))

    def eval_field(self, state, field, out=None):
        """The DG polynomial of field [ne^3, nvar, n1^3] (float64, CUDA) at the particles:
        out [nvar, n] in state's order."""
        self._t(field, "field", torch.float64, self._field_shape(None))
        nvar = field.shape[1]
        if out is None:
            out = torch.empty(nvar, state.n, dtype=torch.float64, device=field.device)
        self._t(out, "out", torch.float64, (nvar, state.n))
        (s,) = self._on(state)
        self._check(library().pc_eval_field(self._h, ctypes.byref(s), _ptr(field), int(nvar), _ptr(out)))
        return out

    def drag_sources(self, state, fluid, mu_f, q=None):
        """Drag sources q [4, n] = (-F, -F.v) from fluid [4, n] = (rho, u) at the particles."""
        self._t(fluid, "fluid", torch.float64, (4, state.n))
        if q is None:
            q = torch.empty(4, state.n, dtype=torch.float64, device=fluid.device)
        self._t(q, "q", torch.float64, (4, state.n))
        (s,) = self._on(state)
        self._check(library().pc_drag_sources(self._h, ctypes.byref(s), _ptr(fluid), float(mu_f), _ptr(q)))
        return q

    def project_idw(self, state, field):
        """field <- the linear corner-node (IDW) deposition of state.q at state.x."""
        self._t(field, "field", torch.float64, self._field_shape())
        (s,) = self._on(state)
        self._check(library().pc_project_idw(self._h, ctypes.byref(s), _ptr(field)))

    def project_dirac(self, state, field):
        """field <- the nearest-DOF (Dirac) deposition of state.q at state.x."""
        self._t(field, "field", torch.float64, self._field_shape())
        (s,) = self._on(state)
        self._check(library().pc_project_dirac(self._h, ctypes.byref(s), _ptr(field)))

    def partner_by_id(self, n_ids, out=None):
        """Device int32 [n_ids]: the partner id of each id in the last collide, or -1."""
        if out is None:
            out = torch.empty(n_ids, dtype=torch.int32, device="cuda:%d" % self.device)
        self._t(out, "out", torch.int32, (n_ids,))
        self._check(library().pc_pairs_to_partner(self._h, _ptr(out), int(n_ids)))
        return out

    def collide_replay(self, src, dst, partner, dt):
        """One step with a fixed pair set (partner: int32 [n], index in the same order)."""
        self._t(partner, "partner", torch.int32, (src.n,))
        a, b = self._on(src, dst)
        self._check(library().pc_collide_replay(self._h, ctypes.byref(a), ctypes.byref(b), _ptr(partner), float(dt)))

    def collide_adjoint(self, pre, partner, dt, gx_out, gv_out, gx_in, gv_in):
        self._t(partner, "partner", torch.int32, (pre.n,))
        for name, g in (("gx_out", gx_out), ("gv_out", gv_out), ("gx_in", gx_in), ("gv_in", gv_in)):
            self._t(g, name, torch.float64, (3, pre.n))
        (a,) = self._on(pre)
        self._check(library().pc_collide_adjoint(self._h, ctypes.byref(a), _ptr(partner), float(dt), _ptr(gx_out),
                                                 _ptr(gv_out), _ptr(gx_in), _ptr(gv_in)))

    def project_adjoint(self, state, G, gq, gx):
        self._t(G, "G", torch.float64, self._field_shape())
        self._t(gq, "gq", torch.float64, (4, state.n))
        self._t(gx, "gx", torch.float64, (3, state.n))
        (a,) = self._on(state)
        self._check(library().pc_project_adjoint(self._h, ctypes.byref(a), _ptr(G), _ptr(gq), _ptr(gx)))

    @property
    def cells_per_side(self):
        return int(library().pc_cells_per_side(self._h))

    def quantize(self, src, dst):
        """FP64 State -> FP32 cell-relative StateF32 (same order)."""
        a, b = self._on(src, dst)
        self._check(library().pc_quantize(self._h, ctypes.byref(a), ctypes.byref(b)))

    def collide_f32(self, src, dst, dt):
        a, b = self._on(src, dst)
        self._check(library().pc_collide_f32(self._h, ctypes.byref(a), ctypes.byref(b), float(dt)))

    def collide_replay_f32(self, src, dst, partner, dt):
        """One mixed step with a fixed pair set (partner: int32 [n], index in the same order)."""
        self._t(partner, "partner", torch.int32, (src.n,))
        a, b = self._on(src, dst)
        self._check(library().pc_collide_replay_f32(self._h, ctypes.byref(a), ctypes.byref(b), _ptr(partner),
                                                    float(dt)))

    def collide_adjoint_f32(self, pre, partner, dt, gx_out, gv_out, gx_in, gv_in):
        self._t(partner, "partner", torch.int32, (pre.n,))
        for name, g in (("gx_out", gx_out), ("gv_out", gv_out), ("gx_in", gx_in), ("gv_in", gv_in)):
            self._t(g, name, torch.float32, (3, pre.n))
        (a,) = self._on(pre)
        self._check(library().pc_collide_adjoint_f32(self._h, ctypes.byref(a), _ptr(partner), float(dt),
                                                     _ptr(gx_out), _ptr(gv_out), _ptr(gx_in), _ptr(gv_in)))

    def project_adjoint_f32(self, state, G, gq, gx):
        self._t(G, "G", torch.float32, self._field_shape())
        self._t(gq, "gq", torch.float32, (4, state.n))
        self._t(gx, "gx", torch.float32, (3, state.n))
        (a,) = self._on(state)
        self._check(library().pc_project_adjoint_f32(self._h, ctypes.byref(a), _ptr(G), _ptr(gq), _ptr(gx)))

    def project_f32(self, state, field, tc="f16"):
        """FP32 field[ne^3, 4, n1^3] <- tensor-core projection (tc = "f16" or "bf16")."""
        self._t(field, "field", torch.float32, self._field_shape())
        (s,) = self._on(state)
        t = PC_TC_BF16 if tc == "bf16" else PC_TC_F16
        self._check(library().pc_project_f32(self._h, ctypes.byref(s), _ptr(field), t))

    def project_curved_f32(self, state, field):
        """FP32 field <- projection on the curved mesh (context made with cutoff="sphere", amp > 0)."""
        self._t(field, "field", torch.float32, self._field_shape())
        (s,) = self._on(state)
        self._check(library().pc_project_curved_f32(self._h, ctypes.byref(s), _ptr(field)))

    def new_field_f32(self):
        return torch.empty(self._field_shape(), dtype=torch.float32, device="cuda:%d" % self.device)

    def new_field(self):
        return torch.empty(self._field_shape(), dtype=torch.float64, device="cuda:%d" % self.device)

    def pairs(self):
        """Pairs of the last collide: (ids[k, 2] smaller first, t[k]) sorted by the smaller id."""
        n = c_i64()
        self._check(library().pc_get_pairs(self._h, c_p(0), c_p(0), 0, ctypes.byref(n)))
        ids = np.zeros((n.value, 2), np.int32)
        t = np.zeros(n.value)
        self._check(library().pc_get_pairs(self._h, ids.ctypes.data_as(c_p), t.ctypes.data_as(c_p), n.value,
                                           ctypes.byref(n)))
        return ids, t

    def stats(self):
        s = PcStats()
        st = library().pc_get_stats(self._h, ctypes.byref(s))
        d = {k: getattr(s, k) for k, _ in PcStats._fields_}
        d["status"] = st
        return d

    def set_timing(self, on=True):
        self._check(library().pc_set_timing(self._h, 1 if on else 0))

    def timing(self):
        """{phase: (ms summed, instances)} since the previous call (waits for the stream)."""
        ms = np.zeros(len(PHASES))
        cnt = np.zeros(len(PHASES), np.int64)
        self._check(library().pc_get_timing(self._h, ms.ctypes.data_as(c_p), cnt.ctypes.data_as(c_p)))
        return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}

    def sync(self):
        self._check(library().pc_sync(self._h))

    def close(self):
        if getattr(self, "_h", None):
            library().pc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_SCRATCH_BYTES = 32 << 20


def project_noalloc(state, field, ne, degree, sigma, cutoff_sigmas=3.0, stream=None):
    """pc_project_noalloc: the projection without a context and without any device
    allocation, for callers that may not allocate (its scratch is a fixed 32 MiB
    device array inside the library). Calls that overlap on the GPU race."""
    if stream is None:
        stream = torch.cuda.current_stream()
    cfg = PcConfig(0, int(ne), int(degree), float(sigma), float(cutoff_sigmas), 0, 0.0, 0.0, 0,
                   c_p(stream.cuda_stream), 0.0)
    _dev(field, "field", torch.float64, (ne ** 3, 4, (degree + 1) ** 3), state.device)
    s = state.struct()
    msg = ctypes.create_string_buffer(256)
    st = library().pc_project_noalloc(ctypes.byref(cfg), ctypes.byref(s), _ptr(field), msg, 256)
    if st != PC_OK:
        raise PcError(st, msg.value.decode())


def reach_of(r, v, dt, margin=1.05):
    """2 r_max + 2 v_max dt with a margin: a good reach_hint for a workload."""
    r = np.asarray(r)
    v = np.asarray(v)
    return margin * (2 * float(r.max()) + 2 * float(np.sqrt((v * v).sum(axis=0)).max()) * dt)
