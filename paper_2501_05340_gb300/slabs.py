"""Slab decomposition of the collision step over ranks (host orchestration).

The periodic unit cube is cut into `world` slabs along x; rank k owns the particles
with x in [k / world, (k + 1) / world). One collision step of the paper's operator
(Sec. 3.3 detection, Sec. 4.3 one collision per particle; the paper shares a halo
region between MPI ranks, Sec. 4.1, 4.3) then runs as:

1. ghost import: every rank sends the particles it owns within `reach` of a slab face
   (reach = 2 r_max + 2 v_max dt, the farthest a colliding partner can start) to the
   neighbour across that face, so each owned particle has all its possible partners
   locally, as owned particles or ghosts;
2. contact search on owned + ghost particles (a local operation);
3. matching rounds: each owned free particle picks its earliest free candidate (ties
   to the smaller id); the picks of owned particles that are ghosts elsewhere go to
   the neighbours; mutual picks become pairs on both sides; the new matched flags go
   to the neighbours; an allreduce of "any pick left" ends the rounds. These are the
   rounds of mutually earliest picks of the single-domain step, so the pairs are the
   same global greedy matching;
4. response and advance of the owned particles (a local operation, computed from
   each particle's own side, so both owners of a pair agree bit for bit);
5. migration: particles whose new x left the slab go to the owning neighbour.

This module only moves data between ranks (torch.distributed point-to-point and
allreduce, any backend); the arithmetic of the step is passed in as `LocalOps`, so
the same orchestration serves any implementation of the local operations. Slabs
must be wider than the reach (checked), so a particle is a ghost of at most the two
neighbouring slabs and migrates at most one slab per step.
"""
from dataclasses import dataclass
from typing import Callable

import numpy as np
import torch

FIELDS = ("x", "v", "r", "m", "id")


@dataclass
class LocalOps:
    """The local operations of a step on a rank's particles (owned first, then ghosts).

    candidates(x, v, r, dt) -> (i, j, t): candidate pairs between local particles
        (local indices, i < j) with their contact times.
    best_free(cand, free, ids) -> best: for every local particle the local index
        of its earliest free candidate partner (ties to the smaller id), or -1;
        `cand` is (i, j, t) and `free` a boolean mask over local particles.
    respond(x, v, m, partner, tc, e, dt) -> (x', v'): response of the given pairs
        (partner[i] local index or -1, tc[i] contact time) and advance of every local
        particle, wrapped into [0, 1).
    """
    candidates: Callable
    best_free: Callable
    respond: Callable


def slab_of(x0, world):
    """Owning rank of each x coordinate in [0, 1)."""
    k = np.floor(np.asarray(x0) * world).astype(np.int64)
    return np.clip(k, 0, world - 1)


class Slabs:
    """Ownership and neighbour exchange on a process group (rank, world)."""

    def __init__(self, dist, group=None):
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.left = (self.rank - 1) % self.world
        self.right = (self.rank + 1) % self.world
        self.lo = self.rank / self.world
        self.hi = (self.rank + 1) / self.world

    # ---- communication -------------------------------------------------------
    def _sendrecv(self, send: np.ndarray, dst: int, src: int) -> np.ndarray:
        """Send a 1-D float64 or int64 array to dst and receive one of the same type
        from src (sizes first)."""
        d = self.dist
        n_out = torch.tensor([send.size], dtype=torch.int64)
        n_in = torch.zeros(1, dtype=torch.int64)
        reqs = [d.isend(n_out, dst, group=self.group), d.irecv(n_in, src, group=self.group)]
        for q in reqs:
            q.wait()
        out = torch.from_numpy(np.ascontiguousarray(send))
        inc = torch.empty(int(n_in.item()), dtype=out.dtype)
        reqs = []
        if out.numel():
            reqs.append(d.isend(out, dst, group=self.group))
        if inc.numel():
            reqs.append(d.irecv(inc, src, group=self.group))
        for q in reqs:
            q.wait()
        return inc.numpy()

    def exchange(self, arrays: dict, to_left: np.ndarray, to_right: np.ndarray) -> dict:
        """Send the selected entries of every per-particle array to the neighbours and
        return what arrives from them (from the right neighbour first, then the left).
        With two ranks both neighbours are the same rank; the two messages stay apart."""
        got = {}
        for key, a in arrays.items():
            a = np.asarray(a)
            lead = a.shape[:-1]
            npdt = np.float64 if a.dtype == np.float64 else np.int64
            parts = []
            for sel, dst, src in ((to_left, self.left, self.right), (to_right, self.right, self.left)):
                flat = a[..., sel].astype(npdt).reshape(-1)
                r = self._sendrecv(flat, dst, src)
                parts.append(r.reshape(lead + (-1,)))
            got[key] = np.concatenate(parts, axis=-1).astype(a.dtype)
        return got

    def allreduce_max(self, value: float) -> float:
        t = torch.tensor([float(value)], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t.item())

    def allreduce_any(self, flag: bool) -> bool:
        t = torch.tensor([1 if flag else 0], dtype=torch.int64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return bool(t.item())

    # ---- geometry -------------------------------------------------------------
    def face_masks(self, x0: np.ndarray, reach: float):
        """Owned particles within reach of the lower and of the upper slab face
        (periodic distances along x)."""
        d_lo = np.mod(x0 - self.lo, 1.0)
        d_hi = np.mod(self.hi - x0, 1.0)
        return d_lo <= reach, d_hi <= reach

    # ---- one step -----------------------------------------------------------
    def collide_step(self, own: dict, e: float, dt: float, ops: LocalOps):
        """One collision step of the owned particles `own` (dict of x[3][n], v[3][n],
        r[n], m[n], id[n]). Returns (new owned dict after migration, pairs), pairs the
        (smaller id, larger id, t) of the collisions whose smaller id this rank owned
        at the start of the step."""
        n_own = own["r"].shape[0]
        rmax = self.allreduce_max(own["r"].max() if n_own else 0.0)
        vmax = self.allreduce_max(np.sqrt((own["v"] ** 2).sum(axis=0)).max() if n_own else 0.0)
        reach = (2.0 * rmax + 2.0 * vmax * dt) * (1.0 + 1e-9) + 1e-12
        if not reach < 1.0 / self.world:
            raise ValueError("slabs of width %g are not wider than the reach %g" % (1.0 / self.world, reach))
        # 1. ghosts (with two ranks both faces lead to the one neighbour: one message)
        to_left, to_right = self.face_masks(own["x"][0], reach)
        if self.world == 2:
            to_left, to_right = to_left | to_right, np.zeros_like(to_left)
        ghosts = self.exchange({k: own[k] for k in FIELDS}, to_left, to_right)
        loc = {k: np.concatenate([own[k], ghosts[k]], axis=-1) for k in FIELDS}
        nl = loc["r"].shape[0]
        ids = loc["id"]
        idx_of = {int(i): k for k, i in enumerate(ids)}
        # 2. candidates on owned + ghost particles
        ci, cj, ct = ops.candidates(loc["x"], loc["v"], loc["r"], dt)
        t_of = {(int(a), int(b)): float(t) for a, b, t in zip(ci, cj, ct)}
        # 3. matching rounds
        free = np.ones(nl, bool)
        partner = np.full(nl, -1, np.int64)
        tc = np.zeros(nl)
        cand = (ci, cj, ct)
        while True:
            best = ops.best_free(cand, free, ids)
            # the picks of the ghosts come from their owners (same masks, same order)
            got = self.exchange({"best_id": np.where(best[:n_own] >= 0, ids[np.maximum(best[:n_own], 0)], -1)},
                                to_left, to_right)
            best_ext = best.copy()
            best_ext[n_own:] = [idx_of.get(int(b), -1) if b >= 0 else -1 for b in got["best_id"]]
            # mutual picks: a pair with an owned member is committed on both sides
            mutual = np.nonzero((best_ext >= 0) & (best_ext[np.maximum(best_ext, 0)] == np.arange(nl)))[0]
            for i in mutual:
                j = int(best_ext[i])
                if free[i] and free[j]:
                    partner[i], partner[j] = j, i
                    tc[i] = tc[j] = t_of[(min(i, j), max(i, j))]
            free = partner < 0
            # matched flags of the ghosts from their owners
            got = self.exchange({"free": free[:n_own].astype(np.int64)}, to_left, to_right)
            free[n_own:] = got["free"].astype(bool)
            left = ops.best_free(cand, free, ids)[:n_own]
            if not self.allreduce_any(bool((left >= 0).any())):
                break
        # 4. response of the owned particles (ghost results are dropped)
        x1, v1 = ops.respond(loc["x"], loc["v"], loc["m"], partner, tc, e, dt)
        pairs = [(int(ids[i]), int(ids[partner[i]]), float(tc[i])) for i in range(n_own)
                 if partner[i] >= 0 and ids[i] < ids[partner[i]]]
        new = {"x": x1[:, :n_own], "v": v1[:, :n_own], "r": own["r"], "m": own["m"], "id": own["id"]}
        # 5. migration
        dest = slab_of(new["x"][0], self.world)
        go_l = dest == self.left
        go_r = (dest == self.right) & ~go_l
        if self.world == 2:
            go_l = dest != self.rank
            go_r = np.zeros_like(go_l)
        arrived = self.exchange({k: new[k] for k in FIELDS}, go_l, go_r)
        stay = dest == self.rank
        out = {k: np.concatenate([new[k][..., stay], arrived[k]], axis=-1) for k in FIELDS}
        if not np.all(slab_of(out["x"][0], self.world) == self.rank):
            raise RuntimeError("a particle migrated by more than one slab")
        return out, pairs
