"""Helpers shared by the GPU tests: oracle comparisons keyed by particle id."""
import numpy as np

import oracle


def by_id(d):
    """Reorder every per-particle array of a state dict into id order."""
    o = np.argsort(d["id"], kind="stable")
    out = {}
    for k, a in d.items():
        out[k] = a[..., o] if isinstance(a, np.ndarray) and a.shape[-1] == len(o) else a
    return out


def oracle_pairs(partner, tc, ids):
    """(ids[k,2], t[k]) of an oracle matching, sorted by the smaller id."""
    i = np.nonzero(partner >= 0)[0]
    j = partner[i]
    keep = ids[i] < ids[j]
    lo, hi, t = ids[i][keep], ids[j][keep], tc[i][keep]
    o = np.argsort(lo, kind="stable")
    return np.stack([lo[o], hi[o]], axis=1).astype(np.int32), t[o]


def field_err(F, R):
    """Normwise error per component: max |F - R| / max |R| over the nodes of that component."""
    F = np.asarray(F)
    R = np.asarray(R)
    num = np.abs(F - R).max(axis=(0, 2))
    den = np.abs(R).max(axis=(0, 2))
    return num / np.maximum(den, 1e-300)


def quad_weights(ne, degree):
    eta, w = np.polynomial.legendre.leggauss(degree + 1)
    h = 1.0 / ne
    return (np.einsum("k,j,i->kji", w, w, w) * (h / 2) ** 3).ravel()
