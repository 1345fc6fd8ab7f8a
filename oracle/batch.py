"""Batch application G^{t-1} -> G^t as a plain edge-set definition (numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper takes G^t as an input and excludes its construction from timing
(Sec. 5.1.5); it defines the batch as deletions E^{t-1} \\ E^t and insertions
E^t \\ E^{t-1} with positive weights, every update applied in both directions
(Sec. 3.5, Sec. 5.1.4).  Readings used here:
  * a deletion (u, v, w) removes the undirected edge {u, v}; w must equal its
    current weight, and the edge must exist;
  * deletions are applied before insertions;
  * an insertion of an edge that exists (or repeats in the batch) adds its
    weight (multi-edges merge);
  * self-loop updates are rejected.
"""
from __future__ import annotations

import numpy as np


def apply_batch(off, idx, w, dels, ins):
    off = np.asarray(off, np.int64)
    idx = np.asarray(idx, np.int64)
    w = np.asarray(w, np.int64)
    n = len(off) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    keys = src * n + idx
    wt = w.copy()
    if len(keys) > 1 and np.any(keys[1:] < keys[:-1]):
        o = np.argsort(keys, kind="stable")
        keys, wt = keys[o], wt[o]
    keep = np.ones(len(keys), bool)
    if dels is not None and len(dels[0]):
        ds, dd, dw = (np.asarray(x, np.int64) for x in dels)
        if np.any(ds == dd):
            raise ValueError("self-loop deletion")
        dk = np.concatenate([ds * n + dd, dd * n + ds])
        dwt = np.concatenate([dw, dw])
        if len(np.unique(dk)) != len(dk):
            raise ValueError("duplicate deletion")
        pos = np.searchsorted(keys, dk)
        ok = (pos < len(keys))
        ok[ok] &= keys[pos[ok]] == dk[ok]
        if not ok.all():
            raise ValueError("deletion of a missing edge")
        if np.any(wt[pos] != dwt):
            raise ValueError("deletion weight mismatch")
        keep[pos] = False
    keys, wt = keys[keep], wt[keep]
    if ins is not None and len(ins[0]):
        is_, id_, iw = (np.asarray(x, np.int64) for x in ins)
        if np.any(is_ == id_):
            raise ValueError("self-loop insertion")
        if np.any(iw <= 0):
            raise ValueError("non-positive insertion weight")
        keys = np.concatenate([keys, is_ * n + id_, id_ * n + is_])
        wt = np.concatenate([wt, iw, iw])
    order = np.argsort(keys, kind="stable")
    keys, wt = keys[order], wt[order]
    first = np.ones(len(keys), bool)
    first[1:] = keys[1:] != keys[:-1]
    starts = np.flatnonzero(first)
    uk = keys[starts]
    uw = np.add.reduceat(wt, starts) if len(starts) else np.zeros(0, np.int64)
    off2 = np.zeros(n + 1, np.int64)
    off2[1:] = np.cumsum(np.bincount(uk // n, minlength=n))
    return off2, (uk % n).astype(np.int32), uw.astype(np.int64)
