"""The at-any-size property checks used on runs too large for the oracle:
they accept a correct result and reject each kind of broken one."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2405_11658_gb300 import synth as S
from tests.props import check_properties, rowsum


def cliques():
    r, k = 10, 5
    g = S.ring_of_cliques(r, k)
    memb = np.arange(r * k) // k
    q = k * (k - 1) / (k * (k - 1) + 2) - 1 / r     # Eq. 1 on the clique partition
    return g, memb, q, r, k


def test_accepts_the_clique_partition():
    (off, idx, w), memb, q, _, _ = cliques()
    inside = int(sum(w[e] for i in range(len(off) - 1) for e in range(off[i], off[i + 1]) if memb[idx[e]] == memb[i]))
    two_m = int(w.sum())
    sig = np.bincount(memb, weights=rowsum(off, w)).astype(np.int64)
    q_exact = float(two_m * inside - int((sig * sig).sum())) / (float(two_m) * float(two_m) * 1.0)
    assert abs(q_exact - q) < 1e-12
    check_properties(off, idx, w, memb, q_exact, Sigma=np.concatenate([sig, np.zeros(len(off) - 1 - len(sig), np.int64)]))


def test_rejects_broken_results():
    (off, idx, w), memb, _, r, k = cliques()
    two_m = int(w.sum())
    sig = np.bincount(memb, weights=rowsum(off, w)).astype(np.int64)
    inside = two_m - 2 * r                            # every edge but the r ring links
    q = float(two_m * inside - int((sig * sig).sum())) / (float(two_m) * float(two_m) * 1.0)
    with pytest.raises(AssertionError):               # wrong modularity
        check_properties(off, idx, w, memb, q + 1e-9)
    bad = memb.copy()
    bad[bad == 2] = 0                                 # cliques 0 and 2 are not adjacent: disconnected
    bad = np.unique(bad, return_inverse=True)[1]
    sig2 = np.bincount(bad, weights=rowsum(off, w)).astype(np.int64)
    inside2 = inside
    q2 = float(two_m * inside2 - int((sig2 * sig2).sum())) / (float(two_m) * float(two_m) * 1.0)
    with pytest.raises(AssertionError):
        check_properties(off, idx, w, bad, q2)
    swapped = memb.copy()                             # labels not in order of smallest member
    swapped[memb == 0], swapped[memb == 1] = 1, 0
    with pytest.raises(AssertionError):
        check_properties(off, idx, w, swapped, q)
    with pytest.raises(AssertionError):               # community totals off by one
        Sg = np.zeros(len(off) - 1, np.int64)
        Sg[:len(sig)] = sig
        Sg[3] += 1
        check_properties(off, idx, w, memb, q, Sigma=Sg)
