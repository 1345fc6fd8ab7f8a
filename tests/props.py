"""Properties of a Leiden result that hold at any graph size, for checking
runs too large for the oracle: canonical labels, modularity equal to an exact
integer recomputation of Eq. 1, community totals equal to the summed degrees,
and every community connected.  Nothing here calls the oracle or the library."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components


def rowsum(off, w):
    n = len(off) - 1
    rows = np.repeat(np.arange(n), np.diff(off))
    # float64 sums of integers far below 2^53 are exact
    return np.bincount(rows, weights=np.asarray(w, np.float64), minlength=n).astype(np.int64)


def check_properties(off, idx, w, memb, q, Sigma=None):
    n = len(off) - 1
    memb = np.asarray(memb, np.int64)
    # canonical labels: community IDs appear in increasing order of their
    # smallest member, densely numbered from 0
    first = np.full(memb.max() + 1, n, np.int64)
    np.minimum.at(first, memb, np.arange(n))
    assert np.all(np.diff(first) > 0) and first[0] == 0
    # Eq. 1 with exact integers (gamma = 1)
    rows = np.repeat(np.arange(n), np.diff(off))
    inside = int(np.asarray(w, np.int64)[memb[rows] == memb[idx]].sum())
    K = rowsum(off, w)
    sig = np.bincount(memb, weights=K.astype(np.float64), minlength=memb.max() + 1).astype(np.int64)
    two_m = int(K.sum())
    assert two_m * two_m < 2**62  # the int64 sum of squares below is exact
    sq = int((sig * sig).sum())
    assert q == float(two_m * inside - sq) / (float(two_m) * float(two_m) * 1.0)
    if Sigma is not None:
        expect = np.zeros(n, np.int64)
        expect[:len(sig)] = sig
        assert np.array_equal(np.asarray(Sigma), expect)
    # every community is connected: the graph restricted to intra-community
    # edges has exactly one component per community
    keep = memb[rows] == memb[idx]
    A = sp.csr_matrix((np.ones(int(keep.sum()), np.int8), (rows[keep], idx[keep])), shape=(n, n))
    ncomp, _ = connected_components(A, directed=False)
    assert ncomp == memb.max() + 1
