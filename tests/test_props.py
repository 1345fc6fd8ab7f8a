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


# ---------------------------------------------------------------------------
# The same checks computed with torch (tests/props_device.py), on CPU tensors.
# ---------------------------------------------------------------------------
torch = pytest.importorskip("torch")
from tests import props_device as PD  # noqa: E402


def _t(*arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)) for a in arrays]


def test_device_checks_accept_the_clique_partition():
    (off, idx, w), memb, _, _, _ = cliques()
    two_m = int(w.sum())
    sig = np.bincount(memb, weights=rowsum(off, w)).astype(np.int64)
    inside = two_m - 2 * 10
    q = float(two_m * inside - int((sig * sig).sum())) / (float(two_m) * float(two_m) * 1.0)
    Sg = np.zeros(len(off) - 1, np.int64)
    Sg[:len(sig)] = sig
    PD.check_properties(*_t(off, idx, w, memb), q, Sigma=torch.from_numpy(Sg))
    check_properties(off, idx, w, memb, q, Sigma=Sg)        # the host version agrees


def test_device_checks_reject_broken_results():
    (off, idx, w), memb, _, r, k = cliques()
    two_m = int(w.sum())
    sig = np.bincount(memb, weights=rowsum(off, w)).astype(np.int64)
    inside = two_m - 2 * r
    q = float(two_m * inside - int((sig * sig).sum())) / (float(two_m) * float(two_m) * 1.0)
    T = _t(off, idx, w)
    with pytest.raises(AssertionError):               # wrong modularity
        PD.check_properties(*T, torch.from_numpy(memb), q + 1e-9)
    bad = memb.copy()
    bad[bad == 2] = 0                                 # cliques 0 and 2 are not adjacent: disconnected
    bad = np.unique(bad, return_inverse=True)[1]
    sig2 = np.bincount(bad, weights=rowsum(off, w)).astype(np.int64)
    q2 = float(two_m * inside - int((sig2 * sig2).sum())) / (float(two_m) * float(two_m) * 1.0)
    with pytest.raises(AssertionError, match="not connected"):
        PD.check_properties(*T, torch.from_numpy(bad), q2)
    swapped = memb.copy()                             # labels not in order of smallest member
    swapped[memb == 0], swapped[memb == 1] = 1, 0
    with pytest.raises(AssertionError):
        PD.check_properties(*T, torch.from_numpy(swapped), q)
    Sg = np.zeros(len(off) - 1, np.int64)
    Sg[:len(sig)] = sig
    Sg[3] += 1
    with pytest.raises(AssertionError):               # community totals off by one
        PD.check_properties(*T, torch.from_numpy(memb), q, Sigma=torch.from_numpy(Sg))


def test_exact_sum_of_squares_is_exact_beyond_int64():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 2**47, size=5000, dtype=np.int64)
    assert PD.exact_sum_of_squares(torch.from_numpy(x)) == sum(int(v) * int(v) for v in x)


def test_components_match_scipy():
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    off, idx, _ = S.kmer(4000, 16, 1.2, seed=3)
    rows = np.repeat(np.arange(4000), np.diff(off))
    lab = PD.components_within(4000, torch.from_numpy(rows), torch.from_numpy(idx.astype(np.int64))).numpy()
    ncomp, ref = connected_components(sp.csr_matrix((np.ones(len(idx)), (rows, idx)), shape=(4000, 4000)))
    # same partition into components, each labelled by its smallest vertex
    assert len(np.unique(lab)) == ncomp
    assert np.array_equal(lab, np.array([np.flatnonzero(ref == ref[v])[0] for v in range(4000)]))
