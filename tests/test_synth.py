"""The seeded input generators: the CSR builder against a plain dictionary
construction, and the shape of each generated graph (symmetric, sorted rows,
no self-loops or duplicate entries, positive weights)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2405_11658_gb300 import synth as S


def dict_csr(n, u, v, w):
    """First weight seen per undirected pair, self-loops dropped, both
    directions, rows sorted by neighbour."""
    first = {}
    for a, b, x in zip(u, v, w):
        if a != b:
            first.setdefault((min(a, b), max(a, b)), x)
    rows = [[] for _ in range(n)]
    for (a, b), x in first.items():
        rows[a].append((b, x))
        rows[b].append((a, x))
    off = np.zeros(n + 1, np.int64)
    idx, wt = [], []
    for i in range(n):
        for j, x in sorted(rows[i]):
            idx.append(j)
            wt.append(x)
        off[i + 1] = len(idx)
    return off, np.asarray(idx, np.int32), np.asarray(wt, np.int32)


@pytest.mark.parametrize("wkind", ["none", "equal", "small", "large"])
@pytest.mark.parametrize("seed", range(4))
def test_edges_to_csr_matches_a_dictionary_construction(wkind, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    m = int(rng.integers(0, 200))
    u = rng.integers(0, n, m)
    v = rng.integers(0, n, m)
    w = {"none": None, "equal": np.full(m, 3), "small": rng.integers(1, 5, m),
         "large": rng.integers(1, 1000, m)}[wkind]
    got = S.edges_to_csr(n, u, v, w)
    want = dict_csr(n, u.tolist(), v.tolist(), [1] * m if w is None else w.tolist())
    for a, b in zip(got, want):
        assert a.dtype == b.dtype and np.array_equal(a, b)


def valid_csr(off, idx, w):
    n = len(off) - 1
    assert off[0] == 0 and np.all(np.diff(off) >= 0) and off[-1] == len(idx) == len(w)
    rows = np.repeat(np.arange(n), np.diff(off))
    assert np.all(rows != idx) and np.all(w > 0)
    key = rows * n + idx
    assert np.all(np.diff(key) > 0)                      # sorted rows, no duplicates
    rkey = idx.astype(np.int64) * n + rows               # the transpose holds the same entries
    order = np.argsort(rkey)
    assert np.array_equal(rkey[order], key) and np.array_equal(w[order], w)


@pytest.mark.parametrize("make", [
    lambda: S.planted_partition(500, 5, 0.05, 0.002, 1), lambda: S.rmat(10, 8, seed=2),
    lambda: S.chung_lu(2000, 8000, 2.1, 1, 4, seed=3), lambda: S.grid(30, 0.05, 0.01, seed=4),
    lambda: S.kmer(3000, 64, 2.1, seed=5), lambda: S.erdos_renyi(60, 0.1, 6, wmax=9),
    lambda: S.ring_of_cliques(6, 4)])
def test_generated_graphs_are_valid_symmetric_csr(make):
    valid_csr(*make())


# ---------------------------------------------------------------------------
# The device generators (torch), run here on the CPU device.
# ---------------------------------------------------------------------------
torch = pytest.importorskip("torch")
from paper_2405_11658_gb300 import synth_device as D  # noqa: E402


@pytest.mark.parametrize("seed", range(3))
def test_device_csr_builder_matches_the_host_builder(seed):
    (off, idx, w), (keys, wk) = D.chung_lu(3000, 12000, 2.1, 1, 4, seed=seed, device="cpu")
    k = keys.numpy()
    assert len(k) == 12000 and np.all(np.diff(k) > 0)      # exactly m distinct edges, sorted
    assert np.all(k // 3000 < k % 3000)                     # a < b: no self-loops
    want = S.edges_to_csr(3000, k // 3000, k % 3000, wk.numpy())
    for a, b in zip((off, idx, w), want):
        assert np.array_equal(a.numpy(), b)
    valid_csr(off.numpy(), idx.numpy(), w.numpy())
    assert wk.min() >= 1 and wk.max() <= 4


def test_device_chung_lu_degrees_follow_the_power_law():
    n, m = 200_000, 2_000_000
    (off, _, _), _ = D.chung_lu(n, m, 2.1, 1, 4, seed=1, device="cpu")
    deg = np.diff(off.numpy())
    # expected degree ~ (i + 10)^(-1/(beta-1)): the log-log slope over the
    # uncapped middle of the ID range is close to -1/1.1
    i = np.array([1000, 3000, 10000, 30000, 100000])
    d = np.array([deg[k - 100:k + 100].mean() for k in i])
    slope = np.polyfit(np.log(i + 10.0), np.log(d), 1)[0]
    assert -1.0 < slope < -0.8, slope
    assert deg.max() <= int(np.sqrt(2 * m)) * 1.2            # the cap holds (up to sampling noise)


@pytest.mark.parametrize("size", [1, 10, 1000])
def test_device_random_batch_is_valid(size):
    n = 5000
    (off, idx, w), (keys, wk) = D.chung_lu(n, 20000, 2.1, 1, 4, seed=4, device="cpu")
    dels, ins = D.random_batch(n, keys, wk, size, seed=9)
    ni = int(round(0.8 * size))
    assert len(ins[0]) == ni and len(dels[0]) == size - ni
    k = keys.numpy()
    dk = dels[0].numpy().astype(np.int64) * n + dels[1].numpy()
    ik = ins[0].numpy().astype(np.int64) * n + ins[1].numpy()
    assert np.all(dels[0].numpy() < dels[1].numpy()) and np.all(ins[0].numpy() < ins[1].numpy())
    assert len(np.unique(dk)) == len(dk) and np.all(np.isin(dk, k))        # distinct existing edges
    assert np.array_equal(dels[2].numpy(), wk.numpy()[np.searchsorted(k, dk)])  # with their weights
    assert len(np.unique(ik)) == len(ik) and not np.any(np.isin(ik, k))    # distinct non-edges
    assert np.all(ins[2].numpy() == 1)


def test_temporal_stream_and_split():
    n, ne = 5000, 60000
    s, d = S.temporal_stream(n, ne, seed=2)
    assert len(s) == len(d) == ne and s.dtype == np.int32
    assert np.all(s != d) and s.min() >= 0 and s.max() < n and d.max() < n
    key = np.minimum(s, d).astype(np.int64) * n + np.maximum(s, d)
    distinct = len(np.unique(key))
    assert 0.35 < 1 - distinct / ne < 0.75                 # many repeated pairs, as in |E_T| vs |E|
    s2, d2 = S.temporal_stream(n, ne, seed=2)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)   # seeded
    g, rest = S.temporal_split(n, s, d, 0.9)
    valid_csr(*g)
    assert len(rest[0]) == ne - 54000
    assert int(g[2].sum()) == 2 * 54000                   # repeats merged by adding unit weights
    bs = S.temporal_batches(rest, 100, 7)
    assert len(bs) == 7 and np.array_equal(bs[3][0], rest[0][300:400]) and np.all(bs[0][2] == 1)
    assert len(S.temporal_batches(rest, 5000, 3)) == 1    # only whole batches
