"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5.1.3-5.1.4).

This module holds input generators only -- none of the method's arithmetic --
so that the tests, the benchmark and the CPU oracle all see the same graphs.
Every generator is deterministic for a given seed (numpy PCG64), on any host.

The paper evaluates on SuiteSparse web / social / road / k-mer graphs and SNAP
temporal graphs (Tables 1-2); none is available here, so these generators
stand in for them:
  * planted partition     -- small graph with clear communities (correctness);
  * R-MAT (a,b,c,d)       -- social networks (com-LiveJournal / Orkut class);
  * Chung-Lu, beta = 2.1  -- web graphs (sk-2005 / it-2004 class);
  * 2D grid + shortcuts   -- road networks (asia_osm / europe_osm class);
  * k-mer-like paths      -- protein k-mer graphs (kmer_A2a / kmer_V1r class).
Random batch updates follow Sec. 5.1.4: 80% insertions between uniformly chosen
vertex pairs and 20% deletions of uniformly chosen existing edges, unit weight,
each undirected pair listed once (the library applies both directions).

All graphs are returned as a symmetric CSR ``(off int64[n+1], idx int32[nnz],
w int32[nnz])`` with sorted rows and no self-loops or duplicate entries.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def edges_to_csr(n: int, u, v, w=None):
    """Symmetric CSR from undirected pairs (u, v); duplicates merged by the
    first weight seen, self-loops dropped."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    if w is None:
        w = np.ones(len(u), np.int64)
    w = np.asarray(w, np.int64)
    keep = u != v
    u, v, w = u[keep], v[keep], w[keep]
    a, b = np.minimum(u, v), np.maximum(u, v)
    key = a * n + b
    if len(w) == 0 or np.all(w == w[0]):
        # every duplicate has the same weight: a plain sort deduplicates
        key = np.sort(key)
        if len(key):
            key = key[np.concatenate([[True], key[1:] != key[:-1]])]
        w = np.full(len(key), w[0] if len(w) else 1, np.int64)
    else:
        key, first = np.unique(key, return_index=True)
        w = w[first]
    a, b = key // n, key % n
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    wt = np.concatenate([w, w])
    ekey = src * n + dst                      # distinct: one per CSR entry
    if len(wt) and wt.min() >= 0 and wt.max() < 8 and n <= (1 << 30):
        # small weights travel in the low bits of the sort key
        packed = np.sort((ekey << 3) | wt)
        ekey, wt = packed >> 3, packed & 7
        src, dst = ekey // n, ekey % n
    else:
        order = np.argsort(ekey, kind="stable")
        src, dst, wt = src[order], dst[order], wt[order]
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(np.bincount(src, minlength=n))
    return off, dst.astype(np.int32), wt.astype(np.int32)


def undirected_pairs(off, idx, w=None):
    """Each undirected edge once as (u < v, w)."""
    off = np.asarray(off, np.int64)
    n = len(off) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    dst = np.asarray(idx, np.int64)
    m = src < dst
    ww = None if w is None else np.asarray(w)[m]
    return src[m], dst[m], ww


def planted_partition(n: int, k: int, p_in: float, p_out: float, seed: int):
    """k equal blocks; each intra-block pair with probability p_in, each
    inter-block pair with probability p_out; unit weights."""
    rng = _rng(seed)
    block = np.arange(n) * k // n
    starts = np.searchsorted(block, np.arange(k + 1))
    us, vs = [], []
    for a in range(k):
        for b in range(a, k):
            na, nb = starts[a + 1] - starts[a], starts[b + 1] - starts[b]
            npairs = na * (na - 1) // 2 if a == b else na * nb
            p = p_in if a == b else p_out
            cnt = rng.binomial(npairs, p)
            if cnt == 0:
                continue
            pick = rng.choice(npairs, size=cnt, replace=False)
            if a == b:
                # unrank pair index -> (x < y) inside the block
                y = np.floor((1 + np.sqrt(1 + 8 * pick.astype(np.float64))) / 2).astype(np.int64)
                y = np.where(y * (y - 1) // 2 > pick, y - 1, y)
                y = np.where((y + 1) * y // 2 <= pick, y + 1, y)
                x = pick - y * (y - 1) // 2
                us.append(starts[a] + x)
                vs.append(starts[a] + y)
            else:
                us.append(starts[a] + pick // nb)
                vs.append(starts[b] + pick % nb)
    if not us:
        return edges_to_csr(n, [], [])
    return edges_to_csr(n, np.concatenate(us), np.concatenate(vs))


def rmat(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, seed: int = 0):
    """R-MAT (Chakrabarti et al.) without noise: edge_factor * 2^scale draws,
    symmetrised, deduplicated, self-loops dropped, unit weights."""
    rng = _rng(seed)
    n = 1 << scale
    m = edge_factor * n
    u = np.zeros(m, np.int64)
    v = np.zeros(m, np.int64)
    ab, abc = a + b, a + b + c
    chunk = 1 << 24
    for s in range(0, m, chunk):
        e = min(m, s + chunk)
        uu = np.zeros(e - s, np.int64)
        vv = np.zeros(e - s, np.int64)
        for _ in range(scale):
            r = rng.random(e - s, dtype=np.float32)
            ubit = r >= ab
            vbit = ((r >= a) & (r < ab)) | (r >= abc)
            uu = (uu << 1) | ubit
            vv = (vv << 1) | vbit
        u[s:e], v[s:e] = uu, vv
    return edges_to_csr(n, u, v)


def chung_lu(n: int, m_target: int, beta: float = 2.1, wmin: int = 1, wmax: int = 4,
             seed: int = 0):
    """Chung-Lu by ball dropping: endpoint i with probability proportional to
    (i + i0)^(-1/(beta-1)), expected degree capped at sqrt(2 m); deduplicate,
    drop loops and resample until m_target undirected edges; integer weights
    uniform in [wmin, wmax]."""
    rng = _rng(seed)
    i0 = 10.0
    x = (np.arange(n, dtype=np.float64) + i0) ** (-1.0 / (beta - 1.0))
    deg = x * (2.0 * m_target / x.sum())
    deg = np.minimum(deg, np.sqrt(2.0 * m_target))
    cdf = np.cumsum(deg)
    cdf /= cdf[-1]
    have = np.zeros(0, np.int64)
    while len(have) < m_target:
        need = int((m_target - len(have)) * 1.1) + 16
        u = np.searchsorted(cdf, rng.random(need))
        v = np.searchsorted(cdf, rng.random(need))
        u, v = np.minimum(u, n - 1), np.minimum(v, n - 1)
        keep = u != v
        a, b = np.minimum(u[keep], v[keep]), np.maximum(u[keep], v[keep])
        have = np.unique(np.concatenate([have, a * n + b]))
    if len(have) > m_target:
        have = rng.permutation(have)[:m_target]
    w = rng.integers(wmin, wmax + 1, size=len(have))
    return edges_to_csr(n, have // n, have % n, w)


def grid(side: int, remove_frac: float = 0.05, shortcut_frac: float = 0.001, seed: int = 0):
    """side x side 4-neighbour lattice, remove_frac of its edges removed
    uniformly, plus shortcut_frac * |V| uniform long-range edges."""
    rng = _rng(seed)
    n = side * side
    ids = np.arange(n, dtype=np.int64).reshape(side, side)
    hu, hv = ids[:, :-1].ravel(), ids[:, 1:].ravel()
    vu, vv = ids[:-1, :].ravel(), ids[1:, :].ravel()
    u = np.concatenate([hu, vu])
    v = np.concatenate([hv, vv])
    keep = rng.random(len(u)) >= remove_frac
    u, v = u[keep], v[keep]
    ns = int(round(shortcut_frac * n))
    su = rng.integers(0, n, size=ns)
    sv = rng.integers(0, n, size=ns)
    return edges_to_csr(n, np.concatenate([u, su]), np.concatenate([v, sv]))


def kmer(n: int, mean_path: float = 64.0, target_degree: float = 2.1, seed: int = 0):
    """Random permutation of the vertices cut into paths of geometric length
    (mean mean_path), plus uniform extra edges until the mean degree reaches
    target_degree."""
    rng = _rng(seed)
    perm = rng.permutation(n).astype(np.int64)
    cut = rng.random(n - 1) < 1.0 / mean_path
    u, v = perm[:-1][~cut], perm[1:][~cut]
    extra = max(0, int(target_degree * n / 2) - len(u))
    eu = rng.integers(0, n, size=extra)
    ev = rng.integers(0, n, size=extra)
    return edges_to_csr(n, np.concatenate([u, eu]), np.concatenate([v, ev]))


def ring_of_cliques(r: int, k: int):
    """r cliques K_k joined in a ring by single edges (clique a's last vertex to
    clique a+1's first)."""
    us, vs = [], []
    for a in range(r):
        base = a * k
        for x in range(k):
            for y in range(x + 1, k):
                us.append(base + x)
                vs.append(base + y)
        us.append(base + k - 1)
        vs.append(((a + 1) % r) * k)
    return edges_to_csr(r * k, us, vs)


def erdos_renyi(n: int, p: float, seed: int, wmax: int = 1):
    rng = _rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    w = rng.integers(1, wmax + 1, size=int(keep.sum()))
    return edges_to_csr(n, iu[keep], ju[keep], w)


def random_batch(off, idx, w, size: int, seed: int, ins_frac: float = 0.8, weight: int = 1,
                 pairs=None):
    """A batch of ``size`` undirected updates: round(ins_frac*size) insertions
    between uniformly chosen vertex pairs (self-loops, existing edges and
    repeats resampled) and the rest deletions of distinct, uniformly chosen
    existing edges.  Returns (dels, ins), each (src, dst, w) int32 arrays.
    ``pairs`` may pass a precomputed ``undirected_pairs(off, idx, w)``."""
    rng = _rng(seed)
    off = np.asarray(off, np.int64)
    n = len(off) - 1
    eu, ev, ew = pairs if pairs is not None else undirected_pairs(off, idx, w)
    ni = int(round(ins_frac * size))
    nd = min(size - ni, len(eu))
    pick = rng.choice(len(eu), size=nd, replace=False) if nd else np.zeros(0, np.int64)
    dels = (eu[pick].astype(np.int32), ev[pick].astype(np.int32),
            np.asarray(ew)[pick].astype(np.int32))
    existing = eu * n + ev
    if len(existing) > 1 and not np.all(existing[1:] > existing[:-1]):
        existing = np.sort(existing)
    got = np.zeros(0, np.int64)
    while len(got) < ni and n > 1:
        need = (ni - len(got)) * 2 + 8
        a = rng.integers(0, n, size=need)
        b = rng.integers(0, n, size=need)
        keep = a != b
        a, b = np.minimum(a[keep], b[keep]), np.maximum(a[keep], b[keep])
        k = a * n + b
        pos = np.searchsorted(existing, k)
        pos = np.minimum(pos, max(len(existing) - 1, 0))
        new = existing[pos] != k if len(existing) else np.ones(len(k), bool)
        k = k[new]
        _, first = np.unique(k, return_index=True)
        k = k[np.sort(first)]
        k = k[~np.isin(k, got)]
        got = np.concatenate([got, k])[:ni]
    ins = ((got // n).astype(np.int32), (got % n).astype(np.int32),
           np.full(len(got), weight, np.int32))
    return dels, ins


def temporal_stream(n: int, n_events: int, comm_size: float = 200.0, p_within: float = 0.8,
                    p_repeat: float = 0.45, beta: float = 2.1, seed: int = 0):
    """A timestamped stream of n_events undirected interactions (src, dst), in
    time order, standing in for the SNAP temporal networks of Sec. 5.3 (Q&A
    and talk-page interactions: heavy-tailed activity, groups that mostly talk
    among themselves, many repeated pairs; |E_T| counts the repeats).

    Vertex activity follows the Chung-Lu weights (i + 10)^(-1/(beta-1)) over a
    random permutation of the IDs; vertices fall into groups of geometric size
    (mean comm_size).  Each event repeats a uniformly chosen earlier event with
    probability p_repeat; otherwise its source is drawn by activity and its
    target by activity, inside the source's group with probability p_within.
    Self-loops are redrawn.  Returns (src, dst) int32 arrays of n_events."""
    rng = _rng(seed)
    act = (np.arange(n, dtype=np.float64) + 10.0) ** (-1.0 / (beta - 1.0))
    act = act[rng.permutation(n)]
    # groups: consecutive runs of a random vertex order, geometric sizes
    order = rng.permutation(n)
    cuts = np.flatnonzero(rng.random(n) < 1.0 / comm_size)
    group = np.zeros(n, np.int64)
    group[order] = np.searchsorted(cuts, np.arange(n), side="right")
    ng = int(group.max()) + 1
    # per-group activity distribution: members sorted by group, prefix sums
    byg = np.argsort(group, kind="stable")
    gstart = np.searchsorted(group[byg], np.arange(ng + 1))
    gcum = np.cumsum(act[byg])
    cdf_all = np.cumsum(act)
    cdf_all /= cdf_all[-1]
    m = n_events
    # fresh events: source by activity, target by activity inside the
    # source's group (p_within) or anywhere
    s = np.minimum(np.searchsorted(cdf_all, rng.random(m)), n - 1)
    t = np.minimum(np.searchsorted(cdf_all, rng.random(m)), n - 1)
    inside = rng.random(m) < p_within
    g = group[s]
    lo, hi = gstart[g], gstart[g + 1]
    base = np.where(lo > 0, gcum[np.maximum(lo - 1, 0)], 0.0)
    span = gcum[hi - 1] - base
    pos = np.clip(np.searchsorted(gcum, base + rng.random(m) * span, side="right"), lo, hi - 1)
    t = np.where(inside, byg[pos], t)
    bad = s == t
    while bad.any():
        t[bad] = np.minimum(np.searchsorted(cdf_all, rng.random(int(bad.sum()))), n - 1)
        bad = s == t
    # repeats: event k copies a uniformly chosen earlier event; chains of
    # repeats resolve to the fresh event at their root (pointer jumping)
    rep = rng.random(m) < p_repeat
    rep[0] = False
    root = np.arange(m, dtype=np.int64)
    root[rep] = np.floor(rng.random(int(rep.sum())) * np.flatnonzero(rep)).astype(np.int64)
    while True:
        nxt = root[root]
        if np.array_equal(nxt, root):
            break
        root = nxt
    return s[root].astype(np.int32), t[root].astype(np.int32)


def temporal_split(n: int, src, dst, preload: float = 0.9):
    """The paper's temporal setup (Sec. 5.3): the first ``preload`` of the
    stream is the initial graph (repeated pairs merge, their unit weights
    adding up), the rest is the sequence of insertions that later batches
    take in order.  Returns (csr, (rest_src, rest_dst))."""
    cut = int(round(preload * len(src)))
    u = np.asarray(src[:cut], np.int64)
    v = np.asarray(dst[:cut], np.int64)
    a, b = np.minimum(u, v), np.maximum(u, v)
    key, cnt = np.unique(a * n + b, return_counts=True)
    g = edges_to_csr(n, key // n, key % n, cnt)
    return g, (np.asarray(src[cut:], np.int32), np.asarray(dst[cut:], np.int32))


def temporal_batches(rest, size: int, count: int):
    """``count`` consecutive insertion batches of ``size`` stream events each
    (unit weight; a pair that exists or repeats adds its weight), taken in
    time order from the events after the preload."""
    s, d = rest
    out = []
    for k in range(count):
        a, b = k * size, (k + 1) * size
        if b > len(s):
            break
        out.append((s[a:b].copy(), d[a:b].copy(), np.ones(size, np.int32)))
    return out
