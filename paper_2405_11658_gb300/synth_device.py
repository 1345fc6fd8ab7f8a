"""Seeded synthetic inputs generated on the device with torch, for the sizes
the host generators of ``synth.py`` cannot reach in reasonable time: the
Chung-Lu web-graph stand-in with 5e7 vertices and 1.0e9 undirected edges
(2.0e9 CSR entries), and random batch updates on it (Sec. 5.1.4).

Like ``synth.py`` this module holds input generators only -- none of the
method's arithmetic.  The recipe is the one of ``synth.chung_lu`` (ball
dropping with endpoint probabilities proportional to (i + i0)^(-1/(beta-1)),
expected degrees capped at sqrt(2 m), deduplication, self-loops dropped,
resampling until exactly m undirected edges, integer weights uniform in
[wmin, wmax]); the endpoint distribution is held as an integer prefix sum, so
sampling is exact; the random numbers come from a torch generator seeded with
``seed`` on the given device, so a graph is reproducible on one machine and
torch build, but is not the same instance as ``synth.chung_lu`` draws on the
host.  Every function also runs on ``device="cpu"`` (used by the CPU tests).

The undirected edges are kept as sorted keys ``a * n + b`` (a < b) with their
weights, from which both the symmetric CSR and the batches are built.
"""
from __future__ import annotations

import math

import torch

# draws per round of the samplers (bounds the temporaries: 16 B per draw)
_CHUNK = 1 << 27


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def chung_lu_edges(n: int, m: int, beta: float = 2.1, wmin: int = 1, wmax: int = 4, seed: int = 0,
                   device="cuda"):
    """m distinct undirected edges of a Chung-Lu graph as (keys, w): keys
    int64 [m] sorted, key = a * n + b with a < b; w int32 [m] in [wmin, wmax]."""
    dev = torch.device(device)
    gen = _gen(seed, dev)
    i0 = 10.0
    x = (torch.arange(n, dtype=torch.float64, device=dev) + i0) ** (-1.0 / (beta - 1.0))
    deg = x * (2.0 * m / float(x.sum()))
    deg.clamp_(max=math.sqrt(2.0 * m))
    # Integer weights and an integer prefix sum: a parallel floating-point
    # scan may add in a different order from run to run, and a last-bit
    # change moves the sampled endpoints.  Integer sums are exact, so the
    # graph depends on the seed alone.
    wint = torch.round(deg * float(1 << 24)).to(torch.int64).clamp_(min=1)
    cdf = torch.cumsum(wint, 0)
    total = int(cdf[-1])
    del x, deg, wint
    have = torch.empty(0, dtype=torch.int64, device=dev)
    while have.numel() < m:
        need = int((m - have.numel()) * 1.1) + 16
        parts = [have]
        for s in range(0, need, _CHUNK):
            k = min(_CHUNK, need - s)
            # endpoint i with probability wint[i] / total: the first i with cdf[i] > r
            u = torch.searchsorted(cdf, torch.randint(0, total, (k,), generator=gen, device=dev), right=True)
            v = torch.searchsorted(cdf, torch.randint(0, total, (k,), generator=gen, device=dev), right=True)
            keep = u != v
            a = torch.minimum(u, v)[keep]
            b = torch.maximum(u, v)[keep]
            del u, v, keep
            parts.append(a * n + b)
            del a, b
        allk = torch.cat(parts)
        del parts, have
        have = torch.unique(allk)            # sorted
        del allk
    if have.numel() > m:
        pick = torch.randperm(have.numel(), generator=gen, device=dev)[:m]
        have = torch.sort(have[pick]).values
        del pick
    w = torch.randint(wmin, wmax + 1, (m,), generator=gen, device=dev, dtype=torch.int32)
    return have, w


def csr_from_edges(n: int, keys: torch.Tensor, w: torch.Tensor):
    """Symmetric CSR (off int64 [n+1], idx int32, w int32) with sorted rows
    from distinct undirected keys a * n + b (a < b), given sorted.

    Row r holds the entries (r, a) of the keys with b = r, all below r, then
    the entries (r, b) of the keys with a = r, all above r.  The second group
    is already in key order; the first comes from one sort of the transposed
    keys.  No sort ever sees more than m elements."""
    dev = keys.device
    m = keys.numel()
    ar = torch.arange(m, dtype=torch.int64, device=dev)

    def starts(rows):
        cnt = torch.bincount(rows, minlength=n)
        first = torch.zeros(n, dtype=torch.int64, device=dev)
        first[1:] = torch.cumsum(cnt, 0)[:-1]
        return cnt, first

    rows_f = keys // n                        # ascending: keys are sorted
    cnt_f, first_f = starts(rows_f)
    t, perm = torch.sort((keys - rows_f * n) * n + rows_f)
    rows_t = t // n
    cnt_t, first_t = starts(rows_t)
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    off[1:] = torch.cumsum(cnt_t + cnt_f, 0)
    idx = torch.empty(2 * m, dtype=torch.int32, device=dev)
    wt = torch.empty(2 * m, dtype=torch.int32, device=dev)
    pos = off[rows_t] + (ar - first_t[rows_t])
    idx[pos] = (t - rows_t * n).to(torch.int32)
    wt[pos] = w[perm].to(torch.int32)
    del t, perm, rows_t, pos
    pos = off[rows_f] + cnt_t[rows_f] + (ar - first_f[rows_f])
    idx[pos] = (keys - rows_f * n).to(torch.int32)
    wt[pos] = w.to(torch.int32)
    return off, idx, wt


def chung_lu(n: int, m: int, beta: float = 2.1, wmin: int = 1, wmax: int = 4, seed: int = 0, device="cuda"):
    """Chung-Lu graph as a device CSR plus its undirected edge keys:
    returns ((off, idx, w), (keys, wkeys))."""
    keys, w = chung_lu_edges(n, m, beta, wmin, wmax, seed, device)
    return csr_from_edges(n, keys, w), (keys, w)


def random_batch(n: int, keys: torch.Tensor, wkeys: torch.Tensor, size: int, seed: int,
                 ins_frac: float = 0.8, weight: int = 1):
    """A batch of ``size`` undirected updates on the graph with sorted edge keys
    ``keys`` (weights ``wkeys``): round(ins_frac * size) insertions between
    uniformly chosen vertex pairs that are not edges (self-loops, existing
    edges and repeats resampled), the rest deletions of distinct, uniformly
    chosen edges.  Returns (dels, ins), each (src, dst, w) int32 tensors on
    the keys' device."""
    dev = keys.device
    gen = _gen(seed, dev)
    m = keys.numel()
    ni = int(round(ins_frac * size))
    nd = min(size - ni, m)
    # deletions: a uniform subset of nd distinct edge positions
    pos = torch.empty(0, dtype=torch.int64, device=dev)
    while pos.numel() < nd:
        extra = torch.randint(0, m, (int((nd - pos.numel()) * 1.1) + 16,), generator=gen, device=dev)
        pos = torch.unique(torch.cat([pos, extra]))
    if pos.numel() > nd:
        pos = pos[torch.randperm(pos.numel(), generator=gen, device=dev)[:nd]]
    dk = keys[pos]
    dels = ((dk // n).to(torch.int32), (dk % n).to(torch.int32), wkeys[pos].to(torch.int32))
    # insertions: distinct non-edges
    got = torch.empty(0, dtype=torch.int64, device=dev)
    while got.numel() < ni and n > 1:
        need = 2 * (ni - got.numel()) + 16
        a = torch.randint(0, n, (need,), generator=gen, device=dev)
        b = torch.randint(0, n, (need,), generator=gen, device=dev)
        keep = a != b
        lo = torch.minimum(a, b)[keep]
        hi = torch.maximum(a, b)[keep]
        k = lo * n + hi
        if m:
            p = torch.searchsorted(keys, k).clamp_(max=m - 1)
            k = k[keys[p] != k]
        k = torch.unique(torch.cat([got, k]))
        if k.numel() > ni:
            # keep the earlier draws, then a uniform subset of the new ones
            fresh = k[~torch.isin(k, got)]
            fresh = fresh[torch.randperm(fresh.numel(), generator=gen, device=dev)[:ni - got.numel()]]
            k = torch.cat([got, fresh])
        got = k
    ins = ((got // n).to(torch.int32), (got % n).to(torch.int32),
           torch.full((got.numel(),), weight, dtype=torch.int32, device=dev))
    return dels, ins
