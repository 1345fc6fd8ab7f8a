"""The at-any-size properties of ``tests/props.py``, computed with torch on
the tensors' own device, for graphs too large to bring to the host (the
2.0e9-entry Chung-Lu workload): canonical labels, modularity equal to an
exact integer recomputation of Eq. 1, community totals equal to the summed
degrees, and every community connected.  Nothing here calls the oracle or
the library; it runs on CPU tensors too (its own tests do)."""
from __future__ import annotations

import torch

# 16-bit limbs: every limb product is below 2^32 and a sum of fewer than 2^31
# of them stays below 2^63, so int64 tensor sums are exact
_LIMB = 16
# CSR entries per chunk of the label gathers
_CHUNK = 1 << 28


def exact_sum_of_squares(x: torch.Tensor) -> int:
    """sum(x_i^2) as an exact Python int for int64 x with 0 <= x < 2^48."""
    assert x.dtype == torch.int64 and x.numel() < 2**31
    if x.numel() == 0:
        return 0
    assert int(x.min()) >= 0 and int(x.max()) < 2**48
    mask = (1 << _LIMB) - 1
    limbs = [(x >> (_LIMB * k)) & mask for k in range(3)]
    total = 0
    for a in range(3):
        for b in range(3):
            total += int((limbs[a] * limbs[b]).sum()) << (_LIMB * (a + b))
    return total


def row_ids(off: torch.Tensor) -> torch.Tensor:
    n = off.numel() - 1
    return torch.repeat_interleave(torch.arange(n, dtype=torch.int32, device=off.device), torch.diff(off))


def row_sums(off: torch.Tensor, w: torch.Tensor, rows: torch.Tensor | None = None) -> torch.Tensor:
    n = off.numel() - 1
    rows = row_ids(off) if rows is None else rows
    K = torch.zeros(n, dtype=torch.int64, device=off.device)
    for e0 in range(0, rows.numel(), _CHUNK):
        K.index_add_(0, rows[e0:e0 + _CHUNK].to(torch.int64), w[e0:e0 + _CHUNK].to(torch.int64))
    return K


def components_within(n: int, src: torch.Tensor, dst: torch.Tensor, max_rounds: int = 400) -> torch.Tensor:
    """Connected-component labels (smallest vertex of the component) of the
    graph with edge list (src, dst), symmetric: min-label propagation with
    pointer jumping."""
    dev = src.device
    lab = torch.arange(n, dtype=torch.int64, device=dev)
    s64, d64 = src.to(torch.int64), dst.to(torch.int64)
    for _ in range(max_rounds):
        new = lab.clone()
        new.scatter_reduce_(0, s64, lab[d64], reduce="amin")
        new = torch.minimum(new, new[new])        # pointer jumping: lab[v] <= v, same component
        if torch.equal(new, lab):
            return lab
        lab = new
    raise AssertionError("component labelling did not converge")


def check_properties(off, idx, w, memb, q, Sigma=None):
    """The checks of tests/props.py on device tensors (gamma = 1)."""
    dev = off.device
    n = off.numel() - 1
    memb = memb.to(torch.int64)
    ncomm = int(memb.max()) + 1 if n else 0
    # canonical labels: community IDs in increasing order of their smallest
    # member, densely numbered from 0
    first = torch.full((ncomm,), n, dtype=torch.int64, device=dev)
    first.scatter_reduce_(0, memb, torch.arange(n, dtype=torch.int64, device=dev), reduce="amin")
    assert int(first[0]) == 0 and bool((torch.diff(first) > 0).all())
    # Eq. 1 with exact integers; the entries are walked in chunks so that the
    # gathered labels stay small next to a graph of 2e9 entries
    rows = row_ids(off)
    m32 = memb.to(torch.int32)
    inside = 0
    srcs, dsts = [], []
    for e0 in range(0, idx.numel(), _CHUNK):
        r = rows[e0:e0 + _CHUNK]
        c = idx[e0:e0 + _CHUNK]
        same = m32[r] == m32[c]
        inside += int(w[e0:e0 + _CHUNK].to(torch.int64)[same].sum())
        srcs.append(r[same])
        dsts.append(c[same])
        del r, c, same
    K = row_sums(off, w, rows)
    sig = torch.zeros(ncomm, dtype=torch.int64, device=dev)
    sig.index_add_(0, memb, K)
    two_m = int(K.sum())
    sq = exact_sum_of_squares(sig)
    assert q == float(two_m * inside - sq) / (float(two_m) * float(two_m) * 1.0)
    if Sigma is not None:
        expect = torch.zeros(n, dtype=torch.int64, device=dev)
        expect[:ncomm] = sig
        assert torch.equal(Sigma.to(torch.int64), expect)
    # every community is connected: over the intra-community edges, all the
    # members of a community share one component label
    del rows
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    del srcs, dsts
    lab = components_within(n, src, dst)
    del src, dst
    comp_of = torch.full((ncomm,), -1, dtype=torch.int64, device=dev)
    comp_of.scatter_reduce_(0, memb, lab, reduce="amax", include_self=False)
    assert torch.equal(comp_of[memb], lab), "a community is not connected"
