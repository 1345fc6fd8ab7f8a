"""The largest single-GPU workload at full size: a Chung-Lu web-graph stand-in
with degree exponent 2.1, 5e7 vertices, 1.0e9 undirected edges (2.0e9 CSR
entries, int64 offsets), integer weights uniform in 1..4, generated on the
device (paper_2405_11658_gb300/synth_device.py), in a context with room for
the benchmark's 1e-1 |E| batch and for an insertion batch that takes G^t past
2^31 entries.

The oracle needs hours at this size, so every run is checked through the
properties that hold at any size (tests/props_device.py, computed on the
device): canonical labels, every community connected, modularity equal to an
exact integer recomputation of Eq. 1 divided in the same double expression,
and for updates Sigma^t equal to the summed degrees and K^t equal to the row
sums of G^t.  The batch's deletions must be gone from G^t and its insertions
present.
"""
from __future__ import annotations

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11658_gb300 as L  # noqa: E402
from paper_2405_11658_gb300 import synth_device as D  # noqa: E402
from tests import props_device as PD  # noqa: E402

N, M = 50_000_000, 1_000_000_000
SEED = 0x1EDE0 + 2
FRAC = 1e-4


BIG_INSERT = 80_000_000   # undirected insertions: 2e9 + 1.6e8 CSR entries > 2^31


def max_nnz_for(nnz, m):
    # room for the benchmark's largest batch (1e-1 |E|, 80% insertions) and
    # for the insertion-only batch below
    return nnz + 2 * max(int(round(0.8 * 0.1 * m)), BIG_INSERT) + 16


@pytest.fixture(scope="module")
def work():
    torch.cuda.empty_cache()
    (off, idx, w), (keys, wk) = D.chung_lu(N, M, 2.1, 1, 4, seed=SEED, device="cuda")
    dels, ins = D.random_batch(N, keys, wk, int(round(FRAC * M)), seed=1)
    del keys, wk
    torch.cuda.empty_cache()
    G = L.Graph(off, idx, w)
    ctx = L.Context(max_n=N, max_nnz=max_nnz_for(G.nnz, M))
    try:
        yield G, dels, ins, ctx
    finally:
        ctx.close()
        del G
        torch.cuda.empty_cache()


def test_the_device_generator_is_reproducible():
    # the graph depends on the seed alone (integer sampling distribution;
    # no floating-point reduction whose order could vary between runs)
    a, ka = D.chung_lu(1_000_000, 10_000_000, 2.1, 1, 4, seed=SEED, device="cuda")
    b, kb = D.chung_lu(1_000_000, 10_000_000, 2.1, 1, 4, seed=SEED, device="cuda")
    assert all(torch.equal(x, y) for x, y in zip(a + ka, b + kb))


def test_the_graph_is_the_configured_one(work):
    G, _, _, _ = work
    assert G.n == N and G.nnz == 2 * M
    assert int(G.w.min()) >= 1 and int(G.w.max()) <= 4


@pytest.fixture(scope="module")
def static_det(work):
    G, _, _, ctx = work
    memb, q = ctx.static(G, L.Opts())
    return memb, q, ctx.stats()


def test_static_det_properties_at_full_size(work, static_det):
    G, _, _, _ = work
    memb, q, st = static_det
    assert st["passes"] >= 2 and st["nnz"][0] == G.nnz
    PD.check_properties(G.off, G.idx, G.w, memb, q)


def test_df_update_properties_at_full_size(work, static_det):
    G, dels, ins, ctx = work
    memb, q_static, _ = static_det
    dE, iE = L.Edges(*dels), L.Edges(*ins)
    Gt = ctx.apply_batch(G, dE, iE, cap_nnz=max_nnz_for(G.nnz, M))
    assert Gt.nnz == G.nnz - 2 * dE.count + 2 * iE.count
    # the batch is applied: deletions gone, insertions present with weight 1
    rows = PD.row_ids(Gt.off).to(torch.int64)
    key = rows * N + Gt.idx.to(torch.int64)
    del rows
    assert bool((torch.diff(key) > 0).all())                  # sorted rows, no duplicates
    for (s, d, ww), present in ((dels, False), (ins, True)):
        for a, b in ((s, d), (d, s)):
            k = a.to(torch.int64) * N + b.to(torch.int64)
            pos = torch.searchsorted(key, k).clamp_(max=key.numel() - 1)
            hit = key[pos] == k
            assert bool(hit.all()) if present else not bool(hit.any())
            if present:
                assert bool((Gt.w[pos] == ww).all())
    del key
    # auxiliary information of the base membership, then DF on G^t
    C0, K0, S0, _ = ctx.update(G, memb, None, None, "ND", L.Opts(), want_q=False)
    m2, K2, S2, q2 = ctx.update(Gt, C0, dE, iE, "DF", L.Opts(), prior_K=K0, prior_Sigma=S0)
    st = ctx.stats()
    assert 0 < st["affected0"] < Gt.n
    assert torch.equal(K2, PD.row_sums(Gt.off, Gt.w))
    PD.check_properties(Gt.off, Gt.idx, Gt.w, m2, q2, Sigma=S2)
    # the paper's soft bar (Sec. 5.2): dynamic modularity close to Static's
    assert q2 >= q_static - 0.02


def test_async_static_properties_at_full_size(work):
    G, _, _, ctx = work
    memb, q = ctx.static(G, L.Opts(sched=L.ASYNC))
    PD.check_properties(G.off, G.idx, G.w, memb, q)


def test_static_past_2_31_entries(work):
    # an insertion-only batch takes G^t past 2^31 CSR entries: offsets and
    # entry positions beyond the 32-bit range in every kernel
    G, _, _, ctx = work
    rows = PD.row_ids(G.off)
    upper = G.idx > rows
    keys = rows[upper].to(torch.int64) * N + G.idx[upper].to(torch.int64)   # sorted: rows are
    del rows, upper
    _, ins = D.random_batch(N, keys, torch.ones_like(keys, dtype=torch.int32), BIG_INSERT, seed=7, ins_frac=1.0)
    del keys
    Gt = ctx.apply_batch(G, None, L.Edges(*ins), cap_nnz=max_nnz_for(G.nnz, M))
    del ins
    assert Gt.nnz == G.nnz + 2 * BIG_INSERT and Gt.nnz > 2**31
    memb, q = ctx.static(Gt, L.Opts())
    assert ctx.stats()["nnz"][0] == Gt.nnz
    PD.check_properties(Gt.off, Gt.idx, Gt.w, memb, q)
