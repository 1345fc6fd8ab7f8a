"""The low-degree workloads at full size, in the benchmark's launch
configuration (DET schedule, 8 colour classes, default tier table):

* a 5000 x 5000 four-neighbour grid with 5% of its edges removed and
  0.1% |V| uniform shortcuts (25M vertices, 9.5e7 CSR entries), standing in
  for road networks: batch application bit-exact, the first pass of Static,
  DS and DF (1e-4 |E| batch) bit-exact with the oracle, full runs checked
  through properties that hold at any size;
* a 1e8-vertex k-mer-like graph (random paths of geometric length, mean 64,
  plus uniform edges up to mean degree 2.1; 2.1e8 CSR entries), standing in
  for protein k-mer graphs: the oracle needs minutes per pass at this size,
  so Static and a DF update (1e-4 |E| batch) are checked through the same
  properties only (canonical labels, Eq. 1 recomputed exactly, Sigma^t equal
  to the summed degrees, K^t equal to the row sums, every community
  connected).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2405_11658_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11658_gb300 as L  # noqa: E402
from tests.props import check_properties, rowsum  # noqa: E402

FRAC = 1e-4


def host(t):
    return t.cpu().numpy()


def batch_of(g, seed):
    size = max(2, int(round(FRAC * len(g[1]) / 2)))
    return S.random_batch(*g, size, seed=seed)


@pytest.fixture(scope="module")
def grid():
    g = S.grid(5000, 0.05, 0.001, seed=0x1EDE0 + 3)
    dels, ins = batch_of(g, 1000)
    gt = O.apply_batch(*g, dels, ins)
    with L.Context(max_n=len(g[0]) - 1, max_nnz=max(len(g[1]), len(gt[1])) + 16) as ctx:
        yield g, gt, dels, ins, ctx


def test_grid_batch_apply_bit_exact(grid):
    g, gt, dels, ins, ctx = grid
    Gt = ctx.apply_batch(L.Graph.from_numpy(*g), L.Edges.from_numpy(dels), L.Edges.from_numpy(ins),
                         cap_nnz=len(gt[1]) + 16)
    for a, b in zip((Gt.off, Gt.idx, Gt.w), gt):
        assert np.array_equal(host(a), b)


def test_grid_static_first_pass_bit_exact(grid):
    g, _, _, _, ctx = grid
    ref = O.static(*g, O.LeidenOpts(max_passes=1))
    memb, q = ctx.static(L.Graph.from_numpy(*g), L.Opts(max_passes=1))
    assert np.array_equal(host(memb), ref.membership)
    assert q == ref.q
    st = ctx.stats()
    for k in ("iters", "nv", "nnz", "moves", "refine_moves"):
        assert st[k][:1] == ref.stats[k][:1], k


@pytest.mark.parametrize("mode", ["DS", "DF"])
def test_grid_update_first_pass_bit_exact(grid, mode):
    g, gt, dels, ins, ctx = grid
    off, idx, w = g
    prior = host(ctx.static(L.Graph.from_numpy(*g), L.Opts(max_passes=1))[0])
    K = rowsum(off, w)
    sig = np.bincount(prior, weights=K.astype(np.float64), minlength=len(K)).astype(np.int64)
    ref = O.update(*gt, prior, K, sig, dels, ins, mode, O.LeidenOpts(max_passes=1))
    Gt = L.Graph.from_numpy(*gt)
    dev = Gt.off.device
    memb, Kt, St, q = ctx.update(Gt, torch.from_numpy(prior).to(dev), L.Edges.from_numpy(dels),
                                 L.Edges.from_numpy(ins), mode, opts=L.Opts(max_passes=1),
                                 prior_K=torch.from_numpy(K).to(dev), prior_Sigma=torch.from_numpy(sig).to(dev))
    assert np.array_equal(host(memb), ref.membership)
    assert np.array_equal(host(Kt), ref.K) and np.array_equal(host(St), ref.Sigma)
    assert q == ref.q
    st = ctx.stats()
    assert st["affected0"] == ref.stats["affected0"] and st["changed0"] == ref.stats["changed0"]


def test_grid_full_runs_properties(grid):
    g, gt, dels, ins, ctx = grid
    off, idx, w = g
    memb, q = ctx.static(L.Graph.from_numpy(*g), L.Opts())
    prior = host(memb)
    check_properties(*g, prior, q)
    K = rowsum(off, w)
    sig = np.bincount(prior, weights=K.astype(np.float64), minlength=len(K)).astype(np.int64)
    Gt = L.Graph.from_numpy(*gt)
    dev = Gt.off.device
    memb, Kt, St, q = ctx.update(Gt, torch.from_numpy(prior).to(dev), L.Edges.from_numpy(dels),
                                 L.Edges.from_numpy(ins), "DF", opts=L.Opts(),
                                 prior_K=torch.from_numpy(K).to(dev), prior_Sigma=torch.from_numpy(sig).to(dev))
    assert np.array_equal(host(Kt), rowsum(gt[0], gt[2]))
    check_properties(*gt, host(memb), q, host(St))


def test_kmer_1e8_static_and_df_properties():
    g = S.kmer(100_000_000, 64.0, 2.1, seed=0x1EDE0 + 4)
    off, idx, w = g
    dels, ins = batch_of(g, 1000)
    n = len(off) - 1
    cap = len(idx) + 2 * len(ins[0]) + 16
    with L.Context(max_n=n, max_nnz=cap) as ctx:
        G0 = L.Graph.from_numpy(*g)
        memb, q = ctx.static(G0, L.Opts())
        prior = host(memb)
        check_properties(*g, prior, q)
        st = ctx.stats()
        assert st["nv"][0] == n and st["nnz"][0] == len(idx)
        K = rowsum(off, w)
        sig = np.bincount(prior, weights=K.astype(np.float64), minlength=n).astype(np.int64)
        dE, iE = L.Edges.from_numpy(dels), L.Edges.from_numpy(ins)
        Gt = ctx.apply_batch(G0, dE, iE, cap_nnz=cap)
        gt = (host(Gt.off), host(Gt.idx), host(Gt.w))
        # the batch landed: deleted pairs absent, inserted pairs present
        rows = np.repeat(np.arange(n), np.diff(gt[0]))
        key = rows.astype(np.int64) * n + gt[1]
        for (s, d, _), present in ((dels, False), (ins, True)):
            k = s.astype(np.int64) * n + d
            pos = np.minimum(np.searchsorted(key, k), len(key) - 1)
            assert np.all((key[pos] == k) == present)
        dev = Gt.off.device
        memb, Kt, St, q = ctx.update(Gt, torch.from_numpy(prior).to(dev), dE, iE, "DF", opts=L.Opts(),
                                     prior_K=torch.from_numpy(K).to(dev), prior_Sigma=torch.from_numpy(sig).to(dev))
        assert np.array_equal(host(Kt), rowsum(gt[0], gt[2]))
        check_properties(*gt, host(memb), q, host(St))
        assert ctx.stats()["affected0"] < n // 100          # DF touched a small frontier
