"""Parity of the persistent many-graph path (leiden_batch_run) with the
oracle: every graph of a batch, run whole inside one thread block of one
CUDA-graph-captured launch, must end with the oracle's membership,
modularity and per-pass statistics (DET), alone or mixed with others."""
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


def star(k):
    return S.edges_to_csr(k + 1, np.zeros(k, np.int64), np.arange(1, k + 1))


def isolated_plus(g, extra):
    off, idx, w = g
    return np.concatenate([off, np.full(extra, off[-1], off.dtype)]), idx, w


SMALL = {
    "pp_2000": lambda: S.planted_partition(2000, 8, 0.02, 0.001, 1),
    "pp_1e4": lambda: S.planted_partition(10000, 20, 0.01, 0.0005, 0x1EDE0),
    "rmat11": lambda: S.rmat(11, 16, seed=2),
    "rmat10_ef32": lambda: S.rmat(10, 32, seed=3),
    "grid": lambda: S.grid(40, 0.05, 0.001, seed=4),
    "kmer": lambda: S.kmer(5000, 32, 2.1, seed=5),
    "ring": lambda: S.ring_of_cliques(12, 5),
    "star": lambda: star(3000),                      # a row far beyond the warp tables
    "er_dense": lambda: S.erdos_renyi(400, 0.4, 6, wmax=5),
    "chung_lu_w": lambda: S.chung_lu(3000, 20000, 2.1, 1, 4, seed=7),
    "isolated": lambda: isolated_plus(S.planted_partition(500, 4, 0.05, 0.002, 8), 37),
    "one_vertex": lambda: (np.zeros(2, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32)),
    "empty": lambda: (np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32)),
}


def stats_equal(r, ref):
    k = ref["passes"]
    assert r["passes"] == k
    for name in ("iters", "nv", "nnz", "moves", "refine_moves"):
        assert r[name][:k] == ref[name][:k], name


@pytest.fixture(scope="module")
def batch():
    with L.Batch(max_graphs=64, max_total_n=1 << 18, max_total_nnz=1 << 23) as b:
        yield b


def test_batch_static_matches_oracle(batch):
    names = list(SMALL)
    graphs = [SMALL[k]() for k in names]
    items = [{"graph": L.Graph.from_numpy(*g), "mode": "static"} for g in graphs]
    outs, res = batch.run(items, L.Opts())
    for name, g, out, r in zip(names, graphs, outs, res):
        ref = O.static(*g, O.LeidenOpts())
        assert r["status"] == 0, name
        assert np.array_equal(out.cpu().numpy(), ref.membership), name
        assert r["q"] == ref.q, name
        stats_equal(r, ref.stats)


@pytest.mark.parametrize("S_,gamma,tol,mp,mi", [(1, 1.0, 1e-2, 10, 20), (32, 0.5, 0.0, 10, 20),
                                                (256, 2.0, 1e-3, 3, 4), (8, 1.0, 1e-2, 1, 20)])
def test_batch_static_options(batch, S_, gamma, tol, mp, mi):
    graphs = [S.rmat(11, 16, seed=21), S.planted_partition(3000, 6, 0.02, 0.002, 5)]
    oo = O.LeidenOpts(det_subsets=S_, gamma=gamma, tol=tol, max_passes=mp, max_iters=mi)
    items = [{"graph": L.Graph.from_numpy(*g)} for g in graphs]
    outs, res = batch.run(items, L.Opts(det_subsets=S_, gamma=gamma, tol=tol, max_passes=mp, max_iters=mi))
    for g, out, r in zip(graphs, outs, res):
        ref = O.static(*g, oo)
        assert np.array_equal(out.cpu().numpy(), ref.membership)
        assert r["q"] == ref.q
        stats_equal(r, ref.stats)


def make_update(name, frac, seed):
    off, idx, w = SMALL[name]()
    prior = O.static(off, idx, w)
    n = len(off) - 1
    K = np.zeros(n, np.int64)
    np.add.at(K, np.repeat(np.arange(n), np.diff(off)), np.asarray(w, np.int64))
    sig = np.zeros(n, np.int64)
    np.add.at(sig, prior.membership, K)
    size = max(2, int(round(frac * len(idx) / 2)))
    dels, ins = S.random_batch(off, idx, w, size, seed=seed)
    gt = O.apply_batch(off, idx, w, dels, ins)
    return gt, prior.membership, K, sig, dels, ins


@pytest.mark.parametrize("mode", ["ND", "DS", "DF"])
def test_batch_updates_match_oracle(batch, mode):
    cases = [("pp_1e4", 1e-3, 1), ("rmat11", 1e-2, 2), ("grid", 1e-3, 3), ("chung_lu_w", 1e-2, 4),
             ("er_dense", 1e-3, 5), ("kmer", 1e-2, 6)]
    ups = [make_update(*c) for c in cases]
    items = []
    for gt, prior, _, _, dels, ins in ups:
        items.append({"graph": L.Graph.from_numpy(*gt), "mode": mode,
                      "prior": torch.from_numpy(prior).cuda(), "dels": L.Edges.from_numpy(dels),
                      "ins": L.Edges.from_numpy(ins)})
    outs, res = batch.run(items, L.Opts())
    for (gt, prior, K, sig, dels, ins), out, r, c in zip(ups, outs, res, cases):
        ref = O.update(*gt, prior, K, sig, dels, ins, mode)
        assert r["status"] == 0, c
        assert np.array_equal(out.cpu().numpy(), ref.membership), c
        assert r["q"] == ref.q, c
        assert r["affected0"] == ref.stats["affected0"] and r["changed0"] == ref.stats["changed0"], c
        stats_equal(r, ref.stats)


def test_each_result_is_the_same_alone_and_in_the_mix(batch):
    graphs = [SMALL[k]() for k in ("pp_2000", "rmat11", "star", "ring", "kmer")]
    up = make_update("pp_1e4", 1e-3, 9)
    mix = [{"graph": L.Graph.from_numpy(*g)} for g in graphs]
    gt, prior, _, _, dels, ins = up
    mix.append({"graph": L.Graph.from_numpy(*gt), "mode": "DF", "prior": torch.from_numpy(prior).cuda(),
                "dels": L.Edges.from_numpy(dels), "ins": L.Edges.from_numpy(ins)})
    outs_mix, res_mix = batch.run(mix, L.Opts())
    for k, it in enumerate(mix):
        outs_one, res_one = batch.run([it], L.Opts())
        assert torch.equal(outs_one[0], outs_mix[k])
        assert res_one[0] == res_mix[k]


def test_batch_replays_and_recaptures(batch):
    g = SMALL["rmat11"]()
    items = [{"graph": L.Graph.from_numpy(*g)}]
    first = batch.run(items, L.Opts())
    for _ in range(3):
        again = batch.run(items, L.Opts())
        assert torch.equal(again[0][0], first[0][0]) and again[1] == first[1]
    other = batch.run(items, L.Opts(gamma=0.5))          # new options: captured again
    ref = O.static(*g, O.LeidenOpts(gamma=0.5))
    assert np.array_equal(other[0][0].cpu().numpy(), ref.membership)
    n0 = L.kernel_launches()
    batch.run(items, L.Opts(gamma=0.5))
    assert L.kernel_launches() - n0 == 1                 # one launch per batch


def test_batch_reports_bad_graphs_per_item(batch):
    good = SMALL["pp_2000"]()
    off, idx, w = SMALL["ring"]()
    bad_idx = idx.copy()
    bad_idx[3] = len(off) + 5                            # neighbour ID out of range
    items = [{"graph": L.Graph.from_numpy(*good)}, {"graph": L.Graph.from_numpy(off, bad_idx, w)}]
    outs, res = batch.run(items, L.Opts())
    assert res[0]["status"] == 0 and res[1]["status"] == -1
    ref = O.static(*good, O.LeidenOpts())
    assert np.array_equal(outs[0].cpu().numpy(), ref.membership)
    with pytest.raises(L.LeidenError):
        batch.run(items[:1], L.Opts(sched=L.ASYNC))      # DET only
    with pytest.raises(L.LeidenError):
        batch.run([items[0]] * 65, L.Opts())             # beyond max_graphs
