"""The serving loop (leiden_server_*): resident graphs, budget admission and
continuous batching of update batches.  Every request's result must be the
oracle's -- Static at admission, then DF on each batch in arrival order --
whether the graph ran alone or mixed with others, on the persistent
many-graph path or on a large-graph worker."""
from __future__ import annotations

import threading

import numpy as np
import pytest

import oracle as O
from paper_2405_11658_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11658_gb300 as L  # noqa: E402

CFG = dict(hbm_budget=8 << 30, large_slots=2, small_max_graphs=16, large_max_n=1 << 16, large_max_nnz=1 << 21,
           small_max_n=12000, small_max_nnz=1 << 18, small_batch_n=1 << 18, small_batch_nnz=1 << 22, growth=0.25)


def rowsum(off, w):
    n = len(off) - 1
    return np.bincount(np.repeat(np.arange(n), np.diff(off)), weights=np.asarray(w, np.float64),
                       minlength=n).astype(np.int64)


def workload():
    graphs = [S.planted_partition(2000, 8, 0.02, 0.001, 1), S.planted_partition(10000, 20, 0.01, 0.0005, 2),
              S.rmat(11, 16, seed=3), S.rmat(10, 8, seed=4), S.grid(50, 0.05, 0.001, seed=5),
              S.rmat(15, 16, seed=6),                        # beyond the small limits: a large worker
              S.planted_partition(30000, 30, 0.002, 0.0001, 7)]
    rng = np.random.default_rng(11)
    seqs = []
    for k, g in enumerate(graphs):
        batches, cur = [], g
        for t in range(3):
            frac = [1e-3, 1e-2, 1e-4][(k + t) % 3]
            size = max(2, int(round(frac * len(cur[1]) / 2)))
            dels, ins = S.random_batch(*cur, size, seed=int(rng.integers(1 << 30)))
            batches.append((dels, ins))
            cur = O.apply_batch(*cur, dels, ins)
        seqs.append(batches)
    return graphs, seqs


def oracle_sequence(g, batches):
    """Memberships and modularities: Static, then DF per batch."""
    r = O.static(*g)
    out = [(r.membership, r.q)]
    cur, C = g, r.membership
    for dels, ins in batches:
        K = rowsum(cur[0], cur[2])
        sig = np.bincount(C, weights=K.astype(np.float64), minlength=len(K)).astype(np.int64)
        nxt = O.apply_batch(*cur, dels, ins)
        u = O.update(*nxt, C, K, sig, dels, ins, "DF")
        out.append((u.membership, u.q))
        cur, C = nxt, u.membership
    return out


@pytest.fixture(scope="module")
def expected():
    graphs, seqs = workload()
    return graphs, seqs, [oracle_sequence(g, b) for g, b in zip(graphs, seqs)]


@pytest.mark.parametrize("min_persistent", [1, 64])    # 64: every small graph runs alone on its worker's context
def test_server_results_match_the_oracle_in_the_mix(expected, min_persistent):
    graphs, seqs, want = expected
    with L.Server(**dict(CFG, min_persistent=min_persistent)) as srv:
        ids, reqs = [], []
        for g in graphs:
            gid, rid = srv.admit(*g)
            ids.append(gid)
            reqs.append([rid])
        # batches arrive from two client threads while earlier ones run
        def client(part):
            for k in part:
                for dels, ins in seqs[k]:
                    reqs[k].append(srv.submit(ids[k], dels, ins))
        ts = [threading.Thread(target=client, args=(range(p, len(graphs), 2),)) for p in range(2)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        paths = set()
        for k, g in enumerate(graphs):
            infos = [srv.wait(r) for r in reqs[k]]
            for step, info in enumerate(infos):
                assert info["status"] == 0, (k, step)
                assert info["q"] == want[k][step][1], (k, step)
                assert info["latency_ms"] >= info["queue_ms"] >= 0
                paths.add(info["path"])
            memb = srv.membership(ids[k], len(g[0]) - 1)
            assert np.array_equal(memb, want[k][-1][0]), k
        assert paths == ({0, 1} if min_persistent == 1 else {1, 2})
        st = srv.stats()
        assert st["completed"] == sum(len(r) for r in reqs) and st["failed"] == 0
        assert st["large_runs"] >= 1 and (st["small_launches"] >= 1) == (min_persistent == 1)


def test_server_result_alone_equals_result_in_the_mix(expected):
    graphs, seqs, want = expected
    for k, trials in ((0, 0), (5, 0), (5, 3)):                # 3: the large graph's tier table autotuned
        with L.Server(**dict(CFG, autotune_trials=trials)) as srv:
            gid, rid = srv.admit(*graphs[k])
            rids = [rid] + [srv.submit(gid, d, i) for d, i in seqs[k]]
            qs = [srv.wait(r)["q"] for r in rids]
            assert qs == [x[1] for x in want[k]]
            assert np.array_equal(srv.membership(gid, len(graphs[k][0]) - 1), want[k][-1][0])


def test_server_admission_by_budget_and_eviction():
    g = S.planted_partition(5000, 10, 0.02, 0.001, 3)
    with L.Server(**dict(CFG, hbm_budget=3 << 30)) as srv:
        ws = srv.stats()["workspace_bytes"]
        assert 0 < ws < 3 << 30
        gid, rid = srv.admit(*g)
        assert srv.wait(rid)["status"] == 0
        used = srv.stats()["resident_bytes"]
        assert used > 0
        big = S.rmat(15, 16, seed=1)
        # a budget that holds the workspaces and this graph but not one more
        with pytest.raises(L.LeidenError):
            with L.Server(**dict(CFG, hbm_budget=ws + used + 1)) as tight:
                tight.admit(*g)
                tight.admit(*big)
        srv.evict(gid)
        assert srv.stats()["resident_bytes"] == 0 and srv.stats()["resident_graphs"] == 0
        with pytest.raises(L.LeidenError):
            srv.submit(gid, None, None)                      # evicted
