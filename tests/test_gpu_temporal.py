"""The temporal workload (Sec. 5.3): a timestamped interaction stream, 90% of
it preloaded as the initial graph, then consecutive insertion batches of
1e-3 |E_T| stream events, each applied to the graph the previous one left.
Every update starts from the membership, K^t and Sigma^t the previous update
returned, so errors in the returned auxiliary information would accumulate.

The library's chain (leiden_apply_batch, then leiden_update with the returned
K and Sigma as prior) must equal the oracle's chain bit for bit at every
step: G^t, membership, K^t, Sigma^t, modularity and the per-pass statistics.
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

N, EVENTS = 20000, 200000


@pytest.fixture(scope="module")
def stream():
    src, dst = S.temporal_stream(N, EVENTS, seed=0x1EDE0 + 5)
    g0, rest = S.temporal_split(N, src, dst, 0.9)
    return g0, rest


def rowsum(off, w):
    K = np.zeros(len(off) - 1, np.int64)
    np.add.at(K, np.repeat(np.arange(len(off) - 1), np.diff(off)), np.asarray(w, np.int64))
    return K


@pytest.mark.parametrize("mode,steps", [("DF", 10), ("DS", 3), ("ND", 3)])
def test_chained_updates_bit_exact(stream, mode, steps):
    g0, rest = stream
    size = int(round(1e-3 * EVENTS))
    batches = S.temporal_batches(rest, size, steps)
    assert len(batches) == steps
    base = O.static(*g0)
    C_ref, K_ref = base.membership, rowsum(g0[0], g0[2])
    S_ref = np.zeros(N, np.int64)
    np.add.at(S_ref, C_ref, K_ref)
    g_ref = g0
    cap = len(g0[1]) + 2 * size * steps + 16
    with L.Context(max_n=N, max_nnz=cap) as ctx:
        G = L.Graph.from_numpy(*g0)
        C = torch.from_numpy(C_ref).cuda()
        K = torch.from_numpy(K_ref).cuda()
        Sg = torch.from_numpy(S_ref).cuda()
        for step, ins in enumerate(batches):
            g_ref = O.apply_batch(*g_ref, None, ins)
            ref = O.update(*g_ref, C_ref, K_ref, S_ref, None, ins, mode)
            C_ref, K_ref, S_ref = ref.membership, ref.K, ref.Sigma
            iE = L.Edges.from_numpy(ins)
            G = ctx.apply_batch(G, None, iE, cap_nnz=cap)
            assert np.array_equal(G.idx.cpu().numpy(), g_ref[1]), step
            assert np.array_equal(G.w.cpu().numpy().astype(np.int64), g_ref[2]), step
            C, K, Sg, q = ctx.update(G, C, None, iE, mode, prior_K=K, prior_Sigma=Sg)
            assert np.array_equal(C.cpu().numpy(), C_ref), step
            assert np.array_equal(K.cpu().numpy(), K_ref), step
            assert np.array_equal(Sg.cpu().numpy(), S_ref), step
            assert q == ref.q, step
            st = ctx.stats()
            assert st["affected0"] == ref.stats["affected0"] and st["changed0"] == ref.stats["changed0"]
            k = ref.stats["passes"]
            for key in ("iters", "nv", "nnz", "moves", "refine_moves"):
                assert st[key][:k] == ref.stats[key], (step, key)
