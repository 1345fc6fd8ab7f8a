"""The allocation-free modularity entry point.

leiden_modularity_noalloc serves callers that cannot allocate device memory
when they need a modularity value (a memory budget that forbids new
allocations, a plugin handed only a stream, a loop that cannot afford the
synchronisation of cudaMalloc/cudaFree).  It keeps its scratch in one fixed
device array instead of a context's workspace.  These tests call it through
the C-ABI: twice in a row on different graphs and memberships, each result
equal to the oracle's Eq. 1 and to leiden_modularity (the entry point that
allocates); malformed labels and column IDs are refused with LEIDEN_EINVAL.
The file is named so that pytest collects it last.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2405_11658_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11658_gb300 as L  # noqa: E402

EINVAL, ENOMEM = -1, -2


def call_noalloc(G, memb, gamma):
    q = C.c_double()
    gc = G.c()
    rc = L.lib().leiden_modularity_noalloc(C.byref(gc), C.c_void_p(memb.data_ptr()), gamma,
                                           C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                           C.byref(q))
    return rc, q.value


def test_noalloc_matches_the_oracle_on_two_calls_in_a_row():
    rng = np.random.default_rng(7)
    cases = [(S.planted_partition(20000, 40, 0.01, 0.0005, 3), 1.0),
             (S.chung_lu(30000, 200000, 2.1, 1, 4, seed=5), 0.5)]
    with L.Context(max_n=30001, max_nnz=500000) as ctx:
        for (off, idx, w), gamma in cases:
            n = len(off) - 1
            G = L.Graph.from_numpy(off, idx, w)
            labels = rng.integers(0, max(1, n // 13), size=n).astype(np.int32)
            memb = torch.from_numpy(labels).cuda()
            q_oracle = O.modularity(off, idx, w, labels, gamma)[0]
            rc, q = call_noalloc(G, memb, gamma)
            assert rc == 0, rc
            # same integer numerator divided by the same double expression
            assert q == q_oracle, (q, q_oracle)
            assert q == ctx.modularity(G, memb, gamma)


def test_noalloc_rejects_a_label_out_of_range():
    off, idx, w = S.planted_partition(500, 5, 0.1, 0.01, 4)
    n = len(off) - 1
    G = L.Graph.from_numpy(off, idx, w)
    labels = np.zeros(n, np.int32)
    labels[n // 2] = n
    rc, _ = call_noalloc(G, torch.from_numpy(labels).cuda(), 1.0)
    assert rc == EINVAL
    # the scratch is clean for the next call
    rc, q = call_noalloc(G, torch.zeros(n, dtype=torch.int32, device="cuda"), 1.0)
    assert rc == 0 and q == O.modularity(off, idx, w, np.zeros(n, np.int32))[0]


def test_noalloc_rejects_a_column_id_out_of_range():
    off, idx, w = S.planted_partition(500, 5, 0.1, 0.01, 4)
    n = len(off) - 1
    bad = idx.copy()
    bad[len(bad) // 3] = n
    G = L.Graph.from_numpy(off, bad, w)
    rc, _ = call_noalloc(G, torch.zeros(n, dtype=torch.int32, device="cuda"), 1.0)
    assert rc == EINVAL


def test_noalloc_rejects_graphs_beyond_its_fixed_scratch():
    n = L.NOALLOC_MAX_N + 1
    G = L.Graph(torch.zeros(n + 1, dtype=torch.int64, device="cuda"),
                torch.zeros(0, dtype=torch.int32, device="cuda"),
                torch.zeros(0, dtype=torch.int32, device="cuda"))
    memb = torch.zeros(n, dtype=torch.int32, device="cuda")
    q = C.c_double()
    gc = G.c()
    rc = L.lib().leiden_modularity_noalloc(C.byref(gc), C.c_void_p(memb.data_ptr()), 1.0, None, C.byref(q))
    assert rc == ENOMEM
