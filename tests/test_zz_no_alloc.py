"""The allocation-free modularity entry point.

leiden_modularity_noalloc serves callers that cannot allocate device memory
when they need a modularity value (a memory budget that forbids new
allocations, a plugin handed only a stream, a loop that cannot afford the
synchronisation of cudaMalloc/cudaFree).  It keeps its scratch in one fixed
device array instead of a context's workspace.  This test calls it through
the C-ABI twice in a row, on different graphs and memberships, and checks each
result against leiden_modularity, the entry point that allocates.  The file is
named so that pytest collects it last.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

from paper_2405_11658_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2405_11658_gb300 as L  # noqa: E402

TOL = 1e-12  # same integer numerator on both paths; tolerance as for modularity elsewhere


def call_noalloc(G, memb, gamma):
    q = C.c_double()
    gc = G.c()
    rc = L.lib().leiden_modularity_noalloc(C.byref(gc), C.c_void_p(memb.data_ptr()), gamma,
                                           C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                           C.byref(q))
    assert rc == 0, rc
    return q.value


def test_noalloc_matches_modularity_on_two_calls_in_a_row():
    rng = np.random.default_rng(7)
    cases = [(S.planted_partition(20000, 40, 0.01, 0.0005, 3), 1.0),
             (S.chung_lu(30000, 200000, 2.1, 1, 4, seed=5), 0.5)]
    with L.Context(max_n=30001, max_nnz=500000) as ctx:
        for (off, idx, w), gamma in cases:
            n = len(off) - 1
            G = L.Graph.from_numpy(off, idx, w)
            memb = torch.from_numpy(rng.integers(0, max(1, n // 13), size=n).astype(np.int32)).cuda()
            q_ref = ctx.modularity(G, memb, gamma)
            q = call_noalloc(G, memb, gamma)
            assert abs(q - q_ref) <= TOL, (q, q_ref)


def test_noalloc_rejects_graphs_beyond_its_fixed_scratch():
    n = L.NOALLOC_MAX_N + 1
    G = L.Graph(torch.zeros(n + 1, dtype=torch.int64, device="cuda"),
                torch.zeros(0, dtype=torch.int32, device="cuda"),
                torch.zeros(0, dtype=torch.int32, device="cuda"))
    memb = torch.zeros(n, dtype=torch.int32, device="cuda")
    q = C.c_double()
    gc = G.c()
    rc = L.lib().leiden_modularity_noalloc(C.byref(gc), C.c_void_p(memb.data_ptr()), 1.0, None, C.byref(q))
    assert rc == -2
