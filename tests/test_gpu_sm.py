"""Contexts restricted to a share of the SMs (leiden_ctx_create_sm: a green
context and its own stream).  The results must not depend on how many SMs run
the kernels: Static and DF on a context of 8, 24 or 80 SMs equal the oracle
bit for bit (DET), like a context on the whole GPU."""
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


@pytest.mark.parametrize("sms", [8, 24, 80])
def test_results_do_not_depend_on_the_sm_count(sms):
    total = torch.cuda.get_device_properties(0).multi_processor_count
    g = S.rmat(14, 16, seed=7)
    ref = O.static(*g, O.LeidenOpts())
    dels, ins = S.random_batch(*g, 300, seed=3)
    gt = O.apply_batch(*g, dels, ins)
    ref_df = O.update(*gt, ref.membership, None, None, dels, ins, "DF")
    with L.Context(max_n=len(g[0]), max_nnz=len(g[1]) + 4096, sm_count=sms) as ctx:
        assert sms <= ctx.sms <= total and ctx.sms % 8 == 0
        G = L.Graph.from_numpy(*g)
        memb, q = ctx.static(G)
        assert np.array_equal(memb.cpu().numpy(), ref.membership) and q == ref.q
        st = ctx.stats()
        assert st["iters"][:ref.stats["passes"]] == ref.stats["iters"]
        Gt = ctx.apply_batch(G, L.Edges.from_numpy(dels), L.Edges.from_numpy(ins))
        m2, _, _, q2 = ctx.update(Gt, memb, L.Edges.from_numpy(dels), L.Edges.from_numpy(ins), "DF")
        assert np.array_equal(m2.cpu().numpy(), ref_df.membership) and q2 == ref_df.q
        assert ctx.modularity(G, memb) == ref.q


def test_sm_count_out_of_range_is_refused():
    total = torch.cuda.get_device_properties(0).multi_processor_count
    for bad in (0, total + 1):
        h = C.c_void_p()
        assert L.lib().leiden_ctx_create_sm(C.byref(h), bad, 100, 100, None) == -1
