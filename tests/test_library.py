"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, and exports every function that include/leiden.h declares."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(leiden_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("leiden_static", "leiden_update", "leiden_modularity", "leiden_apply_batch",
                     "leiden_ctx_create", "leiden_ctx_destroy"):
        assert required in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2405_11658_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2405_11658_gb300 as L
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(L, "_lib", None)
    from paper_2405_11658_gb300 import build
    monkeypatch.setattr(build, "build", lambda *a, **k: (_ for _ in ()).throw(RuntimeError("no nvcc")))
    with pytest.raises(Exception):
        L.lib()


def test_strerror_and_defaults_without_gpu():
    import paper_2405_11658_gb300 as L
    d = L.default_opts()
    assert d["gamma"] == 1.0 and d["tol"] == 0.01 and d["tol_drop"] == 10.0
    assert d["max_iters"] == 20 and d["det_subsets"] == 8
    assert L._strerror(-1) == "invalid argument"


def test_launch_counter_starts_at_zero_without_gpu_work():
    import paper_2405_11658_gb300 as L
    n0 = L.kernel_launches()
    assert n0 >= 0
    L.default_opts()  # host-only calls enqueue nothing
    assert L.kernel_launches() == n0


def _group(lanes, log2_slots, threads, max_degree):
    return {"kind": "group", "lanes": lanes, "log2_slots": log2_slots, "threads": threads, "max_degree": max_degree}


def _block(log2_slots, threads, max_degree):
    return {"kind": "block", "log2_slots": log2_slots, "threads": threads, "max_degree": max_degree}


HUB = {"kind": "hub"}


def test_default_tier_table_validates():
    import paper_2405_11658_gb300 as L
    t = L.default_tiers()
    assert t[-1]["kind"] == "hub" and len(t) <= L.MAX_TIERS
    assert L.validate_tiers(t)
    degs = [x["max_degree"] for x in t[:-1]]
    assert degs == sorted(degs) and len(set(degs)) == len(degs)


@pytest.mark.parametrize("bad", [
    [],                                                             # empty
    [_group(4, 3, 256, 4)],                                         # no hub tier
    [HUB, _group(4, 3, 256, 4)],                                    # hub not last
    [_group(4, 3, 256, 8), HUB],                                    # table 8 slots < 2 * 8
    [_group(4, 5, 256, 4), HUB],                                    # unsupported (lanes, slots)
    [_group(8, 4, 512, 8), HUB],                                    # group block > 256 threads
    [_group(8, 4, 100, 8), HUB],                                    # threads not a multiple of 32
    [_group(8, 4, 256, 8), _group(4, 3, 256, 4), HUB],              # degrees not increasing
    [_block(15, 256, 8192), HUB],                                   # 2^15 slots exceed shared memory
    [_block(12, 32, 2048), HUB],                                    # block tier below 64 threads
    [_block(12, 256, 4096), HUB],                                   # 4096 slots < 2 * 4096
    [_group(32, 10, 256, 512), _block(14, 512, 8192), {"kind": "hub", "threads": 64}],
])
def test_bad_tier_tables_are_rejected(bad):
    import paper_2405_11658_gb300 as L
    assert not L.validate_tiers(bad)


def test_tier_table_variants_are_accepted():
    import paper_2405_11658_gb300 as L
    assert L.validate_tiers([HUB])                                  # every row on the hub path
    assert L.validate_tiers([_group(32, 10, 128, 512), HUB])
    assert L.validate_tiers([_group(4, 4, 256, 4), _group(8, 5, 256, 8), _block(14, 1024, 8192), HUB])
