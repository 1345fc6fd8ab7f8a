"""Python binding of ``libleiden`` -- GB300 (sm_103a) Static / ND / DS / DF
Leiden community detection (arXiv 2405.11658).

This module only marshals arguments to the C-ABI declared in
``include/leiden.h``: every step of the method runs in the library's CUDA
kernels.  PyTorch supplies device memory and the CUDA stream.  There is no CPU
fallback: if ``libleiden.so`` is missing or fails to load, every call raises.

Typical use::

    import torch, paper_2405_11658_gb300 as L
    g = L.Graph.from_numpy(off, idx, w)            # device-resident CSR
    with L.Context(max_n=g.n, max_nnz=g.nnz) as ctx:
        memb, q = ctx.static(g)                     # canonical labels, Eq. 1
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libleiden.so")

LEIDEN_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "EOVERFLOW", -4: "ETIMEOUT", -5: "ECUDA"}
ND, DS, DF = 1, 2, 3
MODES = {"ND": ND, "DS": DS, "DF": DF}
DET, ASYNC = 0, 1
STATS_PASSES = 32


class LeidenError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        self.detail = detail
        extra = f"; {detail}" if detail else ""
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({_strerror(code)}){extra}")


class _Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("off", C.c_void_p),
                ("idx", C.c_void_p), ("w", C.c_void_p)]


class _Edges(C.Structure):
    _fields_ = [("count", C.c_int64), ("src", C.c_void_p), ("dst", C.c_void_p),
                ("w", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("gamma", C.c_double), ("tol", C.c_double), ("tol_drop", C.c_double),
                ("max_iters", C.c_int32), ("max_passes", C.c_int32), ("sched", C.c_int32),
                ("det_subsets", C.c_int32), ("refine_all_first_pass", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class _Stats(C.Structure):
    _fields_ = [("passes", C.c_int32),
                ("iters", C.c_int32 * STATS_PASSES),
                ("nv", C.c_int64 * STATS_PASSES),
                ("nnz", C.c_int64 * STATS_PASSES),
                ("moves", C.c_int64 * STATS_PASSES),
                ("refine_moves", C.c_int64 * STATS_PASSES),
                ("affected0", C.c_int64), ("changed0", C.c_int64),
                ("move_kernel_ms", C.c_double), ("move_kernel_launches", C.c_int64),
                ("move_scanned_entries", C.c_int64), ("move_scanned_vertices", C.c_int64),
                ("move_bytes", C.c_double), ("total_ms", C.c_double),
                ("t_move_ms", C.c_double * STATS_PASSES), ("t_refine_ms", C.c_double * STATS_PASSES),
                ("t_agg_ms", C.c_double * STATS_PASSES), ("t_pass_ms", C.c_double * STATS_PASSES),
                ("move0_kernel_ms", C.c_double), ("move0_kernel_launches", C.c_int64), ("move0_bytes", C.c_double),
                ("wide_passes", C.c_uint32), ("move0_scanned_entries", C.c_int64)]

    def as_dict(self) -> dict:
        k = min(self.passes, STATS_PASSES)
        d = {name: getattr(self, name) for name, _ in self._fields_}
        for name in ("iters", "nv", "nnz", "moves", "refine_moves", "t_move_ms", "t_refine_ms",
                     "t_agg_ms", "t_pass_ms"):
            d[name] = list(getattr(self, name))[:k]
        return d


MAX_TIERS = 11
TIER_KINDS = {"group": 1, "block": 2, "hub": 3}


class _Tier(C.Structure):
    _fields_ = [("kind", C.c_int32), ("lanes", C.c_int32), ("log2_slots", C.c_int32),
                ("threads", C.c_int32), ("max_degree", C.c_int64)]


class _TierTable(C.Structure):
    _fields_ = [("count", C.c_int32), ("reserved", C.c_int32), ("tier", _Tier * MAX_TIERS)]

    @classmethod
    def of(cls, tiers) -> "_TierTable":
        t = cls()
        t.count = len(tiers)
        if t.count > MAX_TIERS:
            raise ValueError(f"at most {MAX_TIERS} tiers")
        for k, d in enumerate(tiers):
            x = t.tier[k]
            x.kind = TIER_KINDS[d["kind"]]
            x.lanes = int(d.get("lanes", 0))
            x.log2_slots = int(d.get("log2_slots", 0))
            x.threads = int(d.get("threads", 0))
            x.max_degree = int(d.get("max_degree", 2**63 - 1))
        return t

    def as_list(self) -> list:
        names = {v: k for k, v in TIER_KINDS.items()}
        return [{"kind": names.get(x.kind, x.kind), "lanes": x.lanes, "log2_slots": x.log2_slots,
                 "threads": x.threads, "max_degree": x.max_degree} for x in self.tier[:self.count]]


class _BatchItem(C.Structure):
    _fields_ = [("g", _Csr), ("mode", C.c_int32), ("reserved", C.c_int32), ("prior", C.c_void_p),
                ("dels", _Edges), ("ins", _Edges), ("out", C.c_void_p)]


class _BatchResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("passes", C.c_int32), ("q", C.c_double),
                ("affected0", C.c_int64), ("changed0", C.c_int64),
                ("iters", C.c_int32 * STATS_PASSES), ("nv", C.c_int64 * STATS_PASSES),
                ("nnz", C.c_int64 * STATS_PASSES), ("moves", C.c_int64 * STATS_PASSES),
                ("refine_moves", C.c_int64 * STATS_PASSES)]

    def as_dict(self) -> dict:
        k = min(self.passes, STATS_PASSES)
        d = {"status": self.status, "passes": self.passes, "q": self.q, "affected0": self.affected0,
             "changed0": self.changed0}
        for name in ("iters", "nv", "nnz", "moves", "refine_moves"):
            d[name] = list(getattr(self, name))[:k]
        return d


class _ServerConfig(C.Structure):
    _fields_ = [("hbm_budget", C.c_int64), ("large_slots", C.c_int32), ("small_max_graphs", C.c_int32),
                ("large_max_n", C.c_int64), ("large_max_nnz", C.c_int64), ("small_max_n", C.c_int64),
                ("small_max_nnz", C.c_int64), ("small_batch_n", C.c_int64), ("small_batch_nnz", C.c_int64),
                ("growth", C.c_double), ("mode", C.c_int32), ("autotune_trials", C.c_int32),
                ("small_workers", C.c_int32), ("min_persistent", C.c_int32), ("opts", _Opts)]


class _RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("graph", C.c_int32), ("path", C.c_int32), ("launch_graphs", C.c_int32),
                ("q", C.c_double), ("queue_ms", C.c_double), ("latency_ms", C.c_double),
                ("n", C.c_int64), ("nnz", C.c_int64)]


class _ServerStats(C.Structure):
    _fields_ = [(name, C.c_int64) for name in ("resident_graphs", "resident_bytes", "workspace_bytes", "budget",
                                                 "completed", "failed", "small_launches", "small_graphs_launched",
                                                 "large_runs")]


_lib = None


def lib():
    """Loads libleiden.so (building it first when nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        from . import build as _build
        _build.build()
    L = C.CDLL(LIB_PATH)
    P, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    L.leiden_opts_default.argtypes = [P]
    L.leiden_opts_default.restype = None
    L.leiden_strerror.argtypes = [C.c_int]
    L.leiden_strerror.restype = C.c_char_p
    L.leiden_ctx_create.argtypes = [P, P, i64, i64]
    L.leiden_ctx_create.restype = C.c_int
    L.leiden_ctx_create_sm.argtypes = [P, i32, i64, i64, P]
    L.leiden_ctx_create_sm.restype = C.c_int
    L.leiden_ctx_sm_count.argtypes = [P, P]
    L.leiden_ctx_sm_count.restype = C.c_int
    L.leiden_ctx_set_agg_policy.argtypes = [P, i32]
    L.leiden_ctx_set_agg_policy.restype = C.c_int
    L.leiden_ctx_destroy.argtypes = [P]
    L.leiden_ctx_destroy.restype = None
    L.leiden_ctx_set_timing.argtypes = [P, i32]
    L.leiden_ctx_set_timing.restype = C.c_int
    L.leiden_ctx_last_error.argtypes = [P]
    L.leiden_ctx_last_error.restype = C.c_char_p
    L.leiden_get_stats.argtypes = [P, P]
    L.leiden_get_stats.restype = C.c_int
    L.leiden_static.argtypes = [P, P, P, P, P]
    L.leiden_static.restype = C.c_int
    L.leiden_update.argtypes = [P, P, P, P, P, P, P, i32, P, P, P, P, P]
    L.leiden_update.restype = C.c_int
    L.leiden_modularity.argtypes = [P, P, P, d, P]
    L.leiden_modularity.restype = C.c_int
    L.leiden_apply_batch.argtypes = [P, P, P, P, P, P, P, i64, P]
    L.leiden_apply_batch.restype = C.c_int
    L.leiden_modularity_noalloc.argtypes = [P, P, d, P, P]
    L.leiden_modularity_noalloc.restype = C.c_int
    L.leiden_tiers_default.argtypes = [P]
    L.leiden_tiers_default.restype = None
    L.leiden_tiers_validate.argtypes = [P]
    L.leiden_tiers_validate.restype = C.c_int
    L.leiden_ctx_set_tiers.argtypes = [P, P]
    L.leiden_ctx_set_tiers.restype = C.c_int
    L.leiden_ctx_get_tiers.argtypes = [P, P]
    L.leiden_ctx_get_tiers.restype = C.c_int
    L.leiden_autotune.argtypes = [P, P, P, i32, i32, P, P]
    L.leiden_autotune.restype = C.c_int
    L.leiden_batch_create.argtypes = [P, P, i32, i64, i64, i32, i32]
    L.leiden_batch_create.restype = C.c_int
    L.leiden_batch_destroy.argtypes = [P]
    L.leiden_batch_destroy.restype = None
    L.leiden_batch_run.argtypes = [P, i32, P, P, P]
    L.leiden_batch_run.restype = C.c_int
    L.leiden_server_config_default.argtypes = [P]
    L.leiden_server_config_default.restype = None
    L.leiden_server_create.argtypes = [P, P]
    L.leiden_server_create.restype = C.c_int
    L.leiden_server_destroy.argtypes = [P]
    L.leiden_server_destroy.restype = None
    L.leiden_server_admit.argtypes = [P, i64, i64, P, P, P, P, P]
    L.leiden_server_admit.restype = C.c_int
    L.leiden_server_submit.argtypes = [P, i32, P, P, P]
    L.leiden_server_submit.restype = C.c_int
    L.leiden_server_wait.argtypes = [P, i64, d, P]
    L.leiden_server_wait.restype = C.c_int
    L.leiden_server_membership.argtypes = [P, i32, P, i64]
    L.leiden_server_membership.restype = C.c_int
    L.leiden_server_evict.argtypes = [P, i32]
    L.leiden_server_evict.restype = C.c_int
    L.leiden_server_get_stats.argtypes = [P, P]
    L.leiden_server_get_stats.restype = C.c_int
    L.leiden_ctx_device_bytes.argtypes = [P, P]
    L.leiden_ctx_device_bytes.restype = C.c_int
    L.leiden_batch_device_bytes.argtypes = [P, P]
    L.leiden_batch_device_bytes.restype = C.c_int
    L.leiden_kernel_launches.argtypes = []
    L.leiden_kernel_launches.restype = C.c_uint64
    _lib = L
    return L


def _strerror(code: int) -> str:
    try:
        return lib().leiden_strerror(code).decode()
    except Exception:  # noqa: BLE001 -- used while formatting another error
        return "?"


def _check(rc: int, what: str, ctx=None):
    if rc != LEIDEN_OK:
        detail = ""
        if ctx:
            try:
                detail = (lib().leiden_ctx_last_error(ctx) or b"").decode()
            except Exception:  # noqa: BLE001
                detail = ""
        raise LeidenError(rc, what, detail)


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(a, dtype, device):
    torch = _torch()
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=dtype).contiguous()
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dtype)


@dataclass
class Opts:
    gamma: float = 1.0
    tol: float = 1e-2
    tol_drop: float = 10.0
    max_iters: int = 20
    max_passes: int = 10
    sched: int = DET
    det_subsets: int = 8
    refine_all_first_pass: int = 0

    def c(self) -> _Opts:
        o = _Opts()
        o.gamma, o.tol, o.tol_drop = self.gamma, self.tol, self.tol_drop
        o.max_iters, o.max_passes, o.sched = self.max_iters, self.max_passes, self.sched
        o.det_subsets, o.refine_all_first_pass = self.det_subsets, self.refine_all_first_pass
        return o


class Graph:
    """Symmetric CSR held in device tensors (int64 off, int32 idx, int32 w)."""

    def __init__(self, off, idx, w):
        self.off, self.idx, self.w = off, idx, w
        self.n = int(off.numel()) - 1
        self.nnz = int(idx.numel())

    @classmethod
    def from_numpy(cls, off, idx, w, device="cuda"):
        torch = _torch()
        return cls(_dev(off, torch.int64, device), _dev(idx, torch.int32, device),
                   _dev(w, torch.int32, device))

    def c(self) -> _Csr:
        return _Csr(self.n, self.nnz, _ptr(self.off), _ptr(self.idx), _ptr(self.w))


class Edges:
    """A batch of undirected pairs (src, dst, w) in device tensors."""

    def __init__(self, src, dst, w):
        self.src, self.dst, self.w = src, dst, w
        self.count = int(src.numel())

    @classmethod
    def from_numpy(cls, triple, device="cuda"):
        torch = _torch()
        s, d, w = triple
        return cls(_dev(s, torch.int32, device), _dev(d, torch.int32, device),
                   _dev(w, torch.int32, device))

    def c(self) -> _Edges:
        return _Edges(self.count, _ptr(self.src), _ptr(self.dst), _ptr(self.w))


class Context:
    """A ``leiden_ctx``: device workspace for graphs up to (max_n, max_nnz),
    bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, max_n: int, max_nnz: int, stream=None, sm_count: int | None = None):
        """With ``sm_count`` the context runs on a share of the GPU's SMs
        (leiden_ctx_create_sm: a green context with its own stream; ``sms``
        holds the count provisioned)."""
        torch = _torch()
        self._h = C.c_void_p()
        if sm_count is not None:
            self.stream = None
            got = C.c_int32()
            _check(lib().leiden_ctx_create_sm(C.byref(self._h), int(sm_count), int(max_n), int(max_nnz),
                                              C.byref(got)), "leiden_ctx_create_sm")
            self.sms = got.value
        else:
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            _check(lib().leiden_ctx_create(C.byref(self._h), C.c_void_p(self.stream.cuda_stream),
                                           int(max_n), int(max_nnz)), "leiden_ctx_create")
            got = C.c_int32()
            _check(lib().leiden_ctx_sm_count(self._h, C.byref(got)), "leiden_ctx_sm_count")
            self.sms = got.value
        self.max_n, self.max_nnz = max_n, max_nnz

    def close(self):
        if self._h:
            lib().leiden_ctx_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def set_timing(self, on: bool):
        _check(lib().leiden_ctx_set_timing(self._h, 1 if on else 0), "leiden_ctx_set_timing")

    def set_tiers(self, tiers=None):
        """Sets the degree-tier table (a list of dicts as default_tiers()
        returns; None restores the default)."""
        t = _TierTable.of(tiers) if tiers is not None else None
        _check(lib().leiden_ctx_set_tiers(self._h, C.byref(t) if t is not None else None),
               "leiden_ctx_set_tiers", self._h)

    def set_agg_policy(self, uniform: bool):
        """Aggregation through size-tiered kernels (False, the default) or one
        bucketed multi-block method for every community (True)."""
        _check(lib().leiden_ctx_set_agg_policy(self._h, 1 if uniform else 0), "leiden_ctx_set_agg_policy", self._h)

    def get_tiers(self) -> list:
        t = _TierTable()
        _check(lib().leiden_ctx_get_tiers(self._h, C.byref(t)), "leiden_ctx_get_tiers", self._h)
        return t.as_list()

    def autotune(self, g: Graph, opts: Opts | None = None, max_trials: int = 16, repeats: int = 3):
        """leiden_autotune: times candidate tier tables on g, keeps the
        fastest on this context and returns (tiers, median ms)."""
        opts = opts or Opts()
        t = _TierTable()
        ms = C.c_double()
        gc, oc = g.c(), opts.c()
        _check(lib().leiden_autotune(self._h, C.byref(gc), C.byref(oc), int(max_trials), int(repeats),
                                     C.byref(t), C.byref(ms)), "leiden_autotune", self._h)
        return t.as_list(), ms.value

    def stats(self) -> dict:
        st = _Stats()
        _check(lib().leiden_get_stats(self._h, C.byref(st)), "leiden_get_stats")
        return st.as_dict()

    def static(self, g: Graph, opts: Opts | None = None, out=None, want_q: bool = True):
        torch = _torch()
        opts = opts or Opts()
        memb = out if out is not None else torch.empty(g.n, dtype=torch.int32, device=g.off.device)
        q = C.c_double()
        gc, oc = g.c(), opts.c()
        _check(lib().leiden_static(self._h, C.byref(gc), C.byref(oc), _ptr(memb),
                                   C.byref(q) if want_q else None), "leiden_static", self._h)
        return memb, (q.value if want_q else None)

    def update(self, g: Graph, prior, dels: Edges | None, ins: Edges | None, mode: str,
               opts: Opts | None = None, prior_K=None, prior_Sigma=None, want_q: bool = True,
               out=None, K_out=None, Sigma_out=None):
        torch = _torch()
        opts = opts or Opts()
        dev = g.off.device
        memb = out if out is not None else torch.empty(g.n, dtype=torch.int32, device=dev)
        K = K_out if K_out is not None else torch.empty(g.n, dtype=torch.int64, device=dev)
        S = Sigma_out if Sigma_out is not None else torch.empty(g.n, dtype=torch.int64, device=dev)
        q = C.c_double()
        gc, oc = g.c(), opts.c()
        dc = dels.c() if dels is not None else None
        ic = ins.c() if ins is not None else None
        _check(lib().leiden_update(self._h, C.byref(gc), _ptr(prior), _ptr(prior_K), _ptr(prior_Sigma),
                                   C.byref(dc) if dc is not None else None,
                                   C.byref(ic) if ic is not None else None,
                                   MODES[mode] if isinstance(mode, str) else int(mode), C.byref(oc),
                                   _ptr(memb), _ptr(K), _ptr(S), C.byref(q) if want_q else None),
               "leiden_update", self._h)
        return memb, K, S, (q.value if want_q else None)

    def modularity(self, g: Graph, memb, gamma: float = 1.0) -> float:
        q = C.c_double()
        gc = g.c()
        _check(lib().leiden_modularity(self._h, C.byref(gc), _ptr(memb), gamma, C.byref(q)),
               "leiden_modularity", self._h)
        return q.value

    def apply_batch(self, g: Graph, dels: Edges | None, ins: Edges | None, cap_nnz: int | None = None):
        torch = _torch()
        dev = g.off.device
        if cap_nnz is None:
            cap_nnz = g.nnz + 2 * (ins.count if ins is not None else 0)
        off = torch.empty(g.n + 1, dtype=torch.int64, device=dev)
        idx = torch.empty(max(cap_nnz, 1), dtype=torch.int32, device=dev)
        w = torch.empty(max(cap_nnz, 1), dtype=torch.int32, device=dev)
        nnz = C.c_int64()
        gc = g.c()
        dc = dels.c() if dels is not None else None
        ic = ins.c() if ins is not None else None
        _check(lib().leiden_apply_batch(self._h, C.byref(gc), C.byref(dc) if dc is not None else None,
                                        C.byref(ic) if ic is not None else None, _ptr(off), _ptr(idx),
                                        _ptr(w), int(cap_nnz), C.byref(nnz)), "leiden_apply_batch", self._h)
        return Graph(off, idx[:nnz.value], w[:nnz.value])


NOALLOC_MAX_N = 1048576


def modularity_noalloc(g: Graph, memb, gamma: float = 1.0, stream=None) -> float:
    """Eq. 1 through leiden_modularity_noalloc: no context and no device
    allocation (for callers that cannot allocate); graphs up to
    NOALLOC_MAX_N vertices.  Calls that overlap on the GPU share one scratch
    array and must not run concurrently."""
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    q = C.c_double()
    gc = g.c()
    _check(lib().leiden_modularity_noalloc(C.byref(gc), _ptr(memb), gamma, C.c_void_p(st.cuda_stream),
                                           C.byref(q)), "leiden_modularity_noalloc")
    return q.value


STATIC = 0


class Batch:
    """A ``leiden_batch``: many small graphs per call, each run whole by one
    thread block of one persistent, CUDA-graph-captured launch."""

    def __init__(self, max_graphs: int, max_total_n: int, max_total_nnz: int, threads: int = 0,
                 blocks_per_sm: int = 0, stream=None):
        torch = _torch()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = C.c_void_p()
        _check(lib().leiden_batch_create(C.byref(self._h), C.c_void_p(self.stream.cuda_stream), int(max_graphs),
                                         int(max_total_n), int(max_total_nnz), int(threads), int(blocks_per_sm)),
               "leiden_batch_create")

    def close(self):
        if self._h:
            lib().leiden_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def run(self, items, opts: Opts | None = None):
        """items: list of dicts {"graph": Graph, "mode": "static" | "ND" | "DF",
        "prior": tensor (updates), "dels": Edges, "ins": Edges, "out": tensor
        (optional)}.  Returns (memberships, results): device tensors and one
        dict per graph (status, q and per-pass statistics)."""
        torch = _torch()
        opts = opts or Opts()
        arr = (_BatchItem * max(1, len(items)))()
        outs = []
        for k, it in enumerate(items):
            g = it["graph"]
            mode = it.get("mode", "static")
            out = it.get("out")
            if out is None:
                out = torch.empty(g.n, dtype=torch.int32, device=g.off.device)
            outs.append(out)
            x = arr[k]
            x.g = g.c()
            x.mode = STATIC if mode == "static" else MODES[mode]
            x.reserved = 0
            x.prior = _ptr(it["prior"]) if it.get("prior") is not None else None
            x.dels = it["dels"].c() if it.get("dels") is not None else _Edges(0, None, None, None)
            x.ins = it["ins"].c() if it.get("ins") is not None else _Edges(0, None, None, None)
            x.out = _ptr(out)
        res = (_BatchResult * max(1, len(items)))()
        oc = opts.c()
        _check(lib().leiden_batch_run(self._h, len(items), arr, C.byref(oc), res), "leiden_batch_run")
        return outs, [res[k].as_dict() for k in range(len(items))]


def _host_ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None and len(a) else None


def _host_edges(b):
    """(src, dst, w) numpy arrays as a leiden_edges of HOST pointers (the
    arrays must outlive the call)."""
    import numpy as np
    if b is None:
        return _Edges(0, None, None, None), None
    arrs = tuple(np.ascontiguousarray(x, dtype=np.int32) for x in b)
    return _Edges(len(arrs[0]), _host_ptr(arrs[0]), _host_ptr(arrs[1]), _host_ptr(arrs[2])), arrs


class Server:
    """A ``leiden_server``: resident graphs, HBM-budget admission and
    continuous batching of update batches (host arrays in, host records out)."""

    def __init__(self, opts: Opts | None = None, mode: str = "DF", **cfg):
        c = _ServerConfig()
        lib().leiden_server_config_default(C.byref(c))
        for k, v in cfg.items():
            if not hasattr(c, k):
                raise TypeError(f"unknown server setting {k}")
            setattr(c, k, v)
        c.mode = MODES[mode]
        if opts is not None:
            c.opts = opts.c()
        self._h = C.c_void_p()
        _check(lib().leiden_server_create(C.byref(self._h), C.byref(c)), "leiden_server_create")

    def close(self):
        if self._h:
            lib().leiden_server_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def admit(self, off, idx, w):
        """Admits a host CSR; returns (graph_id, request_id of its Static run)."""
        import numpy as np
        off = np.ascontiguousarray(off, dtype=np.int64)
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.int32)
        gid, rid = C.c_int32(), C.c_int64()
        _check(lib().leiden_server_admit(self._h, len(off) - 1, len(idx), _host_ptr(off), _host_ptr(idx),
                                         _host_ptr(w), C.byref(gid), C.byref(rid)), "leiden_server_admit")
        return gid.value, rid.value

    def submit(self, graph_id: int, dels=None, ins=None) -> int:
        d, keep_d = _host_edges(dels)
        i, keep_i = _host_edges(ins)
        rid = C.c_int64()
        _check(lib().leiden_server_submit(self._h, int(graph_id), C.byref(d), C.byref(i), C.byref(rid)),
               "leiden_server_submit")
        del keep_d, keep_i
        return rid.value

    def wait(self, request_id: int, timeout_ms: float = -1.0) -> dict:
        info = _RequestInfo()
        _check(lib().leiden_server_wait(self._h, int(request_id), float(timeout_ms), C.byref(info)),
               "leiden_server_wait")
        return {name: getattr(info, name) for name, _ in info._fields_}

    def membership(self, graph_id: int, n: int):
        import numpy as np
        out = np.empty(n, np.int32)
        _check(lib().leiden_server_membership(self._h, int(graph_id), _host_ptr(out) if n else None, int(n)),
               "leiden_server_membership")
        return out

    def evict(self, graph_id: int):
        _check(lib().leiden_server_evict(self._h, int(graph_id)), "leiden_server_evict")

    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib().leiden_server_get_stats(self._h, C.byref(st)), "leiden_server_get_stats")
        return {name: getattr(st, name) for name, _ in st._fields_}


def default_tiers() -> list:
    """The library's default degree-tier table (leiden_tiers_default)."""
    t = _TierTable()
    lib().leiden_tiers_default(C.byref(t))
    return t.as_list()


def validate_tiers(tiers) -> bool:
    """True iff leiden_tiers_validate accepts the table (no GPU needed)."""
    try:
        t = _TierTable.of(tiers)
    except (KeyError, ValueError):
        return False
    return lib().leiden_tiers_validate(C.byref(t)) == LEIDEN_OK


def kernel_launches() -> int:
    """Kernels the library has enqueued in this process so far
    (leiden_kernel_launches); difference two readings to count a region."""
    return int(lib().leiden_kernel_launches())


def default_opts() -> dict:
    o = _Opts()
    lib().leiden_opts_default(C.byref(o))
    return {name: getattr(o, name) for name, _ in o._fields_ if name != "reserved"}


EXPORTED = ("leiden_modularity_noalloc", "leiden_ctx_set_agg_policy", "leiden_ctx_create_sm", "leiden_ctx_sm_count", "leiden_ctx_last_error", "leiden_opts_default", "leiden_ctx_create", "leiden_ctx_destroy", "leiden_static",
            "leiden_update", "leiden_modularity", "leiden_apply_batch", "leiden_get_stats",
            "leiden_ctx_set_timing", "leiden_strerror", "leiden_kernel_launches", "leiden_tiers_default",
            "leiden_tiers_validate", "leiden_ctx_set_tiers", "leiden_ctx_get_tiers", "leiden_autotune",
            "leiden_batch_create", "leiden_batch_destroy", "leiden_batch_run", "leiden_server_create",
            "leiden_server_destroy", "leiden_server_admit", "leiden_server_submit", "leiden_server_wait",
            "leiden_server_membership", "leiden_server_evict", "leiden_server_get_stats",
            "leiden_server_config_default", "leiden_ctx_device_bytes", "leiden_batch_device_bytes")
