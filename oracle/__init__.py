"""Sequential CPU oracle for Static / ND / DS / DF Leiden (arXiv 2405.11658).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its binding) never imports
it, and it imports nothing from the product path.

The arithmetic lives in ``leiden_oracle.c`` (plain C, built with gcc into
``libleiden_oracle.so``).  This module only marshals numpy arrays; the batch
application ``apply_batch`` is a plain edge-set definition in numpy
(``batch.py``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "leiden_oracle.c")
_HDR = os.path.join(_HERE, "leiden_oracle.h")
_LIB = os.path.join(_HERE, "libleiden_oracle.so")

SCHED_DET, SCHED_GS = 0, 1
MODE_STATIC, MODE_ND, MODE_DS, MODE_DF = 0, 1, 2, 3
MODES = {"ND": MODE_ND, "DS": MODE_DS, "DF": MODE_DF}
MAX_PASSES_STATS = 64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: it must build on both
    x86_64 and aarch64 hosts)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call([
        "gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
        "-ffp-contract=off", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


class Opts(C.Structure):
    _fields_ = [("gamma", C.c_double), ("tol", C.c_double), ("tol_drop", C.c_double),
                ("max_iters", C.c_int32), ("max_passes", C.c_int32),
                ("sched", C.c_int32), ("det_subsets", C.c_int32),
                ("refine_all_first_pass", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("passes", C.c_int32),
                ("iters", C.c_int32 * MAX_PASSES_STATS),
                ("nv", C.c_int64 * MAX_PASSES_STATS),
                ("nnz", C.c_int64 * MAX_PASSES_STATS),
                ("moves", C.c_int64 * MAX_PASSES_STATS),
                ("refine_moves", C.c_int64 * MAX_PASSES_STATS),
                ("ncomm", C.c_int64 * MAX_PASSES_STATS),
                ("t_pass", C.c_double * MAX_PASSES_STATS),
                ("affected0", C.c_int64), ("changed0", C.c_int64)]

    def as_dict(self) -> dict:
        k = self.passes
        return {"passes": k, "iters": list(self.iters[:k]), "nv": list(self.nv[:k]),
                "nnz": list(self.nnz[:k]), "moves": list(self.moves[:k]),
                "refine_moves": list(self.refine_moves[:k]),
                "ncomm": list(self.ncomm[:k]), "t_pass": list(self.t_pass[:k]),
                "affected0": self.affected0, "changed0": self.changed0}


@dataclass
class LeidenOpts:
    gamma: float = 1.0
    tol: float = 1e-2
    tol_drop: float = 10.0
    max_iters: int = 20
    max_passes: int = 10
    sched: int = SCHED_DET
    det_subsets: int = 8
    refine_all_first_pass: int = 0

    def c(self) -> Opts:
        return Opts(self.gamma, self.tol, self.tol_drop, self.max_iters, self.max_passes,
                    self.sched, self.det_subsets, self.refine_all_first_pass)


_lib = None
_P = C.c_void_p


def lib():
    global _lib
    if _lib is None:
        # a test may point the wrapper at a deliberately broken build of the
        # oracle (tests/test_oracle_mutations.py) to show the pins catch it
        _lib = C.CDLL(os.environ.get("LEIDEN_ORACLE_LIB") or build())
        L = _lib
        i64, i32, d = C.c_int64, C.c_int32, C.c_double
        L.orc_gamma_ratio.argtypes = [d, _P, _P]; L.orc_gamma_ratio.restype = C.c_int
        L.orc_two_m.argtypes = [i64, _P, _P]; L.orc_two_m.restype = i64
        L.orc_modularity.argtypes = [i64, _P, _P, _P, _P, d, _P, _P]; L.orc_modularity.restype = d
        L.orc_move_score.argtypes = [i64, _P, _P, _P, _P, i32, i32, i64, i64, _P]
        L.orc_move_score.restype = None
        L.orc_det_class.argtypes = [i64, i32]; L.orc_det_class.restype = i32
        L.orc_local_move.argtypes = [i64, _P, _P, _P, _P, _P, _P, _P, _P, _P, i32, i64, i64,
                                     i64, d, i32, i32, i32, _P]
        L.orc_local_move.restype = i32
        L.orc_subset_renumber.argtypes = [i64, _P, _P, _P]; L.orc_subset_renumber.restype = None
        L.orc_break_changed.argtypes = [i64, _P, _P, _P, _P]; L.orc_break_changed.restype = None
        L.orc_refine.argtypes = [i64, _P, _P, _P, _P, _P, _P, _P, _P, i64, i64, i64, i32, i32]
        L.orc_refine.restype = i64
        L.orc_renumber.argtypes = [i64, _P]; L.orc_renumber.restype = i64
        L.orc_aggregate.argtypes = [i64, _P, _P, _P, _P, i64, _P, _P, _P]
        L.orc_aggregate.restype = i64
        L.orc_update_weights.argtypes = [i64, _P, _P, _P, i64, _P, _P, _P, i64, _P, _P, _P]
        L.orc_update_weights.restype = None
        L.orc_changed_communities.argtypes = [i64, _P, _P, i64, _P, _P, i64, _P, _P]
        L.orc_changed_communities.restype = None
        L.orc_mark_df.argtypes = [i64, _P, _P, i64, _P, _P, i64, _P, _P]
        L.orc_mark_df.restype = None
        L.orc_mark_ds.argtypes = [i64, _P, _P, _P, _P, _P, i64, i64, i64, _P,
                                  i64, _P, _P, i64, _P, _P, _P]
        L.orc_mark_ds.restype = None
        L.orc_leiden.argtypes = [i64, _P, _P, _P, _P, _P, _P, _P, i32, _P, i32, _P, _P, _P]
        L.orc_leiden.restype = C.c_int
        L.orc_canonical.argtypes = [i64, _P]; L.orc_canonical.restype = i64
        L.orc_static.argtypes = [i64, _P, _P, _P, _P, _P, _P, _P]; L.orc_static.restype = C.c_int
        L.orc_update.argtypes = [i64, _P, _P, _P, _P, _P, _P, i64, _P, _P, _P, i64, _P, _P, _P,
                                 i32, _P, _P, _P, _P, _P, _P]
        L.orc_update.restype = C.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def _graph(off, idx, w):
    return _c(off, np.int64), _c(idx, np.int32), _c(w, np.int64)


def _i128(lo, hi) -> int:
    return (int(hi) << 64) | (int(lo) & ((1 << 64) - 1))


def gamma_ratio(gamma: float):
    p, q = C.c_int64(), C.c_int64()
    rc = lib().orc_gamma_ratio(gamma, C.byref(p), C.byref(q))
    if rc != 0:
        raise ValueError(f"gamma={gamma!r} is not a multiple of 2^-20")
    return p.value, q.value


def two_m(off, w) -> int:
    off, _, w = _graph(off, np.zeros(0), w)
    return lib().orc_two_m(len(off) - 1, _p(off), _p(w))


def modularity(off, idx, w, C_, gamma: float = 1.0):
    """Eq. 1 at resolution gamma; returns (Q, exact numerator as int)."""
    off, idx, w = _graph(off, idx, w)
    C_ = _c(C_, np.int32)
    lo, hi = C.c_int64(), C.c_int64()
    q = lib().orc_modularity(len(off) - 1, _p(off), _p(idx), _p(w), _p(C_), gamma,
                             C.byref(lo), C.byref(hi))
    return q, _i128(lo.value, hi.value)


def move_score(off, idx, w, C_, i: int, c: int, p: int, q: int) -> int:
    off, idx, w = _graph(off, idx, w)
    C_ = _c(C_, np.int32)
    out = np.zeros(2, np.int64)
    lib().orc_move_score(len(off) - 1, _p(off), _p(idx), _p(w), _p(C_), i, c, p, q, _p(out))
    return _i128(out[0], out[1])


def det_class(i: int, S: int) -> int:
    return lib().orc_det_class(i, S)


def local_move(off, idx, w, C_, K, Sigma, changed, processed, in_range=None, dynamic=0,
               p=1, q=1, tau=0.0, max_iters=20, sched=SCHED_DET, S=8):
    """Alg. leidenlm on numpy state arrays (modified in place). Returns (l_i, moves)."""
    off, idx, w = _graph(off, idx, w)
    tm = lib().orc_two_m(len(off) - 1, _p(off), _p(w))
    moves = C.c_int64()
    li = lib().orc_local_move(len(off) - 1, _p(off), _p(idx), _p(w), _p(C_), _p(K), _p(Sigma),
                              _p(changed), _p(processed), _p(in_range), dynamic, p, q, tm,
                              tau, max_iters, sched, S, C.byref(moves))
    return li, moves.value


def subset_renumber(C_, Sigma, changed):
    lib().orc_subset_renumber(len(C_), _p(C_), _p(Sigma), _p(changed))


def break_changed(C_, K, Sigma, changed):
    lib().orc_break_changed(len(C_), _p(C_), _p(K), _p(Sigma), _p(changed))


def refine(off, idx, w, CB, C_, K, Sigma, changed, p=1, q=1, sched=SCHED_DET, S=8):
    off, idx, w = _graph(off, idx, w)
    tm = lib().orc_two_m(len(off) - 1, _p(off), _p(w))
    return lib().orc_refine(len(off) - 1, _p(off), _p(idx), _p(w), _p(CB), _p(C_), _p(K),
                            _p(Sigma), _p(changed), p, q, tm, sched, S)


def renumber(C_) -> int:
    return lib().orc_renumber(len(C_), _p(C_))


def aggregate(off, idx, w, C_, nc):
    off, idx, w = _graph(off, idx, w)
    C_ = _c(C_, np.int32)
    m = max(int(off[-1]), 1)
    off2 = np.zeros(nc + 1, np.int64)
    idx2 = np.zeros(m, np.int32)
    w2 = np.zeros(m, np.int64)
    m2 = lib().orc_aggregate(len(off) - 1, _p(off), _p(idx), _p(w), _p(C_), nc,
                             _p(off2), _p(idx2), _p(w2))
    return off2, idx2[:m2].copy(), w2[:m2].copy()


def _batch(b):
    if b is None:
        z = np.zeros(0, np.int32)
        return 0, z, z, z
    s, d, wt = (_c(x, np.int32) for x in b)
    return len(s), s, d, wt


def update_weights(Cprev, K, Sigma, dels, ins):
    nd, ds, dd, dw = _batch(dels)
    ni, is_, id_, iw = _batch(ins)
    lib().orc_update_weights(len(Cprev), _p(Cprev), _p(K), _p(Sigma), nd, _p(ds), _p(dd), _p(dw),
                             ni, _p(is_), _p(id_), _p(iw))


def changed_communities(Cprev, dels, ins):
    Cprev = _c(Cprev, np.int32)
    ch = np.zeros(len(Cprev), np.uint8)
    nd, ds, dd, _ = _batch(dels)
    ni, is_, id_, _ = _batch(ins)
    lib().orc_changed_communities(len(Cprev), _p(Cprev), _p(ch), nd, _p(ds), _p(dd),
                                  ni, _p(is_), _p(id_))
    return ch


def mark_df(Cprev, dels, ins):
    Cprev = _c(Cprev, np.int32)
    aff = np.zeros(len(Cprev), np.uint8)
    nd, ds, dd, _ = _batch(dels)
    ni, is_, id_, _ = _batch(ins)
    lib().orc_mark_df(len(Cprev), _p(Cprev), _p(aff), nd, _p(ds), _p(dd), ni, _p(is_), _p(id_))
    return aff


def mark_ds(off, idx, w, Cprev, K, Sigma, dels, ins, gamma=1.0):
    off, idx, w = _graph(off, idx, w)
    Cprev = _c(Cprev, np.int32)
    K = _c(K, np.int64)
    Sigma = _c(Sigma, np.int64)
    p, q = gamma_ratio(gamma)
    tm = lib().orc_two_m(len(off) - 1, _p(off), _p(w))
    aff = np.zeros(len(Cprev), np.uint8)
    nd, ds, dd, _ = _batch(dels)
    ni, is_, id_, iw = _batch(ins)
    lib().orc_mark_ds(len(Cprev), _p(off), _p(idx), _p(Cprev), _p(K), _p(Sigma), p, q, tm,
                      _p(aff), nd, _p(ds), _p(dd), ni, _p(is_), _p(id_), _p(iw))
    return aff


def canonical(C_):
    C_ = np.array(C_, dtype=np.int32, copy=True)
    lib().orc_canonical(len(C_), _p(C_))
    return C_


@dataclass
class Result:
    membership: np.ndarray
    q: float
    stats: dict = field(default_factory=dict)
    K: np.ndarray | None = None
    Sigma: np.ndarray | None = None


def leiden(off, idx, w, Cprev, K, Sigma, affected=None, range_is_affected=0, changed=None,
           dynamic=0, opts: LeidenOpts | None = None):
    """Alg. leiden with explicit lambda state; returns the raw (not canonical) C."""
    opts = opts or LeidenOpts()
    off, idx, w = _graph(off, idx, w)
    n = len(off) - 1
    Cprev, K, Sigma = _c(Cprev, np.int32), _c(K, np.int64), _c(Sigma, np.int64)
    affected, changed = _c(affected, np.uint8), _c(changed, np.uint8)
    out = np.zeros(n, np.int32)
    st = Stats()
    o = opts.c()
    rc = lib().orc_leiden(n, _p(off), _p(idx), _p(w), _p(Cprev), _p(K), _p(Sigma), _p(affected),
                          range_is_affected, _p(changed), dynamic, C.byref(o), _p(out),
                          C.byref(st))
    if rc:
        raise ValueError("oracle leiden failed")
    return out, st.as_dict()


def static(off, idx, w, opts: LeidenOpts | None = None) -> Result:
    opts = opts or LeidenOpts()
    off, idx, w = _graph(off, idx, w)
    n = len(off) - 1
    out = np.zeros(n, np.int32)
    q = C.c_double()
    st = Stats()
    o = opts.c()
    rc = lib().orc_static(n, _p(off), _p(idx), _p(w), C.byref(o), _p(out), C.byref(q),
                          C.byref(st))
    if rc:
        raise ValueError("oracle static failed")
    return Result(out, q.value, st.as_dict())


def update(off, idx, w, Cprev, Kprev, Sprev, dels, ins, mode: str,
           opts: LeidenOpts | None = None) -> Result:
    """ND / DS / DF update on G^t; dels/ins are (src, dst, w) undirected pairs."""
    opts = opts or LeidenOpts()
    off, idx, w = _graph(off, idx, w)
    n = len(off) - 1
    Cprev = _c(Cprev, np.int32)
    Kprev, Sprev = _c(Kprev, np.int64), _c(Sprev, np.int64)
    nd, ds, dd, dw = _batch(dels)
    ni, is_, id_, iw = _batch(ins)
    out = np.zeros(n, np.int32)
    Ko = np.zeros(n, np.int64)
    So = np.zeros(n, np.int64)
    q = C.c_double()
    st = Stats()
    o = opts.c()
    rc = lib().orc_update(n, _p(off), _p(idx), _p(w), _p(Cprev), _p(Kprev), _p(Sprev),
                          nd, _p(ds), _p(dd), _p(dw), ni, _p(is_), _p(id_), _p(iw),
                          MODES[mode], C.byref(o), _p(out), _p(Ko), _p(So), C.byref(q),
                          C.byref(st))
    if rc:
        raise ValueError("oracle update failed")
    return Result(out, q.value, st.as_dict(), Ko, So)


from .batch import apply_batch  # noqa: E402,F401  (plain numpy edge-set definition)
