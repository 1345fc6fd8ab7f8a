"""Brute-force references used to pin the oracle.  Written from the
definitions in Sec. 3 of the paper, in a different form from the oracle (the
pairwise Newman form of modularity, exhaustive partition search, BFS), so a
slip in the oracle's formula shows up as a mismatch here.  Nothing in this
file calls the oracle."""
from __future__ import annotations

from collections import deque
from fractions import Fraction

import numpy as np


def dense(off, idx, w):
    n = len(off) - 1
    A = [[0] * n for _ in range(n)]
    for i in range(n):
        for e in range(off[i], off[i + 1]):
            A[i][int(idx[e])] += int(w[e])
    return A


def q_newman(A, C, p=1, q=1) -> Fraction:
    """Q = (1/2m) sum_ij [A_ij - gamma k_i k_j / 2m] delta(C_i, C_j)."""
    n = len(A)
    k = [sum(r) for r in A]
    two_m = sum(k)
    if two_m == 0:
        return Fraction(0)
    g = Fraction(p, q)
    tot = Fraction(0)
    for i in range(n):
        for j in range(n):
            if C[i] == C[j]:
                tot += A[i][j] - g * Fraction(k[i] * k[j], two_m)
    return tot / two_m


def components_within(off, idx, members) -> int:
    """Connected components of the subgraph induced by ``members``."""
    ms = set(int(x) for x in members)
    seen = set()
    comps = 0
    for s in ms:
        if s in seen:
            continue
        comps += 1
        dq = deque([s])
        seen.add(s)
        while dq:
            u = dq.popleft()
            for e in range(off[u], off[u + 1]):
                v = int(idx[e])
                if v in ms and v not in seen:
                    seen.add(v)
                    dq.append(v)
    return comps


def all_connected(off, idx, C) -> bool:
    C = np.asarray(C)
    for c in np.unique(C):
        if components_within(off, idx, np.flatnonzero(C == c)) != 1:
            return False
    return True


def restricted_growth(n: int) -> np.ndarray:
    """Every set partition of n items as a restricted growth string."""
    rows = np.zeros((1, 1), np.int8)
    mx = np.zeros(1, np.int8)
    for _ in range(1, n):
        reps = (mx + 2).astype(np.int64)
        base = np.repeat(rows, reps, axis=0)
        bmx = np.repeat(mx, reps)
        val = np.concatenate([np.arange(r, dtype=np.int8) for r in reps])
        rows = np.concatenate([base, val[:, None]], axis=1)
        mx = np.maximum(bmx, val)
    return rows


def exhaustive_best(A, p=1, q=1):
    """(Q_opt, argmax partition) over all set partitions, in float64 with an
    exact Fraction recheck of the winner."""
    A = np.asarray(A, np.float64)
    n = len(A)
    k = A.sum(1)
    two_m = k.sum()
    parts = restricted_growth(n).astype(np.int64)
    best_q, best = -np.inf, None
    for s in range(0, len(parts), 20000):
        P = parts[s:s + 20000]
        same = P[:, :, None] == P[:, None, :]
        sig = (same * A[None]).sum((1, 2))
        onehot = P[:, :, None] == np.arange(n)[None, None, :]
        Sg = np.einsum("pic,i->pc", onehot.astype(np.float64), k)
        Q = (sig - (p / q) * (Sg ** 2).sum(1) / two_m) / two_m
        a = int(np.argmax(Q))
        if Q[a] > best_q:
            best_q, best = Q[a], P[a].copy()
    return q_newman(A.astype(np.int64).tolist(), best, p, q), best


def max_single_move_gain(A, C, p=1, q=1) -> Fraction:
    """Largest Q gain of moving one vertex to any existing community or to a
    new singleton, by recomputing Q."""
    n = len(A)
    base = q_newman(A, C, p, q)
    best = Fraction(0)
    labels = sorted(set(C)) + [max(C) + 1]
    for i in range(n):
        for c in labels:
            if c == C[i]:
                continue
            D = list(C)
            D[i] = c
            best = max(best, q_newman(A, D, p, q) - base)
    return best
