"""Model check of the ASYNC refinement's join protocol (Alg. leidenre with the
paper's in-place updates, as `refine_join_async` in csrc/common.cuh does it).

A singleton v leaves its own sub-community only while it is still isolated
(compare-and-swap of Sigma'[v] from K'[v] to a departure marker), then adds
K'[v] to its target's total, and undoes both steps if the total it found says
that the target's own vertex has left.  Every interleaving of the atomic
steps of three threads is enumerated: j leaves for community k while i and m
join j's community (both having read C'[j] = j before j moved, the worst
case).  Invariants at the end: a vertex in community y != itself has y's own
vertex still in y (otherwise the sub-community is held together only by a
vertex outside it), and every community's total is the sum of its members'
K'.  A departure marker of 0 admits an interleaving that breaks both (a
second joiner's add, not yet undone, hides the 0 from a third); a marker far
below any sum of degrees admits none.
"""
from __future__ import annotations

K = {"i": 3, "j": 5, "k": 7, "m": 2}
END = -1


def joiner_step(pc, v, target, loc, Sig, C, mark, has_left):
    """One atomic step of vertex v joining `target`; returns the next pc."""
    if pc == 0:                      # leave v's own community only while isolated
        if Sig[v] != K[v]:
            return END
        Sig[v] = mark
        return 1
    if pc == 1:                      # add K'[v] to the target, remember what was there
        loc["prev"] = Sig[target]
        Sig[target] += K[v]
        return 2
    if pc == 2:
        if has_left(loc["prev"]):    # the target's own vertex has left: undo
            Sig[target] -= K[v]
            return 3
        C[v] = target
        return END
    if pc == 3:
        Sig[v] += K[v] - mark
        return END
    raise AssertionError(pc)


def final_states(mark, has_left):
    threads = (("j", "k"), ("i", "j"), ("m", "j"))
    out = []

    def dfs(Sig, C, pcs, locs):
        live = [t for t in range(len(threads)) if pcs[t] != END]
        if not live:
            out.append((Sig, C))
            return
        for t in live:
            Sig2, C2 = dict(Sig), dict(C)
            locs2 = [dict(x) for x in locs]
            pcs2 = list(pcs)
            v, target = threads[t]
            pcs2[t] = joiner_step(pcs[t], v, target, locs2[t], Sig2, C2, mark, has_left)
            dfs(Sig2, C2, pcs2, locs2)

    dfs(dict(K), {v: v for v in K}, [0, 0, 0], [{}, {}, {}])
    return out


def violations(states, mark):
    bad = []
    for Sig, C in states:
        for v, y in C.items():
            if y != v and C[y] != y:
                bad.append(("member of a community whose own vertex left", v, y))
        for y in K:
            if C[y] == y:
                want = sum(K[v] for v in K if C[v] == y)
                if Sig[y] != want:
                    bad.append(("total", y, Sig[y], want))
            elif Sig[y] not in (0, mark):
                bad.append(("departed total", y, Sig[y]))
    return bad


def test_zero_marker_admits_a_disconnected_sub_community():
    states = final_states(0, lambda prev: prev == 0)
    assert len(states) > 100
    assert any(b[0].startswith("member") for b in violations(states, 0))


def test_negative_marker_admits_none():
    mark = -(1 << 62)
    states = final_states(mark, lambda prev: prev < 0)
    assert len(states) > 100
    assert violations(states, mark) == []
    # and in some interleavings each joiner does get in (j stays, or i/m join)
    assert any(C["i"] == "j" for _, C in states) and any(C["j"] == "k" for _, C in states)
