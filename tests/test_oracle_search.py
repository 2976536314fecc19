"""Pins of the oracle's CB-DFS, IDA* and BTS against BFS distances, closed-form tree counts
and the theorem's properties."""
import numpy as np
import pytest

import workloads as W


def _c0_starts(orc, n=20):
    return [orc.stp_apply_walk(3, W.stp_walk(3, 60, W.seed_for(W.TAG_C0, i))) for i in range(n)]


def _rank(orc, s):
    return orc.perm_rank([(s >> (4 * p)) & 15 for p in range(9)])


def test_ida_md_cost_equals_bfs_distance(orc):
    dist, _, _ = orc.stp3_bfs()
    starts = _c0_starts(orc) + [int(x) for x in W.random_stp_states(3, 30, 3)]
    for s in starts:
        r = orc.ida_star(orc.DOM_STP3, s, orc.Heur(orc.H_MD))
        assert r["cost"] == dist[_rank(orc, s)]
        # the path is legal and reaches the goal
        t = s
        for d in r["path"]:
            t = orc.stp_apply(t, 3, d)
        assert t == orc.stp_goal(3) and len(r["path"]) == r["cost"]


def test_ida_zero_heuristic_is_bfs_on_tiny_instances(orc):
    dist, _, _ = orc.stp3_bfs()
    for i in range(10):
        s = orc.stp_apply_walk(3, W.stp_walk(3, 9, 500 + i))
        r = orc.ida_star(orc.DOM_STP3, s, orc.Heur(orc.H_ZERO))
        assert r["cost"] == dist[_rank(orc, s)]


def test_cbdfs_counts_closed_form_rc_zero_heuristic(orc):
    # With h = 0 and a start far from the goal, every canonical sequence of length <= B is
    # expanded and every one of length B+1 is generated: expanded = sum_{d<=B} T(d),
    # generated = sum_{1<=d<=B+1} T(d), T = 1, 18, 243, 3240, 43254.
    T = [1, 18, 243, 3240, 43254]
    start = orc.rc_apply_seq(W.rc_scramble(16, 99))
    for B in range(0, 4):
        r = orc.cbdfs(orc.DOM_RC3, start, B, orc.Heur(orc.H_ZERO), -1, True)
        assert r.expanded == sum(T[:B + 1])
        assert r.generated == sum(T[1:B + 2])
        assert not r.found and r.minf == B + 1


def test_bound_test_is_inclusive(orc):
    # One blank move from the goal: h(root) = 1 = bound, so the first iteration expands the
    # root (f = 1 <= 1) and reaches the goal child with f = 1 (a strict < would not).
    s = orc.stp_apply_walk(3, [W.DIR_DOWN])
    r = orc.ida_star(orc.DOM_STP3, s, orc.Heur(orc.H_MD))
    assert r["cost"] == 1
    assert r["iters"][0][0] == 1 and r["iters"][0][1] == 1 and len(r["iters"]) == 1


def test_goal_start(orc):
    r = orc.ida_star(orc.DOM_STP4, orc.stp_goal(4), orc.Heur(orc.H_MD))
    assert r["cost"] == 0 and r["iters"] == [(0, 0, 0)]


def test_expansion_limit_cuts(orc):
    s = _c0_starts(orc, 1)[0]
    full = orc.cbdfs(orc.DOM_STP3, s, 20, orc.Heur(orc.H_MD), -1, True)
    cut = orc.cbdfs(orc.DOM_STP3, s, 20, orc.Heur(orc.H_MD), 10, True)
    assert full.expanded > 10 and cut.cut and cut.expanded == 10


def test_stronger_admissible_heuristic_expands_a_subset(orc):
    # Theorem, property 2: h1 <= h2 <= h* gives, at every bound, a tree with h2 inside the
    # tree with h1.  The additive 4-4 PDB dominates Manhattan distance on the 8-puzzle.
    pdb = orc.PDB(3, [[1, 2, 3, 4], [5, 6, 7, 8]],
                  [orc.pdb_build(3, [1, 2, 3, 4]), orc.pdb_build(3, [5, 6, 7, 8])])
    for s in _c0_starts(orc, 8):
        h_md, h_pdb = orc.Heur(orc.H_MD), orc.Heur(orc.H_PDB, pdb=pdb)
        for B in range(orc.stp_md(s, 3), 24, 2):
            a = orc.cbdfs(orc.DOM_STP3, s, B, h_md, -1, True)
            b = orc.cbdfs(orc.DOM_STP3, s, B, h_pdb, -1, True)
            assert b.expanded <= a.expanded and b.generated <= a.generated
        assert orc.ida_star(orc.DOM_STP3, s, h_pdb)["cost"] == \
            orc.ida_star(orc.DOM_STP3, s, h_md)["cost"]


def test_callback_heuristic_matches_builtin(orc):
    s = _c0_starts(orc, 3)[2]
    md = orc.Heur(orc.H_MD)
    cb = orc.Heur(fn=lambda w: orc.stp_md(w[0], 3))
    a, b = orc.ida_star(orc.DOM_STP3, s, md), orc.ida_star(orc.DOM_STP3, s, cb)
    assert a == b


def test_bts_cost_equals_ida_cost(orc):
    for s in _c0_starts(orc, 20):
        ida = orc.ida_star(orc.DOM_STP3, s, orc.Heur(orc.H_MD))
        for n0 in (1, 10, 10000):
            b = orc.bts(orc.DOM_STP3, s, orc.Heur(orc.H_MD), n0=n0)
            assert b["cost"] == ida["cost"]


def test_bts_with_a_real_valued_like_heuristic(orc):
    # A heuristic with many distinct values (MD scaled by 7) makes IDA* take many small
    # iterations; BTS must still return IDA*'s cost, in fewer searches than IDA* iterations
    # once the growth base is small.
    s = orc.rc_apply_seq(W.rc_scramble(5, 1234))
    # admissible on RC: 0 (tree small at depth 5)
    h0 = orc.Heur(orc.H_ZERO)
    ida = orc.ida_star(orc.DOM_RC3, s, h0)
    b = orc.bts(orc.DOM_RC3, s, h0, n0=1)
    assert b["cost"] == ida["cost"] <= 5


@pytest.mark.slow
def test_ida_pdb_cost_equals_md_cost_on_15_puzzle(orc):
    pdb = orc.PDB(4, [[10, 11, 15]], [orc.pdb_build(4, [10, 11, 15])])
    for i in range(3):
        s = orc.stp_apply_walk(4, W.stp_walk(4, 40, W.seed_for(W.TAG_C1, 1000 + i)))
        a = orc.ida_star(orc.DOM_STP4, s, orc.Heur(orc.H_MD))
        # max(MD, a 3-tile PDB) is admissible too; the callback takes the max
        hmax = orc.Heur(fn=lambda w: max(orc.stp_md(w[0], 4), pdb.h(w[0])))
        b = orc.ida_star(orc.DOM_STP4, s, hmax)
        assert a["cost"] == b["cost"]


def test_stored_c0_values_are_bfs_consistent():
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c0_ida_md.json")))
    assert len(gold["instances"]) == 20
    for row in gold["instances"]:
        assert row["cost"] == row["bfs"]
        bounds = [it[0] for it in row["iters"]]
        assert bounds == sorted(bounds) and bounds[-1] == row["cost"]
