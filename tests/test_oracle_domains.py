"""Pins of the oracle's domain code against facts the domains themselves fix."""
import json
import os

import numpy as np

import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "domain_facts.json")))


def test_stp3_bfs_counts(orc):
    dist, reached, maxd = orc.stp3_bfs()
    assert reached == GOLD["stp3_reachable"] == 362880 // 2
    assert maxd == GOLD["stp3_max_distance"]
    assert (dist >= 0).sum() == reached


def test_rc_bfs_depth_counts(orc):
    distinct, tree = orc.rc_bfs_counts(4)
    assert list(distinct) == GOLD["rc_distinct_by_depth"]
    assert list(tree) == GOLD["rc_canonical_sequences_by_depth"]


def test_rc_canonical_counts_closed_form(orc):
    # a = sequences per low face (U R F), b = per high face (D L B):
    # a' = 3(2a + 2b), b' = 3(3a + 2b), a = b = 3 at depth 1.
    a = b = 3
    want = [18]
    for _ in range(3):
        a, b = 3 * (2 * a + 2 * b), 3 * (3 * a + 2 * b)
        want.append(3 * a + 3 * b)
    _, tree = orc.rc_bfs_counts(4)
    assert list(tree[1:]) == want


def _rc_order(orc, seq):
    g = orc.rc_goal()
    s = g
    for k in range(1, 2000):
        for m in seq:
            s = orc.rc_apply(s, m)
        if s == g:
            return k
    return None


def test_rc_group_orders(orc):
    R, U = 3 * 1, 3 * 0
    Ri, Ui = 3 * 1 + 2, 3 * 0 + 2
    for f in range(6):
        assert _rc_order(orc, [3 * f]) == 4
        assert _rc_order(orc, [3 * f + 1]) == 2
    assert _rc_order(orc, [R, U]) == GOLD["rc_order_R_U"]
    assert _rc_order(orc, [R, U, Ri, Ui]) == GOLD["rc_order_R_U_Rinv_Uinv"]


def test_rc_inverse_and_commuting_opposites(orc):
    rng = W.SplitMix64(7)
    for _ in range(50):
        s = orc.rc_apply_seq(W.rc_scramble(10, rng.next()))
        for m in range(18):
            inv = 3 * (m // 3) + (2 - m % 3)
            assert orc.rc_apply(orc.rc_apply(s, m), inv) == s
        for f in range(3):
            a = orc.rc_apply(orc.rc_apply(s, 3 * f), 3 * (f + 3))
            b = orc.rc_apply(orc.rc_apply(s, 3 * (f + 3)), 3 * f)
            assert a == b


def test_rc_invariants_hold_on_scrambles_and_random_states(orc):
    for i in range(50):
        s = orc.rc_apply_seq(W.rc_scramble(14 + i % 3, W.seed_for(W.TAG_C2, i)))
        assert orc.rc_invariants(s) == 0
    for s in W.random_rc_states(500, 11):
        assert orc.rc_invariants(tuple(int(x) for x in s)) == 0
    # a single twisted corner, a single flipped edge and a lone swap all break one
    g = list(orc.rc_goal())
    assert orc.rc_invariants((g[0] + 1, g[1])) & 1
    assert orc.rc_invariants((g[0], g[1] + 1)) & 2
    swapped = (g[0] ^ ((0 ^ 3) << 0) ^ ((3 ^ 0) << 5), g[1])  # corners 0,1 trade slots
    assert orc.rc_invariants(swapped) & 4


def test_stp_moves_and_md(orc):
    for side in (3, 4):
        goal = orc.stp_goal(side)
        assert orc.stp_md(goal, side) == 0
        for i in range(20):
            s = orc.stp_apply_walk(side, W.stp_walk(side, 50, 100 + i))
            for d in range(4):
                c = orc.stp_apply(s, side, d)
                if c is None:
                    continue
                assert orc.stp_apply(c, side, 3 - d) == s
                assert abs(orc.stp_md(c, side) - orc.stp_md(s, side)) == 1
                cells = sorted((c >> (4 * p)) & 15 for p in range(side * side))
                assert cells == list(range(side * side))


def test_random_stp_states_are_reachable(orc):
    dist, _, _ = orc.stp3_bfs()
    for s in W.random_stp_states(3, 300, 5):
        cells = [(int(s) >> (4 * p)) & 15 for p in range(9)]
        assert dist[orc.perm_rank(cells)] >= 0


def test_walks_match_the_packed_goal_and_format(orc):
    assert orc.stp_goal(4) == W.stp_goal(4)
    assert orc.rc_goal() == W.rc_goal()
    # one blank move right from the 3x3 goal swaps cells 0 and 1
    s = orc.stp_apply_walk(3, [W.DIR_RIGHT])
    assert W.stp_cells(s, 3)[:2] == [1, 0]
    assert orc.stp_md(s, 3) == 1
