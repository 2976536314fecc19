"""Pins of the oracle's real-valued CB-DFS, IDA* and BTS (section "Regression-Based Neural
Heuristics": a regression network's h is real, f = g + h is real, IDA*'s next threshold is
the least real f above the bound).

- With an integer-valued h the real search is the integer search (`cbdfs`, pinned by
  BFS distances and closed-form counts in test_oracle_search.py), bound for bound.
- Shifting Manhattan distance down by 1/2 on every non-goal state moves each IDA* bound by
  exactly -1/2 and keeps every iteration's node counts; only the last bound reappears once
  unshifted (the goal's f = g is not shifted).
- Admissible real heuristics on the 8-puzzle give the BFS distance with IDA* and BTS.
- The heuristic rule and the bound test in float64 against values worked by hand."""
import math

import numpy as np

import workloads as W


def _c0_starts(orc, n=20):
    return [orc.stp_apply_walk(3, W.stp_walk(3, 60, W.seed_for(W.TAG_C0, i))) for i in range(n)]


def _rank(orc, s):
    return orc.perm_rank([(s >> (4 * p)) & 15 for p in range(9)])


def _md_real(orc, side, scale=1.0, shift=0.0):
    return orc.HeurReal(lambda w: max(scale * orc.stp_md(w[0], side) + shift, 0.0))


def test_integer_valued_h_gives_the_integer_search(orc):
    md, mdr = orc.Heur(orc.H_MD), _md_real(orc, 4)
    for i in range(6):
        s = orc.stp_apply_walk(4, W.stp_walk(4, 40, W.seed_for(W.TAG_C1, 700 + i)))
        b0 = orc.stp_md(s, 4)
        for b in (b0, b0 + 2, b0 + 6):
            for limit in (-1, 50, 2000):
                a = orc.cbdfs(orc.DOM_STP4, s, b, md, limit)
                r = orc.cbdfs_real(orc.DOM_STP4, s, float(b), mdr, limit)
                assert (a.expanded, a.generated, a.found, a.cost, a.cut) == \
                    (r.expanded, r.generated, r.found, r.cost, r.cut)
                assert (a.minf < 0 and r.minf < 0) or a.minf == r.minf
                assert list(a.path[:a.path_len]) == list(r.path[:r.path_len])


def test_half_shift_moves_every_bound_by_one_half(orc):
    half = _md_real(orc, 4, shift=-0.5)  # non-goal states have MD >= 1
    for i in range(5):
        s = orc.stp_apply_walk(4, W.stp_walk(4, 36, W.seed_for(W.TAG_C1, 800 + i)))
        a = orc.ida_star(orc.DOM_STP4, s, orc.Heur(orc.H_MD))
        r = orc.ida_star_real(orc.DOM_STP4, s, half)
        K = len(a["iters"])
        assert r["cost"] == a["cost"]
        # every iteration before the last: bound - 1/2, the same counts
        for (b, e, g), (rb, re, rg) in zip(a["iters"][:-1], r["iters"]):
            assert rb == b - 0.5 and (re, rg) == (e, g)
        bK, eK, gK = a["iters"][-1]
        tail = r["iters"][K - 1:]
        # the last integer bound is reached either shifted and then unshifted (the least f
        # above bK - 1/2 is the goal's g = bK), or directly when only a goal set it
        assert tail in ([(bK - 0.5, eK, gK), (float(bK), eK, gK)], [(float(bK), eK, gK)])


def test_admissible_real_heuristics_give_bfs_distances(orc):
    dist, _, _ = orc.stp3_bfs()
    starts = _c0_starts(orc, 8) + [int(x) for x in W.random_stp_states(3, 4, 11)]
    for scale, shift in ((0.75, -0.25), (1.0, -2.2), (0.9, 0.05)):
        h = _md_real(orc, 3, scale, shift)
        for s in starts:
            want = dist[_rank(orc, s)]
            r = orc.ida_star_real(orc.DOM_STP3, s, h)
            assert r["cost"] == want
            t = s
            for d in r["path"]:
                t = orc.stp_apply(t, 3, d)
            assert t == orc.stp_goal(3)
            for n0 in (1, 50):
                assert orc.bts_real(orc.DOM_STP3, s, h, n0=n0)["cost"] == want


def test_real_bts_accepts_the_integer_bts_bounds_for_integer_h(orc):
    md, mdr = orc.Heur(orc.H_MD), _md_real(orc, 3)
    for s in _c0_starts(orc, 10):
        for n0 in (1, 20):
            a = orc.bts(orc.DOM_STP3, s, md, n0=n0)
            r = orc.bts_real(orc.DOM_STP3, s, mdr, n0=n0)
            assert r["cost"] == a["cost"]
            # the unlimited searches are the accepted cut ones: the same bounds, same counts
            ua = [(b, e, g) for b, lim, e, g, c, f in a["searches"] if lim < 0]
            ur = [(b, e, g) for b, lim, e, g, c, f in r["searches"] if lim < 0]
            assert ur == [(float(b), e, g) for b, e, g in ua]
            # the search that ends both runs
            assert r["searches"][-1][2:] == a["searches"][-1][2:]


def test_real_valued_h_makes_ida_reexpand_more_than_bts(orc):
    # many distinct f-costs (MD scaled by 0.37): IDA* moves its bound by small steps (86
    # iterations for a cost-20 instance) and re-expands the tree each time; BTS picks bounds
    # whose node counts grow geometrically and expands fewer nodes in all
    h = _md_real(orc, 3, 0.37, -0.1)
    s = _c0_starts(orc, 1)[0]
    ida = orc.ida_star_real(orc.DOM_STP3, s, h)
    bts = orc.bts_real(orc.DOM_STP3, s, h, n0=100)
    assert bts["cost"] == ida["cost"] == 20
    assert len(ida["iters"]) > 4 * 20
    assert sum(x[2] for x in bts["searches"]) < 0.8 * sum(x[1] for x in ida["iters"])


def test_h_real_rule_and_bound_test_by_hand(orc):
    y = np.array([3.7, 1.0, -5.0, 10.2, 7.0])
    md = np.array([4, 1, 3, 0, 6])
    goal = np.array([False, False, False, True, False])
    h = orc.h_real(y, -2.2, md=md, goal=goal)
    # 3.7-2.2 = 1.5 < MD 4; 1.0-2.2 < 0 -> 0, max MD 1; -7.2 -> 0, MD 3; goal 0; 4.8 < 6
    assert np.allclose(h, [4.0, 1.0, 3.0, 0.0, 6.0])
    h2 = orc.h_real(y, -2.2)
    assert np.allclose(h2, [1.5, 0.0, 0.0, 8.0, 4.8])
    g = np.array([10, 0, 2, 1, 3], np.uint8)
    words, minf = orc.bound_test_real(g, h2, 4.8)
    # f = 11.5, 0, 2, 9, 7.8 -> pass: 1, 2 -> bits 0b00110; least f above 4.8 is 7.8
    assert int(words[0]) == 0b00110 and abs(minf - 7.8) < 1e-12
    words, minf = orc.bound_test_real(g, h2, 100.0)
    assert int(words[0]) == 0b11111 and math.isinf(minf)
