"""Pins of the oracle's pattern databases: the all-tiles special case is BFS, additive PDBs
are admissible and dominate Manhattan distance, ranks are a bijection."""
import itertools

import numpy as np
import pytest

import workloads as W


def test_rank_is_a_bijection(orc):
    for n, k in ((5, 2), (6, 3), (7, 7)):
        ranks = sorted(orc.pdb_rank(p, n) for p in itertools.permutations(range(n), k))
        assert ranks == list(range(orc.npk(n, k)))
    # lexicographic: the first placement is rank 0, the last is P-1
    assert orc.pdb_rank([0, 1, 2], 16) == 0
    assert orc.pdb_rank([15, 14, 13], 16) == 16 * 15 * 14 - 1


def test_all_tile_pdb_is_bfs(orc):
    # With every tile in the pattern the abstraction is the puzzle itself.
    dist, _, _ = orc.stp3_bfs()
    tab = orc.pdb_build(3, list(range(1, 9)))
    for perm in itertools.islice(itertools.permutations(range(9)), 0, 362880, 7):
        d = dist[orc.perm_rank(perm)]
        pos = [perm.index(t) for t in range(1, 9)]
        e = tab[orc.pdb_rank(pos, 9)]
        if d >= 0:
            assert e == d
        else:
            assert e == 255


def test_additive_pdb_admissible_and_dominates_md(orc):
    dist, _, _ = orc.stp3_bfs()
    pats = [[1, 2, 3, 4], [5, 6, 7, 8]]
    pdb = orc.PDB(3, pats, [orc.pdb_build(3, p) for p in pats])
    for perm in itertools.islice(itertools.permutations(range(9)), 0, 362880, 11):
        d = dist[orc.perm_rank(perm)]
        if d < 0:
            continue
        s = W.stp_pack(perm)
        h = pdb.h(s)
        assert orc.stp_md(s, 3) <= h <= d


def test_15_puzzle_small_pattern(orc):
    tab = orc.pdb_build(4, [10, 11, 15])
    assert tab.shape == (16 * 15 * 14,)
    assert (tab < 255).all()
    assert tab[orc.pdb_rank([10, 11, 15], 16)] == 0
    # each entry is at least the pattern tiles' Manhattan distance
    for pos in itertools.islice(itertools.permutations(range(16), 3), 0, 3360, 3):
        md = sum(abs(p // 4 - t // 4) + abs(p % 4 - t % 4) for p, t in zip(pos, [10, 11, 15]))
        assert tab[orc.pdb_rank(list(pos), 16)] >= md


@pytest.mark.slow
def test_663_six_tile_table_shape(orc):
    tab = orc.pdb_build(4, [1, 2, 3, 5, 6, 7])
    assert tab.shape == (5765760,)
    assert (tab < 255).all() and tab[orc.pdb_rank([1, 2, 3, 5, 6, 7], 16)] == 0
    assert tab.max() <= 80


@pytest.mark.parametrize("side,tiles,maxd", [(3, [1, 2, 3, 4], 40), (3, [5, 6, 7, 8], 5),
                                             (4, [10, 11, 15], 6), (4, [4, 8, 12, 13], 7),
                                             (4, [1, 2, 4, 5], 4)])
def test_pdb_ball_is_the_table_near_the_goal(orc, side, tiles, maxd):
    # the search stopped after level maxd finds exactly the entries <= maxd of the full table
    # (at maxd 40 the whole 8-puzzle table)
    T = orc.pdb_build(side, tiles)
    ranks, vals = orc.pdb_ball(side, tiles, maxd, cap=1 << 22)
    idx = np.nonzero(T <= maxd)[0]
    assert np.array_equal(ranks, idx)
    assert np.array_equal(vals, T[idx])


# ---- the cube's 8-corner PDB ---------------------------------------------------------------

def test_rc_corner_ball_matches_the_full_table_levels(orc):
    # two independent oracle computations: the ball walks full cube states with or_rc_apply;
    # the stored histogram comes from the full table's own corner-only search
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rc_corner_pdb.json")))
    assert gold["entries"] == orc.RC_CORNER_ENTRIES == 40320 * 2187 == sum(gold["histogram"])
    idx, val = orc.rc_corner_ball(5)
    assert [int((val == d).sum()) for d in range(6)] == gold["histogram"][:6]
    assert len(np.unique(idx)) == len(idx) and idx.min() == 0 and idx.max() < orc.RC_CORNER_ENTRIES
    # sampled entries within the ball agree with the stored table sample
    si, sv = np.array(gold["sample_index"]), np.array(gold["sample_value"])
    pos = np.searchsorted(idx, si)
    inside = (pos < len(idx)) & (idx[np.minimum(pos, len(idx) - 1)] == si)
    assert np.array_equal(val[pos[inside]], sv[inside])
    assert (sv[~inside] > 5).all()


def test_rc_corner_distance_is_admissible_and_consistent(orc):
    idx, val = orc.rc_corner_ball(5)

    def look(s):
        i = orc.rc_corner_index(s)
        p = np.searchsorted(idx, i)
        return int(val[p]) if p < len(idx) and idx[p] == i else None

    assert look(orc.rc_goal()) == 0
    for k in range(40):
        n = 1 + k % 4
        s = orc.rc_apply_seq(W.rc_scramble(n, 900 + k))
        h = look(s)
        assert h is not None and h <= n
        for m in range(18):
            h2 = look(orc.rc_apply(s, m))
            assert h2 is not None and abs(h2 - h) <= 1


def test_rc_corner_index_ignores_edges_and_separates_corners(orc):
    s = orc.rc_apply_seq(W.rc_scramble(6, 4242))
    g = orc.rc_goal()
    assert orc.rc_corner_index((s[0], g[1])) == orc.rc_corner_index(s)
    idx = {orc.rc_corner_index(orc.rc_apply_seq(W.rc_scramble(7, 5000 + k))) for k in range(300)}
    words = {orc.rc_apply_seq(W.rc_scramble(7, 5000 + k))[0] for k in range(300)}
    assert len(idx) == len(words)


# ---- DIV compression -----------------------------------------------------------------------

def test_div_by_hand_and_identity(orc):
    t = np.array([5, 3, 9, 9, 1, 4, 7], np.uint8)
    assert list(orc.pdb_div(t, 2)) == [3, 9, 1, 7]   # the last group holds one entry
    assert list(orc.pdb_div(t, 3)) == [3, 1, 7]
    assert np.array_equal(orc.pdb_div(t, 1), t)
    assert list(orc.pdb_div(t, 7)) == [1]


def test_div_is_a_lower_bound_attained_in_each_group(orc):
    t = orc.pdb_build(3, [1, 2, 3, 4])
    for k in (2, 5, 16):
        d = orc.pdb_div(t, k)
        assert len(d) == -(-len(t) // k)
        assert (d[np.arange(len(t)) // k] <= t).all()
        # every group's value is one of its own entries
        for j in range(0, len(d), 97):
            assert d[j] in t[j * k:(j + 1) * k]


def test_div_heuristic_is_admissible_and_weaker(orc):
    pats = [[1, 2, 3, 4], [5, 6, 7, 8]]
    tabs = [orc.pdb_build(3, p) for p in pats]
    full = orc.PDB(3, pats, tabs)
    dist, _, _ = orc.stp3_bfs()
    for k in (1, 4, 30):
        dt = [orc.pdb_div(t, k) for t in tabs]
        for s in W.random_stp_states(3, 200, 77 + k):
            hd = orc.pdb_div_h(3, pats, dt, k, s)
            assert hd <= full.h(int(s)) <= dist[orc.perm_rank([(int(s) >> (4 * p)) & 15 for p in range(9)])]
            if k == 1:
                assert hd == full.h(int(s))
