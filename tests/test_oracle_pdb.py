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
