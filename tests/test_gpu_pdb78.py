"""The paper's 7-8 additive PDB of the 15-puzzle (tiles 1-7 and 8-15; 57,657,600 and 518,918,400
entries), built by the GPU builder.  The oracle cannot build tables this size in a test, so:

- every entry within distance 11 of the goal is compared with the oracle's search stopped
  after level 11 (pdb_ball: ~146k and ~228k placements, ranks up to 5.1e8), and no other entry
  of the table is <= 11;
- the goal placement is the one and only entry 0, and every placement is reached (no 255);
- each table dominates the Manhattan distance of its own tiles, and a blank move that
  slides a tile of the other pattern leaves the entry unchanged;
- IDA* with the sum finds the cost IDA* with Manhattan distance finds (oracle).

The gather over these tables is compared with the oracle's lookup of the same tables."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2507_11916_b300 as P
    return P


@pytest.fixture(scope="module")
def built(P):
    ctx = P.cbdfs_create(0, max_batch=1 << 16, n_slots=2)
    pats = [list(p) for p in W.PATTERNS_78]
    tabs = [P.pdb_build(ctx, P.DOM_STP4, t) for t in pats]
    ids = [P.cbdfs_pdb_load(ctx, P.DOM_STP4, [p], [t]) for p, t in zip(pats, tabs)]
    both = P.cbdfs_pdb_load(ctx, P.DOM_STP4, pats, tabs)
    yield ctx, pats, tabs, ids, both
    P.cbdfs_destroy(ctx)


def _h(P, ctx, hid, states):
    return P.heur_submit_batch(ctx, hid, P.DOM_STP4, states, np.zeros(len(states), np.uint8), 255)[0].astype(int)


def _md_of(states, tiles):
    tot = np.zeros(len(states), dtype=int)
    for cell in range(16):
        t = ((states >> np.uint64(4 * cell)) & np.uint64(15)).astype(int)
        d = np.abs(cell // 4 - t // 4) + np.abs(cell % 4 - t % 4)
        tot += np.where(np.isin(t, tiles), d, 0)
    return tot


def test_sizes_goal_and_reachability(built, orc):
    _, pats, tabs, _, _ = built
    assert [len(t) for t in tabs] == [57_657_600, 518_918_400]
    for p, t in zip(pats, tabs):
        goal_rank = orc.pdb_rank(p, 16)  # tile t sits on cell t in the goal
        assert t[goal_rank] == 0
        assert np.count_nonzero(t == 0) == 1
        assert t.max() < 255


def test_dominates_manhattan_and_matches_oracle_lookup(P, built, orc):
    ctx, pats, tabs, ids, both = built
    states = W.random_stp_states(4, 50000, 7878)
    hs = [_h(P, ctx, i, states) for i in ids]
    for p, h in zip(pats, hs):
        assert (h >= _md_of(states, p)).all()
    hb = _h(P, ctx, both, states)
    assert np.array_equal(hb, np.minimum(hs[0] + hs[1], 255))
    ref = orc.PDB(4, pats, tabs)
    for i in range(0, 50000, 97):
        assert hb[i] == ref.h(int(states[i]))


def test_entries_near_the_goal_match_oracle(built, orc):
    _, pats, tabs, _, _ = built
    for p, t in zip(pats, tabs):
        ranks, vals = orc.pdb_ball(4, p, 11)
        assert np.array_equal(t[ranks], vals)
        assert np.count_nonzero(t <= 11) == len(ranks)


def test_moves_of_other_tiles_leave_entries_unchanged(P, built):
    ctx, pats, _, ids, _ = built
    s = W.random_stp_states(4, 20000, 4242)
    h0 = [_h(P, ctx, i, s) for i in ids]
    blank = np.zeros(len(s), dtype=int)
    for cell in range(16):
        blank = np.where(((s >> np.uint64(4 * cell)) & np.uint64(15)) == 0, cell, blank)
    for dr, dc in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        r, c = blank // 4 + dr, blank % 4 + dc
        ok = (r >= 0) & (r < 4) & (c >= 0) & (c < 4)
        src, b, o = s[ok], blank[ok], (r * 4 + c)[ok]
        tile = (src >> (4 * o).astype(np.uint64)) & np.uint64(15)
        # the tile on cell o slides onto the blank's cell b
        nxt = (src & ~(np.uint64(15) << (4 * o).astype(np.uint64))) | (tile << (4 * b).astype(np.uint64))
        h1 = [_h(P, ctx, i, nxt) for i in ids]
        tile = tile.astype(int)
        for q, p in enumerate(pats):
            other = ~np.isin(tile, p)
            assert np.array_equal(h1[q][other], h0[q][ok][other])


def test_admissible_and_optimal_cost(P, built, orc):
    ctx, _, _, _, both = built
    for i in range(3):
        walk = W.stp_walk(4, 45, W.seed_for(W.TAG_C1, 9000 + i))
        s = orc.stp_apply_walk(4, walk)
        want = orc.ida_star(orc.DOM_STP4, s, orc.Heur(orc.H_MD))["cost"]
        h = _h(P, ctx, both, np.array([s], np.uint64))[0]
        assert h <= want
        r = P.cbdfs_solve(ctx, P.DOM_STP4, s, P.ALGO_IDA, both, threads=4, work_num=8, batch=1024,
                          timeout_us=200, time_limit_s=60)
        assert r["cost"] == want
