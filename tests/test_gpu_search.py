"""Parity of the batched CB-DFS (cbdfs_solve) with the oracle's serial CB-DFS: the same
solution cost and, per completed iteration, the same expanded and generated counts."""
import json
import os

import numpy as np
import pytest

import workloads as W
from helpers import PREC

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c0_ida_md.json")))


@pytest.fixture(scope="module")
def P():
    import paper_2507_11916_b300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.cbdfs_create(0, max_batch=8192, n_slots=4)
    yield c
    P.cbdfs_destroy(c)


def solve(P, ctx, *a, **kw):
    """cbdfs_solve with a time limit, so that a wrong tree cannot run on for long."""
    kw.setdefault("time_limit_s", 60.0)
    return P.cbdfs_solve(ctx, *a, **kw)


def _iters(r):
    return [list(map(int, t)) for t in r["iters"]]


@pytest.mark.parametrize("threads,work_num,d_init,batch", [(4, 8, -1, 256), (1, 1, 0, 64),
                                                          (3, 5, 4, 18), (8, 32, 2, 1024)])
def test_c0_ida_md_counts_match_oracle(P, ctx, threads, work_num, d_init, batch):
    for row in GOLD["instances"]:
        r = solve(P, ctx, P.DOM_STP3, row["state"], P.ALGO_IDA, P.HEUR_MD, threads=threads,
                          work_num=work_num, d_init=d_init, batch=batch, timeout_us=200)
        assert r["cost"] == row["cost"]
        assert _iters(r) == row["iters"]
        # the path is legal and reaches the goal
        assert P.cbdfs_apply_moves(P.DOM_STP3, row["state"], r["path"]) == W.stp_goal(3)
        assert len(r["path"]) == r["cost"]


def test_c0_network_heuristic_and_fixed_tree(P, ctx, orc):
    # The plain-form network: h = max(rint(y), 0, MD).  Evaluated on every node of the tree
    # that Manhattan distance prunes (fixed tree), and used itself for pruning.
    Ws, bs = W.net_weights(**W.NET_C0)
    hid = P.cbdfs_net_load(ctx, P.DOM_STP3, Ws, bs, PREC["fp32"], P.HEAD_REGRESSION, 1)

    def h_nn(w):
        y = orc.mlp_forward(Ws, bs, orc.one_hot(orc.DOM_STP3, [w[0]]))
        return int(orc.h_regression(y[:, 0], orc.md_states(orc.DOM_STP3, [w[0]]))[0])

    for row in GOLD["instances"][:8]:
        want = orc.ida_star(orc.DOM_STP3, row["state"], orc.Heur(fn=h_nn))
        r = solve(P, ctx, P.DOM_STP3, row["state"], P.ALGO_IDA, hid, threads=4, work_num=8,
                          batch=256, timeout_us=200)
        assert r["cost"] == want["cost"]
        assert _iters(r) == [list(t) for t in want["iters"]]
        f = solve(P, ctx, P.DOM_STP3, row["state"], P.ALGO_IDA, hid, threads=4, work_num=8,
                          batch=256, timeout_us=200, fixed_tree_heur=P.HEUR_MD)
        assert _iters(f) == row["iters"]
        # the network ran on every batch (the initial tree is evaluated once and cached)
        assert f["batches"] > 0 and f["evaluated"] >= f["expanded"]


def test_c0_pdb_heuristic(P, ctx, orc):
    pats = [[1, 2, 3, 4], [5, 6, 7, 8]]
    tabs = [orc.pdb_build(3, p) for p in pats]
    hid = P.cbdfs_pdb_load(ctx, P.DOM_STP3, pats, tabs)
    pdb = orc.PDB(3, pats, tabs)
    for row in GOLD["instances"][:10]:
        want = orc.ida_star(orc.DOM_STP3, row["state"], orc.Heur(orc.H_PDB, pdb=pdb))
        r = solve(P, ctx, P.DOM_STP3, row["state"], P.ALGO_IDA, hid, threads=2, work_num=4,
                          batch=128, timeout_us=200)
        assert r["cost"] == want["cost"] == row["cost"]
        assert _iters(r) == [list(t) for t in want["iters"]]


def test_15_puzzle_md_counts(P, ctx, orc):
    for i in range(6):
        s = orc.stp_apply_walk(4, W.stp_walk(4, 36, W.seed_for(W.TAG_C1, 5000 + i)))
        want = orc.ida_star(orc.DOM_STP4, s, orc.Heur(orc.H_MD))
        r = solve(P, ctx, P.DOM_STP4, s, P.ALGO_IDA, P.HEUR_MD, threads=8, work_num=16,
                          batch=2048, timeout_us=300)
        assert r["cost"] == want["cost"]
        assert _iters(r) == [list(t) for t in want["iters"]]


def test_rc_zero_heuristic_counts(P, ctx, orc):
    for i in range(3):
        s = orc.rc_apply_seq(W.rc_scramble(4, W.seed_for(W.TAG_C2, 100 + i)))
        want = orc.ida_star(orc.DOM_RC3, s, orc.Heur(orc.H_ZERO))
        r = solve(P, ctx, P.DOM_RC3, s, P.ALGO_IDA, P.HEUR_ZERO, threads=4, work_num=16,
                          batch=4096, timeout_us=300)
        assert r["cost"] == want["cost"]
        assert _iters(r) == [list(t) for t in want["iters"]]
        assert P.cbdfs_apply_moves(P.DOM_RC3, s, r["path"]) == W.rc_goal()


def test_rc_classifier_fixed_tree(P, ctx, orc):
    # the cube network evaluated at every node of the tree h = 0 prunes
    Ws, bs = W.net_weights(**W.NET_C2)
    hid = P.cbdfs_net_load(ctx, P.DOM_RC3, Ws, bs, PREC["bf16"], P.HEAD_CLASSIFIER, 0)
    s = orc.rc_apply_seq(W.rc_scramble(4, W.seed_for(W.TAG_C2, 7)))
    want = orc.ida_star(orc.DOM_RC3, s, orc.Heur(orc.H_ZERO))
    r = solve(P, ctx, P.DOM_RC3, s, P.ALGO_IDA, hid, threads=8, work_num=16, batch=4096,
                      timeout_us=300, fixed_tree_heur=P.HEUR_ZERO)
    assert r["cost"] == want["cost"] and _iters(r) == [list(t) for t in want["iters"]]
    assert r["batches"] > 0 and r["evaluated"] >= r["expanded"]
    # every search batch is in exactly one size class of the histogram
    assert sum(r["batch_hist"]) == r["batches"] and len(r["batch_hist"]) == 16


@pytest.mark.parametrize("n0", [1, 10, 10000])
def test_bts_matches_oracle_schedule(P, ctx, orc, n0):
    for row in GOLD["instances"][:10]:
        want = orc.bts(orc.DOM_STP3, row["state"], orc.Heur(orc.H_MD), n0=n0)
        r = solve(P, ctx, P.DOM_STP3, row["state"], P.ALGO_BTS, P.HEUR_MD, threads=4,
                          work_num=8, batch=256, timeout_us=200, bts_n0=n0)
        assert r["cost"] == want["cost"] == row["cost"]
        got = [(b, lim, e, g, c) for (b, e, g), lim, c in zip(r["iters"], r["iter_limit"], r["iter_cut"])]
        exp = [(b, lim, e, g, c) for (b, lim, e, g, c, _f) in want["searches"]]
        assert [(b, lim, c) for b, lim, _, _, c in got] == [(b, lim, c) for b, lim, _, _, c in exp]
        for a, b in zip(got, exp):
            if not a[4]:  # uncut searches expand exactly the oracle's tree
                assert a[2:4] == b[2:4]


def test_solve_errors(P, ctx):
    with pytest.raises(P.CbdfsError):
        solve(P, ctx, P.DOM_RC3, W.rc_goal(), P.ALGO_IDA, P.HEUR_MD)
    with pytest.raises(P.CbdfsError):
        solve(P, ctx, P.DOM_STP3, W.stp_goal(3), P.ALGO_IDA, P.HEUR_MD, threads=0)
    r = solve(P, ctx, P.DOM_STP3, W.stp_goal(3), P.ALGO_IDA, P.HEUR_MD)
    assert r["cost"] == 0 and r["iters"] == [(0, 0, 0)]


def test_node_limit_stops(P, ctx, orc):
    s = orc.stp_apply_walk(4, W.stp_walk(4, 200, W.seed_for(W.TAG_C1, 0)))
    with pytest.raises(P.CbdfsError) as e:
        solve(P, ctx, P.DOM_STP4, s, P.ALGO_IDA, P.HEUR_MD, threads=4, work_num=8,
                      batch=1024, node_limit=20000)
    assert e.value.status == P.CBDFS_ECANCELED
