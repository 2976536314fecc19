"""The cube's 8-corner PDB (Experimental Setup: the cube's h_PDB; section "Fixed-Tree
Evaluation": it prunes while the network is evaluated on every node), built on the GPU.

- the table against the oracle's full breadth-first table: its histogram (all 12 levels) and
  2,000 seeded entries (stored by tests/golden/make_golden.py from the oracle alone), and
  every entry within 6 turns of the solved corners against the oracle's bounded search;
- the gather: h = table[the oracle's index of the state], 0 at the goal, the bound test;
  consistency (a face turn changes h by at most 1);
- IDA* pruned by the table matches the oracle's serial IDA* count for count, and the
  fixed-tree search that evaluates the cube network on every node searches that same tree."""
import json
import os

import numpy as np
import pytest

import workloads as W
from helpers import PREC, fp8_act_scales

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rc_corner_pdb.json")))


@pytest.fixture(scope="module")
def P():
    import paper_2507_11916_b300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.cbdfs_create(0, max_batch=8192, n_slots=3)
    yield c
    P.cbdfs_destroy(c)


@pytest.fixture(scope="module")
def table(P, ctx):
    return P.pdb_build(ctx, P.DOM_RC3, list(range(8)))


@pytest.fixture(scope="module")
def pid(P, ctx):
    return P.cbdfs_pdb_load(ctx, P.DOM_RC3, [list(range(8))])  # built on the device


def test_table_matches_the_oracle(orc, table):
    assert len(table) == GOLD["entries"] == 88_179_840
    assert np.bincount(table, minlength=len(GOLD["histogram"])).tolist() == GOLD["histogram"]
    assert np.array_equal(table[np.array(GOLD["sample_index"])], np.array(GOLD["sample_value"], np.uint8))


def test_entries_near_the_solved_corners(orc, table):
    idx, val = orc.rc_corner_ball(6)
    assert np.array_equal(table[idx], val)
    assert np.count_nonzero(table <= 6) == len(idx)


def _g(n, seed, hi=14):
    return (W.splitmix64_array(seed, n) % np.uint64(hi)).astype(np.uint8)


@pytest.mark.parametrize("n", [1, 31, 129, 1000, 8192])
def test_gather(P, ctx, orc, table, pid, n):
    s = W.random_rc_states(n, 2100 + n)
    s[0] = W.rc_goal()
    if n > 2:
        s[1] = orc.rc_apply_seq(W.rc_scramble(3, 2200 + n))
    g = _g(n, 2300 + n)
    h, mask, minf = P.heur_submit_batch(ctx, pid, P.DOM_RC3, s.reshape(-1), g, 12)
    want = np.array([table[orc.rc_corner_index(tuple(map(int, w)))] for w in s], np.int64)
    want[orc.is_goal_states(orc.DOM_RC3, s.reshape(-1))] = 0
    assert np.array_equal(h, want)
    wm, wf = orc.bound_test(g, want, 12)
    assert np.array_equal(mask, wm) and minf == wf


def test_consistent_under_face_turns(P, ctx, orc, pid):
    s = W.random_rc_states(300, 2400)
    h0 = P.heur_submit_batch(ctx, pid, P.DOM_RC3, s.reshape(-1), np.zeros(300, np.uint8), 255)[0].astype(int)
    for m in range(18):
        t = np.array([orc.rc_apply(tuple(map(int, w)), m) for w in s], np.uint64)
        h1 = P.heur_submit_batch(ctx, pid, P.DOM_RC3, t.reshape(-1), np.zeros(300, np.uint8), 255)[0].astype(int)
        assert (np.abs(h1 - h0) <= 1).all()


def test_errors(P, ctx):
    import torch
    with pytest.raises(P.CbdfsError):  # the cube takes the eight corners only
        P.cbdfs_pdb_load(ctx, P.DOM_RC3, [list(range(7))])
    dev = torch.device("cuda", 0)
    buf = torch.zeros(2 * 65, dtype=torch.int64, device=dev)
    dg = torch.zeros(64, dtype=torch.uint8, device=dev)
    dh = torch.empty(64, dtype=torch.uint8, device=dev)
    dm = torch.empty(2, dtype=torch.int32, device=dev)
    dmin = torch.empty(1, dtype=torch.int32, device=dev)
    with pytest.raises(P.CbdfsError):  # cube states off a 16-byte boundary are refused
        P.heur_eval_device(ctx, P.HEUR_ZERO, P.DOM_RC3, buf[1:], dg, 5, 64, dh, dm, dmin)


def _starts(orc, k, moves=7):
    return [orc.rc_apply_seq(W.rc_scramble(moves, W.seed_for(W.TAG_C2, 300 + i))) for i in range(k)]


def test_ida_with_the_corner_table_and_the_fixed_tree(P, ctx, orc, table, pid):
    href = orc.Heur(fn=lambda w: int(table[orc.rc_corner_index(w)]))
    Ws, bs = W.net_weights(**W.NET_C2)
    nid = P.cbdfs_net_load(ctx, P.DOM_RC3, Ws, bs, PREC["bf16"], P.HEAD_CLASSIFIER, 0)
    for s in _starts(orc, 3):
        want = orc.ida_star(orc.DOM_RC3, s, href)
        r = P.cbdfs_solve(ctx, P.DOM_RC3, s, P.ALGO_IDA, pid, threads=4, work_num=16, batch=2048,
                          timeout_us=200, time_limit_s=60.0)
        assert r["cost"] == want["cost"] <= 7
        assert [tuple(map(int, t)) for t in r["iters"]] == [tuple(t) for t in want["iters"]]
        # the network on every node, the table pruning: the same tree
        f = P.cbdfs_solve(ctx, P.DOM_RC3, s, P.ALGO_IDA, nid, threads=4, work_num=16, batch=2048,
                          timeout_us=200, time_limit_s=60.0, fixed_tree_heur=pid)
        assert f["cost"] == want["cost"]
        assert [tuple(map(int, t)) for t in f["iters"]] == [tuple(t) for t in want["iters"]]
        # the network ran on the batches too (the initial partition's nodes are evaluated once,
        # while `generated` counts them in every iteration)
        assert f["batches"] > 0 and f["evaluated"] > 0


def test_fixed_tree_with_batches_in_flight_on_several_slots(P, orc):
    # 10-turn scrambles searched with four slots and 16 threads: batches of every size class are
    # in flight at once, so chain launches of both tile widths and of CTA pairs (batches of 8 or
    # more row blocks) meet the heads and gathers of other slots on the device.  Every chain
    # launch must have all its CTAs resident (a cooperative launch): a launch only partly
    # started can wait on tiles of CTAs that never start while a full-device launch queued on
    # another stream waits for its SMs.  Short device waits make such a stall an error here.
    ctx = P.cbdfs_create(0, max_batch=8192, n_slots=4, device_wait_ns=300_000_000)
    try:
        dpid = P.cbdfs_pdb_load(ctx, P.DOM_RC3, [list(range(8))])
        Ws, bs = W.net_weights(**W.NET_C2)
        scales = fp8_act_scales(orc, P.DOM_RC3, Ws, bs, W.random_rc_states(1024, 77))
        nets = {"bf16": P.cbdfs_net_load(ctx, P.DOM_RC3, Ws, bs, P.PREC_BF16, P.HEAD_CLASSIFIER, 0),
                "fp8": P.cbdfs_net_load(ctx, P.DOM_RC3, Ws, bs, P.PREC_FP8, P.HEAD_CLASSIFIER, 0,
                                        act_scales=scales)}
        starts = [P.cbdfs_apply_moves(P.DOM_RC3, W.rc_goal(), W.rc_scramble(10, W.seed_for(W.TAG_C2, 100 + i)))
                  for i in range(4)]
        want = [P.cbdfs_solve(ctx, P.DOM_RC3, s, P.ALGO_IDA, dpid, threads=16, work_num=256, batch=4096,
                              timeout_us=500, time_limit_s=60.0) for s in starts]
        for name, nid in nets.items():
            for s, w in zip(starts, want):
                r = P.cbdfs_solve(ctx, P.DOM_RC3, s, P.ALGO_IDA, nid, threads=16, work_num=256, batch=4096,
                                  timeout_us=500, time_limit_s=60.0, fixed_tree_heur=dpid)
                assert r["cost"] == w["cost"] == 10, name
                assert r["iters"] == w["iters"], name
            assert P.cbdfs_device_status(ctx) == 0, name
    finally:
        P.cbdfs_destroy(ctx)
