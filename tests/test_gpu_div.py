"""DIV-compressed pattern databases on the GPU (Background: k adjacent entries grouped by
dividing the index by k keep their minimum; PDB Comparison: h_DIV of the network's size is the
plain-heuristic comparator): the device compression and the gathers against the oracle's
compression of the same full tables, bit-exact, with the bound test."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2507_11916_b300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.cbdfs_create(0, max_batch=8192, n_slots=2)
    yield c
    P.cbdfs_destroy(c)


def _g(n, seed, hi=40):
    return (W.splitmix64_array(seed, n) % np.uint64(hi)).astype(np.uint8)


@pytest.mark.parametrize("k", [2, 7, 64])
@pytest.mark.parametrize("n", [1, 129, 3000])
def test_div_8puzzle(P, ctx, orc, k, n):
    pats = [[1, 2, 3, 4], [5, 6, 7, 8]]
    tabs = [orc.pdb_build(3, p) for p in pats]
    hid = P.cbdfs_pdb_load(ctx, P.DOM_STP3, pats, tabs, div=k)
    dt = [orc.pdb_div(t, k) for t in tabs]
    s = W.random_stp_states(3, n, 3100 + n + k)
    s[0] = W.stp_goal(3)
    g = _g(n, 3200 + n)
    h, mask, minf = P.heur_submit_batch(ctx, hid, P.DOM_STP3, s, g, 20)
    want = np.array([orc.pdb_div_h(3, pats, dt, k, x) for x in s], np.int64)
    assert np.array_equal(h, want)
    wm, wf = orc.bound_test(g, want, 20)
    assert np.array_equal(mask, wm) and minf == wf


def test_div_15puzzle_663_built_on_device(P, ctx, orc):
    pats = [list(p) for p in W.PATTERNS_663]
    full = [P.pdb_build(ctx, P.DOM_STP4, p) for p in pats]
    hid = P.cbdfs_pdb_load(ctx, P.DOM_STP4, pats, div=3)  # built and compressed on the device
    dt = [orc.pdb_div(t, 3) for t in full]
    s = W.random_stp_states(4, 2000, 3300)
    h = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, np.zeros(2000, np.uint8), 255)[0]
    want = np.array([orc.pdb_div_h(4, pats, dt, 3, x) for x in s], np.int64)
    assert np.array_equal(h, want)
    hfull = P.heur_submit_batch(ctx, P.cbdfs_pdb_load(ctx, P.DOM_STP4, pats, full), P.DOM_STP4, s,
                                np.zeros(2000, np.uint8), 255)[0]
    assert (h <= hfull).all() and (h < hfull).any()


def test_div_cube_corners(P, ctx, orc):
    full = P.pdb_build(ctx, P.DOM_RC3, list(range(8)))
    k = 46  # 88.2 MB / 46 = 1.9 MB, the paper's cube network size
    hid = P.cbdfs_pdb_load(ctx, P.DOM_RC3, [list(range(8))], div=k)
    dt = orc.pdb_div(full, k)
    s = W.random_rc_states(3000, 3400)
    s[0] = W.rc_goal()
    g = _g(3000, 3401, 14)
    h, mask, minf = P.heur_submit_batch(ctx, hid, P.DOM_RC3, s.reshape(-1), g, 11)
    want = np.array([dt[orc.rc_corner_index(tuple(map(int, w))) // k] for w in s], np.int64)
    want[0] = 0
    assert np.array_equal(h, want)
    wm, wf = orc.bound_test(g, want, 11)
    assert np.array_equal(mask, wm) and minf == wf
