"""Pins of the oracle's admissibility-preserving heads (Related Work: the quantile of an
ordered classifier, lowered for admissibility; the minimum over an ensemble): hand-worked
values, closed forms for uniform and one-hot-like logits, monotonicity in q."""
import numpy as np

import workloads as W


def test_quantile_by_hand(orc):
    y = np.log(np.array([[0.1, 0.2, 0.3, 0.4]]))
    # cumulative 0.1, 0.3, 0.6, 1.0
    for q, want in ((0.05, 0), (0.2, 1), (0.5, 2), (0.61, 3), (1.0, 3)):
        assert orc.h_quantile(y, q)[0] == want, q


def test_quantile_of_uniform_logits_is_a_closed_form(orc):
    for C in (3, 21, 81):
        y = np.full((1, C), 0.37)
        for q in (0.013, 0.25, 0.5, 0.77, 0.999):
            # cumulative (c+1)/C: the first c with (c+1)/C >= q
            want = int(np.ceil(q * C)) - 1
            assert orc.h_quantile(y, q)[0] == want, (C, q)


def test_quantile_of_a_dominant_class(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        C = int(rng.integers(2, 60))
        k = int(rng.integers(0, C))
        y = rng.normal(size=(1, C))
        y[0, k] = 60.0  # every other class has probability below e^-55
        for q in (1e-6, 0.3, 0.999999):
            assert orc.h_quantile(y, q)[0] == k


def test_quantile_is_monotone_in_q_and_max_md_goal(orc):
    rng = np.random.default_rng(4)
    y = rng.normal(scale=3.0, size=(200, 17))
    qs = [0.01, 0.1, 0.3, 0.5, 0.7, 0.9, 0.99]
    hs = np.stack([orc.h_quantile(y, q) for q in qs])
    assert (np.diff(hs, axis=0) >= 0).all()
    md = rng.integers(0, 17, size=200)
    goal = np.zeros(200, bool)
    goal[5] = True
    h = orc.h_quantile(y, 0.3, md, goal)
    assert h[5] == 0
    keep = ~goal
    assert np.array_equal(h[keep], np.maximum(hs[2], md)[keep])


def test_quantile_margin_flags_near_ties(orc):
    y = np.log(np.array([[0.25, 0.25, 0.5], [0.1, 0.1, 0.8]]))
    m = orc.quantile_margin(y, 0.5, 1e-3)  # row 0 has cumulative exactly 0.5 at class 1
    assert m[0] and not m[1]


def test_combo_by_hand(orc):
    a = np.array([3, 7, 0, 9])
    b = np.array([5, 2, 4, 9])
    c = np.array([1, 1, 1, 1])
    # groups {a, b} and {c}, plus md
    md = np.array([10, 0, 2, 250])
    goal = np.array([False, False, True, False])
    h = orc.h_combo([a, b, c], [2, 1], md, goal)
    assert list(h) == [10 + 3 + 1, 0 + 2 + 1, 0, 255]
    assert list(orc.h_combo([a], [1])) == list(a)
    assert list(orc.h_combo([a, a, a], [3])) == list(a)


def test_combo_of_disjoint_pattern_tables_is_the_additive_pdb(orc):
    # two single-member groups: the sum of two disjoint pattern tables is the additive PDB
    pats = [[1, 2, 3, 4], [5, 6, 7, 8]]
    tabs = [orc.pdb_build(3, p) for p in pats]
    s = W.random_stp_states(3, 500, 8)
    parts = [orc.PDB(3, [p], [t]).hs(s) for p, t in zip(pats, tabs)]
    both = orc.PDB(3, pats, tabs).hs(s)
    assert np.array_equal(orc.h_combo(parts, [1, 1]), np.minimum(both, 255))
    # the minimum of a table and MD never exceeds either
    md = orc.md_states(orc.DOM_STP3, s)
    lo = orc.h_combo([parts[0], md], [2])
    assert (lo <= parts[0]).all() and (lo <= md).all() and ((lo == parts[0]) | (lo == md)).all()
