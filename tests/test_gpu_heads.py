"""Parity of the admissibility-preserving heads (Related Work: the classifier quantile; the
minimum over an ensemble; Experimental Setup: the 15-puzzle h_M adds ensembles to MD).

Quantile head: the logits against the float64 oracle within the precision's tolerance, and
the quantile decision against the oracle's rule applied to the kernel's own logits (the
decision taken on the same numbers; a partial sum within 1e-5 of q is a margin case for the
FP32 sum).  Every finishing kernel is covered: the fused chain epilogue (21 classes), the
register-tiled head (81 classes, BF16 and FP32), the generic head (200 classes).

Composite: bit-exact against the oracle's combination of the members' h, both for members
the oracle computes exactly (PDBs, MD) and for network members (their h from the library,
each member checked above); IDA* with a composite matches the oracle's serial IDA*."""
import numpy as np
import pytest

import workloads as W
from helpers import PREC, check_h, check_logits, oracle_net

pytestmark = pytest.mark.gpu

RAGGED = [1, 33, 129, 1000, 4096]


@pytest.fixture(scope="module")
def P():
    import paper_2507_11916_b300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.cbdfs_create(0, max_batch=8192, n_slots=3)
    yield c
    P.cbdfs_destroy(c)


def _g(n, seed, hi=40):
    return (W.splitmix64_array(seed, n) % np.uint64(hi)).astype(np.uint8)


QNETS = {
    "chain21": (dict(dims=[256, 1024, 1024, 512, 21], init="kaiming", seed=31), "bf16", 0.3),
    "tiled81": (W.NET_C3, "bf16", 0.2),
    "tiled81_fp32": (W.NET_C3, "fp32", 0.5),
    "generic200": (dict(dims=[256, 512, 512, 200], init="kaiming", seed=33), "fp32", 0.1),
}


@pytest.fixture(scope="module")
def qnets(P, ctx):
    out = {}
    for name, (cfg, prec, q) in QNETS.items():
        Ws, bs = W.net_weights(**cfg)
        md = 1 if name == "tiled81" else 0
        hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC[prec], P.HEAD_QUANTILE, md, quantile=q)
        out[name] = (Ws, bs, prec, q, md, hid)
    return out


@pytest.mark.parametrize("name", list(QNETS))
@pytest.mark.parametrize("n", RAGGED)
def test_quantile_head(P, ctx, orc, qnets, name, n):
    Ws, bs, prec, q, md, hid = qnets[name]
    C = Ws[-1].shape[0]
    s = W.random_stp_states(4, n, 1200 + n)
    s[0] = W.stp_goal(4)
    g = _g(n, 1300 + n)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 45, want_y=True, n_out=C)
    y64, _, _ = oracle_net(orc, P.DOM_STP4, Ws, bs, prec, s, "classifier")
    check_logits(y, y64, prec)
    goal = orc.is_goal_states(orc.DOM_STP4, s)
    mdv = orc.md_states(orc.DOM_STP4, s) if md else None
    want = orc.h_quantile(y.astype(np.float64), q, mdv, goal)
    margin = orc.quantile_margin(y.astype(np.float64), q, 1e-5)
    mism = check_h(h, want, margin)
    assert mism <= max(2, n // 200)
    wm, wf = orc.bound_test(g, h, 45)
    assert np.array_equal(mask, wm) and minf == wf


def test_quantile_arguments(P, ctx):
    Ws, bs = W.net_weights(**W.NET_C3)
    for bad in (0.0, -0.1, 1.5, float("nan")):
        with pytest.raises(P.CbdfsError):
            P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_QUANTILE, 0, quantile=bad)
    with pytest.raises(P.CbdfsError):  # a quantile belongs to the quantile head only
        P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_CLASSIFIER, 0, quantile=0.5)


# ---- composites --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def pdb8(orc):
    pats = [[1, 2, 3, 4], [5, 6, 7, 8], [1, 3, 5, 7]]
    return pats, [orc.pdb_build(3, p) for p in pats]


@pytest.mark.parametrize("n", RAGGED)
def test_composite_of_tables_and_md(P, ctx, orc, pdb8, n):
    pats, tabs = pdb8
    ids = [P.cbdfs_pdb_load(ctx, P.DOM_STP3, [p], [t]) for p, t in zip(pats, tabs)]
    # group 1: min(table A, MD); group 2: min(table B, table C); plus nothing
    cid = P.cbdfs_combo_load(ctx, P.DOM_STP3, [[ids[0], P.HEUR_MD], [ids[1], ids[2]]])
    # with MD added: a single-member group
    cid_md = P.cbdfs_combo_load(ctx, P.DOM_STP3, [[ids[2]]], add_md=True)
    s = W.random_stp_states(3, n, 1400 + n)
    s[0] = W.stp_goal(3)
    g = _g(n, 1500 + n)
    goal = orc.is_goal_states(orc.DOM_STP3, s)
    md = orc.md_states(orc.DOM_STP3, s)
    parts = [orc.PDB(3, [p], [t]).hs(s) for p, t in zip(pats, tabs)]
    h, mask, minf = P.heur_submit_batch(ctx, cid, P.DOM_STP3, s, g, 25)
    want = orc.h_combo([parts[0], md, parts[1], parts[2]], [2, 2], None, goal)
    assert np.array_equal(h, want)
    wm, wf = orc.bound_test(g, want, 25)
    assert np.array_equal(mask, wm) and minf == wf
    h2, _, _ = P.heur_submit_batch(ctx, cid_md, P.DOM_STP3, s, g, 25)
    assert np.array_equal(h2, orc.h_combo([parts[2]], [1], md, goal))


def test_composite_of_network_ensembles(P, ctx, orc, qnets):
    # the 15-puzzle h_M shape: MD + min over an ensemble of quantile classifiers + min over a
    # second ensemble (here: two seeds of the 81-class network and the 21-class network)
    Wa, ba = W.net_weights(dims=[256, 1024, 1024, 512, 81], init="kaiming", seed=41)
    Wb, bb = W.net_weights(dims=[256, 1024, 1024, 512, 81], init="kaiming", seed=42)
    ida = P.cbdfs_net_load(ctx, P.DOM_STP4, Wa, ba, PREC["bf16"], P.HEAD_QUANTILE, 0, quantile=0.05)
    idb = P.cbdfs_net_load(ctx, P.DOM_STP4, Wb, bb, PREC["bf16"], P.HEAD_QUANTILE, 0,
                           quantile=0.05)
    idc = qnets["chain21"][5]
    idd = qnets["tiled81"][5]
    cid = P.cbdfs_combo_load(ctx, P.DOM_STP4, [[ida, idb], [idc, idd]], add_md=True)
    for n in (1, 777, 8192):
        s = W.random_stp_states(4, n, 1600 + n)
        s[0] = W.stp_goal(4)
        g = _g(n, 1700 + n)
        members = [P.heur_submit_batch(ctx, i, P.DOM_STP4, s, g, 255)[0] for i in (ida, idb, idc, idd)]
        h, mask, minf = P.heur_submit_batch(ctx, cid, P.DOM_STP4, s, g, 60)
        want = orc.h_combo(members, [2, 2], orc.md_states(orc.DOM_STP4, s), orc.is_goal_states(orc.DOM_STP4, s))
        assert np.array_equal(h, want)
        wm, wf = orc.bound_test(g, want, 60)
        assert np.array_equal(mask, wm) and minf == wf


def test_composite_errors(P, ctx, pdb8):
    pats, tabs = pdb8
    pid = P.cbdfs_pdb_load(ctx, P.DOM_STP3, [pats[0]], [tabs[0]])
    with pytest.raises(P.CbdfsError):  # a member of another domain
        P.cbdfs_combo_load(ctx, P.DOM_STP4, [[pid]])
    with pytest.raises(P.CbdfsError):  # nine members in one group
        P.cbdfs_combo_load(ctx, P.DOM_STP3, [[pid] * 9])
    cid = P.cbdfs_combo_load(ctx, P.DOM_STP3, [[pid]])
    with pytest.raises(P.CbdfsError):  # nesting
        P.cbdfs_combo_load(ctx, P.DOM_STP3, [[cid]])
    with pytest.raises(P.CbdfsError):  # MD on the cube
        P.cbdfs_combo_load(ctx, P.DOM_RC3, [[P.HEUR_ZERO]], add_md=True)


def test_ida_with_a_composite_matches_oracle(P, ctx, orc, pdb8):
    pats, tabs = pdb8
    ids = [P.cbdfs_pdb_load(ctx, P.DOM_STP3, [p], [t]) for p, t in zip(pats, tabs)]
    cid = P.cbdfs_combo_load(ctx, P.DOM_STP3, [[ids[0], P.HEUR_MD], [ids[1]]])
    A, B = (orc.PDB(3, [p], [t]) for p, t in zip(pats[:2], tabs[:2]))

    def h(w):
        s = w[0]
        return min(A.h(s), orc.stp_md(s, 3)) + B.h(s)

    dist, _, _ = orc.stp3_bfs()
    for i in range(6):
        s = orc.stp_apply_walk(3, W.stp_walk(3, 60, W.seed_for(W.TAG_C0, 50 + i)))
        want = orc.ida_star(orc.DOM_STP3, s, orc.Heur(fn=h))
        r = P.cbdfs_solve(ctx, P.DOM_STP3, s, P.ALGO_IDA, cid, threads=4, work_num=8, batch=256,
                          timeout_us=200, time_limit_s=60.0)
        assert r["cost"] == want["cost"] == dist[orc.perm_rank([(s >> (4 * p)) & 15 for p in range(9)])]
        assert [tuple(map(int, t)) for t in r["iters"]] == [tuple(t) for t in want["iters"]]


@pytest.mark.parametrize("C", [81, 40, 128])
def test_tensor_core_head_is_fp32_accurate(P, ctx, orc, C):
    # 256 -> 256 -> C with an identity hidden layer: the stored BF16 activations are the one-hot
    # rows exactly, so y_c = b_c + the sum of W2[c, i] over the 16 active inputs, in float64.  The
    # head's three BF16 parts of W2 leave only the FP32 accumulation's rounding, a few 2^-24 of
    # the summed magnitudes (a plain BF16 last layer would be off by ~1e-3 relative)
    rng = np.random.default_rng(C)
    W1 = np.eye(256, dtype=np.float32)
    b1 = np.zeros(256, np.float32)
    W2 = rng.normal(size=(C, 256)).astype(np.float32)
    b2 = rng.normal(size=C).astype(np.float32)
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, [W1, W2], [b1, b2], PREC["bf16"], P.HEAD_CLASSIFIER, 0)
    n = 3000
    s = W.random_stp_states(4, n, 1800 + C)
    g = np.zeros(n, np.uint8)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 255, want_y=True, n_out=C)
    X = orc.one_hot(orc.DOM_STP4, s)
    terms = X[:, None, :] * W2.astype(np.float64)[None, :, :]
    y64 = terms.sum(axis=2) + b2.astype(np.float64)
    scale = np.abs(terms).sum(axis=2) + np.abs(b2)
    err = np.abs(y.astype(np.float64) - y64) / scale
    assert err.max() < 2e-6, err.max()
    want = orc.h_classifier(y.astype(np.float64), None, orc.is_goal_states(orc.DOM_STP4, s))
    assert np.array_equal(h, np.minimum(want, 255))


def test_grouped_ensemble_equals_its_members(P, ctx, orc):
    # four 81-class quantile networks of one shape in one group: run as one grouped network
    # (stacked first layer, grouped hidden layers, grouped tensor-core heads), the minimum must
    # be exactly the minimum of the members evaluated one by one
    ids = []
    for seed in (51, 52, 53, 54):
        Wq, bq = W.net_weights(dims=[256, 1024, 1024, 512, 81], init="kaiming", seed=seed)
        ids.append(P.cbdfs_net_load(ctx, P.DOM_STP4, Wq, bq, PREC["bf16"], P.HEAD_QUANTILE, 0, quantile=0.1))
    cid = P.cbdfs_combo_load(ctx, P.DOM_STP4, [ids], add_md=False)
    for n in (1, 129, 3001, 8192):
        s = W.random_stp_states(4, n, 1900 + n)
        g = _g(n, 1950 + n)
        members = [P.heur_submit_batch(ctx, i, P.DOM_STP4, s, g, 255)[0] for i in ids]
        h, mask, minf = P.heur_submit_batch(ctx, cid, P.DOM_STP4, s, g, 40)
        want = orc.h_combo(members, [4], None, orc.is_goal_states(orc.DOM_STP4, s))
        assert np.array_equal(h, want)
        wm, wf = orc.bound_test(g, want, 40)
        assert np.array_equal(mask, wm) and minf == wf
