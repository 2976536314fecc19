"""Parity of the GPU heuristic path with the oracle: built-in Manhattan distance, additive
PDB gather, the FP32 and BF16 network forms, the integer-h epilogue and the bound test."""
import numpy as np
import pytest

import workloads as W
from helpers import (PREC, check_h, check_logits, fp8_act_scales, logit_ratio, md_plus_net, normwise,
                     oracle_net, plain_mismatches, report)

pytestmark = pytest.mark.gpu

RAGGED = [1, 31, 33, 127, 129, 300, 1000]


@pytest.fixture(scope="module")
def P():
    import paper_2507_11916_b300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.cbdfs_create(0, max_batch=16384, n_slots=2)
    yield c
    P.cbdfs_destroy(c)


def _g(n, seed, hi=40):
    return (W.splitmix64_array(seed, n) % np.uint64(hi)).astype(np.uint8)


def _check_bound(orc, h, g, bound, mask, minf):
    want_mask, want_minf = orc.bound_test(g, h, bound)
    assert np.array_equal(mask, want_mask)
    assert minf == want_minf


@pytest.mark.parametrize("n", RAGGED)
def test_manhattan(P, ctx, orc, n):
    for side, dom in ((3, P.DOM_STP3), (4, P.DOM_STP4)):
        s = W.random_stp_states(side, n, 10 + n)
        s[0] = W.stp_goal(side)
        g = _g(n, n)
        h, mask, minf = P.heur_submit_batch(ctx, P.HEUR_MD, dom, s, g, 45)
        want = orc.md_states(dom, s)
        want[0] = 0
        assert np.array_equal(h, want)
        _check_bound(orc, h, g, 45, mask, minf)


def test_empty_batch(P, ctx):
    h, mask, minf = P.heur_submit_batch(ctx, P.HEUR_MD, P.DOM_STP4, np.zeros(0, np.uint64),
                                        np.zeros(0, np.uint8), 10)
    assert len(h) == 0 and minf == 0xFFFFFFFF


def test_rejects_bad_arguments(P, ctx):
    with pytest.raises(P.CbdfsError):
        P.heur_submit_batch(ctx, 99, P.DOM_STP4, np.zeros(4, np.uint64), np.zeros(4, np.uint8), 1)
    with pytest.raises(P.CbdfsError):
        P.heur_submit_batch(ctx, P.HEUR_MD, P.DOM_RC3, np.zeros(8, np.uint64), np.zeros(4, np.uint8), 1)
    with pytest.raises(P.CbdfsError):
        big = 16385
        P.heur_submit_batch(ctx, P.HEUR_MD, P.DOM_STP4, np.zeros(big, np.uint64), np.zeros(big, np.uint8), 1)


@pytest.fixture(scope="module")
def pdb8(orc):
    pats = [[1, 2, 3, 4], [5, 6, 7, 8]]
    return pats, [orc.pdb_build(3, p) for p in pats]


@pytest.fixture(scope="module")
def pdb15(orc):
    pats = [[1, 2, 3, 5, 6], [4, 8, 9, 12, 13], [7, 10, 11, 14, 15]]
    return pats, [orc.pdb_build(4, p) for p in pats]


@pytest.mark.parametrize("n", RAGGED)
def test_pdb_gather(P, ctx, orc, pdb8, pdb15, n):
    for side, dom, (pats, tabs) in ((3, P.DOM_STP3, pdb8), (4, P.DOM_STP4, pdb15)):
        hid = P.cbdfs_pdb_load(ctx, dom, pats, tabs)
        s = W.random_stp_states(side, n, 20 + n)
        g = _g(n, 7 * n)
        h, mask, minf = P.heur_submit_batch(ctx, hid, dom, s, g, 50)
        want = orc.PDB(side, pats, tabs).hs(s)
        want[orc.is_goal_states(dom, s)] = 0
        assert np.array_equal(h, want)
        _check_bound(orc, h, g, 50, mask, minf)


@pytest.mark.parametrize("tiles", [[1, 2, 3, 4], [5, 6, 7, 8], [1, 3, 5, 7, 8]])
def test_pdb_build_8puzzle(P, ctx, orc, tiles):
    assert np.array_equal(P.pdb_build(ctx, P.DOM_STP3, tiles), orc.pdb_build(3, tiles))


def test_pdb_build_15puzzle_small(P, ctx, orc):
    for tiles in ([10, 11, 15], [1, 2, 3, 5], [4, 8, 12, 13, 14]):
        assert np.array_equal(P.pdb_build(ctx, P.DOM_STP4, tiles), orc.pdb_build(4, tiles))


@pytest.mark.slow
def test_pdb_build_663(P, ctx, orc):
    for tiles in orc.PATTERNS_663:
        assert np.array_equal(P.pdb_build(ctx, P.DOM_STP4, tiles), orc.pdb_build(4, tiles))


# ---- network heuristic ------------------------------------------------------------------

def _net(P, ctx, cfg, dom, prec, head, md):
    Ws, bs = W.net_weights(**cfg)
    hid = P.cbdfs_net_load(ctx, dom, Ws, bs, PREC[prec], head, md)
    return Ws, bs, hid


@pytest.mark.parametrize("n", RAGGED)
def test_c0_fp32_regression(P, ctx, orc, n):
    Ws, bs, hid = _net(P, ctx, W.NET_C0, P.DOM_STP3, "fp32", P.HEAD_REGRESSION, 1)
    s = W.random_stp_states(3, n, 40 + n)
    g = _g(n, n + 1)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP3, s, g, 30, want_y=True)
    y64, h64, margin = oracle_net(orc, 0, Ws, bs, "fp32", s, "regression", True)
    check_logits(y, y64, "fp32")
    check_h(h, h64, margin)
    _check_bound(orc, h, g, 30, mask, minf)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("n", [1, 31, 129, 2000, 5000])
def test_c0_chain_8puzzle(P, ctx, orc, prec, n):
    # the 8-puzzle network 81-256-256-1 in the fused chain (the one-hot rows 81 wide, padded to
    # 128; 16-row pre-pass units), against the oracle on the same rounded weights
    Ws, bs = W.net_weights(**W.NET_C0)
    kw = {}
    if prec == "fp8":
        kw["act_scales"] = fp8_act_scales(orc, 0, Ws, bs, W.random_stp_states(3, 4096, 12))
    hid = P.cbdfs_net_load(ctx, P.DOM_STP3, Ws, bs, PREC[prec], P.HEAD_REGRESSION, 1, **kw)
    s = W.random_stp_states(3, n, 45 + n)
    s[0] = W.stp_goal(3)
    g = _g(n, n + 7)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP3, s, g, 30, want_y=True)
    y64, h64, margin = oracle_net(orc, 0, Ws, bs, prec, s, "regression", True, **kw)
    check_logits(y, y64, prec)
    check_h(h, h64, margin)
    report(f"c0 {prec} n={n}", h, h64, margin, plain_mismatches(orc, 0, Ws, bs, prec, s, h, "regression", True))
    assert h[0] == 0
    _check_bound(orc, h, g, 30, mask, minf)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("n", [1, 127, 129, 1000])
def test_c1_regression(P, ctx, orc, prec, n):
    Ws, bs, hid = _net(P, ctx, W.NET_C1, P.DOM_STP4, prec, P.HEAD_REGRESSION, 1)
    s = W.random_stp_states(4, n, 50 + n)
    g = _g(n, n + 2)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 60, want_y=True)
    y64, h64, margin = oracle_net(orc, 1, Ws, bs, prec, s, "regression", True)
    check_logits(y, y64, prec)
    check_h(h, h64, margin)
    _check_bound(orc, h, g, 60, mask, minf)


def test_c1_regression_without_md_exposes_rounding(P, ctx, orc):
    # without the max with Manhattan distance the integer h is the network's own rounding
    Ws, bs = W.net_weights(**W.NET_C1)
    Ws[-1] = Ws[-1] * 20.0  # spread y over many integers
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_REGRESSION, 0)
    n = 2000
    s = W.random_stp_states(4, n, 77)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, np.zeros(n, np.uint8), 255,
                                           want_y=True)
    y64, h64, margin = oracle_net(orc, 1, Ws, bs, "bf16", s, "regression", False)
    check_logits(y, y64, "bf16")
    assert len(set(h64.tolist())) > 5
    check_h(h, h64, margin)
    report("c1 x20 bf16 no MD", h, h64, margin, plain_mismatches(orc, 1, Ws, bs, "bf16", s, h))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("n", [1, 129, 700, 1000])
def test_c2_classifier(P, ctx, orc, prec, n):
    # 700 states: six row blocks of 64-wide tiles (192 per 2048-wide layer), 1000: CTA pairs
    Ws, bs, hid = _net(P, ctx, W.NET_C2, P.DOM_RC3, prec, P.HEAD_CLASSIFIER, 0)
    s = W.random_rc_states(n, 60 + n)
    s[0] = W.rc_goal()
    g = _g(n, n + 3, 20)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_RC3, s.reshape(-1), g, 25, want_y=True,
                                           n_out=21)
    y64, h64, margin = oracle_net(orc, 2, Ws, bs, prec, s, "classifier", False)
    check_logits(y, y64, prec)
    check_h(h, h64, margin)
    assert h[0] == 0
    _check_bound(orc, h, g, 25, mask, minf)
    report(f"c2 {prec} n={n}", h, h64, margin,
           plain_mismatches(orc, 2, Ws, bs, prec, s, h, "classifier") if prec != "fp32" else None)


def test_c1_full_batch_sampled(P, ctx, orc):
    """The bench's launch shape (8192 states, BF16): every h checked against the rule on the
    GPU's own y, and a sample of rows against the oracle."""
    Ws, bs, hid = _net(P, ctx, W.NET_C1, P.DOM_STP4, "bf16", P.HEAD_REGRESSION, 1)
    n = 8192
    s = W.random_stp_states(4, n, 8192)
    g = _g(n, 5)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 60, want_y=True)
    idx = np.random.default_rng(0).choice(n, 512, replace=False)
    y64, h64, margin = oracle_net(orc, 1, Ws, bs, "bf16", s[idx], "regression", True)
    check_logits(y[idx], y64, "bf16")
    check_h(h[idx], h64, margin)
    _check_bound(orc, h, g, 60, mask, minf)


# A network of the 15-puzzle regression shape whose output decides h on most rows: Manhattan
# distance plus four times the seeded network's output plus 1.5 (helpers.md_plus_net).  With
# the seeded network alone, y stays within (-1, 1) and the max with MD decides every h.

@pytest.fixture(scope="module")
def c1_md_plus(orc):
    Ws, bs = md_plus_net(*W.net_weights(**W.NET_C1), 4)
    sc = fp8_act_scales(orc, 1, Ws, bs, W.random_stp_states(4, 4096, 11))
    return Ws, bs, sc


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("n", [1, 129, 1000, 1500, 8192])
def test_c1_network_decides_h(P, ctx, orc, c1_md_plus, prec, n):
    Ws, bs, sc = c1_md_plus
    kw = {"act_scales": sc} if prec == "fp8" else {}
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC[prec], P.HEAD_REGRESSION, 1, **kw)
    s = W.random_stp_states(4, n, 3100 + n)
    s[0] = W.stp_goal(4)
    g = _g(n, 3200 + n, 20)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 60, want_y=True)
    ye, he, margin = oracle_net(orc, 1, Ws, bs, prec, s, "regression", True, **kw)
    check_logits(y, ye, prec)
    check_h(h, he, margin)
    assert h[0] == 0
    if n >= 1000:  # the network, not the max with MD, decides most rows
        assert (he > orc.md_states(orc.DOM_STP4, s)).mean() > 0.4
    _check_bound(orc, h, g, 60, mask, minf)
    report(f"c1 MD-plus {prec} n={n}", h, he, margin,
           plain_mismatches(orc, 1, Ws, bs, prec, s, h, "regression", True))


def test_device_entry_matches_host_entry(P, ctx):
    import torch
    Ws, bs, hid = _net(P, ctx, W.NET_C1, P.DOM_STP4, "bf16", P.HEAD_REGRESSION, 1)
    n = 3000
    s = W.random_stp_states(4, n, 99)
    g = _g(n, 9)
    h, mask, minf = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 55)
    dev = torch.device("cuda:0")
    ds = torch.from_numpy(s.view(np.int64)).to(dev)
    dg = torch.from_numpy(g).to(dev)
    dh = torch.empty(n, dtype=torch.uint8, device=dev)
    dm = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    dmin = torch.empty(1, dtype=torch.int32, device=dev)
    for _ in range(2):
        P.heur_eval_device(ctx, hid, P.DOM_STP4, ds, dg, 55, n, dh, dm, dmin,
                           stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert np.array_equal(dh.cpu().numpy(), h)
        assert np.array_equal(dm.cpu().numpy().view(np.uint32), mask)
        assert int(dmin.cpu().numpy().view(np.uint32)[0]) == minf
    assert P.cbdfs_device_status(ctx) == 0


# FP8 (E4M3 weights with a per-tensor scale, E4M3 activations with static per-layer scales):
# per-logit parity is checked against the oracle's emulation of that storage (float64
# arithmetic on the E4M3 values); against plain float64 on the same weights the error is the
# format's own and is bounded normwise.

@pytest.mark.parametrize("n", [1, 129, 1000])
def test_c1_fp8(P, ctx, orc, n):
    Ws, bs = W.net_weights(**W.NET_C1)
    sc = fp8_act_scales(orc, 1, Ws, bs, W.random_stp_states(4, 4096, 11))
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["fp8"], P.HEAD_REGRESSION, 1, act_scales=sc)
    s = W.random_stp_states(4, n, 70 + n)
    g = _g(n, n + 4)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 60, want_y=True)
    ye, he, margin = oracle_net(orc, 1, Ws, bs, "fp8", s, "regression", True, act_scales=sc)
    check_logits(y, ye, "fp8")
    check_h(h, he, margin)
    y64, _, _ = oracle_net(orc, 1, Ws, bs, "fp8", s, "regression", True, emulate=False)
    if n > 1:
        assert normwise(y, y64) <= 6e-2
    _check_bound(orc, h, g, 60, mask, minf)
    print(f"c1 fp8 n={n}: per-logit error vs plain float64 {logit_ratio(y, y64, 'fp8'):.2f} x tolerance (reported)")


@pytest.mark.parametrize("n", [129, 700, 1000])
def test_c2_fp8(P, ctx, orc, n):
    Ws, bs = W.net_weights(**W.NET_C2)
    sc = fp8_act_scales(orc, 2, Ws, bs, W.random_rc_states(4096, 12))
    hid = P.cbdfs_net_load(ctx, P.DOM_RC3, Ws, bs, PREC["fp8"], P.HEAD_CLASSIFIER, 0, act_scales=sc)
    s = W.random_rc_states(n, 80 + n)
    g = _g(n, n + 5, 20)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_RC3, s.reshape(-1), g, 25, want_y=True,
                                           n_out=21)
    ye, he, margin = oracle_net(orc, 2, Ws, bs, "fp8", s, "classifier", False, act_scales=sc)
    check_logits(y, ye, "fp8")
    check_h(h, he, margin)
    y64, _, _ = oracle_net(orc, 2, Ws, bs, "fp8", s, "classifier", False, emulate=False)
    err = normwise(y, y64)
    assert err <= 6e-2
    _check_bound(orc, h, g, 25, mask, minf)
    report(f"c2 fp8 n={n}", h, he, margin, plain_mismatches(orc, 2, Ws, bs, "fp8", s, h, "classifier"))
    print(f"normwise error vs plain float64 {err:.4f}; per logit {logit_ratio(y, y64, 'fp8'):.2f} x tolerance")


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_fused_chain_matches_per_layer_kernels(P, ctx, orc, prec):
    """The persistent chain (device-buffer entry) and the per-layer kernels (the static-scratch
    entry) evaluate the same network: outputs agree to the precision, integers exactly."""
    import torch
    Ws, bs = W.net_weights(**W.NET_C1)
    sc = fp8_act_scales(orc, 1, Ws, bs, W.random_stp_states(4, 4096, 11)) if prec == "fp8" else None
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC[prec], P.HEAD_REGRESSION, 1, act_scales=sc)
    dev = torch.device("cuda:0")
    n = 5000
    s = W.random_stp_states(4, n, 4321)
    g = _g(n, 17)
    ds = torch.from_numpy(s.view(np.int64)).to(dev)
    dg = torch.from_numpy(g).to(dev)
    outs = []
    for fn in (P.heur_eval_device, P.heur_eval_device_static):
        dh = torch.empty(n, dtype=torch.uint8, device=dev)
        dm = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
        dmin = torch.empty(1, dtype=torch.int32, device=dev)
        fn(ctx, hid, P.DOM_STP4, ds, dg, 55, n, dh, dm, dmin, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        outs.append((dh.cpu().numpy(), dm.cpu().numpy(), int(dmin.cpu()[0])))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1]) and outs[0][2] == outs[1][2]
    assert P.cbdfs_device_status(ctx) == 0


# The 81-class network of the training configuration: wider than the fused head, so the chain
# stores its last hidden layer (BF16) and the register-tiled FP32 head kernel runs after it.

@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("n", [1, 129, 1000])
def test_c3_classifier_81(P, ctx, orc, prec, n):
    Ws, bs = W.net_weights(**W.NET_C3)
    sc = fp8_act_scales(orc, 1, Ws, bs, W.random_stp_states(4, 4096, 13)) if prec == "fp8" else None
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC[prec], P.HEAD_CLASSIFIER, 1, act_scales=sc)
    s = W.random_stp_states(4, n, 90 + n)
    s[0] = W.stp_goal(4)
    g = _g(n, n + 6, 60)
    h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 70, want_y=True, n_out=81)
    ye, he, margin = oracle_net(orc, 1, Ws, bs, prec, s, "classifier", True, act_scales=sc)
    check_logits(y, ye, prec)
    check_h(h, he, margin)
    assert h[0] == 0
    _check_bound(orc, h, g, 70, mask, minf)
    report(f"c3 {prec} n={n}", h, he, margin, plain_mismatches(orc, 1, Ws, bs, prec, s, h, "classifier", True))


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_c3_chain_matches_per_layer_kernels(P, ctx, orc, prec):
    """Chain + separate head against the per-layer kernels + the CUDA-core head: both store the
    last hidden layer in BF16 after the same tensor-core arithmetic."""
    import torch
    Ws, bs = W.net_weights(**W.NET_C3)
    sc = fp8_act_scales(orc, 1, Ws, bs, W.random_stp_states(4, 4096, 13)) if prec == "fp8" else None
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC[prec], P.HEAD_CLASSIFIER, 1, act_scales=sc)
    dev = torch.device("cuda:0")
    n = 4000
    s = W.random_stp_states(4, n, 5432)
    g = _g(n, 18, 60)
    ds = torch.from_numpy(s.view(np.int64)).to(dev)
    dg = torch.from_numpy(g).to(dev)
    outs = []
    for fn in (P.heur_eval_device, P.heur_eval_device_static):
        dh = torch.empty(n, dtype=torch.uint8, device=dev)
        dm = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
        dmin = torch.empty(1, dtype=torch.int32, device=dev)
        fn(ctx, hid, P.DOM_STP4, ds, dg, 70, n, dh, dm, dmin, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        outs.append((dh.cpu().numpy(), dm.cpu().numpy(), int(dmin.cpu()[0])))
    # the last layer: the chain's tensor-core head (split FP32 weights) and the per-layer path's
    # CUDA-core FP32 head round their accumulations in different orders, so h may differ only
    # where the two largest logits lie within 1e-4 of each other
    y64, _, _ = oracle_net(orc, P.DOM_STP4, Ws, bs, prec, s, "classifier", True, sc)
    tie = orc.classifier_margin(y64, 1e-4)
    assert np.array_equal(outs[0][0][~tie], outs[1][0][~tie])
    for h, mask, minf in outs:  # each path's bound test is that of its own h
        wm, wf = orc.bound_test(g, h, 70)
        assert np.array_equal(mask.view(np.uint32), wm) and (minf & 0xFFFFFFFF) == wf
    assert P.cbdfs_device_status(ctx) == 0


def test_page_locked_buffers_read_and_written_in_place(P, ctx, orc):
    # the host-buffer call with page-locked states, g, h and mask (the kernels read and write
    # them over the bus) gives what the staged call gives, for a network and for the cube
    import torch
    Ws, bs = W.net_weights(**W.NET_C1)
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_REGRESSION, 1)
    for n in (1, 1000, 8192):
        s = W.random_stp_states(4, n, 6600 + n)
        g = _g(n, 6700 + n, 60)
        want = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 50)
        ps = torch.from_numpy(s.view(np.int64)).pin_memory().numpy().view(np.uint64)
        pg = torch.from_numpy(g).pin_memory().numpy()
        ph = torch.zeros(n, dtype=torch.uint8).pin_memory().numpy()
        pm = torch.zeros((n + 31) // 32, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        h, mask, minf = P.heur_submit_batch(ctx, hid, P.DOM_STP4, ps, pg, 50, out=(ph, pm))
        assert h is ph and np.array_equal(ph, want[0]) and np.array_equal(pm, want[1]) and minf == want[2]
    pids = P.cbdfs_pdb_load(ctx, P.DOM_RC3, [list(range(8))])
    rs = W.random_rc_states(500, 6800).reshape(-1)
    rg = _g(500, 6801, 14)
    want = P.heur_submit_batch(ctx, pids, P.DOM_RC3, rs, rg, 12)
    prs = torch.from_numpy(rs.view(np.int64)).pin_memory().numpy().view(np.uint64)
    ph = torch.zeros(500, dtype=torch.uint8).pin_memory().numpy()
    pm = torch.zeros(16, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    h, mask, minf = P.heur_submit_batch(ctx, pids, P.DOM_RC3, prs, torch.from_numpy(rg).pin_memory().numpy(), 12,
                                        out=(ph, pm))
    assert np.array_equal(ph, want[0]) and np.array_equal(pm, want[1]) and minf == want[2]


def test_async_batches_and_wait(P, orc):
    # three batches in flight on three host slots, waited on in reverse order; each is what the
    # synchronous call gives.  A collected ticket is unknown afterwards.
    import torch
    ctx = P.cbdfs_create(0, max_batch=8192, n_slots=4)
    try:
        Ws, bs = W.net_weights(**W.NET_C1)
        hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_REGRESSION, 1)
        jobs = []
        for k, (heur, n) in enumerate(((hid, 8192), (P.HEUR_MD, 3000), (hid, 129))):
            s = W.random_stp_states(4, n, 7100 + k)
            g = _g(n, 7200 + k, 60)
            want = P.heur_submit_batch(ctx, heur, P.DOM_STP4, s, g, 50)
            ps = torch.from_numpy(s.view(np.int64)).pin_memory().numpy().view(np.uint64)
            pg = torch.from_numpy(g).pin_memory().numpy()
            out = (torch.zeros(n, dtype=torch.uint8).pin_memory().numpy(),
                   torch.zeros((n + 31) // 32, dtype=torch.int32).pin_memory().numpy().view(np.uint32))
            jobs.append((P.heur_submit_batch_async(ctx, heur, P.DOM_STP4, ps, pg, 50, out=out), want))
        for job, want in reversed(jobs):
            try:
                h, mask, minf = job.wait(timeout_us=1)   # may still be running: the ticket stays
            except P.CbdfsError as e:
                assert e.status == P.CBDFS_ETIMEDOUT
                h, mask, minf = job.wait()
            assert np.array_equal(h, want[0]) and np.array_equal(mask, want[1]) and minf == want[2]
        with pytest.raises(P.CbdfsError):
            jobs[0][0].wait()
    finally:
        P.cbdfs_destroy(ctx)


@pytest.mark.parametrize("net", ["c1", "c1_md_plus"])
@pytest.mark.parametrize("n", [65536, 262144])
def test_chain_at_the_kernel_micro_sizes_sampled(P, orc, n, net):
    # many tiles per CTA (the persistent schedule's later rounds, counters reused across row
    # blocks): a seeded sample of rows against the oracle, the bound test over every row, in BF16
    # and E4M3; the seeded network (h = MD on every row) and the one whose output decides h
    ctx = P.cbdfs_create(0, max_batch=n, n_slots=2)
    try:
        Ws, bs = W.net_weights(**W.NET_C1)
        if net == "c1_md_plus":
            Ws, bs = md_plus_net(Ws, bs, 4)
        sc = fp8_act_scales(orc, 1, Ws, bs, W.random_stp_states(4, 4096, 11))
        s = W.random_stp_states(4, n, 9000 + n)
        g = _g(n, 9100 + n, 60)
        idx = np.random.default_rng(n).choice(n, 400, replace=False)
        for prec in ("bf16", "fp8"):
            hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC[prec], P.HEAD_REGRESSION, 1,
                                   act_scales=sc if prec == "fp8" else None)
            h, mask, minf, y = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 55, want_y=True)
            y64, h64, margin = oracle_net(orc, 1, Ws, bs, prec, s[idx], "regression", True,
                                          sc if prec == "fp8" else None)
            check_logits(y[idx], y64, prec)
            check_h(h[idx], h64, margin)
            report(f"{net} {prec} n={n} (sample of 400)", h[idx], h64, margin)
            # every row: h follows the rule on the kernel's own y, and the bound test is exact
            own = orc.h_regression(y[:, 0], orc.md_states(orc.DOM_STP4, s), orc.is_goal_states(orc.DOM_STP4, s))
            assert np.array_equal(h, own)
            _check_bound(orc, h, g, 55, mask, minf)
        assert P.cbdfs_device_status(ctx) == 0
    finally:
        P.cbdfs_destroy(ctx)


@pytest.mark.parametrize("net", ["c1_bf16", "c1_fp8", "c2_bf16", "c3_bf16"])
def test_chain_counts_left_zero_between_launches(P, orc, net):
    # the fused kernel's dependency counts are zeroed by the launch itself (each count once
    # nothing reads it any more): a batch evaluated after launches of other sizes on the same
    # slot gives what the first launch of a fresh context gives, bit for bit (a count left
    # behind would let a layer start early or make a wait run out)
    cfg, dom, head, md = {"c1": (W.NET_C1, P.DOM_STP4, P.HEAD_REGRESSION, 1),
                          "c2": (W.NET_C2, P.DOM_RC3, P.HEAD_CLASSIFIER, 0),
                          "c3": (W.NET_C3, P.DOM_STP4, P.HEAD_CLASSIFIER, 1)}[net[:2]]
    prec = net[3:]
    Ws, bs = W.net_weights(**cfg)
    kw = {}
    if prec == "fp8":
        kw["act_scales"] = fp8_act_scales(orc, 1, Ws, bs, W.random_stp_states(4, 4096, 11))

    def batch(n, seed):
        s = W.random_rc_states(n, seed).reshape(-1) if dom == P.DOM_RC3 else W.random_stp_states(4, n, seed)
        return s, _g(n, seed + 1, 40)

    def fresh(s, g):
        c = P.cbdfs_create(0, max_batch=8192, n_slots=2)
        try:
            hid = P.cbdfs_net_load(c, dom, Ws, bs, PREC[prec], head, md, **kw)
            return P.heur_submit_batch(c, hid, dom, s, g, 30)
        finally:
            P.cbdfs_destroy(c)

    ctx = P.cbdfs_create(0, max_batch=8192, n_slots=2)
    try:
        hid = P.cbdfs_net_load(ctx, dom, Ws, bs, PREC[prec], head, md, **kw)
        for k, n in enumerate((8192, 129, 1, 4096, 8192, 300, 2000)):
            s, g = batch(n, 8800 + k)
            got = P.heur_submit_batch(ctx, hid, dom, s, g, 30)
            if k in (0, 2, 4, 6):
                want = fresh(s, g)
                assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]) and got[2] == want[2]
        assert P.cbdfs_device_status(ctx) == 0
    finally:
        P.cbdfs_destroy(ctx)
