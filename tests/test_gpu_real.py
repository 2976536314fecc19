"""Parity of the real-valued regression heuristic (CBDFS_HEAD_REAL; section "Regression-Based
Neural Heuristics", Experimental Setup: the regression model's predictions minus 2.2) and of
the batched search with real thresholds.

- h = max(y + offset, 0) (max'ed with MD when asked, 0 at the goal) against the float64
  oracle on the same quantised weights, within the precision's tolerance on y; the bound
  test exactly, given the kernel's FP32 h (the decision is taken in FP32 on both sides).
- A network that computes 3/4 of Manhattan distance exactly (integer weights, one path
  through the hidden layers): with offset -9/4 every h and f is a multiple of 1/4, exact in
  FP32 and float64, so IDA* and BTS with real thresholds must match the oracle's serial
  searches bound for bound and count for count."""
import math

import numpy as np
import pytest

import workloads as W
from helpers import PREC, RTOL, fp8_act_scales, oracle_net

pytestmark = pytest.mark.gpu

OFFSET = -2.2
RAGGED = [1, 31, 129, 1000, 8192]
NET_CUBE_REAL = dict(dims=[480, 2048, 2048, 1024, 1], init="kaiming", seed=12)


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


def _check_bound_fp32(orc, g, h, bound, mask, minf):
    want_mask, want_minf = orc.bound_test_real(g, h, bound, np.float32)
    assert np.array_equal(mask, want_mask)
    assert minf == want_minf or (math.isinf(minf) and math.isinf(want_minf))


CASES = [("stp4", "bf16", 0), ("stp4", "bf16", 1), ("stp4", "fp8", 0), ("stp4", "fp32", 1),
         ("rc", "bf16", 0)]


@pytest.fixture(scope="module")
def nets(P, ctx, orc):
    out = {}
    for dom_name, prec, md in CASES:
        dom = P.DOM_STP4 if dom_name == "stp4" else P.DOM_RC3
        Ws, bs = W.net_weights(**(W.NET_C1 if dom_name == "stp4" else NET_CUBE_REAL))
        scales = None
        if prec == "fp8":
            scales = fp8_act_scales(orc, dom, Ws, bs, W.random_stp_states(4, 2048, 77))
        hid = P.cbdfs_net_load(ctx, dom, Ws, bs, PREC[prec], P.HEAD_REAL, md, act_scales=scales,
                               h_offset=OFFSET)
        out[(dom_name, prec, md)] = (dom, Ws, bs, scales, hid)
    return out


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("n", RAGGED)
def test_real_h_and_bound_test(P, ctx, orc, nets, case, n):
    dom_name, prec, md = case
    dom, Ws, bs, scales, hid = nets[case]
    if dom_name == "stp4":
        s = W.random_stp_states(4, n, 300 + n)
        s[0] = W.stp_goal(4)
    else:
        s = W.random_rc_states(n, 300 + n)
        s[0] = W.rc_goal()
    g = _g(n, 900 + n)
    y64, _, _ = oracle_net(orc, dom, Ws, bs, prec, s, "regression", bool(md), scales)
    goal = orc.is_goal_states(dom, s)
    mdv = orc.md_states(dom, s) if md else None
    h64 = orc.h_real(y64[:, 0], OFFSET, mdv, goal)
    f64 = g + h64
    bound = float(np.median(f64)) if n > 1 else 1e9
    h, mask, minf = P.heur_submit_batch_real(ctx, hid, dom, s, g, bound)
    assert h.dtype == np.float32 and h[0] == 0.0
    # h is 1-Lipschitz in y (the clamp and the max with MD), so y's tolerance bounds it
    scale = np.maximum(np.abs(y64[:, 0]), np.sqrt(np.mean(y64[:, 0] ** 2)))
    err = np.abs(h.astype(np.float64) - h64) / scale
    assert err.max() <= RTOL[prec], f"worst {err.max() / RTOL[prec]:.3f} x tolerance"
    _check_bound_fp32(orc, g, h, bound, mask, minf)


def test_device_entry_and_no_f_above(P, ctx, orc, nets):
    import torch
    dom, Ws, bs, scales, hid = nets[("stp4", "bf16", 1)]
    n = 3000
    s = W.random_stp_states(4, n, 4040)
    g = _g(n, 4041)
    h, mask, minf = P.heur_submit_batch_real(ctx, hid, dom, s, g, 55.5)
    dev = torch.device("cuda", 0)
    ds = torch.from_numpy(s.view(np.int64)).to(dev)
    dg = torch.from_numpy(g).to(dev)
    dh = torch.empty(n, dtype=torch.float32, device=dev)
    dm = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    dmin = torch.empty(1, dtype=torch.float32, device=dev)
    P.heur_eval_device_real(ctx, hid, dom, ds, dg, 55.5, n, dh, dm, dmin)
    torch.cuda.synchronize()
    assert np.array_equal(dh.cpu().numpy(), h)
    assert np.array_equal(dm.cpu().numpy().view(np.uint32), mask)
    assert float(dmin.cpu()[0]) == minf
    # nothing above an infinite bound: every bit set; the host call returns +inf, the device
    # call leaves the bit pattern 0xFFFFFFFF
    h2, mask2, minf2 = P.heur_submit_batch_real(ctx, hid, dom, s, g, float("inf"))
    assert np.array_equal(h2, h) and math.isinf(minf2) and minf2 > 0
    assert np.array_equal(mask2, orc.bound_test_real(g, h, float("inf"), np.float32)[0])
    P.heur_eval_device_real(ctx, hid, dom, ds, dg, float("inf"), n, dh, dm, dmin)
    torch.cuda.synchronize()
    assert dmin.cpu().numpy().view(np.uint32)[0] == 0xFFFFFFFF


def test_refusals(P, ctx, nets):
    dom, Ws, bs, scales, hid = nets[("stp4", "bf16", 0)]
    s = W.random_stp_states(4, 8, 1)
    g = np.zeros(8, np.uint8)
    with pytest.raises(P.CbdfsError):  # the integer entry with a real-valued network
        P.heur_submit_batch(ctx, hid, dom, s, g, 40)
    with pytest.raises(P.CbdfsError):  # the real entry with an integer heuristic
        P.heur_submit_batch_real(ctx, P.HEUR_MD, dom, s, g, 40.0)
    for bad in (-1.0, float("nan")):
        with pytest.raises(P.CbdfsError):
            P.heur_submit_batch_real(ctx, hid, dom, s, g, bad)
    Ws1, bs1 = W.net_weights(**W.NET_C1)
    with pytest.raises(P.CbdfsError):  # an offset is for the real-valued head only
        P.cbdfs_net_load(ctx, dom, Ws1, bs1, PREC["bf16"], P.HEAD_REGRESSION, 0, h_offset=-2.2)


# ---- exact search parity -------------------------------------------------------------

def md_linear_net(scale):
    """256-1024-1024-512-1 weights with y = scale * MD: hidden unit 0 of the first layer sums
    the Manhattan contribution of each (tile, cell) one-hot input (index tile*16 + cell), the
    next two layers pass unit 0 on, the last layer multiplies it by `scale`."""
    dims = [256, 1024, 1024, 512, 1]
    Ws = [np.zeros((dims[i + 1], dims[i]), np.float32) for i in range(4)]
    bs = [np.zeros(dims[i + 1], np.float32) for i in range(4)]
    for t in range(1, 16):
        for c in range(16):
            Ws[0][0, t * 16 + c] = abs(c // 4 - t // 4) + abs(c % 4 - t % 4)
    Ws[1][0, 0] = 1.0
    Ws[2][0, 0] = 1.0
    Ws[3][0, 0] = scale
    return Ws, bs


@pytest.fixture(scope="module")
def mdlin(P, ctx, orc):
    Ws, bs = md_linear_net(0.75)
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_REAL, 0, h_offset=-2.25)
    # the oracle's float64 forward of these weights is 3/4 of MD exactly
    s = W.random_stp_states(4, 500, 5150)
    y = orc.mlp_forward(Ws, bs, orc.one_hot(orc.DOM_STP4, s))[:, 0]
    assert np.array_equal(y, 0.75 * orc.md_states(orc.DOM_STP4, s))
    href = orc.HeurReal(lambda w: max(0.75 * orc.stp_md(w[0], 4) - 2.25, 0.0))
    return hid, href


def _starts(orc, k, moves=26, base=6100):
    return [orc.stp_apply_walk(4, W.stp_walk(4, moves, W.seed_for(W.TAG_C1, base + i))) for i in range(k)]


def test_md_linear_values_exact(P, ctx, orc, mdlin):
    hid, _ = mdlin
    s = W.random_stp_states(4, 4096, 5151)
    g = _g(4096, 5152)
    h, mask, minf = P.heur_submit_batch_real(ctx, hid, P.DOM_STP4, s, g, 40.25)
    want = orc.h_real(0.75 * orc.md_states(orc.DOM_STP4, s), -2.25, None, orc.is_goal_states(orc.DOM_STP4, s))
    assert np.array_equal(h.astype(np.float64), want)
    wm, wf = orc.bound_test_real(g, want, 40.25)
    assert np.array_equal(mask, wm) and minf == wf


@pytest.mark.parametrize("threads,work_num,batch", [(4, 8, 1024), (2, 3, 64)])
def test_ida_real_thresholds_match_oracle(P, ctx, orc, mdlin, threads, work_num, batch):
    hid, href = mdlin
    for s in _starts(orc, 3):
        want = orc.ida_star_real(orc.DOM_STP4, s, href)
        r = P.cbdfs_solve(ctx, P.DOM_STP4, s, P.ALGO_IDA, hid, threads=threads, work_num=work_num,
                          batch=batch, timeout_us=200, time_limit_s=60.0)
        assert r["real_valued"] and r["cost"] == want["cost"]
        assert [(float(b), e, g) for b, e, g in r["iters"]] == [(float(b), e, g) for b, e, g in want["iters"]]
        # bounds are multiples of 1/4: several per integer step of f
        assert any(b != math.floor(b) for b, _, _ in r["iters"])
        assert P.cbdfs_apply_moves(P.DOM_STP4, s, r["path"]) == W.stp_goal(4)


@pytest.mark.parametrize("n0", [10, 1000])
def test_bts_real_thresholds_match_oracle(P, ctx, orc, mdlin, n0):
    hid, href = mdlin
    for s in _starts(orc, 3, moves=28, base=6100):
        want = orc.bts_real(orc.DOM_STP4, s, href, n0=n0)
        r = P.cbdfs_solve(ctx, P.DOM_STP4, s, P.ALGO_BTS, hid, threads=4, work_num=8, batch=1024,
                          timeout_us=200, bts_n0=n0, time_limit_s=60.0)
        assert r["cost"] == want["cost"]
        got = [(float(b), lim, e, g, c) for (b, e, g), lim, c in zip(r["iters"], r["iter_limit"], r["iter_cut"])]
        exp = [(float(b), lim, e, g, int(c)) for (b, lim, e, g, c, _f) in want["searches"]]
        assert [(b, lim, c) for b, lim, _, _, c in got] == [(b, lim, c) for b, lim, _, _, c in exp]
        for a, b in zip(got, exp):
            if not a[4]:  # uncut searches expand exactly the oracle's tree
                assert a[2:4] == b[2:4]
