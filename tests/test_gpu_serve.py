"""Continuous batching: requests of uneven sizes from many threads, for several networks,
coalesced into size-bucket launches that overlap on the device.  Every request's result must
be exactly what it gets alone."""
import concurrent.futures as cf

import numpy as np
import pytest

import workloads as W
from helpers import PREC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2507_11916_b300 as P
    return P


def _mix(P, n_req, seed):
    rng = W.SplitMix64(seed)
    reqs = []
    for i in range(n_req):
        size = int(round(32 * (4096 / 32) ** rng.uniform()))  # log-uniform 32..4096
        kind = rng.below(3)
        bound = 30 + rng.below(30)
        reqs.append((kind, size, bound, 5000 + i))
    return reqs


def _inputs(P, kind, size, seed):
    if kind == 1:  # cube
        s = W.random_rc_states(size, seed).reshape(-1)
        dom = P.DOM_RC3
    else:
        s = W.random_stp_states(4, size, seed)
        dom = P.DOM_STP4
    g = (W.splitmix64_array(seed + 7, size) % np.uint64(25)).astype(np.uint8)
    return dom, s, g


@pytest.mark.parametrize("coalesce", [1, 0])
def test_each_request_same_alone_and_in_the_mix(P, coalesce):
    ctx = P.cbdfs_create(0, max_batch=8192, n_slots=4)
    try:
        W1, b1 = W.net_weights(**W.NET_C1)
        W2, b2 = W.net_weights(**W.NET_C2)
        ids = {0: P.cbdfs_net_load(ctx, P.DOM_STP4, W1, b1, PREC["bf16"], P.HEAD_REGRESSION, 1),
               1: P.cbdfs_net_load(ctx, P.DOM_RC3, W2, b2, PREC["bf16"], P.HEAD_CLASSIFIER, 0),
               2: P.HEUR_MD}
        reqs = _mix(P, 60, 77 + coalesce)
        alone = []
        for kind, size, bound, seed in reqs:
            dom, s, g = _inputs(P, kind, size, seed)
            alone.append(P.heur_submit_batch(ctx, ids[kind], dom, s, g, bound))
        inputs = [_inputs(P, kind, size, seed) for kind, size, bound, seed in reqs]
        P.cbdfs_server_start(ctx, max_inflight=3, bucket_max=4096, coalesce=coalesce)

        # half the requests from 8 threads, half as one burst from this thread (so that
        # requests queue up behind the launches in flight and are merged)
        def run(i):
            kind, size, bound, seed = reqs[i]
            dom, s, g = inputs[i]
            return i, P.heur_request_submit(ctx, ids[kind], dom, s, g, bound).wait()

        with cf.ThreadPoolExecutor(8) as ex:
            got = dict(ex.map(run, range(len(reqs) // 2)))
        burst = [(i, P.heur_request_submit(ctx, ids[reqs[i][0]], inputs[i][0], inputs[i][1], inputs[i][2],
                                           reqs[i][2])) for i in range(len(reqs) // 2, len(reqs))]
        for i, r in burst:
            got[i] = r.wait()
        for i, (h, mask, minf) in got.items():
            ah, amask, aminf = alone[i]
            assert np.array_equal(h, ah), f"request {i}: h differs"
            assert np.array_equal(mask, amask) and minf == aminf, f"request {i}: bound test differs"
        st = P.cbdfs_server_get_stats(ctx)
        print("server stats", st)
        assert st["requests"] == len(reqs)
        assert st["states"] == sum(r[1] for r in reqs)
        assert 0 < st["launches"] <= len(reqs)
        if coalesce:
            assert st["launches"] < len(reqs)  # the burst was merged into fewer launches
        assert 0 < st["p50_us"] <= st["p99_us"]
        P.cbdfs_server_stop(ctx)
    finally:
        P.cbdfs_destroy(ctx)


def test_memory_budget_and_errors(P):
    ctx = P.cbdfs_create(0, max_batch=8192, n_slots=3)
    try:
        W1, b1 = W.net_weights(**W.NET_C1)
        hid = P.cbdfs_net_load(ctx, P.DOM_STP4, W1, b1, PREC["bf16"], P.HEAD_REGRESSION, 1)
        # a budget below one launch: admission serialises, everything still completes
        P.cbdfs_server_start(ctx, max_inflight=2, mem_budget=1, coalesce=1)
        rs = []
        for i in range(10):
            s = W.random_stp_states(4, 500 + 37 * i, 40 + i)
            g = np.zeros(len(s), np.uint8)
            rs.append((P.heur_request_submit(ctx, hid, P.DOM_STP4, s, g, 50), s, g))
        for r, s, g in rs:
            h, mask, minf = r.wait()
            assert np.array_equal(h, P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 50)[0])
        # a collected ticket is unknown afterwards; too large a request is refused
        with pytest.raises(P.CbdfsError):
            rs[0][0].wait()
        with pytest.raises(P.CbdfsError):
            P.heur_request_submit(ctx, hid, P.DOM_STP4, np.zeros(5000, np.uint64), np.zeros(5000, np.uint8), 1)
        # a load could move the scratch the server's graphs were captured on: refused while it runs
        W2, b2 = W.net_weights(**W.NET_C2)
        with pytest.raises(P.CbdfsError):
            P.cbdfs_net_load(ctx, P.DOM_RC3, W2, b2, PREC["bf16"], P.HEAD_CLASSIFIER, 0)
        P.cbdfs_server_stop(ctx)
        # after a wider network moved the scratch, a new server serves the first network unchanged
        P.cbdfs_net_load(ctx, P.DOM_RC3, W2, b2, PREC["bf16"], P.HEAD_CLASSIFIER, 0)
        s = W.random_stp_states(4, 3000, 99)
        g = np.zeros(len(s), np.uint8)
        want = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 50)[0]
        P.cbdfs_server_start(ctx, max_inflight=2, coalesce=1)
        h, _, _ = P.heur_request_submit(ctx, hid, P.DOM_STP4, s, g, 50).wait()
        assert np.array_equal(h, want)
        P.cbdfs_server_stop(ctx)
        with pytest.raises(P.CbdfsError):
            P.heur_request_submit(ctx, hid, P.DOM_STP4, np.zeros(8, np.uint64), np.zeros(8, np.uint8), 1)
    finally:
        P.cbdfs_destroy(ctx)


@pytest.mark.parametrize("threads,depth", [(64, 1), (8, 8)])
def test_native_clients_mixed_burst(P, threads, depth):
    # a burst of 15-puzzle (81-class and regression networks, Manhattan distance) and cube
    # requests from native client threads; requests queue behind the launch in flight, are
    # packed at 32-row boundaries and bound-tested on the device with their own bounds: each
    # result is bit for bit the one the request gets alone
    ctx = P.cbdfs_create(0, max_batch=8192, n_slots=4)
    try:
        W1, b1 = W.net_weights(**W.NET_C3)
        W2, b2 = W.net_weights(**W.NET_C2)
        ids = {0: P.cbdfs_net_load(ctx, P.DOM_STP4, W1, b1, PREC["bf16"], P.HEAD_CLASSIFIER, 1),
               1: P.cbdfs_net_load(ctx, P.DOM_RC3, W2, b2, PREC["bf16"], P.HEAD_CLASSIFIER, 0),
               2: P.HEUR_MD}
        reqs = _mix(P, 300, 901 + threads)
        inputs = [_inputs(P, kind, size, seed) for kind, size, bound, seed in reqs]
        alone = [P.heur_submit_batch(ctx, ids[kind], dom, s, g, bound)
                 for (kind, size, bound, seed), (dom, s, g) in zip(reqs, inputs)]
        P.cbdfs_server_start(ctx, max_inflight=2, bucket_max=8192, coalesce=1)
        secs, got = P.cbdfs_server_drive(
            ctx, [(ids[kind], dom, s, g, bound) for (kind, size, bound, seed), (dom, s, g) in zip(reqs, inputs)],
            threads=threads, depth=depth)
        st = P.cbdfs_server_get_stats(ctx)
        P.cbdfs_server_stop(ctx)
        for i, ((h, mask, minf), (ah, amask, aminf)) in enumerate(zip(got, alone)):
            assert np.array_equal(h, ah), f"request {i}: h differs"
            assert np.array_equal(mask, amask) and minf == aminf, f"request {i}: bound test differs"
        print(f"{threads} clients x {depth}: {st['launches']} launches for {len(reqs)} requests, "
              f"{st['states'] / secs / 1e6:.1f} M states/s, p50 {st['p50_us']:.0f} us")
        assert st["requests"] == len(reqs) and st["launches"] < len(reqs)  # requests were merged
        assert P.cbdfs_device_status(ctx) == 0
    finally:
        P.cbdfs_destroy(ctx)


def test_request_sizes_at_the_bucket_limit(P):
    # requests whose 32-row packing reaches the largest bucket, with a bucket limit that is not
    # a multiple of 32: every one is served and equals its stand-alone result
    ctx = P.cbdfs_create(0, max_batch=4096, n_slots=2)
    try:
        ids = {2: P.HEUR_MD}
        P.cbdfs_server_start(ctx, max_inflight=1, bucket_min=24, bucket_max=1000, coalesce=1)
        reqs = [(2, n, 40, 7000 + n) for n in (1, 31, 33, 1000, 999, 968, 500, 501, 32, 64)]
        inputs = [_inputs(P, kind, size, seed) for kind, size, bound, seed in reqs]
        alone = [P.heur_submit_batch(ctx, P.HEUR_MD, dom, s, g, bound)
                 for (kind, size, bound, seed), (dom, s, g) in zip(reqs, inputs)]
        secs, got = P.cbdfs_server_drive(
            ctx, [(ids[kind], dom, s, g, bound) for (kind, size, bound, seed), (dom, s, g) in zip(reqs, inputs)],
            threads=2, depth=5)
        P.cbdfs_server_stop(ctx)
        for (h, mask, minf), (ah, amask, aminf) in zip(got, alone):
            assert np.array_equal(h, ah) and np.array_equal(mask, amask) and minf == aminf
    finally:
        P.cbdfs_destroy(ctx)
