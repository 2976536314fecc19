"""Failure detection on the device without a fault: a bounded wait inside the fused network
kernel is made to run out, and the host reads the status.

cbdfs_debug_withhold_publish makes the next launch skip one row block's first-layer
completion count, so the second layer's tiles of that row block wait for rows that never come
(a flag that nothing sets).  With a 5 ms bound their wait runs out; the kernel records the code
in the context's error flag, winds down (every other wait sees the flag and gives up) and ends.
The call reports CBDFS_ETIMEDOUT, cbdfs_device_status returns the dependency-wait code and
clears the flag and the counts left behind, and the next launch on the same context and slot
is bit-identical to a fresh context's."""
import numpy as np
import pytest

import workloads as W
from helpers import PREC

pytestmark = pytest.mark.gpu

DEVERR_DEPENDENCY = 5  # a chain tile waited for the previous layer's row block


@pytest.fixture(scope="module")
def P():
    import paper_2507_11916_b300 as P
    return P


def _batch(n, seed):
    s = W.random_stp_states(4, n, seed)
    g = (W.splitmix64_array(seed + 1, n) % np.uint64(50)).astype(np.uint8)
    return s, g


def _fresh(P, Ws, bs, s, g, bound):
    c = P.cbdfs_create(0, max_batch=8192, n_slots=1)
    try:
        hid = P.cbdfs_net_load(c, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_REGRESSION, 1)
        return P.heur_submit_batch(c, hid, P.DOM_STP4, s, g, bound)
    finally:
        P.cbdfs_destroy(c)


@pytest.mark.parametrize("row_block", [0, 37])
def test_dependency_wait_runs_out_and_the_context_recovers(P, row_block):
    Ws, bs = W.net_weights(**W.NET_C1)
    ctx = P.cbdfs_create(0, max_batch=8192, n_slots=1, device_wait_ns=5_000_000)
    try:
        hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_REGRESSION, 1)
        s, g = _batch(8192, 4400 + row_block)
        # an ordinary launch stays well inside the 5 ms bound
        first = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 50)
        assert P.cbdfs_device_status(ctx) == 0
        P.cbdfs_debug_withhold_publish(ctx, row_block)
        with pytest.raises(P.CbdfsError) as e:
            P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 50)
        assert e.value.status == P.CBDFS_ETIMEDOUT
        assert P.cbdfs_device_status(ctx) == DEVERR_DEPENDENCY
        assert P.cbdfs_device_status(ctx) == 0
        # the same slot again: bit for bit what the first launch and a fresh context give
        again = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 50)
        s2, g2 = _batch(3000, 4500 + row_block)
        other = P.heur_submit_batch(ctx, hid, P.DOM_STP4, s2, g2, 45)
        want = _fresh(P, Ws, bs, s2, g2, 45)
        for a, b in ((again, first), (other, want)):
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
        assert P.cbdfs_device_status(ctx) == 0
    finally:
        P.cbdfs_destroy(ctx)


def test_withhold_is_one_launch_only_and_validates(P):
    with pytest.raises(P.CbdfsError):
        P.cbdfs_debug_withhold_publish(None, 0)
    Ws, bs = W.net_weights(**W.NET_C1)
    ctx = P.cbdfs_create(0, max_batch=8192, n_slots=1, device_wait_ns=5_000_000)
    try:
        hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_REGRESSION, 1)
        s, g = _batch(1000, 4600)
        P.cbdfs_debug_withhold_publish(ctx, 3)
        P.cbdfs_debug_withhold_publish(ctx, -1)  # cleared again: nothing is held
        P.heur_submit_batch(ctx, hid, P.DOM_STP4, s, g, 50)
        assert P.cbdfs_device_status(ctx) == 0
    finally:
        P.cbdfs_destroy(ctx)
