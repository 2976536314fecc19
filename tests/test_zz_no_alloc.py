"""heur_eval_device_static: the allocation-free evaluation entry point, for callers that
cannot allocate device memory while they evaluate a batch.  Its results must equal those of
heur_eval_device (the same kernels on the same inputs, so the integers are identical) on two
calls in a row, and a batch beyond its fixed scratch limit must be refused.  This file is
collected last and must pass both alone and after the other tests."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_static_entry_matches_allocating_entry():
    import torch

    import paper_2507_11916_b300 as P
    dev = torch.device("cuda:0")
    ctx = P.cbdfs_create(0, max_batch=16384, n_slots=1)
    try:
        Ws, bs = W.net_weights(**W.NET_C1)
        hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, P.PREC_BF16, P.HEAD_REGRESSION, 1)
        stream = torch.cuda.current_stream()
        # two calls in a row, of different sizes: the second must not see the first's scratch
        for call, n in enumerate((8192, 1000)):
            s = W.random_stp_states(4, n, 555 + call)
            g = (W.splitmix64_array(556 + call, n) % np.uint64(60)).astype(np.uint8)
            ds = torch.from_numpy(s.view(np.int64)).to(dev)
            dg = torch.from_numpy(g).to(dev)
            out = []
            for fn in (P.heur_eval_device, P.heur_eval_device_static):
                dh = torch.empty(n, dtype=torch.uint8, device=dev)
                dm = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
                dmin = torch.empty(1, dtype=torch.int32, device=dev)
                fn(ctx, hid, P.DOM_STP4, ds, dg, 50, n, dh, dm, dmin, stream=stream)
                torch.cuda.synchronize()
                out.append((dh.cpu().numpy(), dm.cpu().numpy(), int(dmin.cpu().numpy()[0])))
            assert np.array_equal(out[0][0], out[1][0]), f"h differs on call {call}"
            assert np.array_equal(out[0][1], out[1][1]), f"mask differs on call {call}"
            assert out[0][2] == out[1][2]
        # beyond the 16 MiB per-buffer limit: 8320 states x 1024 x 2 bytes
        n = 8320
        ds = torch.zeros(n, dtype=torch.int64, device=dev)
        dg = torch.zeros(n, dtype=torch.uint8, device=dev)
        dh = torch.empty(n, dtype=torch.uint8, device=dev)
        dm = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
        dmin = torch.empty(1, dtype=torch.int32, device=dev)
        with pytest.raises(P.CbdfsError) as e:
            P.heur_eval_device_static(ctx, hid, P.DOM_STP4, ds, dg, 50, n, dh, dm, dmin, stream=stream)
        assert e.value.status == P.CBDFS_EINVAL and "at most 8192 states" in str(e.value)
        assert P.cbdfs_device_status(ctx) == 0
    finally:
        P.cbdfs_destroy(ctx)
