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


def _eval_both(P, ctx, hid, dom, s, g, bound, n, stream, dev):
    import torch
    ds = torch.from_numpy(np.ascontiguousarray(s).reshape(-1).view(np.int64)).to(dev)
    dg = torch.from_numpy(g).to(dev)
    out = []
    for fn in (P.heur_eval_device, P.heur_eval_device_static):
        dh = torch.empty(n, dtype=torch.uint8, device=dev)
        dm = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
        dmin = torch.empty(1, dtype=torch.int32, device=dev)
        fn(ctx, hid, dom, ds, dg, bound, n, dh, dm, dmin, stream=stream)
        torch.cuda.synchronize()
        out.append((dh.cpu().numpy(), dm.cpu().numpy().view(np.uint32), int(dmin.cpu().numpy().view(np.uint32)[0])))
    return out


def test_static_entry_fp32_network_and_its_limit():
    # An FP32 network stores its activations in FP32 (4 bytes): the 16 MiB buffer holds 4096
    # states of a 1024-wide network, and both entries run the same CUDA-core kernels.
    import torch

    import paper_2507_11916_b300 as P
    dev = torch.device("cuda:0")
    ctx = P.cbdfs_create(0, max_batch=8192, n_slots=1)
    try:
        Ws, bs = W.net_weights(**W.NET_C1)
        hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, P.PREC_FP32, P.HEAD_REGRESSION, 1)
        stream = torch.cuda.current_stream()
        for call, n in enumerate((4096, 777)):
            s = W.random_stp_states(4, n, 651 + call)
            g = (W.splitmix64_array(652 + call, n) % np.uint64(60)).astype(np.uint8)
            a, b = _eval_both(P, ctx, hid, P.DOM_STP4, s, g, 50, n, stream, dev)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
        n = 4097
        z = np.zeros(n, np.uint64)
        with pytest.raises(P.CbdfsError) as e:
            _eval_both(P, ctx, hid, P.DOM_STP4, z, np.zeros(n, np.uint8), 50, n, stream, dev)
        assert e.value.status == P.CBDFS_EINVAL and "at most 4096 states" in str(e.value)
        assert P.cbdfs_device_status(ctx) == 0
    finally:
        P.cbdfs_destroy(ctx)


def test_static_entry_cube_classifier(orc):
    # The cube network (two 64-bit words per state, 480-wide one-hot rows, 21 classes): the
    # allocating entry runs the fused chain and the tensor-core head, the static entry the
    # per-layer kernels and the CUDA-core head.  Their last layers round in different orders, so
    # h may differ only where the two largest logits lie within 1e-4; each mask and least f is
    # the bound test of its own h.
    import torch

    import paper_2507_11916_b300 as P
    from helpers import oracle_net
    dev = torch.device("cuda:0")
    ctx = P.cbdfs_create(0, max_batch=8192, n_slots=1)
    try:
        Ws, bs = W.net_weights(**W.NET_C2)
        hid = P.cbdfs_net_load(ctx, P.DOM_RC3, Ws, bs, P.PREC_BF16, P.HEAD_CLASSIFIER, 0)
        stream = torch.cuda.current_stream()
        for call, n in enumerate((2000, 129)):
            s = W.random_rc_states(n, 661 + call)
            g = (W.splitmix64_array(662 + call, n) % np.uint64(20)).astype(np.uint8)
            a, b = _eval_both(P, ctx, hid, P.DOM_RC3, s, g, 25, n, stream, dev)
            y64, _, _ = oracle_net(orc, P.DOM_RC3, Ws, bs, "bf16", s, "classifier")
            tie = orc.classifier_margin(y64, 1e-4)
            assert np.array_equal(a[0][~tie], b[0][~tie])
            for h, mask, minf in (a, b):
                wm, wf = orc.bound_test(g, h, 25)
                assert np.array_equal(mask, wm) and minf == wf
        # a 2048-wide BF16 network fits 4096 states in a 16 MiB buffer; 4097 are refused
        n = 4097
        with pytest.raises(P.CbdfsError) as e:
            _eval_both(P, ctx, hid, P.DOM_RC3, np.zeros((n, 2), np.uint64), np.zeros(n, np.uint8), 25, n, stream, dev)
        assert e.value.status == P.CBDFS_EINVAL and "at most 4096 states" in str(e.value)
        assert P.cbdfs_device_status(ctx) == 0
    finally:
        P.cbdfs_destroy(ctx)
