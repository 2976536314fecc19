"""Pins of the oracle's network heuristic, quantisers and training math against closed
forms and library routines."""
import numpy as np
import pytest
import torch

import workloads as W


def _md_net(side):
    N = side * side
    w = np.zeros((1, N * N))
    for t in range(1, N):
        for p in range(N):
            w[0, t * N + p] = abs(p // side - t // side) + abs(p % side - t % side)
    return w


def test_linear_net_reproduces_manhattan(orc):
    # One linear layer whose weight at (tile t, cell p) is that tile's distance from home
    # computes Manhattan distance exactly: pins the one-hot layout and the forward pass.
    for side, dom in ((3, orc.DOM_STP3), (4, orc.DOM_STP4)):
        states = W.random_stp_states(side, 200, 17)
        y = orc.mlp_forward([_md_net(side)], [np.zeros(1)], orc.one_hot(dom, states))
        want = [orc.stp_md(int(s), side) for s in states]
        assert np.array_equal(y[:, 0], np.array(want, float))
        # through a ReLU identity layer too
        N2 = side ** 4
        y2 = orc.mlp_forward([np.eye(N2), _md_net(side)], [np.zeros(N2), np.zeros(1)],
                             orc.one_hot(dom, states))
        assert np.array_equal(y2, y)


def test_rc_one_hot_counts_misplaced_cubies(orc):
    w = np.zeros((1, 480))
    for c in range(8):
        for f in range(24):
            w[0, c * 24 + f] = float(f // 3 != c)
    for e in range(12):
        for f in range(24):
            w[0, 192 + e * 24 + f] = float(f // 2 != e)
    g = orc.rc_goal()
    one_u = orc.rc_apply(g, 0)     # U moves 4 corners and 4 edges
    y = orc.mlp_forward([w], [np.zeros(1)], orc.one_hot(orc.DOM_RC3, [g, one_u]))
    assert list(y[:, 0]) == [0.0, 8.0]
    X = orc.one_hot(orc.DOM_RC3, W.random_rc_states(64, 3))
    assert (X.sum(axis=1) == 20).all()


def test_forward_matches_torch_float64(orc):
    Ws, bs = W.net_weights([81, 256, 256, 1], "uniform", 0)
    X = orc.one_hot(orc.DOM_STP3, W.random_stp_states(3, 100, 1))
    y = orc.mlp_forward(Ws, bs, X)
    t = torch.tensor(X, dtype=torch.float64)
    for l, (w, b) in enumerate(zip(Ws, bs)):
        t = torch.nn.functional.linear(t, torch.tensor(w, dtype=torch.float64),
                                       torch.tensor(b, dtype=torch.float64))
        if l < len(Ws) - 1:
            t = torch.relu(t)
    assert np.allclose(y, t.numpy(), rtol=1e-12, atol=1e-12)


def test_integer_h_rules(orc):
    y = np.array([2.5, 3.5, -0.7, 0.49, 7.51, 300.0, 1.0])
    md = np.array([0, 0, 0, 0, 0, 0, 5])
    assert list(orc.h_regression(y, md)) == [2, 4, 0, 0, 8, 255, 5]
    goal = np.array([False] * 6 + [True])
    assert orc.h_regression(y, md, goal)[-1] == 0
    logits = np.array([[0.1, 0.3, 0.3], [1.0, -1.0, 0.0]])
    assert list(orc.h_classifier(logits)) == [1, 0]
    assert list(orc.h_classifier(logits, md=np.array([0, 4]))) == [1, 4]
    assert list(orc.regression_margin(np.array([2.495, 2.48, 0.5]))) == [True, False, True]


def test_bound_test(orc):
    g = np.arange(40) % 7
    h = (np.arange(40) * 5) % 11
    words, minf = orc.bound_test(g, h, 8)
    f = g + h
    for i in range(40):
        assert bool((int(words[i // 32]) >> (i % 32)) & 1) == (f[i] <= 8)
    assert minf == f[f > 8].min()
    assert orc.bound_test([0], [0], 5)[1] == 0xFFFFFFFF


def test_bf16_round_matches_torch(orc):
    x = np.concatenate([W._normal_array(5, 20000).astype(np.float32) * 3,
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8], np.float32)])
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(orc.bf16_round(x), ref)
    assert orc.bf16_round(np.float32(1 + 2 ** -8)) == 1.0


def test_e4m3_round_matches_torch(orc):
    x = np.concatenate([W._normal_array(6, 20000).astype(np.float32) * 40,
                        np.array([0.0, 1.0625, 1.1875, 448.0, -300.0, 2 ** -9], np.float32)])
    x = np.clip(x, -448, 448).astype(np.float32)
    ref = torch.tensor(x).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    assert np.array_equal(orc.e4m3_round(x), ref)
    assert orc.e4m3_round(np.float32(1000.0)) == 448.0


def _tiny(seed):
    Ws, bs = W.net_weights([16, 8, 4], "uniform", seed)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((5, 16))
    return [w.astype(np.float64) for w in Ws], [b.astype(np.float64) for b in bs], X


@pytest.mark.parametrize("loss", ["ce", "mse"])
def test_gradients_match_finite_differences(orc, loss):
    Ws, bs, X = _tiny(3)
    if loss == "mse":
        Ws[-1], bs[-1] = Ws[-1][:1], bs[-1][:1]
        labels = np.array([0.5, 1.0, -2.0, 3.0, 0.0])
    else:
        labels = np.array([0, 3, 1, 2, 3])
    L, gW, gb = orc.train_forward_backward(Ws, bs, X, labels, loss)
    eps = 1e-6
    for l in range(2):
        for arr, g in ((Ws[l], gW[l]), (bs[l], gb[l])):
            num = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + eps
                Lp = orc.train_forward_backward(Ws, bs, X, labels, loss)[0]
                arr[idx] = old - eps
                Lm = orc.train_forward_backward(Ws, bs, X, labels, loss)[0]
                arr[idx] = old
                num[idx] = (Lp - Lm) / (2 * eps)
            assert np.linalg.norm(num - g) <= 1e-6 * max(1.0, np.linalg.norm(g))


def test_cross_entropy_of_uniform_logits(orc):
    Ws = [np.zeros((7, 16))]
    bs = [np.zeros(7)]
    L, _, _ = orc.train_forward_backward(Ws, bs, np.ones((3, 16)), np.array([0, 1, 6]))
    assert abs(L - np.log(7)) < 1e-12


def test_adam_matches_torch(orc):
    rng = np.random.default_rng(0)
    w0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(5)]
    # first step closed form: m_hat = g, v_hat = g^2
    w1, _, _ = orc.adam_step(w0, grads[0], np.zeros(50), np.zeros(50), 1)
    assert np.allclose(w1, w0 - 1e-3 * grads[0] / (np.abs(grads[0]) + 1e-8), rtol=0, atol=1e-15)
    p = torch.nn.Parameter(torch.tensor(w0))
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, 1):
        p.grad = torch.tensor(g)
        opt.step()
        w, m, v = orc.adam_step(w, g, m, v, t)
    assert np.allclose(w, p.detach().numpy(), rtol=0, atol=1e-14)


def test_fp8_quantised_weights_within_grid(orc):
    Ws, _ = W.net_weights([64, 32], "kaiming", 9)
    q = orc.quantise_weights(Ws, "fp8")[0]
    s = orc.fp8_weight_scale(Ws[0])
    assert np.abs(q).max() <= 448 * s * (1 + 1e-6)
    # relative error of E4M3 rounding is at most 2^-4 for normal values
    big = np.abs(Ws[0]) > 2 ** -6 * s
    assert (np.abs(q - Ws[0])[big] <= 2 ** -4 * np.abs(Ws[0])[big] + 1e-12).all()


def test_e4m3_activation_emulation(orc):
    # Activations that are exactly representable in E4M3 at the given scale are unchanged
    # by the emulation; others move by at most 2^-4 of their value (round to nearest).
    W1 = np.zeros((4, 16))
    W1[0, 0], W1[1, 1], W1[2, 2], W1[3, 3] = 2.0, 3.0, 0.5, 448.0
    Ws = [W1, np.eye(4), np.ones((1, 4))]
    bs = [np.zeros(4), np.zeros(4), np.zeros(1)]
    X = np.eye(16)[:4]
    plain = orc.mlp_forward(Ws, bs, X)
    emu = orc.mlp_forward(Ws, bs, X, act_scales=[1.0, 1.0])
    assert np.array_equal(plain, emu)
    W1[0, 0] = 2.3  # 2.3 is between E4M3 neighbours 2.25 and 2.5
    emu = orc.mlp_forward(Ws, bs, X, act_scales=[1.0, 1.0])
    assert emu[0, 0] == 2.25
    rng = np.random.default_rng(1)
    Ws2, bs2 = W.net_weights([16, 32, 32, 1], "kaiming", 5)
    X2 = rng.random((50, 16))
    _, hp = orc.mlp_forward(Ws2, bs2, X2, return_hidden=True)
    _, he = orc.mlp_forward(Ws2, bs2, X2, return_hidden=True, act_scales=[0.01, 0.01])
    big = hp[0] > 2 ** -6 * 0.01
    assert (np.abs(he[0] - hp[0])[big] <= 2 ** -4 * hp[0][big] + 1e-12).all()


def test_bf16_activation_storage_emulation(orc):
    # Stored activations that bfloat16 represents exactly are unchanged by the emulation.
    W1 = np.zeros((3, 16))
    W1[0, 0], W1[1, 1], W1[2, 2] = 2.0, 1.5, 0.375
    Ws = [W1, np.eye(3), np.ones((1, 3))]
    bs = [np.zeros(3), np.zeros(3), np.zeros(1)]
    X = np.eye(16)[:3]
    plain = orc.mlp_forward(Ws, bs, X)
    assert np.array_equal(plain, orc.mlp_forward(Ws, bs, X, bf16_acts=True, store_last=True))
    # Hand-worked: one input 1; first hidden layer a0 = (1 + 2^-8, 1 + 2^-7 + 2^-9);
    # second hidden layer a1 = a0[0] + a0[1] + 2^-10; y = a1.
    #  - plain float64: y = 2.013671875 + 2^-10 = 2.0146484375
    #  - bf16_acts: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 and goes to the even
    #    mantissa, 1.0; 1.009765625 is nearer 1.0078125 than 1.015625; a1 = 2.0087890625
    #  - store_last as well: at 2 the bfloat16 step is 2^-6, and 2.0087890625 is nearer
    #    2.015625 than 2.0, so y = 2.015625
    Ws = [np.array([[1 + 2 ** -8], [1 + 2 ** -7 + 2 ** -9]]), np.array([[1.0, 1.0]]), np.array([[1.0]])]
    bs = [np.zeros(2), np.array([2 ** -10]), np.zeros(1)]
    X = np.ones((1, 1))
    assert orc.mlp_forward(Ws, bs, X)[0, 0] == 2.0146484375
    assert orc.mlp_forward(Ws, bs, X, bf16_acts=True)[0, 0] == 2.0087890625
    assert orc.mlp_forward(Ws, bs, X, bf16_acts=True, store_last=True)[0, 0] == 2.015625
    # E4M3 activations (scale 1: step 1/8 at 1) with a BF16-stored last hidden layer:
    # a0 -> (1, 1), a1 = 2 + 2^-10 -> 2.0
    assert orc.mlp_forward(Ws, bs, X, act_scales=[1.0], store_last=True)[0, 0] == 2.0
    # and a random network: every stored value within half a bfloat16 step of the float64 one
    Ws2, bs2 = W.net_weights([16, 32, 32, 1], "kaiming", 5)
    X2 = np.random.default_rng(2).random((50, 16))
    _, hp = orc.mlp_forward(Ws2, bs2, X2, return_hidden=True)
    _, he = orc.mlp_forward(Ws2, bs2, X2, return_hidden=True, bf16_acts=True)
    assert (np.abs(he[0] - hp[0]) <= 2 ** -8 * hp[0] + 1e-30).all()
    assert np.array_equal(he[0], orc.bf16_round(hp[0].astype(np.float32)))


def test_bf16_storage_emulation(orc):
    # with every stored value exactly representable in bfloat16 the emulation changes nothing
    Ws = [np.array([[1.0, 0.5], [0.25, -1.0]]), np.array([[2.0, -0.5], [1.0, 1.0]]),
          np.array([[1.0, 1.0], [0.5, -1.0]])]
    bs = [np.zeros(2), np.array([0.5, 0.0]), np.zeros(2)]
    X = np.array([[1.0, 2.0], [3.0, 0.0]])
    a = orc.train_forward_backward(Ws, bs, X, np.array([0, 1]), "ce")
    b = orc.train_forward_backward(Ws, bs, X, np.array([0, 1]), "ce", bf16_storage=True)
    assert a[0] == b[0]
    # the first hidden layer's gradient only involves exact values here
    assert np.array_equal(a[1][0], b[1][0]) or np.allclose(a[1][0], b[1][0], rtol=2 ** -8)
    # and a random network moves by at most a few bfloat16 ulps per stored value
    Ws2, bs2 = W.net_weights([16, 32, 32, 4], "kaiming", 4)
    X2 = np.random.default_rng(0).random((20, 16))
    lab = np.arange(20) % 4
    g1 = orc.train_forward_backward(Ws2, bs2, X2, lab, "ce")
    g2 = orc.train_forward_backward(Ws2, bs2, X2, lab, "ce", bf16_storage=True)
    assert abs(g1[0] - g2[0]) < 1e-2 * abs(g1[0])


def test_md_plus_network_construction(orc):
    # The test network "Manhattan distance plus the seeded network's output" computes exactly
    # MD when the seeded part is scaled to zero, in float64 and with BF16 storage emulated.
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from helpers import md_plus_net
    Ws, bs = md_plus_net(*W.net_weights([256, 1024, 1024, 512, 1], "kaiming", 1), 4, scale=0.0, shift=0.0)
    s = W.random_stp_states(4, 100, 5)
    X = orc.one_hot(orc.DOM_STP4, s)
    md = orc.md_states(orc.DOM_STP4, s)
    assert np.array_equal(orc.mlp_forward(Ws, bs, X)[:, 0], md)
    Wq = orc.quantise_weights(Ws[:-1], "bf16") + [Ws[-1]]
    assert np.array_equal(orc.mlp_forward(Wq, bs, X, bf16_acts=True)[:, 0], md)
