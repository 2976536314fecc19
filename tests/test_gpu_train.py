"""The learned heuristic: label walks, gradients of the BF16 training step against the
float64 oracle, the Adam update, and what a network trained on additive-PDB labels gains in
the search over Manhattan distance alone."""
import numpy as np
import pytest

import workloads as W
from helpers import PREC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2507_11916_b300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.cbdfs_create(0, max_batch=8192, n_slots=4)
    yield c
    P.cbdfs_destroy(c)


def _normwise(a, b):
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def test_walk_states_match_oracle(P, ctx, orc):
    tag, first, n = W.TAG_C3, 17, 3000
    gpu = P.cbdfs_gen_walk_states(ctx, P.DOM_STP4, tag, first, n, 250)
    for i in range(0, n, 61):
        dirs = W.stp_walk_random_length(4, 250, W.seed_for(tag, first + i))
        assert int(gpu[i]) == orc.stp_apply_walk(4, dirs)
    gpu3 = P.cbdfs_gen_walk_states(ctx, P.DOM_STP3, 7, 0, 200, 30)
    for i in range(0, 200, 13):
        assert int(gpu3[i]) == orc.stp_apply_walk(3, W.stp_walk_random_length(3, 30, W.seed_for(7, i)))


def _grad_case(P, ctx, orc, cfg, dom, head, loss, n, seed, label_hi):
    Ws, bs = W.net_weights(**cfg)
    hid = P.cbdfs_net_load(ctx, dom, Ws, bs, PREC["bf16"], head, 0)
    s = W.random_stp_states(4, n, seed)
    labels = (W.splitmix64_array(seed + 1, n) % np.uint64(label_hi)).astype(np.uint8)
    L, gw, gb = P.cbdfs_train_grad(ctx, hid, s, labels, cfg["dims"], loss)
    Wq = orc.quantise_weights(Ws[:-1], "bf16") + [Ws[-1]]
    kind = "ce" if loss == P.LOSS_CE else "mse"
    X = orc.one_hot(dom, s)
    ref64 = orc.train_forward_backward(Wq, bs, X, labels, kind)
    emu = orc.train_forward_backward(Wq, bs, X, labels, kind, bf16_storage=True)
    return hid, s, labels, Ws, bs, L, gw, gb, ref64, emu


# The training step stores hidden activations and hidden dZ in BF16.  Against the oracle's
# emulation of exactly that storage the gradients agree to 1e-2 normwise (the remaining
# difference is FP32 versus float64 accumulation); against plain float64 the BF16 storage
# itself moves them (ReLU units within a rounding step of 0 change side), by up to 0.1.
def _check_grads(L, gw, gb, ref64, emu):
    L64, gW64, gb64 = ref64
    Le, gWe, gbe = emu
    assert abs(L - Le) <= 1e-3 * abs(Le)
    for l in range(len(gw)):
        ew, eb = _normwise(gw[l], gWe[l]), _normwise(gb[l], gbe[l])
        fw = _normwise(gw[l], gW64[l])
        print(f"layer {l}: dW vs emulation {ew:.2e}, db {eb:.2e}; dW vs float64 {fw:.2e}")
        assert ew <= 1e-2 and eb <= 1e-2
        assert fw <= 0.1


@pytest.mark.parametrize("n", [300, 1024])
def test_gradients_match_oracle_ce(P, ctx, orc, n):
    _, _, _, _, _, L, gw, gb, ref64, emu = _grad_case(
        P, ctx, orc, W.NET_C3, P.DOM_STP4, P.HEAD_CLASSIFIER, P.LOSS_CE, n, 900 + n, 81)
    _check_grads(L, gw, gb, ref64, emu)


def test_gradients_match_oracle_mse(P, ctx, orc):
    _, _, _, _, _, L, gw, gb, ref64, emu = _grad_case(
        P, ctx, orc, W.NET_C1, P.DOM_STP4, P.HEAD_REGRESSION, P.LOSS_MSE, 640, 4242, 60)
    _check_grads(L, gw, gb, ref64, emu)


def test_adam_step_matches_oracle(P, ctx, orc):
    # the update is pinned given the gradients: one step of net_train on the whole set (one
    # batch) equals the oracle's Adam applied to the library's own gradients
    hid, s, labels, Ws, bs, L, gw, gb, _, _ = _grad_case(
        P, ctx, orc, W.NET_C3, P.DOM_STP4, P.HEAD_CLASSIFIER, P.LOSS_CE, 512, 77, 81)
    rep = P.net_train(ctx, hid, s, labels, batch=512, epochs=1, lr=1e-3, seed=5)
    assert rep["steps"] == 1
    Wn, bn = P.cbdfs_net_read(ctx, hid, W.NET_C3["dims"])
    # net_train visits the set in a permuted order, so its FP32 sums differ from the
    # natural-order gradient in the last bits; Adam's first step is about -lr*sign(g), so
    # gradients within that noise of zero (|g| < 1e-7, a handful of elements) may step either
    # way: those are held only to the step bound lr
    for got_all, w0_all, g_all in ((Wn, Ws, gw), (bn, bs, gb)):
        for l in range(len(Ws)):
            w0, g, got = w0_all[l].astype(np.float64), g_all[l].astype(np.float64), got_all[l]
            z = np.zeros_like(w0)
            want, _, _ = orc.adam_step(w0, g, z, z, 1)
            sig = np.abs(g) >= 1e-7
            assert np.allclose(got[sig], want[sig], rtol=1e-5, atol=2e-6)
            assert (np.abs(got[~sig] - w0[~sig]) <= 1e-3 * 1.001).all()
            zero = g == 0  # no gradient, no step
            assert np.array_equal(got[zero], w0[zero].astype(np.float32))
            assert ((~sig) & ~zero).mean() < 1e-2  # the exempt set stays small


def test_training_on_pdb_labels_gains_over_manhattan(P, ctx, orc):
    # labels: the additive 6-6-3 PDB on states of random walks from the goal (lengths 1..250)
    pats = [list(p) for p in orc.PATTERNS_663]
    tabs = [P.pdb_build(ctx, P.DOM_STP4, t) for t in pats]
    pdb = P.cbdfs_pdb_load(ctx, P.DOM_STP4, pats, tabs)
    n = 409600
    states = P.cbdfs_gen_walk_states(ctx, P.DOM_STP4, W.TAG_C3, 0, n, 250)
    labels = np.concatenate([
        P.heur_submit_batch(ctx, pdb, P.DOM_STP4, states[o:o + 8192], np.zeros(min(8192, n - o), np.uint8), 255)[0]
        for o in range(0, n, 8192)])
    assert labels.max() <= 80
    Ws, bs = W.net_weights(**W.NET_C3)
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_CLASSIFIER, 1)
    rep = P.net_train(ctx, hid, states, labels, batch=8192, epochs=3, lr=1e-3, seed=3)
    print("train report", rep)
    assert rep["last_loss"] < 0.6 * rep["first_loss"]
    # held-out states: predicted class (network alone) against the PDB value
    held = P.cbdfs_gen_walk_states(ctx, P.DOM_STP4, W.TAG_C3, 10_000_000, 8192, 250)
    plain = P.cbdfs_net_load(ctx, P.DOM_STP4, *P.cbdfs_net_read(ctx, hid, W.NET_C3["dims"]),
                             PREC["bf16"], P.HEAD_CLASSIFIER, 0)
    h_nn = P.heur_submit_batch(ctx, plain, P.DOM_STP4, held, np.zeros(8192, np.uint8), 255)[0]
    h_pdb = P.heur_submit_batch(ctx, pdb, P.DOM_STP4, held, np.zeros(8192, np.uint8), 255)[0]
    md = np.array([orc.stp_md(int(x), 4) for x in held])
    err = np.abs(h_nn.astype(int) - h_pdb.astype(int))
    print(f"held-out: mean |h_nn - h_pdb| {err.mean():.2f}, exact {np.mean(err == 0):.3f}, "
          f"inadmissible vs PDB {np.mean(h_nn > h_pdb):.3f}, mean MD {md.mean():.1f}, "
          f"mean PDB {h_pdb.mean():.1f}, mean NN {h_nn.mean():.1f}")
    assert np.mean(np.abs(h_nn.astype(int) - h_pdb.astype(int))) < np.mean(h_pdb.astype(int) - md)
    # the search: max(network, MD) expands fewer nodes than MD alone
    tot_md = tot_nn = 0
    for i in range(6):
        s = orc.stp_apply_walk(4, W.stp_walk(4, 50, W.seed_for(W.TAG_C1, 7000 + i)))
        a = P.cbdfs_solve(ctx, P.DOM_STP4, s, P.ALGO_IDA, P.HEUR_MD, threads=8, work_num=16,
                          batch=2048, timeout_us=300, time_limit_s=60)
        b = P.cbdfs_solve(ctx, P.DOM_STP4, s, P.ALGO_IDA, hid, threads=8, work_num=16,
                          batch=2048, timeout_us=300, time_limit_s=60)
        assert b["cost"] >= a["cost"]
        tot_md += a["expanded"]
        tot_nn += b["expanded"]
        print(f"instance {i}: MD cost {a['cost']} expanded {a['expanded']}; "
              f"network cost {b['cost']} expanded {b['expanded']}")
    assert tot_nn < tot_md


def test_checkpoint_resume_continues_exactly(P, ctx, orc, tmp_path):
    # train, save, train on: a second network loaded from the checkpoint and trained on the same
    # way ends with the same weights bit for bit, and right after the load it evaluates exactly
    # as the first network did when it was saved (its BF16 weights and FP32 head rewritten)
    dims = W.NET_C3["dims"]
    Ws, bs = W.net_weights(**W.NET_C3)
    s = W.random_stp_states(4, 3072, 321)
    labels = (W.splitmix64_array(322, 3072) % np.uint64(81)).astype(np.uint8)
    probe = W.random_stp_states(4, 1000, 323)
    g0 = np.zeros(1000, np.uint8)
    a = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_CLASSIFIER, 0)
    P.net_train(ctx, a, s, labels, batch=1024, epochs=1, lr=1e-3, seed=5)
    path = tmp_path / "c3.ckpt"
    P.cbdfs_train_save(ctx, a, path)
    h_saved, _, _, y_saved = P.heur_submit_batch(ctx, a, P.DOM_STP4, probe, g0, 255, want_y=True, n_out=81)
    W_saved, b_saved = P.cbdfs_net_read(ctx, a, dims)
    P.net_train(ctx, a, s, labels, batch=1024, epochs=1, lr=1e-3, seed=6)
    Wa, ba = P.cbdfs_net_read(ctx, a, dims)

    b = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, PREC["bf16"], P.HEAD_CLASSIFIER, 0)
    P.cbdfs_train_load(ctx, b, path)
    Wl, bl = P.cbdfs_net_read(ctx, b, dims)
    assert all(np.array_equal(x, y) for x, y in zip(Wl + bl, W_saved + b_saved))
    h_loaded, _, _, y_loaded = P.heur_submit_batch(ctx, b, P.DOM_STP4, probe, g0, 255, want_y=True, n_out=81)
    assert np.array_equal(h_loaded, h_saved) and np.array_equal(y_loaded, y_saved)
    P.net_train(ctx, b, s, labels, batch=1024, epochs=1, lr=1e-3, seed=6)
    Wb, bb = P.cbdfs_net_read(ctx, b, dims)
    assert all(np.array_equal(x, y) for x, y in zip(Wb + bb, Wa + ba))

    # another shape, or a damaged file, is refused and leaves the network as it was
    c1 = P.cbdfs_net_load(ctx, P.DOM_STP4, *W.net_weights(**W.NET_C1), PREC["bf16"], P.HEAD_REGRESSION, 1)
    with pytest.raises(P.CbdfsError):
        P.cbdfs_train_load(ctx, c1, path)
    raw = bytearray(path.read_bytes())
    raw[-5] ^= 0x40
    (tmp_path / "bad.ckpt").write_bytes(bytes(raw))
    with pytest.raises(P.CbdfsError):
        P.cbdfs_train_load(ctx, b, tmp_path / "bad.ckpt")
    assert all(np.array_equal(x, y) for x, y in zip(P.cbdfs_net_read(ctx, b, dims)[0], Wb))


def _fresh_c3(P, ctx):
    Ws, bs = W.net_weights(**W.NET_C3)
    return P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, P.PREC_BF16, P.HEAD_CLASSIFIER, 0)


def _same_weights(P, ctx, a, b):
    wa, ba = P.cbdfs_net_read(ctx, a, W.NET_C3["dims"])
    wb, bb = P.cbdfs_net_read(ctx, b, W.NET_C3["dims"])
    return all(np.array_equal(x, y) for x, y in zip(wa + ba, wb + bb))


def test_step_graph_matches_eager_steps(P, ctx):
    # a full batch is one replay of the captured step; a batch smaller than the configured
    # batch size runs the same kernels launched one by one.  512 states with batch 512 (three
    # replays) and with batch 640 (three eager steps of the same 512 rows in the same
    # permutations) must end bit-identical
    s = W.random_stp_states(4, 512, 41)
    labels = (W.splitmix64_array(42, 512) % np.uint64(81)).astype(np.uint8)
    a, b = _fresh_c3(P, ctx), _fresh_c3(P, ctx)
    ra = P.net_train(ctx, a, s, labels, batch=512, epochs=3, lr=1e-3, seed=7)
    rb = P.net_train(ctx, b, s, labels, batch=640, epochs=3, lr=1e-3, seed=7)
    assert ra["steps"] == rb["steps"] == 3
    assert ra["last_loss"] == rb["last_loss"]
    assert _same_weights(P, ctx, a, b)
    assert P.cbdfs_device_status(ctx) == 0


def test_epochs_with_a_partial_batch_are_deterministic(P, ctx):
    # 1124 states in batches of 512: two replays and one partial eager step per epoch, the next
    # epoch's order drawn while the current one runs; two runs end bit-identical, and a step
    # limit stops inside an epoch
    s = W.random_stp_states(4, 1124, 43)
    labels = (W.splitmix64_array(44, 1124) % np.uint64(81)).astype(np.uint8)
    a, b, c = _fresh_c3(P, ctx), _fresh_c3(P, ctx), _fresh_c3(P, ctx)
    ra = P.net_train(ctx, a, s, labels, batch=512, epochs=3, lr=1e-3, seed=9)
    rb = P.net_train(ctx, b, s, labels, batch=512, epochs=3, lr=1e-3, seed=9)
    assert ra["steps"] == rb["steps"] == 9
    assert np.isfinite(ra["last_loss"]) and ra["last_loss"] < ra["first_loss"]
    assert _same_weights(P, ctx, a, b)
    rc = P.net_train(ctx, c, s, labels, batch=512, epochs=3, lr=1e-3, seed=9, max_steps=4)
    assert rc["steps"] == 4
    assert not _same_weights(P, ctx, a, c)
    assert P.cbdfs_device_status(ctx) == 0
