"""Shared test helpers: oracle-side expected values for the network heuristic, and the
tolerance rules the parity tests use.

Expected values come from the oracle's float64 forward pass on the same quantised weights,
with the activations the library stores between layers rounded to the library's storage
format (BF16, or E4M3 with static per-layer scales; BF16 for a last hidden layer that a
separate last-layer step reads back).  The workload statement's standards then apply as
written:

* per logit, |y - y_oracle| <= rtol * max(|y_oracle|, rms(y_oracle)) with rtol 1e-4 (FP32),
  2e-2 (BF16) or 6e-2 (FP8): relative, with the batch's RMS logit as the floor for logits
  near zero (a relative bound alone is undefined at y = 0);
* integer h equal to the oracle's, except margin cases: rows whose pre-rounding value, or
  top-two logit gap, lies within exactly 1e-2 of a boundary that changes the final h (after
  the max with Manhattan distance).  Margin cases are counted, not failed.

Against plain float64 (no storage rounding) the integer h is compared too, and its mismatches
are counted and reported, not exempted."""
import numpy as np

import workloads as W

# per-logit tolerance against float64 on the same quantised weights (workload statement)
RTOL = {"fp32": 1e-4, "bf16": 2e-2, "fp8": 6e-2}
PREC = {"fp32": 0, "bf16": 1, "fp8": 2}
MARGIN = 1e-2  # the workload statement's integer-h margin


def last_hidden_stored(prec, head, C, dims=None, per_layer=False):
    """Whether the library writes the last hidden layer to memory (in BF16) before the last
    layer runs: always on the per-layer path; on the fused chain only when the last layer is
    a separate step (classifier heads of more than 16 outputs, regression heads of more than
    32) or when a hidden width is not a multiple of 256 (no fused chain).  FP32 networks keep
    FP32 throughout."""
    if prec == "fp32":
        return False
    if per_layer or (dims is not None and any(d % 256 for d in dims[1:-1])):
        return True
    if head in ("regression", "real"):
        return C > 32
    return C > 16


def oracle_forward(orc, dom, Ws, bs, prec, states, head="regression", act_scales=None,
                   emulate=True, per_layer=False):
    """The oracle's float64 outputs on the weights the precision evaluates (the hidden layers'
    weights rounded to `prec`, the last layer float32).  emulate: round the activations the
    library stores (BF16, or E4M3 with act_scales, between hidden layers; BF16 for a stored
    last hidden layer)."""
    Wq = orc.quantise_weights(Ws[:-1], prec) + [np.asarray(Ws[-1], np.float32)]
    kw = {}
    if emulate and prec != "fp32":
        C = np.asarray(Ws[-1]).shape[0]
        dims = [np.asarray(Ws[0]).shape[1]] + [np.asarray(w).shape[0] for w in Ws]
        kw = dict(act_scales=act_scales, bf16_acts=act_scales is None,
                  store_last=last_hidden_stored(prec, head, C, dims, per_layer))
    return orc.mlp_forward(Wq, bs, orc.one_hot(dom, states), **kw)


def h_margin(orc, y, head, md=None, goal=None, width=MARGIN):
    """Rows whose final integer h could change if the pre-rounding value (regression) or any
    logit within `width` of the largest (classifier) decided it: the integer rule applied at
    y - width and y + width differs (regression; h is nondecreasing in y), or the classes
    whose logits lie within `width` of the largest do not all give the same final h after
    the max with Manhattan distance (classifier).  The goal row is never a margin case."""
    y = np.asarray(y, np.float64)
    if head == "regression":
        lo = orc.h_regression(y[:, 0] - width, md, goal)
        hi = orc.h_regression(y[:, 0] + width, md, goal)
        return lo != hi
    top = y.max(axis=1, keepdims=True)
    near = y > top - width
    mdv = np.zeros(len(y), np.int64) if md is None else np.asarray(md, np.int64)
    cls = np.arange(y.shape[1])[None, :]
    final = np.minimum(np.maximum(cls, mdv[:, None]), 255)
    fmin = np.where(near, final, 1 << 30).min(axis=1)
    fmax = np.where(near, final, -1).max(axis=1)
    m = fmin != fmax
    if goal is not None:
        m &= ~np.asarray(goal, bool)
    return m


def oracle_net(orc, dom, Ws, bs, prec, states, head="regression", max_with_md=False,
               act_scales=None, emulate=True, per_layer=False):
    """Float64 outputs (storage emulated, see oracle_forward), the integer h of the oracle's
    rule and the margin flags (exactly 1e-2)."""
    y = oracle_forward(orc, dom, Ws, bs, prec, states, head, act_scales, emulate, per_layer)
    goal = orc.is_goal_states(dom, states)
    md = orc.md_states(dom, states) if max_with_md else None
    if head == "regression":
        h = orc.h_regression(y[:, 0], md, goal)
    else:
        h = orc.h_classifier(y, md, goal)
    return y, h, h_margin(orc, y, head, md, goal)


def plain_mismatches(orc, dom, Ws, bs, prec, states, h_gpu, head="regression",
                     max_with_md=False):
    """Integer-h mismatches against plain float64 (no storage rounding) on the same quantised
    weights: (mismatches, of which inside the 1e-2 margin).  Reported, not failed."""
    y, h, m = oracle_net(orc, dom, Ws, bs, prec, states, head, max_with_md, emulate=False)
    diff = np.asarray(h_gpu, np.int64) != h
    return int(diff.sum()), int((diff & m).sum())


def logit_ratio(y_gpu, y64, prec):
    """Worst |y - y64| / (rtol * max(|y64|, rms(y64))) over the logits."""
    y_gpu = np.asarray(y_gpu, np.float64)
    y64 = np.asarray(y64, np.float64)
    floor = np.sqrt(np.mean(y64 ** 2)) + 1e-30
    return float((np.abs(y_gpu - y64) / np.maximum(np.abs(y64), floor)).max()) / RTOL[prec]


def check_logits(y_gpu, y64, prec):
    """Per logit |y - y64| <= rtol * max(|y64|, rms(y64)); returns the worst ratio."""
    worst = logit_ratio(y_gpu, y64, prec)
    assert worst <= 1.0, f"logit error {worst:.3f} x tolerance ({prec})"
    return worst


def check_h(h_gpu, h64, margin):
    """Integer h equal except margin cases; returns the number of margin mismatches."""
    diff = np.asarray(h_gpu, np.int64) != np.asarray(h64, np.int64)
    assert not (diff & ~margin).any(), f"h differs outside the margin at {np.nonzero(diff & ~margin)[0][:10]}"
    return int(diff.sum())


def report(tag, h_gpu, h64, margin, plain=None):
    """One line of counts for the log: rows, margin cases, mismatches inside the margin, and
    the mismatches against plain float64 when given."""
    diff = np.asarray(h_gpu, np.int64) != np.asarray(h64, np.int64)
    line = f"{tag}: rows {len(diff)}, margin cases {int(margin.sum())}, mismatches (all in margin) {int(diff.sum())}"
    if plain is not None:
        line += f"; vs plain float64 {plain[0]} ({plain[1]} in margin)"
    print(line)


def md_plus_net(Ws, bs, side, scale=4.0, shift=1.5):
    """A network of the given shape whose output is Manhattan distance plus the seeded
    network's own output scaled by `scale`, plus `shift`: y = MD(s) + scale * y_net(s) +
    shift.  Hidden unit 0 of the first layer sums the tiles' distances from home (one-hot
    index tile*N + cell), later hidden layers pass unit 0 on with weight 1 and keep it out of
    the other units, and the last layer reads it with weight 1.  With the max with MD the
    network then decides h wherever y_net(s) > (0.5 - shift) / scale: most states, for the
    defaults.  Exact in every precision for the Manhattan part up to the weight rounding of
    the precision (E4M3 rounds the unit weights)."""
    Ws = [np.array(w, np.float32, copy=True) for w in Ws]
    bs = [np.array(b, np.float32, copy=True) for b in bs]
    N = side * side
    w0 = np.zeros(Ws[0].shape[1], np.float32)
    for t in range(1, N):
        for p in range(N):
            w0[t * N + p] = abs(p // side - t // side) + abs(p % side - t % side)
    Ws[0][0, :] = w0
    bs[0][0] = 0.0
    for l in range(1, len(Ws) - 1):
        Ws[l][:, 0] = 0.0
        Ws[l][0, :] = 0.0
        Ws[l][0, 0] = 1.0
        bs[l][0] = 0.0
    Ws[-1] = Ws[-1] * np.float32(scale)
    Ws[-1][:, 0] = 1.0
    bs[-1] = bs[-1] * np.float32(scale) + np.float32(shift)
    return Ws, bs


def stp_states(side, n, seed):
    return W.random_stp_states(side, n, seed)


def rc_states(n, seed):
    return W.random_rc_states(n, seed)


def fp8_act_scales(orc, dom, Ws, bs, states, margin=1.0):
    """Static per-layer activation scales for the FP8 form: the largest float64 activation of
    each hidden layer over calibration states (on the E4M3-rounded weights), divided by 448."""
    Wq = orc.quantise_weights(Ws[:-1], "fp8") + [np.asarray(Ws[-1], np.float32)]
    _, hidden = orc.mlp_forward(Wq, bs, orc.one_hot(dom, states), return_hidden=True)
    return np.array([max(float(a.max()), 1e-6) * margin / 448.0 for a in hidden], np.float32)


def normwise(y_gpu, y64):
    y64 = np.asarray(y64, np.float64)
    return float(np.linalg.norm(np.asarray(y_gpu, np.float64) - y64) / np.linalg.norm(y64))


def cube_classifier_net(Ws, bs, noise=0.3):
    """A cube classifier of the given shape (480 -> H1 -> H2 -> H3 -> C, C >= 21) whose class
    logits are -|c - x(s)| plus `noise` times the seeded network's own logits, with x(s) =
    (cubies not in their home slot with zero twist or flip) / 8.  A face turn moves 8 cubies,
    so ceil(x) never exceeds the distance to the goal; the argmax lies near x, and the noise
    moves it where two classes are close, so the network, not a fixed rule, decides h.
    Hidden unit 0 of the first layer computes x (weight 1/8 on every one-hot entry other than
    a cubie's home entry); units 1..2C of the second compute relu(x - c) and relu(c - x);
    the third passes them on; the last layer adds each class's pair with weight -1.  Every
    weight and stored value of that part is exact in BF16."""
    Ws = [np.array(w, np.float32, copy=True) for w in Ws]
    bs = [np.array(b, np.float32, copy=True) for b in bs]
    C = Ws[-1].shape[0]
    k = 1 + 2 * C  # units carrying the construction in the second and third hidden layers
    w0 = np.full(Ws[0].shape[1], 0.125, np.float32)
    for c in range(8):
        w0[c * 24 + c * 3] = 0.0            # corner cubie c home: slot c, twist 0
    for e in range(12):
        w0[192 + e * 24 + e * 2] = 0.0      # edge cubie e home: slot e, flip 0
    Ws[0][0, :] = w0
    bs[0][0] = 0.0
    W1, b1 = Ws[1], bs[1]
    W1[:k, :] = 0.0
    W1[k:, 0] = 0.0
    b1[:k] = 0.0
    for c in range(C):
        W1[1 + 2 * c, 0], b1[1 + 2 * c] = 1.0, -float(c)
        W1[2 + 2 * c, 0], b1[2 + 2 * c] = -1.0, float(c)
    for l in range(2, len(Ws) - 1):
        Ws[l][:k, :] = 0.0
        Ws[l][k:, :k] = 0.0
        for j in range(1, k):
            Ws[l][j, j] = 1.0
        bs[l][:k] = 0.0
    WL = Ws[-1] * np.float32(noise)
    WL[:, :k] = 0.0
    for c in range(C):
        WL[c, 1 + 2 * c] = -1.0
        WL[c, 2 + 2 * c] = -1.0
    Ws[-1] = WL
    bs[-1] = bs[-1] * np.float32(noise)
    return Ws, bs
