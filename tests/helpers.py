"""Shared test helpers: oracle-side expected values for the network heuristic, and the
tolerance rule the parity tests use."""
import numpy as np

import workloads as W

# per-logit tolerance against float64 on the same quantised weights (workload statement)
RTOL = {"fp32": 1e-4, "bf16": 2e-2, "fp8": 6e-2}
PREC = {"fp32": 0, "bf16": 1, "fp8": 2}


def oracle_net(orc, dom, Ws, bs, prec, states, head="regression", max_with_md=False,
               act_scales=None):
    """Float64 outputs and integer h of the oracle, with the hidden layers' weights rounded
    to `prec` (the last layer stays float32, as the library keeps it).  With act_scales the
    E4M3 storage of the activations between tensor-core layers is emulated too."""
    Wq = orc.quantise_weights(Ws[:-1], prec) + [np.asarray(Ws[-1], np.float32)]
    y = orc.mlp_forward(Wq, bs, orc.one_hot(dom, states), act_scales=act_scales)
    goal = orc.is_goal_states(dom, states)
    md = orc.md_states(dom, states) if max_with_md else None
    # A rounding or argmax decision counts as a margin case when the boundary lies within
    # 1e-2 of the float64 value, or within the precision's own logit tolerance band.
    band = RTOL[prec] * (np.abs(y) + np.sqrt(np.mean(y ** 2)))
    if head == "regression":
        h = orc.h_regression(y[:, 0], md, goal)
        margin = orc.regression_margin(y[:, 0], np.maximum(1e-2, band[:, 0]))
    else:
        h = orc.h_classifier(y, md, goal)
        top = np.max(band, axis=1)
        margin = orc.classifier_margin(y, np.maximum(1e-2, 2 * top))
    return y, h, margin


def check_logits(y_gpu, y64, prec):
    """|y - y64| <= rtol * (|y64| + rms(y64)) elementwise; returns the worst ratio."""
    y_gpu = np.asarray(y_gpu, np.float64)
    scale = np.abs(y64) + np.sqrt(np.mean(y64 ** 2)) + 1e-30
    ratio = np.abs(y_gpu - y64) / scale
    worst = float(ratio.max()) / RTOL[prec]
    assert worst <= 1.0, f"logit error {worst:.3f} x tolerance ({prec})"
    return worst


def check_h(h_gpu, h64, margin):
    """Integer h equal except margin cases; returns the number of margin mismatches."""
    diff = np.asarray(h_gpu, np.int64) != np.asarray(h64, np.int64)
    assert not (diff & ~margin).any(), f"h differs outside the margin at {np.nonzero(diff & ~margin)[0][:10]}"
    return int(diff.sum())


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
