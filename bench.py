#!/usr/bin/env python3
"""Throughput of the batched neural-heuristic hot path of Batch CB-DFS on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (the 15-puzzle regression configuration): a batch of 8192 packed 15-puzzle states
resident in HBM, each with its path cost g, evaluated by the 256 -> 1024 -> 1024 -> 512 -> 1
ReLU network (Kaiming-normal weights, seed 1) in BF16 with FP32 accumulation and an FP32
last layer, then h = max(rint(y), 0, Manhattan distance) and the bound test g + h <= 50 with
the least f above the bound.  One step = one pass of that whole path over the batch (packed
state decode + one-hot encode, three tensor-core layers, the fused head), replayed from a
CUDA graph; the L2 is flushed (a 512 MB write) before every timed step, outside the timing.
Prints one JSON line.  With torchrun (N > 1) every rank evaluates its own batch (weak
scaling, replicas, no collective on the data path).

The reference arm (--impl reference) times the oracle -- the float64 CPU statement of the
same computation -- on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
import workloads as W  # noqa: E402

BATCH = 8192
BOUND = 50
FLUSH_BYTES = 512 << 20
METRIC = "NN heuristic states/s (15-puzzle regression net, BF16)"
CONFIG = {"workload": "15-puzzle regression heuristic: 256-1024-1024-512-1 BF16 MLP + "
                      "max(rint(y),0,MD) + bound test, 8192 packed states per step",
          "batch": BATCH, "bound": BOUND, "l2": "flushed before every timed step (512 MB write)",
          "inputs": "seeded uniformly random solvable 15-puzzle states, g uniform in 0..59"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"],
                    src="measured")
    return dict(hbm=6400.0, bf16=1800.0, bf16_sus=1400.0, src="fallback")


class Clocks:
    """nvidia-smi sampled every 100 ms while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for name, v in zip(names, r[2:6]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_traffic(key):
    """DRAM bytes per launch of the fused chain kernel from the committed ncu summary, if the
    kernel source is the one the counters were taken on; else None."""
    path = os.path.join(ROOT, "profiles", "chain_c1_bf16_b8192.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    h = hashlib.sha256()
    for f in ("mlp_chain.cu", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2507_11916_b300", "csrc", f), "rb").read())
    want = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith(("source_sha256", f"{key}_dram_bytes")):
            k, v = line.split(":", 1)
            want[k.strip()] = v.strip()
    if want.get("source_sha256") != h.hexdigest()[:16]:
        return None
    v = want.get(f"{key}_dram_bytes")
    return float(v) if v else None


def blas_threads():
    """Threads the oracle's numpy BLAS runs with."""
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except ImportError:
        for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            if os.environ.get(v, "").isdigit():
                return int(os.environ[v])
        return len(os.sched_getaffinity(0))


def cpu_oracle_rate(seconds=10.0, chunk=1024):
    """The oracle's float64 evaluation of the same workload on the host cores."""
    import oracle
    Ws, bs = W.net_weights(**W.NET_C1)
    Wq = oracle.quantise_weights(Ws[:-1], "bf16") + [Ws[-1]]
    states = W.random_stp_states(4, chunk, 4242)
    g = (W.splitmix64_array(4243, chunk) % np.uint64(60)).astype(np.uint8)
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        y = oracle.mlp_forward(Wq, bs, oracle.one_hot(oracle.DOM_STP4, states))
        h = oracle.h_regression(y[:, 0], oracle.md_states(oracle.DOM_STP4, states),
                                oracle.is_goal_states(oracle.DOM_STP4, states))
        oracle.bound_test(g, h, BOUND)
        n += chunk
    dt = time.perf_counter() - t0
    threads = blas_threads()
    return {"value": n / dt, "unit": "states/s", "cores": threads, "kind": "oracle",
            "sample": f"{n} states of the workload in chunks of {chunk} (float64 numpy forward, "
                      f"integer-h rule and bound test), {dt:.1f} s"}


def run_reference(args):
    """The oracle as the reference arm: each step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    Ws, bs = W.net_weights(**W.NET_C1)
    Wq = oracle.quantise_weights(Ws[:-1], "bf16") + [Ws[-1]]
    # size each step's sample so that the whole run takes about a minute
    probe = W.random_stp_states(4, 256, 4241)
    t0 = time.perf_counter()
    oracle.mlp_forward(Wq, bs, oracle.one_hot(oracle.DOM_STP4, probe))
    oracle.md_states(oracle.DOM_STP4, probe)
    per_state = (time.perf_counter() - t0) / 256
    chunk = int(max(1, min(1024, 60.0 / ((args.steps + args.warmup) * per_state))))
    states = W.random_stp_states(4, chunk, 4242)
    g = (W.splitmix64_array(4243, chunk) % np.uint64(60)).astype(np.uint8)

    def step():
        y = oracle.mlp_forward(Wq, bs, oracle.one_hot(oracle.DOM_STP4, states))
        h = oracle.h_regression(y[:, 0], oracle.md_states(oracle.DOM_STP4, states),
                                oracle.is_goal_states(oracle.DOM_STP4, states))
        oracle.bound_test(g, h, BOUND)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    threads = blas_threads()
    v = chunk * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "states/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(CONFIG, sample=f"{chunk} states per step"),
        "cpu_baseline": {"value": v, "unit": "states/s", "cores": threads, "kind": "oracle",
                         "sample": f"{chunk} states per step, {args.steps} steps"},
        "e2e": {"value": v, "unit": "states/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def search_rates(P, ctx, hid_bf16, hid_fp32, seconds):
    """IDA* nodes/s with the network heuristic (BF16 vs FP32) at equal solution cost."""
    out = {}
    starts = [P.cbdfs_apply_moves(P.DOM_STP4, W.stp_goal(4), W.stp_walk(4, 60, W.seed_for(W.TAG_C1, i)))
              for i in range(4)]
    threads = min(32, os.cpu_count() or 4)
    for name, hid in (("bf16", hid_bf16), ("fp32", hid_fp32)):
        costs, exp, gen, secs, nb, ev = [], 0, 0, 0.0, 0, 0
        for s in starts:
            r = P.cbdfs_solve(ctx, P.DOM_STP4, s, P.ALGO_IDA, hid, partial_ok=True, threads=threads,
                              work_num=64, batch=8192, timeout_us=500, time_limit_s=seconds)
            costs.append(r["cost"] if r["status"] == 0 else None)
            exp += r["expanded"]
            gen += r["generated"]
            secs += r["seconds"]
            nb += r["batches"]
            ev += r["evaluated"]
        out[name] = {"costs": costs, "expanded_per_s": exp / secs, "generated_per_s": gen / secs,
                     "avg_batch": ev / max(nb, 1), "seconds": secs, "threads": threads}
    out["equal_cost"] = out["bf16"]["costs"] == out["fp32"]["costs"]
    out["instances"] = "4 seeded 60-move 15-puzzle walks, h = max(rint(y), 0, MD)"
    return out


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    import paper_2507_11916_b300 as P

    B = BATCH
    ctx = P.cbdfs_create(local, max_batch=B, n_slots=2)
    Ws, bs = W.net_weights(**W.NET_C1)
    hid = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, P.PREC_BF16, P.HEAD_REGRESSION, 1)
    hid32 = P.cbdfs_net_load(ctx, P.DOM_STP4, Ws, bs, P.PREC_FP32, P.HEAD_REGRESSION, 1)
    states = W.random_stp_states(4, B, W.seed_for(W.TAG_C1, 1_000_000 + rank))
    g = (W.splitmix64_array(W.seed_for(W.TAG_C1, 2_000_000 + rank), B) % np.uint64(60)).astype(np.uint8)
    ds = torch.from_numpy(states.view(np.int64)).to(dev)
    dg = torch.from_numpy(g).to(dev)
    dh = torch.empty(B, dtype=torch.uint8, device=dev)
    dm = torch.empty((B + 31) // 32, dtype=torch.int32, device=dev)
    dmin = torch.empty(1, dtype=torch.int32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(dev)

    def enqueue(h):
        P.heur_eval_device(ctx, h, P.DOM_STP4, ds, dg, BOUND, B, dh, dm, dmin, stream=stream)

    def graph_of(h, warm):
        with torch.cuda.stream(stream):
            for _ in range(warm):
                enqueue(h)
        stream.synchronize()
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=stream):
            enqueue(h)
        return gr

    def timed(gr, K):
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        with torch.cuda.stream(stream):
            for k in range(K):
                flush.zero_()
                e0[k].record(stream)
                gr.replay()
                e1[k].record(stream)
        stream.synchronize()
        return sum(a.elapsed_time(b) for a, b in zip(e0, e1))

    gr = graph_of(hid, max(3, args.warmup))
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            flush.zero_()
            gr.replay()
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = timed(gr, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    clk = clocks.stop()
    value = world * B * args.steps / (ms / 1e3)
    # the graph replays the same pipeline: check its result against a host-buffer call
    h_ref, mask_ref, minf_ref = P.heur_submit_batch(ctx, hid, P.DOM_STP4, states, g, BOUND)
    assert np.array_equal(dh.cpu().numpy(), h_ref), "graph replay result differs"
    assert P.cbdfs_device_status(ctx) == 0

    # FP32 form of the same workload (SIMT path), fewer steps
    K32 = max(10, min(args.steps, 200))
    gr32 = graph_of(hid32, 3)
    ms32 = timed(gr32, K32)
    fp32_rate = B * K32 / (ms32 / 1e3)

    # per-kernel device time of the BF16 pipeline (events between launches, same stream)
    stage = []
    for _ in range(20):
        with torch.cuda.stream(stream):
            flush.zero_()
        stage.append(P.cbdfs_eval_profile(ctx, hid, P.DOM_STP4, ds, dg, BOUND, B, dh, dm, dmin,
                                          stream=stream))
    stage_ms = np.mean(np.array(stage), axis=0)
    dims = W.NET_C1["dims"]
    layer_flops = [2 * B * dims[l] * dims[l + 1] for l in range(len(dims) - 1)]
    if len(stage_ms) == 1:
        # the fused chain: one launch runs every layer and the head
        names = ["k_chain (256-1024-1024-512-1, one launch)"]
        flops = [sum(layer_flops)]
        traffic_key = "chain"
    else:
        names = ["layer1_onehot_256x1024", "layer2_1024x1024", "layer3_1024x512", "head_512x1"]
        flops = layer_flops
        traffic_key = None
    top = int(np.argmax(stage_ms))
    pk = peaks()
    achieved = flops[top] / (stage_ms[top] / 1e3) / 1e12
    roof = {"kernel": names[top], "bound": "tensor", "achieved": achieved,
            "peak": pk["bf16"], "unit": "TFLOP/s", "frac": achieved / pk["bf16"],
            "peak_source": f"{pk['src']} bf16 dense (burst)",
            "traffic": kernel_traffic(traffic_key) if traffic_key else None,
            "algorithmic_flops_per_launch": flops[top],
            "algorithmic_flops_onehot_as_gather": flops[top] - layer_flops[0] + 2 * B * 16 * dims[1],
            "launch_ms": float(stage_ms[top]),
            "stages_ms": {n: float(t) for n, t in zip(names, stage_ms)},
            "step_share": float(stage_ms[top] / stage_ms.sum())}
    launches_per_step = len(stage_ms)

    # end to end through the public host-buffer call (copies in and out every step)
    pin_s = torch.from_numpy(states.view(np.int64)).pin_memory()
    pin_g = torch.from_numpy(g).pin_memory()
    s_np, g_np = pin_s.numpy().view(np.uint64), pin_g.numpy()
    Ke = max(10, min(args.steps, 500))
    for _ in range(3):
        P.heur_submit_batch(ctx, hid, P.DOM_STP4, s_np, g_np, BOUND)
    t0 = time.perf_counter()
    for _ in range(Ke):
        P.heur_submit_batch(ctx, hid, P.DOM_STP4, s_np, g_np, BOUND)
    e2e = B * Ke / (time.perf_counter() - t0)
    if dist:
        t = torch.tensor([e2e], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        e2e = float(t.item()) * world

    line = {
        "metric": METRIC, "value": value, "unit": "states/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": dict(CONFIG, parallelism=f"replicas x{world}"),
        "gpu_launches": launches_per_step * args.steps,
        "e2e": {"value": e2e, "unit": "states/s", "h2d_bytes_per_step": B * 8 + B,
                "d2h_bytes_per_step": B + (B + 31) // 32 * 4 + 4},
        "roofline": roof, "clocks": clk,
        "fp32_states_per_s": fp32_rate, "bf16_over_fp32": value / world / fp32_rate,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate(args.cpu_seconds)
    if rank == 0 and not args.no_search:
        line["search"] = search_rates(P, ctx, hid, hid32, args.search_seconds)
    P.cbdfs_destroy(ctx)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline leg")
    ap.add_argument("--no-search", action="store_true", help="skip the IDA* nodes/s leg")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--search-seconds", type=float, default=3.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
