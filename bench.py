"""Benchmark: exact k-NN graph rows/s on one GB300 (or N replicas), one JSON line.

Workload (default): k-NN graph of N = 262144 unit-norm Gaussian directions in
d = 1024 with 1% exact duplicate points, k = 64, squared Euclidean distance. A step
is one full knng_build call (prep, distance GEMM, select, exact re-rank, any
fallback) over that input, already resident in HBM. The input (1.07 GB) is larger
than L2, so no flush is needed between steps.

Arms:
  --impl ours (default)   the CUDA engine through its C ABI;
  --impl reference        the FP64 CPU oracle on the host cores, on a bounded sample
                          of the same workload's rows per step.

Multi-GPU (torchrun): every rank builds the same graph on its own GPU (weak
scaling, replicas, no data-path collective); value = rows of all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact k-NNG rows/s & % roofline, fused BF16 vs plain FP32, N=262144 d=1024 k=64"
N_DEFAULT, D_DEFAULT, K_DEFAULT, M_EXTRA = 262144, 1024, 64, 32
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["auto", "fused", "plain"], default="auto")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--d", type=int, default=D_DEFAULT)
    ap.add_argument("--k", type=int, default=K_DEFAULT)
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP32 and FP8 comparison steps")
    ap.add_argument("--compare-repeats", type=int, default=3,
                    help="timed repeats (after one warm-up call) of each comparison form; the median is reported")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--mode", choices=["knng", "plain", "fp8", "select", "select_sweep", "batch", "mlp", "metric",
                                       "streamed"],
                    default="knng",
                    help="fp8: FP8 e4m3 against BF16 on 262144 near-duplicate points (2048 groups of 128) in d=1024; "
                         "plain: the plain FP32 form on the integer lattice (--workload lattice: N=4096, d=128, k=16) "
                         "or the Gaussian mixture (--workload mixture: N=65536, d=256, k=32); "
                         "select: the quick multi-select alone on a Q x n uniform random matrix (paper's experiments); "
                         "metric: the cosine and Pearson similarity graphs of the headline data; "
                         "streamed: search of 65536 queries against a 4M x 256 corpus read from pinned host "
                         "memory in 1M-row chunks, against the same search with the corpus resident; "
                         "select_sweep: the select alone over the paper's selection experiment shapes "
                         "(n = 2^20 with Q 8..256; n Q = 2^27 with n/Q 2^-3..2^19; Q = 256 with n 2^16..2^20); "
                         "batch: 512 independent search problems of uneven shape in one graph; "
                         "mlp: k-NN graph of a 524288 x 768 anisotropic mixture, k=100, with learned per-row "
                         "thresholds against the same graph without them")
    ap.add_argument("--workload", choices=sorted(PLAIN_WORKLOADS), default="lattice", help="plain mode: workload")
    ap.add_argument("--max-workspace-mb", type=int, default=0,
                    help="plain mode: workspace cap in MiB (sizes the distance-matrix slabs; 0 = library default)")
    ap.add_argument("--train-rows", type=int, default=50000, help="mlp mode: training rows")
    ap.add_argument("--epochs", type=int, default=40, help="mlp mode: training epochs")
    ap.add_argument("--problems", type=int, default=512, help="batch mode: number of problems")
    ap.add_argument("--batch-k", type=str, default="",
                    help="batch mode: keep only the problems whose k is in this comma list (same shapes and seeds)")
    ap.add_argument("--batch-d", type=str, default="",
                    help="batch mode: keep only the problems whose d is in this comma list")
    ap.add_argument("--q", type=int, default=16384, help="select mode: rows")
    ap.add_argument("--cols", type=int, default=65536, help="select mode: row length n")
    return ap.parse_args()


SCHEDULE_NAMES = {0: "fused", 1: "plain-fp32", 2: "fused-no-speculation", 3: "fused-speculation",
                  4: "fused-128-no-speculation", 5: "fused-128-speculation"}


def autotune_table(path: str) -> dict:
    """The autotuner's cache file as {"device": tag, "buckets": {bucket: schedule name}}."""
    try:
        raw = json.load(open(path))
    except (OSError, ValueError):
        return {"unavailable": f"no cache at {path}"}
    dev = raw.pop("_device", None)
    return {"device": dev, "buckets": {k: SCHEDULE_NAMES.get(v, v) for k, v in sorted(raw.items())},
            "counts": {name: sum(1 for v in raw.values() if SCHEDULE_NAMES.get(v) == name)
                       for name in SCHEDULE_NAMES.values()}}


def run_batch(args):
    """512 independent k-NN search problems (M~U[256,16384], N~U[1024,65536], d in {64,128,256,768},
    k in {1,8,32,128,512}, N(0,1) FP32 data) answered by one knn_search_batched call (one CUDA graph)."""
    import tempfile
    # a fresh autotuner cache for this run, read back afterwards for the choice table
    tune_dir = tempfile.mkdtemp(prefix="knn_tune_")
    os.environ["KNN_AUTOTUNE_CACHE"] = os.path.join(tune_dir, "autotune.json")
    import torch
    from paper_1309_5478_gb300 import binding as kb
    from paper_1309_5478_gb300 import inputs
    shapes = inputs.batch_problems(count=args.problems)
    keep_k = {int(v) for v in args.batch_k.split(",") if v}
    keep_d = {int(v) for v in args.batch_d.split(",") if v}
    g = torch.Generator(device="cuda").manual_seed(20130904)
    probs = []
    kept = []
    for pr in shapes:
        Q = torch.randn((pr.M, pr.d), device="cuda", generator=g, dtype=torch.float32)
        C = torch.randn((pr.N, pr.d), device="cuda", generator=g, dtype=torch.float32)
        if (keep_k and pr.k not in keep_k) or (keep_d and pr.d not in keep_d):
            del Q, C  # drawn all the same, so a subset keeps the full batch's data
            continue
        kept.append(pr)
        probs.append({"Q": Q, "C": C, "k": pr.k,
                      "out_idx": torch.empty((pr.M, pr.k), dtype=torch.int32, device="cuda"),
                      "out_dist": torch.empty((pr.M, pr.k), dtype=torch.float32, device="cuda")})
    subset = len(kept) != len(shapes)
    shapes = kept
    rows = sum(pr.M for pr in shapes)
    pairs = sum(pr.M * pr.N for pr in shapes)
    flops = sum(2.0 * pr.M * pr.N * pr.d for pr in shapes)
    t0 = time.perf_counter()
    kb.knn_search_batched(probs)  # autotune (first time per bucket) + capture
    torch.cuda.synchronize()
    first_call_s = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        kb.knn_search_batched(probs)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    stats = None
    for _ in range(args.steps):
        _, stats = kb.knn_search_batched(probs, return_stats=True)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    P = peaks()
    kinds = {}
    for pr in shapes:
        kinds[pr.k] = kinds.get(pr.k, 0) + 1
    line = {"metric": "exact k-NN search rows/s over a batch of independent problems", "value": rows / (ms / 1e3),
            "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"{len(shapes)} independent k-NN search problems, M~U[256,16384], N~U[1024,65536], "
                                   "d in {64,128,256,768}, k in {1,8,32,128,512}, N(0,1) FP32"
                                   + (f" (subset: k in {sorted(keep_k) or 'all'}, d in {sorted(keep_d) or 'all'})"
                                      if subset else ""),
                       "rows": rows, "pairs": pairs, "gemm_tflop": flops / 1e12, "k_histogram": kinds,
                       "l2": "inputs ~26 GB > L2"},
            "pairs_per_s": pairs / (ms / 1e3), "effective_tflops": flops / (ms / 1e3) / 1e12,
            "frac_of_bf16_sustained": flops / (ms / 1e3) / 1e12 / P["bf16_sustained"],
            "first_call_s": first_call_s, "clocks": clk,
            "batch_stats": {k: stats[k] for k in ("rows", "candidates", "rows_uncertified", "rows_fallback",
                                                   "fused_used", "kernel_launches")},
            "phases_ms": {"call_host_total": stats["ms_total"], "graph": stats["ms_gemm"],
                          "prep_bounds": stats["ms_prep"], "fused": stats["ms_select"],
                          "rerank": stats["ms_rerank"], "plain_problems": stats["ms_fallback"]},
            "autotuner": autotune_table(os.environ["KNN_AUTOTUNE_CACHE"])}
    # oracle on a few rows of a few problems
    import oracle
    sample = []
    t_cpu = 0.0
    nrows = 0
    for pr, pb in list(zip(shapes, probs))[:: max(1, len(shapes) // 8)]:
        Qh, Ch = pb["Q"][:8].cpu().numpy(), pb["C"].cpu().numpy()
        t0 = time.perf_counter()
        oracle.knn(Qh, Ch, pr.k)
        t_cpu += time.perf_counter() - t0
        nrows += Qh.shape[0]
    line["cpu_baseline"] = {"value": nrows / t_cpu, "unit": "rows/s", "cores": oracle.threads(), "kind": "oracle",
                            "sample": f"8 query rows of each of {len(shapes[::max(1, len(shapes)//8)])} problems"}
    print(json.dumps(line), flush=True)


def run_mlp(args):
    """k-NN graph with learned per-row thresholds: N=524288 points of a 256-component anisotropic
    Gaussian mixture in d=768 (diagonal scales log-uniform in [0.1, 2]), k=100, fused BF16 form.
    The network is trained on 50000 seeded rows whose targets (log k-th squared distance without
    the row itself) come from the engine; a step is features + prediction + knng_build with the
    proposed thresholds, against knng_build alone on the same data."""
    import torch
    from paper_1309_5478_gb300 import binding as kb
    from paper_1309_5478_gb300 import inputs
    n = args.n if args.n != N_DEFAULT else 524288
    d = args.d if args.d != D_DEFAULT else 768
    k = args.k if args.k != K_DEFAULT else 100
    X = inputs.anisotropic_mixture(n=n, d=d)
    Xd = torch.from_numpy(X).cuda()
    P = peaks()
    F = kb.MLP_FEATURES
    # training
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = Xd[torch.from_numpy(inputs.sample_rows(n, F - 1, seed=501)).cuda()].contiguous()
    rows = torch.from_numpy(inputs.sample_rows(n, args.train_rows, seed=502)).cuda()
    _, dt = kb.knn_search(Xd[rows].contiguous(), Xd, k + 1, precision="bf16")
    targets = torch.log(dt[:, k].contiguous())
    feats = kb.mlp_features(Xd, S)
    torch.cuda.synchronize()
    t_targets = time.perf_counter() - t0
    params = torch.zeros(kb.mlp_param_count(), dtype=torch.float32, device="cuda")
    gen = torch.Generator().manual_seed(503)
    params[:kb.MLP_TRAINED] = (torch.randn(kb.MLP_TRAINED, generator=gen) * 0.02).cuda()
    # training rows in a seeded shuffled order (the hold-out is the tail)
    perm = torch.from_numpy(inputs.permutation(504, 0, args.train_rows)).cuda()
    t1 = time.perf_counter()
    hist = kb.mlp_train(feats[rows[perm]].contiguous(), targets[perm].contiguous(), params,
                        epochs=args.epochs, batch=1024, lr=1e-3, holdout=0.1, margin_quantile=0.99)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1

    oi = torch.empty((n, k), dtype=torch.int32, device="cuda")
    od = torch.empty((n, k), dtype=torch.float32, device="cuda")
    oi2 = torch.empty_like(oi)
    od2 = torch.empty_like(od)
    fbuf = torch.empty((n, F), dtype=torch.float32, device="cuda")
    thr = torch.empty(n, dtype=torch.float32, device="cuda")

    def with_mlp():
        kb.mlp_features(Xd, S, out=fbuf)
        _, t = kb.mlp_predict(fbuf, params)
        thr.copy_(t)
        return kb.knng_build(Xd, k, out_idx=oi, out_dist=od, precision="bf16", fused=1, row_threshold=thr,
                             flags=kb.KNN_FLAG_CHECK_FINITE | kb.KNN_FLAG_TIMING, return_stats=True)[2]

    def without_mlp():
        return kb.knng_build(Xd, k, out_idx=oi2, out_dist=od2, precision="bf16", fused=1,
                             flags=kb.KNN_FLAG_CHECK_FINITE | kb.KNN_FLAG_TIMING, return_stats=True)[2]

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        st = [fn() for _ in range(args.steps)]
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / args.steps, st

    clocks = ClockSampler(0)
    clocks.start()
    ms_with, st_with = timed(with_mlp)
    ms_without, st_without = timed(without_mlp)
    # the method without any speculation (plain running thresholds), with and without the
    # network: what the learned thresholds gain over the method alone
    variants = {}
    prev = os.environ.get("KNN_SPECULATE")
    os.environ["KNN_SPECULATE"] = "0"
    try:
        for name, fn in (("running_threshold_only", without_mlp), ("learned_threshold_only", with_mlp)):
            ms_v, st_v = timed(fn)
            sv = st_v[-1]
            variants[name] = {"ms_per_step": ms_v, "rows_per_s": n / (ms_v / 1e3), "ms_select": sv["ms_select"],
                              "inserted_per_row": sv["candidates_inserted"] / n,
                              "ms_rerank": sv["ms_rerank"], "ms_fallback": sv["ms_fallback"],
                              "rows_fallback": int(sv["rows_fallback"])}
    finally:
        if prev is None:
            os.environ.pop("KNN_SPECULATE", None)
        else:
            os.environ["KNN_SPECULATE"] = prev
    variants["speculative_only"] = {"ms_per_step": ms_without, "ms_select": st_without[-1]["ms_select"]}
    variants["speculative_and_learned"] = {"ms_per_step": ms_with, "ms_select": st_with[-1]["ms_select"]}
    clk = clocks.stop()
    identical = bool(torch.equal(oi, oi2) and torch.equal(od, od2))
    s1, s0 = st_with[-1], st_without[-1]
    dk = od2[:, k - 1].double()
    lr = torch.log(thr.double() / dk)
    flops = float(s1["gemm_flops"])
    ach = flops / (float(np.mean([s["ms_gemm"] for s in st_with])) / 1e3) / 1e12
    line = {"metric": "exact k-NNG rows/s with learned per-row thresholds, N=524288 d=768 k=100",
            "value": n / (ms_with / 1e3), "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_with, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": f"k-NN graph, N={n} points of a 256-component anisotropic Gaussian mixture in "
                                   f"d={d} (diagonal scales log-uniform in [0.1,2]), k={k}, learned thresholds "
                                   f"from a 257-128-1 network trained on {args.train_rows} rows",
                       "N": n, "d": d, "k": k, "train_rows": args.train_rows, "epochs": args.epochs,
                       "l2": "input 1.6 GB > L2: no flush needed"},
            "without_mlp": {"rows_per_s": n / (ms_without / 1e3), "ms_per_step": ms_without,
                            "candidates_per_row": s0["candidates"] / n, "ms_select": s0["ms_select"],
                            "inserted_per_row": s0["candidates_inserted"] / n,
                            "ms_rerank": s0["ms_rerank"]},
            "with_mlp": {"candidates_per_row": s1["candidates"] / n, "ms_select": s1["ms_select"],
                         "inserted_per_row": s1["candidates_inserted"] / n,
                         "ms_rerank": s1["ms_rerank"], "ms_fallback": s1["ms_fallback"],
                         "threshold_misses": int(s1["threshold_misses"]),
                         "rows_uncertified": int(s1["rows_uncertified"]), "rows_fallback": int(s1["rows_fallback"])},
            "speedup_vs_without": ms_without / ms_with,
            "variants": variants,
            "learned_gain_over_running_threshold": (variants["running_threshold_only"]["ms_per_step"] /
                                                    variants["learned_threshold_only"]["ms_per_step"]),
            "identical_to_without": identical,
            "pass_rate": 1.0 - (s1["rows_uncertified"] + s1["threshold_misses"]) / n,
            "proposal_log_ratio": {"median": float(lr.median()), "p01": float(torch.quantile(lr.float(), 0.01)),
                                   "frac_at_or_above_kth": float((lr >= 0).double().mean())},
            "training": {"targets_and_features_s": t_targets, "train_s": t_train, "loss_first": hist[0],
                         "loss_last": hist[-1], "margin": float(params[-1])},
            "roofline": {"bound": "tensor", "achieved": ach, "peak": P["bf16_sustained"], "unit": "TFLOP/s",
                         "frac": ach / P["bf16_sustained"], "traffic": None, "kernel": "knn_fused_gemm_select",
                         "peak_source": f"{P['source']} bf16 sustained"},
            "clocks": clk,
            # engine launches of the graph builds, plus the feature (2 norm + 2 per 65536-row slab) and
            # prediction (2) kernels of every step
            "gpu_launches": int(sum(s["kernel_launches"] for s in st_with)) + args.steps * (4 + 2 * -(-n // 65536))}
    if not args.no_cpu_baseline:
        cb = oracle_sample_rate(X, k, args.cpu_seconds, seed=505)
        rows, ri, rd = cb.pop("_rows"), cb.pop("_idx"), cb.pop("_dist")
        line["cpu_baseline"] = cb
        line["oracle_check"] = oracle_check(X, rows, oi.cpu().numpy()[rows], od.cpu().numpy()[rows], ri, rd)
    print(json.dumps(line), flush=True)


def run_select_only(args):
    """Quick multi-select alone: k smallest of every row of a Q x n uniform random FP32 matrix."""
    import torch
    from paper_1309_5478_gb300 import binding as kb
    P = peaks()
    g = torch.Generator(device="cuda").manual_seed(20130906)
    D = torch.rand((args.q, args.cols), device="cuda", generator=g, dtype=torch.float32)
    k = args.k
    oi = torch.empty((args.q, k), dtype=torch.int32, device="cuda")
    ov = torch.empty((args.q, k), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        kb.knn_select(D, k, out_idx=oi, out_val=ov)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        kb.knn_select(D, k, out_idx=oi, out_val=ov)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    bytes_alg = args.q * args.cols * 4 + args.q * k * 8
    gbs = bytes_alg / (ms / 1000.0) / 1e9
    line = {"metric": "quick multi-select rows/s (selection only, uniform random values)", "value": args.q / (ms / 1000),
            "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"select k={k} smallest of {args.q} rows x {args.cols} uniform FP32 values",
                       "Q": args.q, "n": args.cols, "k": k, "l2": "matrix > L2: no flush needed"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": P["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / P["hbm_gbs"],
                         "traffic": (recorded_traffic("select_rows_kernel", ["paper_1309_5478_gb300/csrc/select.cu"])
                                     if (args.q, args.cols, k) == (16384, 65536, 64) else None),
                         "kernel": "select_rows_kernel", "peak_source": P["source"]},
            "clocks": clk, "gpu_launches": args.steps}
    print(json.dumps(line), flush=True)


PLAIN_WORKLOADS = {
    # name: (generator, k, description)
    "lattice": (lambda: __import__("paper_1309_5478_gb300.inputs", fromlist=["x"]).integer_lattice(), 16,
                "k-NN graph, N=4096 integer points uniform in [-8,8]^128, k=16"),
    "mixture": (lambda: __import__("paper_1309_5478_gb300.inputs", fromlist=["x"]).gaussian_mixture(), 32,
                "k-NN graph, N=65536 points of a 64-component Gaussian mixture in d=256 "
                "(means N(0,4I), sigma 0.5), k=32"),
}


def run_plain(args):
    """The plain FP32 form (SIMT distance GEMM writing the d' matrix in row slabs, the unfused
    quick multi-select over it, exact re-rank) on the two smaller graph configurations. Each
    step is one knng_build call, timed by CUDA events, with a 256 MB L2 flush before it
    (outside the timed region). Reports rows/s, the select's achieved HBM bandwidth on the
    d' slabs (4 bytes per matrix entry read once, over the select launches' device time), the
    GEMM's FP32 rate, and the output checked against the FP64 oracle."""
    import torch
    import oracle
    from paper_1309_5478_gb300 import binding as kb
    gen, k, desc = PLAIN_WORKLOADS[args.workload]
    X = gen()
    n, d = X.shape
    P = peaks()
    Xd = torch.from_numpy(X).cuda()
    oi = torch.empty((n, k), dtype=torch.int32, device="cuda")
    od = torch.empty((n, k), dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def call():
        return kb.knng_build(Xd, k, out_idx=oi, out_dist=od, precision="fp32", fused=0,
                             flags=kb.KNN_FLAG_CHECK_FINITE | kb.KNN_FLAG_TIMING, return_stats=True,
                             max_workspace_bytes=args.max_workspace_mb << 20)[2]

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    times, stats = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        stats.append(call())
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    clk = clocks.stop()
    ms = float(np.sum(times)) / args.steps
    ms_sel = float(np.mean([s["ms_select"] for s in stats]))
    ms_gemm = float(np.mean([s["ms_gemm"] for s in stats]))
    ms_rr = float(np.mean([s["ms_rerank"] for s in stats]))
    sel_bytes = 4.0 * n * n
    sel_gbs = sel_bytes / (ms_sel / 1000.0) / 1e9
    alu_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * P["sm_max_mhz"] * 1e6 / 1e12
    gemm_tf = 2.0 * n * n * d / (ms_gemm / 1000.0) / 1e12
    idx, dist = oi.cpu().numpy(), od.cpu().numpy()
    from paper_1309_5478_gb300 import inputs
    rows = np.arange(n) if args.workload == "lattice" else inputs.sample_rows(n, 256, seed=78)
    t0 = time.perf_counter()
    ri, rd = oracle.knng(X, k, rows=rows)
    t_cpu = time.perf_counter() - t0
    check = oracle_check(X, rows, idx[rows], dist[rows], ri, rd)
    if args.workload == "lattice":
        check["bit_exact"] = bool(np.array_equal(idx.astype(np.int64), ri) and np.array_equal(dist.astype(np.float64), rd))
    line = {"metric": f"exact k-NNG rows/s, plain FP32 form ({args.workload})", "value": n / (ms / 1000.0),
            "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "N": n, "d": d, "k": k, "form": "plain-fp32",
                       "max_workspace_mb": args.max_workspace_mb,
                       "l2": "256 MB written between steps (outside the timed region)"},
            "roofline": {"bound": "hbm", "achieved": sel_gbs, "peak": P["hbm_gbs"], "unit": "GB/s",
                         "frac": sel_gbs / P["hbm_gbs"], "kernel": "select_rows_kernel",
                         "traffic": None, "peak_source": P["source"],
                         "algorithmic_bytes": sel_bytes, "launch_ms": ms_sel},
            "gemm": {"kernel": "gemm_dprime_kernel", "ms": ms_gemm, "tflops": gemm_tf, "alu_peak_tflops": alu_peak,
                     "frac": gemm_tf / alu_peak},
            "phases_ms": {"gemm": ms_gemm, "select": ms_sel, "rerank": ms_rr, "prep": stats[-1]["ms_prep"],
                          "fallback": stats[-1]["ms_fallback"]},
            "clocks": clk, "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
            "oracle_check": check,
            "cpu_baseline": {"value": len(rows) / t_cpu, "unit": "rows/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{len(rows)} rows of the same graph, {t_cpu:.1f} s"}}
    print(json.dumps(line), flush=True)


def run_fp8(args):
    """FP8 e4m3 against BF16 on a workload whose FP8 error bound still separates the answer:
    the k-NN graph (k = 64) of 262144 points in d = 1024 made of 2048 groups of 128
    near-duplicates (unit-norm centres, members within about 1e-2 of their centre). The band
    of either form is the point's own group, so both certify their rows in the first pass, and
    FP8 halves the tensor work. Each form: one untimed call, then the median of the timed
    steps (CUDA events); inputs (1.07 GB) exceed L2."""
    import torch
    import oracle
    from paper_1309_5478_gb300 import binding as kb
    from paper_1309_5478_gb300 import inputs
    n, d, k = 262144, 1024, 64
    X = inputs.tight_groups(n=n, d=d, group=128)
    Xd = torch.from_numpy(X).cuda()
    oi = torch.empty((n, k), dtype=torch.int32, device="cuda")
    od = torch.empty((n, k), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    P = peaks()
    forms = {}
    outs = {}
    clocks = ClockSampler(0)
    clocks.start()
    for prec in ("bf16", "fp8"):
        def call():
            return kb.knng_build(Xd, k, out_idx=oi, out_dist=od, precision=prec, rerank_extra=M_EXTRA, fused=1,
                                 flags=kb.KNN_FLAG_CHECK_FINITE | kb.KNN_FLAG_TIMING, return_stats=True)[2]
        ms, st = timed_calls(call, stream, args.steps)
        outs[prec] = (oi.cpu().numpy(), od.cpu().numpy())
        forms[prec] = {"ms_per_step": ms, "rows_per_s": n / (ms / 1000.0), "ms_gemm": st["ms_gemm"],
                       "gemm_tflops": st["gemm_flops"] / (st["ms_gemm"] / 1000.0) / 1e12,
                       "rows_certified_first_pass": int(n - st["rows_uncertified"]),
                       "rows_fallback": int(st["rows_fallback"]), "symmetric": bool(st["symmetric"]),
                       "candidates_per_row": st["candidates"] / n, "max_error_ratio": float(st["max_error_ratio"]),
                       "phases_ms": {"prep": st["ms_prep"], "gemm_select": st["ms_select"],
                                     "rerank": st["ms_rerank"], "fallback": st["ms_fallback"]}}
    clk = clocks.stop()
    rows = inputs.sample_rows(n, 64, seed=79)
    ri, rd = oracle.knng(X, k, rows=rows)
    for prec in forms:
        forms[prec]["oracle_check"] = oracle_check(X, rows, outs[prec][0][rows], outs[prec][1][rows], ri, rd)
    line = {"metric": "exact k-NNG rows/s, FP8 e4m3 against BF16 (near-duplicate groups)",
            "value": forms["fp8"]["rows_per_s"], "unit": "rows/s", "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": forms["fp8"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp8-e4m3", "data": "synthetic",
            "config": {"workload": f"k-NN graph, N={n} points in d={d}: 2048 groups of 128 near-duplicates "
                                   "(unit-norm centres, members c + 0.01 z / sqrt(d)), k=64, squared Euclidean",
                       "N": n, "d": d, "k": k, "seed": 20130909, "l2": "input 1.07 GB > L2"},
            "forms": forms, "fp8_vs_bf16": forms["bf16"]["ms_per_step"] / forms["fp8"]["ms_per_step"],
            "clocks": clk, "peak_bf16_sustained": P["bf16_sustained"]}
    print(json.dumps(line), flush=True)


def run_metric(args):
    """Cosine and Pearson similarity graphs (k most similar, exact) of the headline data,
    timed like the Euclidean step; beside each, the Euclidean graph of the same rows already
    normalised (the engine part of the similarity path), and a sampled check of the similarity
    rows against the FP64 oracle."""
    import torch
    import oracle
    from paper_1309_5478_gb300 import binding as kb
    from paper_1309_5478_gb300 import inputs
    X = workload(args.n, args.d)
    k = args.k
    Xd = torch.from_numpy(X).cuda()
    oi = torch.empty((args.n, k), dtype=torch.int32, device="cuda")
    ov = torch.empty((args.n, k), dtype=torch.float32, device="cuda")
    out = {}
    for metric in ("cosine", "pearson"):
        for _ in range(args.warmup):
            kb.knng_build_metric(Xd, k, metric, out_idx=oi, out_val=ov)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            _, _, st = kb.knng_build_metric(Xd, k, metric, out_idx=oi, out_val=ov, return_stats=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        clk = clocks.stop()
        # the Euclidean graph of the unit rows alone (the same engine work)
        Xc = X.astype(np.float64)
        if metric == "pearson":
            Xc = Xc - Xc.mean(axis=1, keepdims=True)
        U = torch.from_numpy((Xc / np.linalg.norm(Xc, axis=1, keepdims=True)).astype(np.float32)).cuda()
        kb.knng_build(U, k + 32, rerank_extra=32)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            kb.knng_build(U, k + 32, rerank_extra=32)
        e1.record()
        torch.cuda.synchronize()
        ms_unit = e0.elapsed_time(e1) / args.steps
        del U
        rows = inputs.sample_rows(args.n, 64, seed=606)
        t0 = time.perf_counter()
        ref_idx, ref_sim = oracle.knng_sim(X, k, metric, rows=rows)
        dt = time.perf_counter() - t0
        gi, gv = oi.cpu().numpy()[rows], ov.cpu().numpy()[rows]
        same = int(sum(np.array_equal(gi[r].astype(np.int64), ref_idx[r]) for r in range(len(rows))))
        max_ulps = float(max((np.max(np.abs(gv[r].astype(np.float64) - ref_sim[r]) /
                                     np.spacing(np.abs(ref_sim[r]).astype(np.float32)).astype(np.float64))
                              for r in range(len(rows)) if np.array_equal(gi[r].astype(np.int64), ref_idx[r])),
                             default=float("nan")))
        out[metric] = {"ms_per_step": ms, "rows_per_s": args.n / (ms / 1e3), "ms_euclidean_unit_rows": ms_unit,
                       "ms_similarity_overhead": ms - ms_unit, "rows_uncertified": st["rows_uncertified"],
                       "rows_fallback": st["rows_fallback"], "precision_used": st["precision_used"],
                       "oracle_check": {"rows": len(rows), "rows_identical_indices": same,
                                        "max_value_error_fp32_ulps": max_ulps},
                       "cpu_baseline": {"value": len(rows) / dt, "unit": "rows/s", "cores": oracle.threads(),
                                        "kind": "oracle", "sample": f"{len(rows)} seeded rows, {dt:.1f} s"},
                       "clocks": clk}
    line = {"metric": "exact cosine / Pearson k-NN graph rows/s", "value": out["cosine"]["rows_per_s"],
            "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["cosine"]["ms_per_step"], "higher_is_better": True, "dtype": "bf16+f32pair+f64",
            "data": "synthetic", "config": {"workload": f"similarity graph N={args.n} d={args.d} k={k}, unit "
                                                        "directions + 1% duplicates", "N": args.n, "d": args.d,
                                            "k": k}, "metrics": out}
    print(json.dumps(line), flush=True)


def run_streamed(args):
    """k-NN search of 65536 queries against a 4194304 x 256 Gaussian-mixture corpus (4 GB) that
    stays in page-locked host memory and is read in 1048576-row chunks, against the same search
    with the corpus resident on the device; both answers compared."""
    import torch
    from paper_1309_5478_gb300 import binding as kb
    from paper_1309_5478_gb300 import inputs
    n, d, m, k, chunk = 1 << 22, 256, 1 << 16, 32, 1 << 20
    g = torch.Generator(device="cuda").manual_seed(20130907)
    centers = torch.randn((64, d), device="cuda", generator=g) * 2.0
    C = centers[torch.randint(0, 64, (n,), device="cuda", generator=g)] + torch.randn((n, d), device="cuda", generator=g)
    Q = centers[torch.randint(0, 64, (m,), device="cuda", generator=g)] + torch.randn((m, d), device="cuda", generator=g)
    Ch = C.cpu().pin_memory()
    oi = torch.empty((m, k), dtype=torch.int32, device="cuda")
    od = torch.empty((m, k), dtype=torch.float32, device="cuda")
    ri = torch.empty_like(oi)
    rd = torch.empty_like(od)
    res = {}
    for name, fn in (("resident", lambda: kb.knn_search(Q, C, k, out_idx=ri, out_dist=rd)),
                     ("streamed", lambda: kb.knn_search_streamed(Q, Ch, k, chunk_rows=chunk, out_idx=oi, out_dist=od))):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / args.steps
    # the host link alone: one chunk copied from the same pinned corpus, CUDA events
    dst = torch.empty((chunk, d), device="cuda")
    link = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.copy_(Ch[:chunk], non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        link.append(e0.elapsed_time(e1))
    link_gbs = chunk * d * 4 / (min(link) / 1e3) / 1e9
    same_idx = bool(torch.equal(oi, ri))
    rel = float(((od.double() - rd.double()).abs() / rd.double().clamp_min(1e-30)).max())
    h2d_gbs = n * d * 4 / (res["streamed"] / 1e3) / 1e9
    line = {"metric": "k-NN search rows/s with the corpus streamed from host memory", "value": m / (res["streamed"] / 1e3),
            "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["streamed"], "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"search M={m} against N={n} d={d} k={k}, corpus in pinned host memory, "
                                   f"chunks of {chunk} rows"},
            "ms_resident": res["resident"], "streamed_over_resident": res["streamed"] / res["resident"],
            "corpus_bytes_per_step_time_gbs": h2d_gbs, "h2d_link_gbs": link_gbs,
            "ms_corpus_copy_at_link_rate": n * d * 4 / (link_gbs * 1e9) * 1e3, "indices_identical_to_resident": same_idx,
            "max_rel_distance_difference": rel}
    print(json.dumps(line), flush=True)


def select_sweep_shapes():
    """(family, Q, n, k) of the paper's selection experiments: time per query against Q at
    n = 2^20 (Fig. 8), a constant n Q = 2^27 with n / Q from 2^-3 to 2^19 (Fig. 6), and Q = 256
    with n from 2^16 to 2^20 (Fig. 9)."""
    out = []
    for k in (16, 128, 1024):
        for q in (8, 16, 32, 64, 128, 256):
            out.append(("n=2^20", q, 1 << 20, k))
    for k in (2, 32, 512):
        for r in range(-3, 20, 2):
            ln = (27 + r) // 2
            out.append(("nQ=2^27", 1 << (27 - ln), 1 << ln, k))
    for k in (2, 32, 1024):
        for ln in (16, 18, 20):
            out.append(("Q=256", 256, 1 << ln, k))
    return out


def run_select_sweep(args):
    """The quick multi-select alone over the paper's selection experiment shapes, on uniform
    random FP32 values; each call runs alone after an L2 flush (many of these matrices fit in
    L2). ms is the device time of the select kernels (events inside the call, KNN_FLAG_TIMING),
    ms_call the whole synchronous call from Python (launch and host overheads included). Row
    0 of every shape is checked against a sort on the host."""
    import torch
    from paper_1309_5478_gb300 import binding as kb
    P = peaks()
    g = torch.Generator(device="cuda").manual_seed(20130906)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MB > L2
    clocks = ClockSampler(0)
    clocks.start()
    rows = []
    for fam, q, n, k in select_sweep_shapes():
        D = torch.rand((q, n), device="cuda", generator=g, dtype=torch.float32)
        oi = torch.empty((q, k), dtype=torch.int32, device="cuda")
        ov = torch.empty((q, k), dtype=torch.float32, device="cuda")
        for _ in range(max(args.warmup, 1)):
            kb.knn_select(D, k, out_idx=oi, out_val=ov)
        times, dev_ms, launches = [], [], 0
        for _ in range(max(args.steps, 3)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, _, st = kb.knn_select(D, k, out_idx=oi, out_val=ov, return_stats=True, timing=True)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            dev_ms.append(st["ms_select"])
            launches = st["kernel_launches"]
        ms_call = float(np.median(times))
        ms = float(np.median(dev_ms))
        r0 = D[0].cpu().numpy()
        ref = np.lexsort((np.arange(n), r0))[:k]
        ok = bool(np.array_equal(oi[0].cpu().numpy(), ref) and np.array_equal(ov[0].cpu().numpy(), r0[ref]))
        gbs = (q * n * 4 + q * k * 8) / (ms / 1000.0) / 1e9
        rows.append({"family": fam, "Q": q, "n": n, "k": k, "ms": round(ms, 4), "ms_call": round(ms_call, 4),
                     "launches": launches,
                     "us_per_query": round(ms * 1000.0 / q, 3), "GB_s": round(gbs, 1),
                     "frac": round(gbs / P["hbm_gbs"], 3), "row0_exact": ok})
        del D, oi, ov
    clk = clocks.stop()
    line = {"metric": "quick multi-select device time over the paper's selection shapes", "unit": "ms",
            "higher_is_better": False, "dtype": "f32", "data": "synthetic uniform [0,1) FP32",
            "config": {"workload": "select sweep (n=2^20 Q 8..256; nQ=2^27; Q=256 n 2^16..2^20)",
                       "l2": "256 MB written before each timed call"},
            "peak_hbm_gbs": P["hbm_gbs"], "peak_source": P["source"], "clocks": clk,
            "all_row0_exact": all(r["row0_exact"] for r in rows), "shapes": rows}
    print(json.dumps(line), flush=True)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16": p["bf16_tflops"], "bf16_sustained": p["bf16_tflops_sustained"],
                "sm_max_mhz": p.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash(*files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, src_files) -> float | None:
    """DRAM bytes per launch from a committed ncu summary, if the kernel source is unchanged since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    e = t.get(kernel)
    if not e or e.get("source_hash") != source_hash(*src_files):
        return None
    return e.get("dram_bytes_per_launch")


def workload(n: int, d: int):
    from paper_1309_5478_gb300 import inputs
    X, targets, sources = inputs.unit_directions_with_duplicates(n=n, d=d, dup_fraction=0.01)
    return X


def oracle_sample_rate(X: np.ndarray, k: int, seconds: float, seed: int) -> dict:
    """Oracle rows/s on a bounded row sample of the same k-NN graph (all host cores)."""
    import oracle
    from paper_1309_5478_gb300 import inputs
    n = X.shape[0]
    threads = oracle.threads()
    probe = inputs.sample_rows(n, threads, seed=seed)  # one row per thread
    t0 = time.perf_counter()
    oracle.knng(X, k, rows=probe)
    rate = len(probe) / max(time.perf_counter() - t0, 1e-6)
    want = int(min(8192, max(threads, seconds * rate)))
    want = max(threads, (want // threads) * threads)
    rows = inputs.sample_rows(n, want, seed=seed + 1)
    t0 = time.perf_counter()
    ref_idx, ref_dist = oracle.knng(X, k, rows=rows)
    dt = time.perf_counter() - t0
    return {"value": len(rows) / dt, "unit": "rows/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(rows)} seeded rows of the same {n}-point graph (FP64 direct difference, qsort per row), "
                      f"{dt:.1f} s", "_rows": rows, "_idx": ref_idx, "_dist": ref_dist}


def oracle_check(X: np.ndarray, rows, idx: np.ndarray, dist: np.ndarray, ref_idx, ref_dist, rel: float = 1e-5) -> dict:
    """The engine's rows against the FP64 oracle's (same rows): distance error and the acceptance
    rule (every oracle neighbour below tau (1 - rel) reported; every reported neighbour within
    tau (1 + rel) in FP64; rows ascending; self absent)."""
    max_err = 0.0
    same = 0
    ok = 0
    for r, i in enumerate(rows):
        gi, gd = idx[r].astype(np.int64), dist[r].astype(np.float64)
        if np.array_equal(gi, ref_idx[r]):
            same += 1
            exact = ref_dist[r]
        else:
            diff = X[gi].astype(np.float64) - X[i].astype(np.float64)
            exact = np.einsum("ij,ij->i", diff, diff)
        err = np.abs(gd - exact) / np.maximum(exact, 1e-30)
        err[exact == 0] = np.abs(gd[exact == 0])
        max_err = max(max_err, float(err.max()))
        tau = ref_dist[r, -1]
        must = set(ref_idx[r][ref_dist[r] < tau * (1 - rel)].tolist())
        good = (must <= set(gi.tolist()) and bool(np.all(exact <= tau * (1 + rel) + 1e-30)) and
                bool(np.all(np.diff(gd) >= 0)) and i not in gi and float(err.max()) <= rel)
        ok += 1 if good else 0
    return {"rows": len(rows), "max_rel_dist_err": max_err, "rows_identical_indices": same,
            "rows_pass_acceptance": ok}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    X = workload(args.n, args.d)
    k = args.k
    import oracle
    rates = []
    steps = []
    per_step_seconds = max(3.0, min(12.0, 150.0 / max(1, args.steps + args.warmup)))
    for s in range(args.warmup + args.steps):
        r = oracle_sample_rate(X, k, per_step_seconds, seed=1000 + s)
        if s >= args.warmup:
            rates.append(r["value"])
            steps.append(r)
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * args.n / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, "oracle-fp64"),
            "cpu_baseline": {"value": value, "unit": "rows/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": steps[-1]["sample"]},
            "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(value: float, world: int, device="cuda") -> float:
    """The largest of every rank's value (the slowest rank's time); the value itself on one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_rate(rows_per_rank: int, world: int, seconds_slowest: float) -> float:
    """Whole-job rows/s of weak scaling: every rank answers rows_per_rank rows, the job ends with
    the slowest rank."""
    return world * rows_per_rank / seconds_slowest


def timed_calls(fn, stream, repeats: int):
    """One untimed call, then `repeats` calls each timed by CUDA events on `stream`;
    returns (median ms, the last call's result)."""
    import torch
    fn()
    times, out = [], None
    for _ in range(max(1, repeats)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return float(np.median(times)), out


def workload_config(args, form: str) -> dict:
    return {"workload": f"k-NN graph, N={args.n} unit-norm Gaussian directions in d={args.d} with 1% exact "
                        f"duplicates, k={args.k}, squared Euclidean", "N": args.n, "d": args.d, "k": args.k,
            "rerank_extra": M_EXTRA, "form": form, "l2": "input 1.07 GB > L2 (129 MB): no flush needed",
            "seed": 20130903}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.mode in ("plain", "fp8", "select", "select_sweep", "batch", "mlp", "metric", "streamed"):
        import torch
        torch.cuda.set_device(local)
        {"plain": run_plain, "fp8": run_fp8, "select": run_select_only, "select_sweep": run_select_sweep, "batch": run_batch,
         "mlp": run_mlp, "metric": run_metric, "streamed": run_streamed}[args.mode](args)
        return

    import torch
    import torch.distributed as dist
    from paper_1309_5478_gb300 import binding as kb

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    X = workload(args.n, args.d)
    Xd = torch.from_numpy(X).cuda()
    k = args.k
    oi = torch.empty((args.n, k), dtype=torch.int32, device="cuda")
    od = torch.empty((args.n, k), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    form = args.form
    if form == "auto":
        form = "fused"
    precision = "bf16" if form == "fused" else "fp32"
    fused = 1 if form == "fused" else 0

    def step(prec, fz, stats=False):
        return kb.knng_build(Xd, k, out_idx=oi, out_dist=od, precision=prec, rerank_extra=M_EXTRA, fused=fz,
                             flags=kb.KNN_FLAG_CHECK_FINITE | kb.KNN_FLAG_TIMING, return_stats=True)

    try:
        step(precision, fused)
    except kb.KnnError as e:
        if e.status != kb.KNN_EUNSUPPORTED or args.form == "fused":
            raise
        form, precision, fused = "plain", "fp32", 0
        step(precision, fused)
    for _ in range(max(0, args.warmup - 1)):
        step(precision, fused)

    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step(precision, fused)[2])
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    fused_idx, fused_dist = oi.cpu().numpy(), od.cpu().numpy()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world)
    ms_step = ms_total / args.steps
    rows_per_s = weak_scaling_rate(args.n, world, ms_step / 1000.0)

    P = peaks()
    s0 = stats[-1]
    ms_gemm = float(np.mean([s["ms_gemm"] for s in stats]))
    launches_gemm = max(1, int(s0["gemm_launches"]))
    flops = float(s0["gemm_flops"])
    if form == "fused":
        peak = P["bf16_sustained"]
        achieved = flops / (ms_gemm / 1000.0) / 1e12
        kern = "knn_fused_gemm_select"
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"{P['source']} bf16 sustained", "kernel": kern}
        src = ["paper_1309_5478_gb300/csrc/gemm_tc.cu", "paper_1309_5478_gb300/csrc/rerank_core.cuh",
               "paper_1309_5478_gb300/csrc/select_core.cuh", "paper_1309_5478_gb300/csrc/tc_fused.h",
               "paper_1309_5478_gb300/csrc/common.cuh"]
    else:
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * P["sm_max_mhz"] * 1e6 / 1e12
        achieved = flops / (ms_gemm / 1000.0) / 1e12
        kern = "gemm_dprime_kernel"
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop x {P['sm_max_mhz']:.0f} MHz", "kernel": kern}
        src = ["paper_1309_5478_gb300/csrc/gemm_simt.cu"]
    tr = recorded_traffic(kern, src)
    roof["traffic"] = tr * 1.0 if tr is not None else None
    roof["launch_ms"] = ms_gemm / launches_gemm
    roof["share_of_step"] = ms_gemm / ms_step
    # whole-path roofline of the method: the slower of the distance product the form computes at
    # tensor peak (the symmetric graph form computes each pair's product once: about N^2 d, not
    # 2 N^2 d) and the compulsory bytes at HBM bandwidth
    compulsory = args.n * args.d * 4 + args.n * k * 8 + (args.n * args.d * 2 * 2 if form == "fused" else 0)
    if form == "plain":
        compulsory += 8 * args.n * args.n
    t_roof = max(flops / (P["bf16_sustained"] * 1e12), compulsory / (P["hbm_gbs"] * 1e9))
    path_frac = t_roof / (ms_step / 1000.0)

    line = {"metric": METRIC, "value": rows_per_s, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if form == "fused" else "f32", "data": "synthetic",
            "config": workload_config(args, ("fused-bf16-symmetric" if s0.get("symmetric", 0) else "fused-bf16")
                                      if form == "fused" else "plain-fp32"),
            "pairs_per_s": world * args.n * (args.n - 1) / (ms_step / 1000.0),
            "path_roofline_frac": path_frac,
            "path_roofline": {"t_roof_ms": t_roof * 1000.0, "gemm_flops": flops,
                              "symmetric": bool(s0.get("symmetric", 0)),
                              "full_product_flops": 2.0 * args.n * args.n * args.d,
                              # the full product at tensor peak: the floor of a form without the
                              # symmetric halving, which this step is compared against
                              "t_full_product_ms": 2.0 * args.n * args.n * args.d / (P["bf16_sustained"] * 1e12) * 1e3,
                              # the exact re-rank's gathers (candidates x 4 d bytes) at HBM bandwidth,
                              # serial after the GEMM: the floor of this form's design
                              "rerank_gather_bytes": s0["candidates"] * args.d * 4.0,
                              "t_gemm_then_rerank_ms": (t_roof + s0["candidates"] * args.d * 4.0
                                                        / (P["hbm_gbs"] * 1e9)) * 1e3},
            "roofline": roof, "clocks": clk,
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
            "exactness": {"rows_uncertified": int(s0["rows_uncertified"]), "rows_fallback": int(s0["rows_fallback"]),
                          "rows_fp64_ties": int(s0["rows_fp64_ties"]), "rows_truncated": int(s0["rows_truncated"]),
                          "candidates_per_row": s0["candidates"] / max(1, s0["rows"]),
                          "inserted_per_row": s0["candidates_inserted"] / max(1, s0["rows"]),
                          "rows_reranked_in_sweep": int(s0["rows_reranked_in_sweep"]),
                          "list_capacity": int(s0["list_capacity"]),
                          "max_error_ratio": float(s0["max_error_ratio"])},
            "phases_ms": {"prep": s0["ms_prep"], "gemm_select": s0["ms_select"], "rerank": s0["ms_rerank"],
                          "fallback": s0["ms_fallback"], "gemm": s0["ms_gemm"]}}

    # the plain FP32 form on the same data, for the reported factor: one warm-up call, then the
    # median of the timed repeats (CUDA events on the call's stream), like the headline
    if form == "fused" and not args.no_compare and rank == 0:
        ms_p, sp = timed_calls(lambda: step("fp32", 0)[2], stream, args.compare_repeats)
        line["plain_fp32"] = {"rows_per_s": args.n / (ms_p / 1000.0), "ms_per_step": ms_p,
                              "gemm_ms": sp["ms_gemm"], "repeats": args.compare_repeats, "warmup": 1}
        line["fused_vs_plain"] = rows_per_s / world / (args.n / (ms_p / 1000.0))

    # the FP8 e4m3 form on the same data: time, how many rows its first pass certified, fallback
    fp8_out = None
    if form == "fused" and not args.no_compare and rank == 0:
        try:
            ms8, s8 = timed_calls(lambda: step("fp8", 1)[2], stream, args.compare_repeats)
            fp8_out = (oi.cpu().numpy(), od.cpu().numpy())
            line["fp8"] = {"rows_per_s": args.n / (ms8 / 1000.0), "ms_per_step": ms8, "ms_gemm": s8["ms_gemm"],
                           "rows_certified_first_pass": int(args.n - s8["rows_uncertified"]),
                           "rows_fallback": int(s8["rows_fallback"]), "candidates_per_row": s8["candidates"] / args.n,
                           "max_error_ratio": float(s8["max_error_ratio"]),
                           "repeats": args.compare_repeats, "warmup": 1}
        except kb.KnnError as e:
            line["fp8"] = {"unavailable": str(e)}

    # end to end through the public API with host buffers (pinned)
    if not args.no_e2e:
        Xh = torch.from_numpy(X).pin_memory()
        oih = torch.empty((args.n, k), dtype=torch.int32).pin_memory()
        odh = torch.empty((args.n, k), dtype=torch.float32).pin_memory()
        kb.knng_build(Xh, k, out_idx=oih, out_dist=odh, precision=precision, fused=fused)
        torch.cuda.synchronize()
        e_steps = max(1, min(args.steps, 3))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            kb.knng_build(Xh, k, out_idx=oih, out_dist=odh, precision=precision, fused=fused)
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / e_steps, world)
        line["e2e"] = {"value": weak_scaling_rate(args.n, world, dt), "unit": "rows/s",
                       "h2d_bytes_per_step": args.n * args.d * 4,
                       "d2h_bytes_per_step": args.n * k * 8}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample_rate(X, k, args.cpu_seconds, seed=77)
        rows, ri, rd = cb.pop("_rows"), cb.pop("_idx"), cb.pop("_dist")
        line["cpu_baseline"] = cb
        # the timed output against the FP64 oracle on the oracle's rows
        line["oracle_check"] = oracle_check(X, rows, fused_idx[rows], fused_dist[rows], ri, rd)
        if fp8_out is not None and "fp8" in line:
            line["fp8"]["oracle_check"] = oracle_check(X, rows, fp8_out[0][rows], fp8_out[1][rows], ri, rd)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
