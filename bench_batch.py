"""Uneven batch benchmark: 4096 random recursive trees, sizes log-uniform in
[64, 65536] (integer edge lengths 1..8, grid step 1), d = 16 FP32 N(0,1),
f(x) = 1/(1 + 0.1 x)^2; forward + backward per step.

The forest is planned once (leaf cutoff s0 and the shared-memory FFT tile chosen by
the library autotuner, tfi_autotune, on a subset of the trees)
and a whole step is captured in one CUDA graph: every tree's calls share the
same launches. It is compared with a per-tree launch loop (one plan and two
applies per tree) on the same GPU, and spot-checked against the FP64 oracle.
Prints one JSON line.

    python bench_batch.py [--count 4096] [--steps 10] [--warmup 3]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--loop-trees", type=int, default=0, help="trees in the per-tree loop (0 = all)")
    a = ap.parse_args()
    import torch

    import paper_2609_34025_b300 as tfi
    from paper_2609_34025_b300 import build as tbuild
    import workloads as W
    from workloads import trees as T

    tbuild.build()
    d = 16
    cfg = W.configs.uneven_batch(count=a.count, d=d)
    forest, offs, sizes = cfg["tree"], cfg["offsets"], cfg["sizes"]
    spec, delta = cfg["kernel"], cfg["delta"]
    n = forest.n

    def timed(fn, k, w=2):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    # the library autotuner: leaf cutoff and shared-memory FFT tile timed on the first 256 trees
    # (a representative size mix), then the whole forest planned once with the winner
    t0 = time.perf_counter()
    plan, tuned = tfi.Plan.autotune(forest, delta, spec, d, leaf_candidates=[64, 128, 256, 512],
                                    sample_trees=min(256, a.count), reps=5)
    plan_s = time.perf_counter() - t0
    best = tuned["leaf_max"]
    F = torch.from_numpy(W.normal_field(n, d, seed=123)).cuda()
    G = torch.from_numpy(W.normal_field(n, d, seed=124)).cuda()
    out, gF = torch.empty_like(F), torch.empty_like(F)
    graph = tfi.Graph(plan, F, out, G, gF)
    step_ms = timed(graph.launch, a.steps, a.warmup)
    # the step against HBM: the hot-path byte model and the stage model's bytes (bin-sum and table
    # rows written and read between stages too), two applies per step
    from bench import measured_peaks, step_bytes_8d
    pk, pk_src = measured_peaks()
    b8d = step_bytes_8d(plan, n, d)
    b_stages = sum(b for b, _ in plan.stage_model(d).values())
    t_step = step_ms / 1e3
    hbm = {"bytes_per_apply_model": b8d, "bytes_per_apply_stages": b_stages,
           "achieved_gbs": 2 * b8d / t_step / 1e9, "frac": 2 * b8d / t_step / 1e9 / pk["hbm_gbs"],
           "frac_stage_bytes": 2 * b_stages / t_step / 1e9 / pk["hbm_gbs"], "peak": pk["hbm_gbs"],
           "unit": "GB/s", "peak_source": f"{pk_src} (MEASURED_PEAKS.json hbm_gbs)"}
    # spot check against the oracle
    from oracle import brute
    rng = np.random.default_rng(0)
    tgt = np.sort(rng.choice(n, 64, replace=False)).astype(np.int32)
    graph.launch()
    torch.cuda.synchronize()
    ref = brute.integrate(forest, delta, spec, F.cpu().numpy().astype(np.float64), targets=tgt)
    y = out.cpu().numpy()[tgt].astype(np.float64)
    err = float((np.abs(y - ref).max(0) / np.abs(ref).max(0)).max())
    # per-tree launch loop: one plan per tree, forward + backward applies tree by tree
    nloop = a.count if a.loop_trees <= 0 else min(a.loop_trees, a.count)
    plans, views = [], []
    t1 = time.perf_counter()
    for i in range(nloop):
        lo, hi = int(offs[i]), int(offs[i + 1])
        e0, e1 = lo - i, hi - i - 1
        ti = T.Tree(hi - lo, forest.u[e0:e1] - lo, forest.v[e0:e1] - lo, forest.w[e0:e1])
        plans.append(tfi.Plan.from_spec(ti, delta, spec, leaf_max=best, max_channels=d))
        views.append((F[lo:hi], out[lo:hi], G[lo:hi], gF[lo:hi]))
    loop_plan_s = time.perf_counter() - t1

    def loop_step():
        for p, (f, o, g, q) in zip(plans, views):
            p.apply(f, o)
            p.apply_backward(g, q)

    loop_ms = timed(loop_step, max(1, a.steps // 5), 1)
    loop_n = int(offs[nloop])
    line = {
        "metric": "vertex.channel integrations/s (N*d/s), fwd+bwd, uneven batch", "value": n * d / (step_ms / 1e3),
        "unit": "vertex.channel/s", "ms_per_step": step_ms, "steps": a.steps, "warmup": a.warmup,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"uneven_batch_{a.count}_trees", "trees": a.count, "n_total": int(n),
                   "sizes": "log-uniform [64, 65536]", "weights": "integers 1..8", "delta": 1.0, "d": d,
                   "kernel": "1/(1+0.1x)^2", "autotuned": tuned, "autotune_trees": min(256, a.count),
                   "autotune_and_plan_seconds": round(plan_s, 2), "launch": "one CUDA graph per fwd+bwd step"},
        "per_tree_loop": {"trees": nloop, "n": loop_n, "ms_per_step": loop_ms,
                          "value": loop_n * d / (loop_ms / 1e3), "plan_seconds": round(loop_plan_s, 2)},
        "speedup_vs_loop": (loop_n * d / (loop_ms / 1e3)) and (n * d / (step_ms / 1e3)) / (loop_n * d / (loop_ms / 1e3)),
        "parity": {"sampled_targets": 64, "max_normwise_err": err},
        "hbm": hbm,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
