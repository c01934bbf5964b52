"""Attention-width benchmark: one tree per head (12 heads, random spanning trees
of the 14 x 14 patch grid, unit edges, N = 196), d = 64 images x 64 channels =
4096 BF16 channels, f = 8-term exponential sum per head. One step = forward and
backward (K G) for every head, plus the learnable-f gradient with --grad. The
heads are independent: each head's step is one CUDA graph replayed on its own
stream, and the step ends when all streams have joined.

Compares the cross-table evaluators: FFT / direct (default), the Hankel-matrix
product on tensor cores chosen by the cost model ("auto") or for every
qualifying table ("all"), dense leaves on the FP32 ALUs instead of the tensor
cores ("alu_leaf"), and the dense f(D) F path on tensor cores. The leaf cutoff
s0 is tuned per variant. Outputs of head 0 are checked against the
FP64 oracle. Prints one JSON line.

    python bench_attention.py [--steps 20] [--warmup 3] [--grad]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--heads", type=int, default=12)
    ap.add_argument("--grad", action="store_true", help="include the learnable-f gradient in the step")
    ap.add_argument("--modes", default="default,auto,all,alu_leaf", help="comma-separated variants to run")
    ap.add_argument("--s0", type=int, default=0, help="fixed leaf cutoff (0: tune per variant)")
    ap.add_argument("--no-dense", dest="dense", action="store_false", help="skip the dense tensor-core path")
    a = ap.parse_args()
    import torch

    import paper_2609_34025_b300 as tfi
    from paper_2609_34025_b300 import build as tbuild
    import workloads as W
    from oracle import brute

    tbuild.build()
    cfg = W.configs.attention(heads=a.heads)
    heads = cfg["heads"]
    d = cfg["d"]
    n = heads[0]["tree"].n
    gen = torch.Generator(device="cuda").manual_seed(123)
    X = [torch.randn(n, d, device="cuda", generator=gen).to(torch.bfloat16) for _ in heads]
    G = [torch.randn(n, d, device="cuda", generator=gen).to(torch.bfloat16) for _ in heads]
    Y = [torch.empty_like(x) for x in X]
    GX = [torch.empty_like(x) for x in X]

    def timed(fn, k, w):
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

    def make(mode, s0):
        return [tfi.Plan.from_spec(h["tree"], 1.0, h["kernel"], leaf_max=s0, max_channels=d,
                                   hankel=mode if mode in ("auto", "all") else None,
                                   leaf_alu=mode == "alu_leaf") for h in heads]

    # the heads are independent: each replays its graph on its own stream, joined at the end of the step
    streams = [torch.cuda.Stream() for _ in heads]

    def step_fn(plans, graphs):
        def run():
            cur = torch.cuda.current_stream()
            start = torch.cuda.Event()
            start.record(cur)
            for st, g in zip(streams, graphs):
                st.wait_event(start)
                g.launch(stream=st)
            if a.grad:
                # dL/df per head on its stream, parameter gradients left on the device
                for p, g, x, st in zip(plans, G, X, streams):
                    p.kernel_grad(g, x, stream=st, device_dtheta=True)
            for st in streams:
                cur.wait_stream(st)
        return run

    results = {}
    for mode in a.modes.split(","):
        best = None
        for s0 in ((a.s0,) if a.s0 > 0 else (1, 4, 16, 64, 196)):
            plans = make(mode, s0)
            graphs = [tfi.Graph(p, x, y, g, gx) for p, x, y, g, gx in zip(plans, X, Y, G, GX)]
            ms = timed(step_fn(plans, graphs), max(3, a.steps // 4), 2)
            if best is None or ms < best[0]:
                best = (ms, s0)
            for g in graphs:
                g.close()
        plans = make(mode, best[1])
        graphs = [tfi.Graph(p, x, y, g, gx) for p, x, y, g, gx in zip(plans, X, Y, G, GX)]
        ms = timed(step_fn(plans, graphs), a.steps, a.warmup)
        info = [p.info() for p in plans]
        # per-stage device time of one forward per head
        for p in plans:
            p.profile(True)
        for p, x, y in zip(plans, X, Y):
            p.apply(x, y)
        prof = {}
        for p in plans:
            for k, (t, ln) in p.profile_read().items():
                prof[k] = prof.get(k, 0.0) + t
            p.profile(False)
        model = {}
        for p in plans:
            for k, (b, f) in p.stage_model(d, tfi.DTYPE_BF16).items():
                mb, mf = model.get(k, (0.0, 0.0))
                model[k] = (mb + b, mf + f)
        # parity of head 0 against the FP64 oracle
        y0 = plans[0].apply(X[0]).float().cpu().numpy().astype(np.float64)
        ref = brute.integrate(heads[0]["tree"], 1.0, heads[0]["kernel"], X[0].float().cpu().numpy().astype(np.float64))
        err = float((np.abs(y0 - ref).max(0) / np.maximum(np.abs(ref).max(0), 1e-300)).max())
        results[mode] = dict(
            s0=best[1], ms_per_step=ms, value=a.heads * n * d / (ms * 1e-3),
            n_jobs_hankel=sum(i["n_jobs_hankel"] for i in info), n_jobs_direct=sum(i["n_jobs_direct"] for i in info),
            n_jobs_fft=sum(i["n_jobs_fft"] for i in info), stage_ms={k: round(v, 4) for k, v in prof.items() if v > 0},
            hankel_tflops=(model["hankel"][1] / (prof["hankel"] * 1e-3) / 1e12) if prof.get("hankel") else None,
            parity_head0=err, device_errors=sum(i["device_errors"] for i in info))
        for g in graphs:
            g.close()
    # dense f(D) F on tensor cores, forward and backward per head (synchronises per call)
    dense_ms = None
    if a.dense:
        plans = make("default", 64)
        dense_ms = timed(lambda: [(p.dense_apply(x, y), p.dense_apply(g, gx)) for p, x, y, g, gx in
                                  zip(plans, X, Y, G, GX)], a.steps, a.warmup)
    out = dict(metric="vertex.channel integrations/s (fwd+bwd" + (" + f grad" if a.grad else "") + ")",
               unit="vertex.channel/s", workload=f"attention_{a.heads}heads_n{n}_d{d}_bf16_expsum8",
               dtype="bf16", data="synthetic", evaluators=results,
               dense_tensor_core=None if dense_ms is None else
               dict(ms_per_step=dense_ms, value=a.heads * n * d / (dense_ms * 1e-3)))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
