"""Per-operation throughput of the library on one grid level (CUDA events).

    python opbench.py --op all --shape 256 256 --frames 200

Each operation is timed through the C ABI on device-resident data (the call,
including its host work) and reported as achieved GB/s of its algorithmic bytes (every array it must read or write
counted once, per pixel-frame, fp32; see the table in each result) against
the measured HBM copy bandwidth; "kernel_us_per_launch" gives the device
time of each kernel class from the library's own CUDA-event profiling.
Inputs are larger than L2 at the default size, and L2 is flushed before every
timed call.

    python opbench.py --op net_forward --shape 256 256 --frames 32

times the learned predictor's forward pass on a batch of `frames` canvases
(TFLOP/s of its 3x3 convolutions against the measured BF16 peak);
`--op net_train` one training step (forward, input and weight gradients,
Adam) on `frames` crops of the given shape.

    python opbench.py --op batch --frames 8

registers `frames` sequences of uneven length and size (the first of the
batching workload's seeded draws, scaled down by 4 in each axis) with the
persistent batched solver and reports the time of each stage.

    python opbench.py --op coop_floor

sets the cooperative PCG solves of the paper-scale registration (the small
levels) against the latency floor of their grid barriers and reductions.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _peak():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        return 6800.0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="all",
                    choices=["all", "hessvec", "eval", "objective", "trial", "predict_ls", "net_forward",
                             "net_train", "batch", "coop_floor"])
    ap.add_argument("--shape", type=int, nargs="+", default=[256, 256])
    ap.add_argument("--frames", type=int, default=200)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    args = ap.parse_args(argv)

    import torch
    import paper_2001_06613_gb300 as S
    from paper_2001_06613_gb300 import synthetic
    S.load()
    dev = torch.device("cuda", 0)
    if args.op == "net_forward":
        return net_forward(S, torch, synthetic, dev, args)
    if args.op == "net_train":
        return net_train(S, torch, synthetic, dev, args)
    if args.op == "batch":
        return batch(S, torch, synthetic, dev, args)
    if args.op == "coop_floor":
        return coop_floor(S, torch, synthetic, dev, args)
    shape = tuple(args.shape)
    d = len(shape)
    n = args.frames
    N = int(np.prod(shape))
    rng = np.random.default_rng(0)
    R = torch.rand((n,) + shape, device=dev, dtype=torch.float32)
    prm = S.stml_default_params(n_levels=1, n_tlevels=1)
    ctx = S.Context(prm)
    S.stml_load_sequence(ctx.ptr, R)
    S.stml_build_pyramid(ctx.ptr)
    frames = list(range(n))
    u = torch.from_numpy(synthetic.random_field(rng, 1, d, shape, amp=2.0, rough=0.3)).to(dev)
    u = u.expand(n, *u.shape[1:]).contiguous()
    v = torch.randn((n, d) + shape, device=dev)
    g = torch.empty_like(v)
    # a smooth search direction for the trial objective (like a Gauss-Newton step)
    dirn = torch.from_numpy(synthetic.random_field(rng, 1, d, shape, amp=0.7, rough=0.3)).to(dev)
    dirn = dirn.expand(n, *dirn.shape[1:]).contiguous()
    dT = torch.empty_like(v)
    Hv = torch.empty_like(v)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    peak = _peak()
    pf = n * N
    S.stml_eval(ctx.ptr, 0, frames, u, g, dT)

    def timed(fn, nbytes, name, per_pf):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        S.stml_profile_enable(ctx.ptr, 1)   # CUDA events around every library launch
        for _ in range(args.iters):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        kernels = {}
        for r in S.stml_profile_report(ctx.ptr):
            kernels[r["kernel"]] = round(1e3 * r["ms"] / max(1, r["launches"]), 3)
        S.stml_profile_enable(ctx.ptr, 0)
        ms = float(np.median(ts))
        gbs = nbytes / (ms / 1e3) / 1e9
        print(json.dumps({"op": name, "shape": list(shape), "frames": n, "ms": ms, "GB/s": gbs,
                          "frac_of_measured_hbm": gbs / peak, "bytes_per_pixel_frame": per_pf,
                          "kernel_us_per_launch": kernels}), flush=True)

    ops = [args.op] if args.op != "all" else ["hessvec", "eval", "objective", "trial", "predict_ls"]
    for op in ops:
        if op == "hessvec":
            b = 12 * d                     # read v, read grad T, write Hv
            timed(lambda: S.stml_hessvec(ctx.ptr, 0, frames, dT, v, Hv), b * pf, op, b)
        elif op == "eval":
            b = 4 + 4 * d + 12 * d         # read T, read u; write grad T, g, M^-1
            timed(lambda: S.stml_eval(ctx.ptr, 0, frames, u, g, dT), b * pf, op, b)
        elif op == "objective":
            b = 4 + 4 * d                  # read T, read u
            timed(lambda: S.stml_eval(ctx.ptr, 0, frames, u), b * pf, op, b)
        elif op == "trial":
            b = 4 + 8 * d                  # read T, u, d
            timed(lambda: S.stml_eval_trial(ctx.ptr, 0, frames, u, dirn, 0.5), b * pf, op, b)
            b = 4 + 16 * d                 # and g, d for <g, d> (first Armijo trial)
            timed(lambda: S.stml_eval_trial(ctx.ptr, 0, frames, u, dirn, 1.0, g), b * pf, "trial_gd", b)
        elif op == "predict_ls":
            K = list(range(0, n, 4))
            if K[-1] != n - 1:
                K.append(n - 1)
            eta = torch.randn((len(K), d) + shape, device=dev)
            omega = torch.randn((n, d) + shape, device=dev)
            zeta = torch.empty_like(omega)
            b = 16 + 8 * len(K) / n        # omega (all + K), zeta x3 (in-place sweep), eta on K
            timed(lambda: S.stml_predict_ls(eta, K, omega, zeta, n, 1e-5, d * N), b * d * pf, op, b * d)
    ctx.close()


def net_forward(S, torch, synthetic, dev, args):
    """Forward pass of the predictor network on B = --frames canvases."""
    H, W = args.shape[0], args.shape[1]
    B = args.frames
    rng = np.random.default_rng(0)
    f = torch.from_numpy(synthetic.random_field(rng, 2 * B, 2, (H, W), amp=2.0)).to(dev)
    T = torch.rand((3, B, H, W), device=dev)
    out = torch.empty((B, 2, H, W), device=dev)
    net = S.Net(synthetic.net_init_params(0, head_scale=1.0), max_batch=B, max_h=H, max_w=W)
    smp = S.net_samples(f[:B].contiguous(), f[B:].contiguous(), T[0], T[1], T[2], 1.0, 0.5, out=out)
    convs = [(0, 7, 32), (0, 32, 32), (1, 32, 64), (1, 64, 64), (2, 64, 96), (2, 96, 96), (3, 96, 128),
             (3, 128, 128), (2, 224, 96), (2, 96, 96), (1, 160, 64), (1, 64, 64), (0, 96, 32), (0, 32, 32)]
    H8, W8 = (H + 7) // 8 * 8, (W + 7) // 8 * 8
    flops = sum(2.0 * B * (H8 >> lv) * (W8 >> lv) * 9 * ci * co for lv, ci, co in convs)
    for _ in range(args.warmup):
        S.stml_net_forward(net, smp, H, W)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        S.stml_net_forward(net, smp, H, W)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    net.close()
    ms = float(np.median(ts))
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
    except Exception:
        peak = 1900.0
    tf = flops / (ms / 1e3) / 1e12
    print(json.dumps({"op": "net_forward", "batch": B, "shape": [H, W], "ms": ms, "GFLOP": flops / 1e9,
                      "TFLOP/s": tf, "frac_of_measured_bf16": tf / peak}), flush=True)
    return 0



def net_train(S, torch, synthetic, dev, args):
    """One Adam step of the predictor network on B = --frames crops."""
    H, W = args.shape[0], args.shape[1]
    B = args.frames
    rng = np.random.default_rng(1)
    f = torch.from_numpy(synthetic.random_field(rng, 3 * B, 2, (H, W), amp=2.0)).to(dev)
    T = torch.rand((3, B, H, W), device=dev)
    net = S.Net(synthetic.net_init_params(0, head_scale=0.1), max_batch=B, max_h=H, max_w=W)
    smp = S.net_samples(f[:B].contiguous(), f[B:2 * B].contiguous(), T[0], T[1], T[2], 1.0, 0.5,
                        target=f[2 * B:].contiguous())
    for _ in range(args.warmup):
        S.stml_net_train_step(net, smp, H, W, lr=1e-6, want_loss=False)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.iters):
        S.stml_net_train_step(net, smp, H, W, lr=1e-6, want_loss=False)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.iters
    convs = [(0, 7, 32), (0, 32, 32), (1, 32, 64), (1, 64, 64), (2, 64, 96), (2, 96, 96), (3, 96, 128),
             (3, 128, 128), (2, 224, 96), (2, 96, 96), (1, 160, 64), (1, 64, 64), (0, 96, 32), (0, 32, 32)]
    flops = sum(2.0 * B * (H >> lv) * (W >> lv) * 9 * ci * co * (2 if i == 0 else 3)
                for i, (lv, ci, co) in enumerate(convs))
    print(json.dumps({"op": "net_train", "batch": B, "shape": [H, W], "ms": ms,
                      "tflops_algorithmic": flops / (ms / 1e3) / 1e12}), flush=True)
    net.close()


def batch(S, torch, synthetic, dev, args):
    """stml_batch_register on --frames sequences: 20-300 frames of 32^2-128^2."""
    rng = np.random.default_rng(1000)
    seqs = []
    for i in range(args.frames):
        n = int(rng.integers(20, 301))
        m = int(rng.choice([32, 48, 64, 96, 128]))
        seqs.append(torch.from_numpy(synthetic.make_sequence(synthetic.SequenceSpec(
            n=n, shape=(m, m), n_modes=4, amp=1.0, periods=[(16.0, 0.0)], noise_sd=0.01, seed=1000 + i)))
            .to(dev))
    prm = S.stml_default_params(n_levels=3, n_tlevels=3)
    ctxs = [S.Context(prm) for _ in seqs]
    for c, R in zip(ctxs, seqs):
        S.stml_load_sequence(c.ptr, R)
        S.stml_build_pyramid(c.ptr)
    bt = S.Batch(ctxs)
    for _ in range(max(1, args.warmup)):
        bt.register(0)
    torch.cuda.synchronize()
    reports = []
    for _ in range(max(1, args.iters)):
        for c, R in zip(ctxs, seqs):
            S.stml_load_sequence(c.ptr, R)
            S.stml_build_pyramid(c.ptr)
        bt.register(0)
        reports.append(bt.report())
    torch.cuda.synchronize()
    print(json.dumps({"op": "batch", "sequences": len(seqs), "frames": sum(int(r.shape[0]) for r in seqs),
                      "shapes": [list(r.shape) for r in seqs], "stages": reports}), flush=True)
    bt.close()
    for c in ctxs:
        c.close()


def _coop_blocks(shape, nK, sms):
    """CTAs of the cooperative PCG solve of nK frames on a 2-D level `shape`:
    the larger of its (frame, 1024-pixel chunk) items and its pixel tiles
    (16 pixels with the float4 path), at most two per SM -- the grid rule of
    the solve's launcher."""
    N = int(np.prod(shape))
    vec = 4 if shape[-1] % 4 == 0 else 1
    tpr = 4 if vec == 4 else 8
    items = -(-N // (256 * vec)) * nK
    tiles = -(-N // (tpr * vec))
    return max(1, min(max(items, tiles), 2 * sms))


def coop_floor(S, torch, synthetic, dev, args):
    """The cooperative PCG solves of the paper-scale STML registration (200
    frames of 256^2, 4 spatial and 3 temporal levels) against their latency
    floor: per level, the solve's device time per CG step (each solve's start
    and end amortised over its steps; every launch timed with CUDA events) and
    the time of the synchronisation alone (stml_coop_sync_floor) on the grid
    of each GIR, weighted by the GIR's CG steps."""
    L, Q = 4, 3
    R = torch.from_numpy(synthetic.make_sequence(synthetic.spec_paper_scale())).to(dev)
    finest = tuple(R.shape[1:])
    ctx = S.Context(S.stml_default_params(n_levels=L, n_tlevels=Q))

    def run():
        S.stml_load_sequence(ctx.ptr, R)
        S.stml_build_pyramid(ctx.ptr)
        return S.stml_register(ctx.ptr, S.MODE_STML)

    for _ in range(max(1, args.warmup)):
        run()
    torch.cuda.synchronize()
    S.stml_profile_enable(ctx.ptr, 1)
    stats = run()
    table = S.stml_profile_report(ctx.ptr)
    S.stml_profile_enable(ctx.ptr, 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    for lev in range(L):
        shape = tuple(m >> (L - 1 - lev) for m in finest)
        N = int(np.prod(shape))
        rows = [r for r in table if r["kernel"] == "pcg_solve_cooperative" and r["level"] == lev]
        girs = [s for s in stats if s["level"] == lev and N * s["n_frames"] <= (1 << 21)]
        if not rows or not girs:
            continue
        cg = sum(s["cg_iters"] for s in girs)
        blocks = [_coop_blocks(shape, s["n_frames"], sms) for s in girs]
        floors = [S.stml_coop_sync_floor(b, 20 * args.iters) for b in blocks]
        floor = sum(f * s["cg_iters"] for f, s in zip(floors, girs)) / max(1, cg)
        us = 1e3 * sum(r["ms"] for r in rows) / max(1, cg)
        print(json.dumps({"op": "coop_floor", "level": lev, "shape": list(shape),
                          "frames": [s["n_frames"] for s in girs], "cg_steps": [s["cg_iters"] for s in girs],
                          "solves": sum(r["launches"] for r in rows), "blocks": blocks,
                          "floor_us_per_step": [round(f, 3) for f in floors],
                          "us_per_cg_step": round(us, 3), "floor_us_per_cg_step": round(floor, 3),
                          "floor_share": round(floor / us, 3)}), flush=True)
    ctx.close()


if __name__ == "__main__":
    sys.exit(main())
