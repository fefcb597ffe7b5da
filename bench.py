"""Benchmark: frames registered per second by spatio-temporal multilevel (STML)
registration of a 200-frame 256x256 OCT-like sequence (4 spatial x 3 temporal
levels), with the Gauss-Newton Hessian-product kernel's HBM throughput.

One step = one full registration of the sequence through the C ABI
(pyramid build, predictor-corrector sweep over all levels, Gauss-Newton/PCG),
inputs resident in device memory.  Run with no flags for 1 GPU; under
torchrun every rank registers its own replica (no data-path collective).

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (the method has no other reference implementation).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames registered/s at fixed objective tol; GN-matvec HBM GB/s vs peak"

WORKLOADS = {
    # name: (n, shape, levels, tlevels, spec factory name)
    "paper-scale": (200, (256, 256), 4, 3, "spec_paper_scale"),
    "tiny": (16, (64, 64), 2, 2, "spec_tiny"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="paper-scale", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="stml", choices=["stml", "spml"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-spml", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-affine", action="store_true")
    ap.add_argument("--no-volume", action="store_true")
    ap.add_argument("--no-ugrid", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="let the library time launch shapes and PCG paths on first use (warm-up steps)")
    ap.add_argument("--cpu-sample-frames", type=int, default=25)
    ap.add_argument("--batch-sequences", type=int, default=8,
                    help="sequences of the batching workload (the first N of its 64 seeded draws)")
    ap.add_argument("--image-dtype", default="f32", choices=["f32", "f16", "bf16"],
                    help="storage of the image pyramid and of the solver's grad T (arithmetic stays FP32)")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
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
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


MATVEC_SOURCES = ("k_gn.cu", "gn_items.cuh")   # the Hessian-product kernel and its per-item body


def matvec_source_digest():
    h = hashlib.sha256()
    for name in MATVEC_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2001_06613_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def matvec_traffic_per_pixel_frame():
    """DRAM bytes per pixel-frame of the Hessian-product kernel from the ncu
    capture recorded in profiles/gn_matvec_paper_scale.json, if that capture
    was taken on the current kernel source (same hash of csrc/k_gn.cu and
    csrc/gn_items.cuh)."""
    path = os.path.join(ROOT, "profiles", "gn_matvec_paper_scale.json")
    try:
        rec = json.load(open(path))
        if rec.get("kernel_source_sha256_16") != matvec_source_digest():
            return None
        return float(rec["dram_bytes_per_pixel_frame"])
    except Exception:
        return None


def make_sequence(workload: str, seed_offset: int = 0):
    from paper_2001_06613_gb300 import synthetic
    n, shape, L, Q, factory = WORKLOADS[workload]
    spec = getattr(synthetic, factory)()
    spec.seed += seed_offset
    return synthetic.make_sequence(spec), spec


# ----------------------------------------------------------------- CPU oracle
def _oracle_register_chunk(job):
    """One oracle registration of frames [lo, hi) (runs in a spawned worker)."""
    workload, lo, hi, mode = job
    from oracle import Params, multilevel
    n, shape, L, Q, _ = WORKLOADS[workload]
    R, _ = make_sequence(workload)
    sub = R[lo:hi].astype(np.float64)
    t0 = time.perf_counter()
    multilevel.register(sub, Params(n_levels=L, n_tlevels=Q), mode)
    return hi - lo, time.perf_counter() - t0


def oracle_sample(R: np.ndarray, workload: str, frames: int, mode: str = "stml"):
    """Register the first `frames` frames (full spatial size, same level
    structure) with the FP64 oracle on one thread; returns (frames/s, seconds)."""
    from oracle import Params, multilevel
    n, shape, L, Q, _ = WORKLOADS[workload]
    p = Params(n_levels=L, n_tlevels=Q)
    sub = R[:frames].astype(np.float64)
    t0 = time.perf_counter()
    multilevel.register(sub, p, mode)
    dt = time.perf_counter() - t0
    return frames / dt, dt


def host_cpu():
    """(logical cores, model name) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return os.cpu_count() or 1, model or "unknown"


def oracle_sample_all_cores(workload: str, frames: int, mode: str = "stml"):
    """The oracle on all host cores: the sequence is cut into consecutive
    chunks of `frames` frames, each registered by its own single-threaded
    worker process (started with spawn), all at once.  Returns (frames/s over
    the longest worker's registration time, workers, that time, frames
    registered)."""
    import multiprocessing as mp
    n = WORKLOADS[workload][0]
    cores, _ = host_cpu()
    chunks = [(lo, min(lo + frames, n)) for lo in range(0, n, frames)]
    chunks = [c for c in chunks if c[1] - c[0] == frames][:max(1, cores)]
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"       # one thread per worker; inherited by the spawned processes
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(len(chunks)) as pool:
            res = pool.map(_oracle_register_chunk, [(workload, lo, hi, mode) for lo, hi in chunks])
        wall = max(t for _, t in res)   # the workers register at the same time; input generation excluded
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    done = sum(f for f, _ in res)
    return done / wall, len(chunks), wall, done


def oracle_op_ns(workload: str, frames: int, reps: int = 3):
    """FP64 oracle's per-operation cost on the finest level of `frames`
    frames (seeded inputs, one thread), in nanoseconds per pixel-frame:
    the Gauss-Newton Hessian product, the objective + gradient pass (warp,
    grad T, residual, regulariser, penalty) and the least-squares predictor
    of eq. (2) over all frames of the sequence.  The CPU side of the
    per-operation comparison in the bench line."""
    from oracle import Params, grid, objective, predictor
    n, shape, L, Q, _ = WORKLOADS[workload]
    rng = np.random.default_rng(5)
    d = len(shape)
    N = float(np.prod(shape))
    p = Params(n_levels=L, n_tlevels=Q)
    K = list(range(frames))
    out = {}

    def timed(f):
        f()
        t0 = time.perf_counter()
        for _ in range(reps):
            f()
        return (time.perf_counter() - t0) / reps

    dT = rng.normal(size=(frames, d) + tuple(shape))
    v = rng.normal(size=(frames, d) + tuple(shape))
    dt = timed(lambda: objective.hessvec(dT, v, K, 1.0, p))
    out["gn_hessian_product"] = {"oracle_ns_per_pixel_frame": 1e9 * dt / (frames * N),
                                 "sample": f"finest level, {frames} frames, mean of {reps} calls ({dt:.2f} s each)"}
    R, _ = make_sequence(workload)
    T = R[:frames].astype(np.float64)
    u = 0.5 * rng.normal(size=(frames, d) + tuple(shape))
    dt = timed(lambda: objective.evaluate(T, u, K, 1.0, p))
    out["gradient_pass"] = {"oracle_ns_per_pixel_frame": 1e9 * dt / (frames * N),
                            "sample": f"finest level, {frames} frames, objective and gradient, mean of {reps} "
                                      f"calls ({dt:.2f} s each)"}
    Kq = grid.temporal_sets(n, Q)[Q - 2] if Q > 1 else list(range(n))
    omega = rng.normal(size=(n, d) + tuple(shape))
    eta = omega[Kq] + rng.normal(size=(len(Kq), d) + tuple(shape))
    dt = timed(lambda: predictor.predict_ls(eta, omega, Kq, p.beta))
    out["predict_ls_eq2"] = {"oracle_ns_per_pixel_frame": 1e9 * dt / (n * N),
                             "sample": f"finest level, all {n} frames from |K| = {len(Kq)}, mean of {reps} calls "
                                       f"({dt:.2f} s each)"}
    return out


def workload_label(args) -> str:
    """The workload as both arms name it in their config."""
    n, shape, L, Q, _ = WORKLOADS[args.workload]
    return (f"{args.workload}: {n} frames {shape[0]}x{shape[1]} fp32, "
            f"{L} spatial x {Q} temporal levels, {args.mode.upper()}")


def run_reference(args):
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    n = WORKLOADS[args.workload][0]
    # frames per chunk: the whole run (warm-up and timed steps) within about
    # 2.5 minutes at the oracle's measured ~0.55 s per frame and core of this
    # workload (between 4 and --cpu-sample-frames frames)
    per_step_s = 150.0 / max(1, args.steps + args.warmup)
    frames = max(4, min(args.cpu_sample_frames, n, int(per_step_s / 0.55)))
    for _ in range(args.warmup):
        oracle_sample_all_cores(args.workload, frames, args.mode)
    times, done = [], 0
    for _ in range(args.steps):
        _, workers, wall, f = oracle_sample_all_cores(args.workload, frames, args.mode)
        times.append(wall)
        done += f
    total = sum(times)
    value = done / total
    host_cores, model = host_cpu()
    sample = (f"{workers} chunks of {frames} consecutive frames of {n} at full size, same spatial/temporal "
              f"levels, each registered by its own single-threaded numpy FP64 worker process, all at once; "
              f"one such batch per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_label(args), "n_frames": n,
                       "shape": list(WORKLOADS[args.workload][1]), "levels": WORKLOADS[args.workload][2],
                       "tlevels": WORKLOADS[args.workload][3], "mode": args.mode, "sample_frames": frames},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": workers, "kind": "oracle",
                             "sample": sample, "host_cores": host_cores, "cpu_model": model},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------- batched serving
BATCH_LEVELS = (4, 3)


class RawStreams:
    """Distinct CUDA streams, one per context (torch's stream pool repeats
    after 32 streams, and contexts of stml_register_batch may not share one)."""

    def __init__(self, torch, n: int):
        import ctypes
        self.rt = None
        for name in ("libcudart.so", "libcudart.so.13", "libcudart.so.12"):
            try:
                self.rt = ctypes.CDLL(name)
                break
            except OSError:
                continue
        self.handles = []
        if self.rt is None:   # fall back to torch streams when n fits its pool
            if n > 32:
                raise RuntimeError("no CUDA runtime library to create more than 32 streams")
            self.torch_streams = [torch.cuda.Stream() for _ in range(n)]
            self.handles = [st.cuda_stream for st in self.torch_streams]
            return
        for _ in range(n):
            h = ctypes.c_void_p()
            if self.rt.cudaStreamCreateWithFlags(ctypes.byref(h), 1) != 0:   # cudaStreamNonBlocking
                raise RuntimeError("cudaStreamCreateWithFlags failed")
            self.handles.append(h.value)

    def close(self):
        if self.rt is not None:
            import ctypes
            for h in self.handles:
                self.rt.cudaStreamDestroy(ctypes.c_void_p(h))
        self.handles = []


def batch_specs(count: int):
    """The batching workload: 64 seeded sequences, frame counts uniform in
    20-300, sizes drawn from 128^2 ... 512^2, each with its own smooth motion
    of the tiny workload's kind (4 Fourier modes, 2 px, sin(2 pi t / 16)); the
    first `count` of the 64 draws."""
    from paper_2001_06613_gb300 import synthetic
    rng = np.random.default_rng(1000)
    out = []
    for i in range(64):
        n = int(rng.integers(20, 301))
        m = int(rng.choice([128, 192, 256, 384, 512]))
        out.append(synthetic.SequenceSpec(n=n, shape=(m, m), n_modes=4, amp=2.0, periods=[(16.0, 0.0)],
                                          noise_sd=0.01, seed=1000 + i))
    return out[:count]


def run_batch_small(S, torch, dev, mode, count: int = 64):
    """Many small sequences (seeded: 20-60 frames of 32^2, 48^2 or 64^2, the
    tiny workload's kind of motion, 3 x 3 levels), where each registration is
    bound by launch and synchronisation latency rather than by bytes:
    sequential, streams and persistent forms as in run_batch."""
    from paper_2001_06613_gb300 import synthetic
    rng = np.random.default_rng(2000)
    seqs = []
    for i in range(count):
        n = int(rng.integers(20, 61))
        m = int(rng.choice([32, 48, 64]))
        seqs.append(torch.from_numpy(synthetic.make_sequence(synthetic.SequenceSpec(
            n=n, shape=(m, m), n_modes=4, amp=1.5, periods=[(16.0, 0.0)], noise_sd=0.01, seed=2000 + i),
            device=dev)).to(dev))
    frames = sum(int(r.shape[0]) for r in seqs)
    torch.cuda.synchronize()   # the contexts' streams do not wait for torch's stream
    raw = RawStreams(torch, len(seqs))
    ctxs = [S.Context(S.stml_default_params(n_levels=3, n_tlevels=3), st) for st in raw.handles]

    def timed(fn):
        for _ in range(2):
            for c, R in zip(ctxs, seqs):
                S.stml_load_sequence(c.ptr, R)
                S.stml_build_pyramid(c.ptr)
            torch.cuda.synchronize()
            a = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            t = time.perf_counter() - a
        return t

    t_seq = timed(lambda: [S.stml_register(c.ptr, mode) for c in ctxs])
    bt = S.Batch(ctxs)
    t_per = timed(lambda: bt.register(mode))
    steps = sum(r["steps"] for r in bt.report() if "steps" in r)
    bt.close()
    for c in ctxs:
        S.stml_set_params(c.ptr, S.stml_default_params(n_levels=3, n_tlevels=3, pcg_cooperative=0))
    t_str = timed(lambda: S.stml_register_batch(ctxs, mode))
    for c in ctxs:
        c.close()
    torch.cuda.synchronize()
    raw.close()
    return {"sequences": count, "frames": frames, "sizes": "20-60 frames of 32^2/48^2/64^2, 3 x 3 levels",
            "sequential_frames_per_s": frames / t_seq, "streams_frames_per_s": frames / t_str,
            "persistent_frames_per_s": frames / t_per, "persistent_kernel_steps": steps,
            "timing": "host wall clock around the registrations (pyramids built before), second of two rounds"}


def run_batch(S, torch, dev, mode, count: int, with_combined: bool):
    """Batched serving on the batching workload (device-resident frames; every
    arm's timed region loads, builds the pyramids and registers all sequences):
      sequential -- one context per sequence, stml_register one after another;
      streams    -- stml_register_batch (a host thread and a stream per context);
      persistent -- stml_batch_register (one persistent kernel per stage);
      combined   -- persistent + BF16 image storage + the learned predictor,
                    each sequence with target_J = its sequential final
                    objective (equal final objective within 1e-5 when reached).
    Final objectives are evaluated over all frames on FP32 frames."""
    from paper_2001_06613_gb300 import synthetic
    L, Q = BATCH_LEVELS
    specs = batch_specs(count)
    t0 = time.perf_counter()
    seqs = [torch.from_numpy(synthetic.make_sequence(sp, device=dev)).to(dev) for sp in specs]
    torch.cuda.synchronize()   # the contexts' streams do not wait for torch's stream
    gen_s = time.perf_counter() - t0
    frames = sum(sp.n for sp in specs)
    pixel_frames = sum(sp.n * sp.shape[0] * sp.shape[1] for sp in specs)
    raw = RawStreams(torch, len(seqs))
    streams = raw.handles
    prm = S.stml_default_params(n_levels=L, n_tlevels=Q)
    ctxs = [S.Context(prm, st) for st in streams]

    def load_all(cs):
        for c, R in zip(cs, seqs):
            S.stml_load_sequence(c.ptr, R)
            S.stml_build_pyramid(c.ptr)

    def final_J(c, R):
        n = int(R.shape[0])
        y = torch.empty((n, 2) + tuple(R.shape[1:]), device=dev)
        S.stml_get_field(c.ptr, L - 1, y)
        return y, float(S.stml_eval(c.ptr, L - 1, list(range(n)), y)[0])

    def timed(fn, cs):
        load_all(cs)
        fn()                                   # warm-up: workspaces, graphs
        torch.cuda.synchronize()
        a = time.perf_counter()
        load_all(cs)
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - a

    t_seq = timed(lambda: [S.stml_register(c.ptr, mode) for c in ctxs], ctxs)
    y_seq, J_seq = zip(*[final_J(c, R) for c, R in zip(ctxs, seqs)])
    batch = S.Batch(ctxs)
    t_per = timed(lambda: batch.register(mode), ctxs)
    rep = batch.report()
    J_per = [final_J(c, R)[1] for c, R in zip(ctxs, seqs)]
    batch.close()
    for c in ctxs:
        S.stml_set_params(c.ptr, S.stml_default_params(n_levels=L, n_tlevels=Q, pcg_cooperative=0))
    t_str = timed(lambda: S.stml_register_batch(ctxs, mode), ctxs)
    J_str = [final_J(c, R)[1] for c, R in zip(ctxs, seqs)]
    out = {"sequences": len(specs), "frames": frames, "pixel_frames": pixel_frames,
           "sizes": "frame counts 20-300, 128^2-512^2 (first %d of 64 seeded draws)" % len(specs),
           "levels": [L, Q], "generation_s": gen_s,
           "sequential_frames_per_s": frames / t_seq, "streams_frames_per_s": frames / t_str,
           "persistent_frames_per_s": frames / t_per,
           "persistent_over_sequential": t_seq / t_per, "persistent_over_streams": t_str / t_per,
           "streams_over_sequential": t_seq / t_str,
           "persistent_final_J_rel_diff": [a / b - 1.0 for a, b in zip(J_per, J_seq)],
           "streams_final_J_max_rel_diff": max(abs(a / b - 1.0) for a, b in zip(J_str, J_seq)),
           "persistent_stages": [r for r in rep if "steps" in r],
           "timing": "host wall clock around load + pyramid + registration of all sequences, "
                     "device-resident frames, after one warm-up round"}
    if with_combined and os.path.exists(WEIGHTS):
        # combined: streams + BF16 image storage + learned predictor, against
        # the plain form (sequential, FP32, classical predictors) at equal
        # final objective: both are run again to a common target per sequence,
        # the higher of their two natural final objectives (on the FP32
        # frames), which each reaches on its own path.  The combined form
        # solves on BF16 frames, so its target is shifted by the BF16 - FP32
        # objective difference measured at its own natural result.
        params = np.fromfile(WEIGHTS, dtype=np.float32)
        cprm = lambda **kw: S.stml_default_params(n_levels=L, n_tlevels=Q, image_dtype=2, pcg_cooperative=0, **kw)
        comb = [S.Context(cprm(), st) for st in streams]
        nets = [S.Net(params, max_batch=32, max_h=256, max_w=256, stream=st) for st in streams]
        for c, net in zip(comb, nets):
            S.stml_set_predictor_net(c, net)
        t_comb = timed(lambda: S.stml_register_batch(comb, mode), comb)
        J_comb, offset = [], []
        for c, cf, R in zip(ctxs, comb, seqs):
            y, Jb = final_J(cf, R)
            Jf = float(S.stml_eval(c.ptr, L - 1, list(range(int(R.shape[0]))), y)[0])
            J_comb.append(Jf)
            offset.append(Jb - Jf)
        target = [max(a, b) for a, b in zip(J_seq, J_comb)]
        for c, t in zip(ctxs, target):
            S.stml_set_params(c.ptr, S.stml_default_params(n_levels=L, n_tlevels=Q, target_J=t))
        t_seq_T = timed(lambda: [S.stml_register(c.ptr, mode) for c in ctxs], ctxs)
        J_seq_T = [final_J(c, R)[1] for c, R in zip(ctxs, seqs)]
        def comb_fp32():
            out_J = []
            for c, cf, R in zip(ctxs, comb, seqs):
                y, _ = final_J(cf, R)
                out_J.append(float(S.stml_eval(c.ptr, L - 1, list(range(int(R.shape[0]))), y)[0]))
            return out_J

        # calibration (untimed): land on target + offset, then correct the BF16
        # target by how far the FP32 objective of the landed point missed
        for c, t, o in zip(comb, target, offset):
            S.stml_set_params(c.ptr, cprm(target_J=t + o))
        load_all(comb)
        S.stml_register_batch(comb, mode)
        miss = [a - t for a, t in zip(comb_fp32(), target)]
        for c, t, o, e in zip(comb, target, offset, miss):
            S.stml_set_params(c.ptr, cprm(target_J=t + o - e))
        t_comb_T = timed(lambda: S.stml_register_batch(comb, mode), comb)
        J_comb_T = comb_fp32()
        for c in comb:
            c.close()
        for net in nets:
            net.close()
        rel = [a / b - 1.0 for a, b in zip(J_comb_T, J_seq_T)]
        out["combined"] = {
            "form": "stml_register_batch (streams) + BF16 image storage + learned predictor",
            "natural": {"frames_per_s": frames / t_comb, "over_sequential": t_seq / t_comb,
                        "final_J_rel_diff": [a / b - 1.0 for a, b in zip(J_comb, J_seq)]},
            "equal_objective": {
                "how": "both forms run to a common target per sequence: the higher of their natural final "
                       "objectives over all frames on the FP32 frames (regula falsi landing within 1e-5); the "
                       "combined form lands on its BF16 frames, its target shifted by the BF16 - FP32 objective "
                       "difference at its natural result and corrected once by an untimed calibration run",
                "plain_frames_per_s": frames / t_seq_T, "combined_frames_per_s": frames / t_comb_T,
                "combined_over_plain": t_seq_T / t_comb_T,
                "final_J_rel_diff": rel, "within_1e-4": sum(abs(r) <= 1e-4 for r in rel), "of": len(rel),
                "max_abs_rel_diff": max(abs(r) for r in rel)}}
    for c in ctxs:
        c.close()
    torch.cuda.synchronize()
    raw.close()
    return out


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2001_06613_gb300", "weights",
                       "predictor_500x100x256.f32")


def net_train_flops(B: int, H: int, W: int):
    """(algorithmic, executed) FLOPs of one training step of the predictor
    network on B canvases of H x W: forward, input gradient (not of the first
    layer) and weight gradient of every 3x3 convolution, 2 FLOPs per MAC; the
    executed count has the first layer's 7 input channels padded to 32."""
    convs = [(0, 7, 32), (0, 32, 32), (1, 32, 64), (1, 64, 64), (2, 64, 96), (2, 96, 96), (3, 96, 128),
             (3, 128, 128), (2, 224, 96), (2, 96, 96), (1, 160, 64), (1, 64, 64), (0, 96, 32), (0, 32, 32)]
    alg = exe = 0.0
    for i, (lv, ci, co) in enumerate(convs):
        P = B * (H >> lv) * (W >> lv)
        passes = 2 if i == 0 else 3
        alg += 2.0 * P * 9 * ci * co * passes
        exe += 2.0 * P * 9 * (32 if i == 0 else ci) * co * passes
    return alg, exe


def run_learned(S, torch, dev, peaks):
    """The learned temporal predictor: training throughput of its kernels and
    what the trained network (500 sequences of 100 frames of 256^2, committed
    weights) changes in STML registration on held-out 16-frame 64^2 sequences
    and on the paper-scale sequence."""
    from paper_2001_06613_gb300 import predictor_training as PT
    from paper_2001_06613_gb300 import synthetic
    params = np.fromfile(WEIGHTS, dtype=np.float32) if os.path.exists(WEIGHTS) else None
    trained = params is not None
    if params is None:
        params = synthetic.net_init_params(1000)
    net = S.Net(params, max_batch=64, max_h=256, max_w=256)
    # training throughput: 32 crops of 64^2 from registered fields of 4 sequences
    prm = S.stml_default_params(n_levels=3, n_tlevels=3)
    data = PT.collect(S, [synthetic.make_sequence(PT.training_spec(5000 + i, 64, 128), device="cuda")
                          for i in range(4)], prm)
    if not trained:
        PT.train(S, net, data, 1500, batch=32, crop=64, lr=5e-4, seed=1)
    rng = np.random.default_rng(7)
    batches = [PT.sample_batch([d for d in data if d.T.shape[1] >= 64], rng, 32, 64) for _ in range(20)]
    # the timed steps train a copy: restore the committed parameters afterwards
    for smp, H, W in batches[:5]:
        S.stml_net_train_step(net, smp, H, W, lr=1e-6, want_loss=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for smp, H, W in batches[5:]:
        S.stml_net_train_step(net, smp, H, W, lr=1e-6, want_loss=False)
    torch.cuda.synchronize()
    step_s = (time.perf_counter() - t0) / 15
    S.stml_net_set_params(net, params)
    alg, exe = net_train_flops(32, 64, 64)
    # forward pass alone (what a registration runs) on 16 canvases of 256^2
    fb, fh = 16, 256
    fld = torch.from_numpy(synthetic.random_field(np.random.default_rng(3), 2 * fb, 2, (fh, fh), amp=2.0)).to(dev)
    img = torch.rand((3, fb, fh, fh), device=dev)
    fout = torch.empty((fb, 2, fh, fh), device=dev)
    fsmp = S.net_samples(fld[:fb].contiguous(), fld[fb:].contiguous(), img[0], img[1], img[2], 1.0, 0.5, out=fout)
    for _ in range(3):
        S.stml_net_forward(net, fsmp, fh, fh)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(10):
        S.stml_net_forward(net, fsmp, fh, fh)
    ev1.record()
    torch.cuda.synchronize()
    fwd_ms = ev0.elapsed_time(ev1) / 10
    convs = [(0, 7, 32), (0, 32, 32), (1, 32, 64), (1, 64, 64), (2, 64, 96), (2, 96, 96), (3, 96, 128),
             (3, 128, 128), (2, 224, 96), (2, 96, 96), (1, 160, 64), (1, 64, 64), (0, 96, 32), (0, 32, 32)]
    fwd_flops = sum(2.0 * fb * (fh >> lv) * (fh >> lv) * 9 * ci * co for lv, ci, co in convs)
    peak = peaks.get("bf16_tflops") if peaks else None
    peak = peak or 1900.0
    tiny = [synthetic.make_sequence(synthetic.spec_tiny(seed=300 + i)) for i in range(8)]
    ev_tiny = PT.compare(S, net, tiny, S.stml_default_params(n_levels=2, n_tlevels=2), repeats=3)
    R, _ = make_sequence("paper-scale")
    ev_paper = PT.compare(S, net, [R], S.stml_default_params(n_levels=4, n_tlevels=3), repeats=2)
    net.close()
    # the same network on a 128 x 128 canvas: the finest 256^2 level keeps the classical predictor
    net128 = S.Net(params, max_batch=64, max_h=128, max_w=128)
    ev_paper128 = PT.compare(S, net128, [R], S.stml_default_params(n_levels=4, n_tlevels=3), repeats=2)
    net128.close()
    return {"weights": "trained: 500 seqs x 100 frames x 256^2, 4000 Adam steps" if trained else
            "untrained fallback (weights file missing): 1500 steps on 4 sequences",
            "train_step_ms": 1e3 * step_s, "train_batch": "32 crops of 64x64",
            "train_tflops_algorithmic": alg / step_s / 1e12, "train_tflops_executed": exe / step_s / 1e12,
            "tensor_roofline": {"bound": "tensor", "achieved": alg / step_s / 1e12, "peak": peak,
                                "unit": "TFLOP/s", "frac": alg / step_s / 1e12 / peak,
                                "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured)" if peaks
                                else "fallback 1.9 PFLOP/s (of fallback)",
                                "note": "whole training step (tcgen05 BF16 convolutions and weight "
                                        "gradients plus the FP32 elementwise and reduction kernels)"},
            "forward": {"batch": "16 canvases of 256x256", "ms": fwd_ms,
                        "tflops_algorithmic": fwd_flops / (fwd_ms / 1e3) / 1e12,
                        "frac_of_bf16_peak": fwd_flops / (fwd_ms / 1e3) / 1e12 / peak,
                        "kernel": "tcgen05 implicit-GEMM 3x3 convolutions on halo tiles (conv3_kernel)"},
            "held_out_16x64x64_2x2": ev_tiny, "paper_scale_200x256x256_4x3": ev_paper,
            "paper_scale_canvas128": ev_paper128}


def run_volume(S, torch, dev, peak_gbs: float):
    """Three-dimensional sequence: 40 volumes of 64x128x128 (depth first; 6
    modes, 4 voxel max, sin(2 pi t / 40)), 3 spatial x 3 temporal levels,
    STML, with the image pyramid and grad T stored in FP32, FP16 and BF16
    (arithmetic in FP32).  Per storage type: frames/s (one warm-up, then the
    mean of two registrations, L2 flushed before each), the Hessian
    product's achieved bandwidth (36 B per voxel-frame, 30 with 16-bit
    grad T) over all its launches and on the finest level, and for the
    16-bit types the final objective on the FP32 volumes and the field
    difference against the FP32 run."""
    from paper_2001_06613_gb300 import synthetic
    spec = synthetic.spec_volume()
    t0 = time.perf_counter()
    R = synthetic.make_sequence(spec, device=dev)
    gen_s = time.perf_counter() - t0
    n, shape, L, Q = spec.n, tuple(spec.shape), 3, 3
    d = len(shape)
    stream = torch.cuda.current_stream(dev)
    R_dev = torch.from_numpy(R).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"workload": f"{n} volumes {shape[0]}x{shape[1]}x{shape[2]} fp32, 6 modes, 4 voxel max, "
                       f"{L} spatial x {Q} temporal levels, STML", "generation_s": gen_s, "runs": {}}
    ctx32 = None
    y32 = None
    J32 = None
    try:
        for name, code in (("f32", 0), ("f16", 1), ("bf16", 2)):
            ctx = S.Context(S.stml_default_params(n_levels=L, n_tlevels=Q, image_dtype=code), stream.cuda_stream)

            def reg():
                S.stml_load_sequence(ctx.ptr, R_dev)
                S.stml_build_pyramid(ctx.ptr)
                return S.stml_register(ctx.ptr, S.MODE_STML)

            reg()
            S.stml_profile_enable(ctx.ptr, 2)
            times = []
            for _ in range(2):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                stats = reg()
                b.record(stream)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
            prof = S.stml_profile_read(ctx.ptr)
            levels = S.stml_profile_report(ctx.ptr)
            S.stml_profile_enable(ctx.ptr, 0)
            y = torch.empty((n, d) + shape, dtype=torch.float32, device=dev)
            S.stml_get_field(ctx.ptr, L - 1, y)
            fin = [r for r in levels if r["kernel"] == "gn_hessian_product" and r["level"] == L - 1]
            gbs = prof["bytes"] / (prof["ms"] / 1e3) / 1e9 if prof["ms"] > 0 else None
            fgbs = fin[0]["bytes"] / (fin[0]["ms"] / 1e3) / 1e9 if fin and fin[0]["ms"] > 0 else None
            row = {"frames_per_s": n / (statistics.mean(times) / 1e3), "ms": times,
                   "hessian_product": {"GB/s": gbs, "frac": gbs / peak_gbs if gbs else None,
                                       "finest_GB/s": fgbs, "finest_frac": fgbs / peak_gbs if fgbs else None,
                                       "bytes_per_voxel_frame": (8.0 + (4.0 if code == 0 else 2.0)) * d,
                                       "launches": prof["launches"]},
                   "gn_iters": sum(s["gn_iters"] for s in stats), "cg_iters": sum(s["cg_iters"] for s in stats)}
            if code == 0:
                ctx32, y32 = ctx, y
                J32 = S.stml_eval(ctx32.ptr, L - 1, list(range(n)), y32)[0]
                row["final_J"] = J32
            else:
                ctx.close()
                J = S.stml_eval(ctx32.ptr, L - 1, list(range(n)), y)[0]
                row["final_J_on_fp32_volumes"] = J
                row["final_J_rel_diff"] = (J - J32) / J32
                row["field_rms_diff_vs_fp32"] = float(torch.sqrt(torch.mean((y - y32) ** 2)).item())
                row["field_max_diff_vs_fp32"] = float(torch.max(torch.abs(y - y32)).item())
            out["runs"][name] = row
    finally:
        if ctx32 is not None:
            ctx32.close()
    return out


def run_ugrid(S, torch, dev, R_dev, n, shape, L, Q, s: int = 1, repeats: int = 2):
    """The paper-scale sequence registered (STML) with the unknowns of every
    level on its image grid coarsened by 2^s (params.u_coarsen): frames/s
    (one warm-up, then the mean of `repeats` registrations, L2 flushed before
    each), Gauss-Newton / CG counts and the final objective of that
    discretisation, beside the field-grid size."""
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx = S.Context(S.stml_default_params(n_levels=L, n_tlevels=Q, u_coarsen=s), stream.cuda_stream)
    try:
        def reg():
            S.stml_load_sequence(ctx.ptr, R_dev)
            S.stml_build_pyramid(ctx.ptr)
            return S.stml_register(ctx.ptr, S.MODE_STML)

        reg()
        times = []
        for _ in range(repeats):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            stats = reg()
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        cshape = tuple(m // 2 ** s for m in shape)
        w = torch.empty((n, len(shape)) + cshape, dtype=torch.float32, device=dev)
        S.stml_get_field(ctx.ptr, L - 1, w)
        J = S.stml_eval_ugrid(ctx.ptr, L - 1, list(range(n)), w)[0]
        return {"workload": f"{n} frames {'x'.join(map(str, shape))} fp32, {L} spatial x {Q} temporal levels, "
                            f"STML, unknowns on the image grid coarsened by 2^{s} (finest {'x'.join(map(str, cshape))})",
                "u_coarsen": s, "frames_per_s": n / (statistics.mean(times) / 1e3), "ms": times,
                "final_J": J, "gn_iters": sum(t["gn_iters"] for t in stats),
                "cg_iters": sum(t["cg_iters"] for t in stats),
                "note": "J is the coarse-grid objective (S and P on the coarse grid), not comparable with the "
                        "headline's"}
    finally:
        ctx.close()


def run_affine(S, torch, dev, repeats: int = 2):
    """The paper's own setting (Sec. 4): one affine-linear map per frame,
    L-BFGS (Sec. 2), 129 frames with |K_0| = 17, |K_1| = 33 (4 temporal
    levels), STML against SpML on 256^2 OCT-like frames under a planted
    affine motion (4 spatial levels), with the stopping rule eq. (3) at the
    default eps = 1e-3 and at 1e-2: frames/s, L-BFGS iterations, whether
    eq. (3) ended levels early, and the final objective (finest level, all
    frames)."""
    from paper_2001_06613_gb300 import synthetic
    n, shape = 129, (256, 256)
    spec = synthetic.SequenceSpec(n=n, shape=shape, n_modes=8, amp=0.0, periods=[(37.0, 0.0)],
                                  noise_sd=0.02, seed=11)
    R = torch.from_numpy(synthetic.make_affine_sequence(spec, rot_deg=2.0, scale=0.02, shift=3.0)).to(dev)
    out = {"workload": f"{n} frames {shape[0]}x{shape[1]} fp32, planted affine motion (2 deg, 2 %, 3 px), "
                       "4 spatial x 4 temporal levels (|K_0| = 17, |K_1| = 33, |K_2| = 65)",
           "transform": "affine, L-BFGS (m = 5)"}
    for name, mode, eps in (("stml", S.MODE_STML, 1e-3), ("stml_eps1e-2", S.MODE_STML, 1e-2),
                            ("spml", S.MODE_SPML, 1e-3)):
        ctx = S.Context(S.stml_default_params(n_levels=4, n_tlevels=4, transform=1, eps_stop=eps))
        S.stml_load_sequence(ctx.ptr, R)
        S.stml_build_pyramid(ctx.ptr)
        S.stml_register(ctx.ptr, mode)                    # warm-up (allocations)
        best, stats = float("inf"), None
        for _ in range(repeats):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            stats = S.stml_register(ctx.ptr, mode)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        y = torch.empty((n, 2) + shape, device=dev)
        S.stml_get_field(ctx.ptr, 3, y)
        J = float(S.stml_eval(ctx.ptr, 3, list(range(n)), y)[0])
        ctx.close()
        out[name] = {"frames_per_s": n / best, "seconds": best, "final_J": J,
                     "lbfgs_iterations": sum(s["gn_iters"] for s in stats), "girs": len(stats),
                     "levels_ended_by_eq3": sum(s["stopped_early"] for s in stats),
                     "per_gir": [(s["level"], s["tlevel"], s["n_frames"], s["gn_iters"]) for s in stats]}
    out["stml_over_spml_speedup"] = out["stml"]["frames_per_s"] / out["spml"]["frames_per_s"]
    out["stml_eps1e-2_over_spml_speedup"] = out["stml_eps1e-2"]["frames_per_s"] / out["spml"]["frames_per_s"]
    # the correlation distance on the same motion with per-frame brightness and contrast changes
    ks = np.arange(n)
    gain = 1.0 + 0.2 * np.sin(2 * np.pi * ks / 29.0)
    offset = 0.1 * np.cos(2 * np.pi * ks / 17.0)
    Rc = torch.from_numpy(synthetic.make_affine_sequence(spec, rot_deg=2.0, scale=0.02, shift=3.0,
                                                         gain=gain, offset=offset)).to(dev)
    for name, mode in (("nc_stml", S.MODE_STML), ("nc_spml", S.MODE_SPML)):
        ctx = S.Context(S.stml_default_params(n_levels=4, n_tlevels=4, transform=1, distance=1, lam=1e-3))
        S.stml_load_sequence(ctx.ptr, Rc)
        S.stml_build_pyramid(ctx.ptr)
        S.stml_register(ctx.ptr, mode)
        best, stats = float("inf"), None
        for _ in range(repeats):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            stats = S.stml_register(ctx.ptr, mode)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        th = S.stml_get_affine(ctx.ptr, n, 2)
        outJ, _ = S.stml_eval_affine(ctx.ptr, 3, list(range(n)), th, want_grad=False)
        ctx.close()
        out[name] = {"frames_per_s": n / best, "seconds": best, "final_J": float(outJ[0]),
                     "final_D_nc": float(outJ[1]), "lbfgs_iterations": sum(s["gn_iters"] for s in stats),
                     "girs": len(stats), "levels_ended_by_eq3": sum(s["stopped_early"] for s in stats)}
    out["nc_workload"] = ("the same frames with per-frame gain 1 + 0.2 sin(2 pi k / 29) and offset "
                          "0.1 cos(2 pi k / 17), normalised-correlation distance, lambda = 1e-3")
    out["paper_speedup"] = "2.5x on average (Sec. 4, Table 1; 4D-OCT data, affine L-BFGS, CPU MATLAB/FAIR)"
    return out


# ----------------------------------------------------------------- GPU arm
def run_native(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2001_06613_gb300 as S
    S.load()

    n, shape, L, Q, _ = WORKLOADS[args.workload]
    R, spec = make_sequence(args.workload, seed_offset=rank)
    mode = S.MODE_STML if args.mode == "stml" else S.MODE_SPML
    prm = S.stml_default_params(n_levels=L, n_tlevels=Q,
                                image_dtype={"f32": 0, "f16": 1, "bf16": 2}[args.image_dtype],
                                autotune=int(args.autotune))
    stream = torch.cuda.current_stream(dev)
    ctx = S.Context(prm, stream.cuda_stream)
    R_dev = torch.from_numpy(R).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2

    def step():
        S.stml_load_sequence(ctx.ptr, R_dev)          # device-to-device: inputs already in HBM
        S.stml_build_pyramid(ctx.ptr)
        return S.stml_register(ctx.ptr, mode)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = S.stml_launch_count()
    S.stml_profile_enable(ctx.ptr, 2)          # events around the Hessian-product launches only
    stats = None
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        for i in range(args.steps):
            flush.zero_()                                 # evict the previous step from L2
            ev[i][0].record(stream)
            stats = step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = S.stml_launch_count() - launches0
    prof = S.stml_profile_read(ctx.ptr)
    hess_levels = S.stml_profile_report(ctx.ptr)   # timed region, Hessian product per level
    S.stml_profile_enable(ctx.ptr, 1)          # one more (untimed) step with every launch timed
    step()
    table = S.stml_profile_report(ctx.ptr)
    S.stml_profile_enable(ctx.ptr, 0)
    tuning = S.stml_tuning_report(ctx.ptr) if args.autotune else None
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    ms_total = max_over_ranks(sum(ms_steps), world, dev)
    frames_all = sum_over_ranks(float(n * args.steps), world, dev)
    value = frames_all / (ms_total / 1e3)

    # final objective over all frames on the finest level
    y = torch.empty((n, len(shape)) + tuple(shape), dtype=torch.float32, device=dev)
    S.stml_get_field(ctx.ptr, L - 1, y)
    outJ = S.stml_eval(ctx.ptr, L - 1, list(range(n)), y)

    # end to end through the public API with host buffers
    R_host = torch.from_numpy(R).pin_memory()
    y_host = torch.empty((n, len(shape)) + tuple(shape), dtype=torch.float32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        S.stml_load_sequence(ctx.ptr, R_host)
        S.stml_build_pyramid(ctx.ptr)
        S.stml_register(ctx.ptr, mode)
        S.stml_get_field(ctx.ptr, L - 1, y_host)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_value = sum_over_ranks(float(n * e2e_steps), world, dev) / e2e_s

    # spatial-only multilevel on the same data (the paper's comparison), each
    # strategy with its own stopping tests, then at equal final objective:
    # STML with target_J = SpML's final objective (its last GIR over all
    # frames stops where J reaches that value, within target_tol)
    spml = None
    if not args.no_spml and mode == S.MODE_STML:
        sp_steps = max(2, min(args.steps, 3))

        def timed_register(m, prm_run):
            S.stml_set_params(ctx.ptr, prm_run)
            t = []
            for _ in range(sp_steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                S.stml_load_sequence(ctx.ptr, R_dev)
                S.stml_build_pyramid(ctx.ptr)
                st = S.stml_register(ctx.ptr, m)
                b.record(stream)
                torch.cuda.synchronize()
                t.append(a.elapsed_time(b))
            S.stml_get_field(ctx.ptr, L - 1, y)
            J = S.stml_eval(ctx.ptr, L - 1, list(range(n)), y)[0]
            return statistics.median(t), J, st

        sp_ms, J_sp, st_sp = timed_register(S.MODE_SPML, prm)
        prm_t = S.stml_default_params(n_levels=L, n_tlevels=Q,
                                      image_dtype={"f32": 0, "f16": 1, "bf16": 2}[args.image_dtype],
                                      autotune=int(args.autotune), target_J=J_sp)
        st_ms, J_st, st_st = timed_register(S.MODE_STML, prm_t)
        S.stml_set_params(ctx.ptr, prm)
        spml_fps = n / (sp_ms / 1e3)
        spml = {"frames_per_s": spml_fps, "final_J": J_sp, "stml_final_J": outJ[0],
                "stml_over_spml_speedup": (value / world) / spml_fps if world else None,
                "note": "each strategy with the same stopping tests (its own final objective)",
                "gn_iters": sum(x["gn_iters"] for x in st_sp),
                "matched": {"target_J": J_sp, "spml_final_J": J_sp, "stml_final_J": J_st,
                            "rel_diff": abs(J_st - J_sp) / abs(J_sp), "spml_ms": sp_ms, "stml_ms": st_ms,
                            "stml_frames_per_s": n / (st_ms / 1e3), "spml_frames_per_s": spml_fps,
                            "stml_over_spml_speedup": sp_ms / st_ms,
                            "stml_last_gir_gn_iters": st_st[-1]["gn_iters"],
                            "how": "STML with target_J = SpML's final objective over all frames on the finest "
                                   "level (the step that crosses it is shortened until |J - target| <= 1e-5 "
                                   "target); median of %d registrations each" % sp_steps},
                "paper_speedup": "2.5x average (Sec. 4, Table 1; hardware not stated)"}

    batch = None
    if not args.no_batch and rank == 0 and world == 1:
        batch = run_batch(S, torch, dev, mode, args.batch_sequences, with_combined=not args.no_learned)
        batch["small_sequences"] = run_batch_small(S, torch, dev, mode)
    learned = None
    if not args.no_learned and rank == 0 and world == 1 and args.mode == "stml":
        learned = run_learned(S, torch, dev, measured_peaks())
    affine = None
    if not args.no_affine and rank == 0 and world == 1:
        affine = run_affine(S, torch, dev)
    volume = None
    if not args.no_volume and rank == 0 and world == 1:
        pk = measured_peaks()
        volume = run_volume(S, torch, dev, pk["hbm_gbs"] if pk else 6800.0)

    ugrid = None
    if not args.no_ugrid and rank == 0 and world == 1 and args.image_dtype == "f32":
        ugrid = run_ugrid(S, torch, dev, R_dev, n, shape, L, Q)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        frames = min(args.cpu_sample_frames, n)
        fps1, dt1 = oracle_sample(R, args.workload, frames, args.mode)
        fpsN, workers, wall, done = oracle_sample_all_cores(args.workload, frames, args.mode)
        host_cores, model = host_cpu()
        cpu = {"value": fpsN, "unit": "frames/s", "cores": workers, "kind": "oracle",
               "sample": f"{workers} chunks of {frames} consecutive frames ({done} of {n}) at full size, same "
                         f"levels, each registered by its own single-threaded numpy FP64 worker process, all at "
                         f"once; {wall:.1f} s wall",
               "host_cores": host_cores, "cpu_model": model,
               "single_core": {"value": fps1, "unit": "frames/s", "cores": 1,
                               "sample": f"first {frames} of {n} frames, one thread; {dt1:.1f} s"},
               "ops": oracle_op_ns(args.workload, frames)}

    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = prof["bytes"] / (prof["ms"] / 1e3) / 1e9 if prof["ms"] > 0 else None
    tpf = matvec_traffic_per_pixel_frame()
    finest = [r for r in hess_levels if r["kernel"] == "gn_hessian_product" and r["level"] == L - 1]
    fin = None
    if finest and finest[0]["ms"] > 0:
        fgbs = finest[0]["bytes"] / (finest[0]["ms"] / 1e3) / 1e9
        fin = {"achieved": fgbs, "frac": fgbs / peak, "launches": finest[0]["launches"],
               "avg_us": 1e3 * finest[0]["ms"] / finest[0]["launches"],
               "bytes_per_launch": finest[0]["bytes"] / finest[0]["launches"]}
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": (tpf * prof["pixel_frames"] / prof["launches"]) if tpf and prof["launches"] else None,
            "kernel": "GN Hessian product (apply_kernel: read v, grad T; write Hv; 24 B per pixel-frame)",
            "algorithmic_bytes_per_launch": prof["bytes"] / max(1, prof["launches"]),
            "launches": prof["launches"], "ms_total": prof["ms"], "finest_level": fin,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s (of fallback)"}
    if cpu:
        # GPU side of each per-operation entry: finest-level device time per
        # pixel-frame from the kernel table (objective + gradient for the
        # oracle's evaluate, which computes both)
        def gpu_ns(kernel):
            rows = [r for r in table if r["kernel"] == kernel and r["level"] == L - 1 and r["pixel_frames"] > 0]
            return 1e6 * sum(r["ms"] for r in rows) / sum(r["pixel_frames"] for r in rows) if rows else None
        per_pf = {"gn_hessian_product": [gpu_ns("gn_hessian_product")],
                  "gradient_pass": [gpu_ns("gradient_pass"), gpu_ns("objective_pass")],
                  "predict_ls_eq2": [gpu_ns("predict_ls_eq2")]}
        for name, op in cpu["ops"].items():
            vals = per_pf.get(name, [None])
            if all(v is not None for v in vals):
                op["gpu_ns_per_pixel_frame"] = sum(vals)
                op["oracle_over_gpu"] = op["oracle_ns_per_pixel_frame"] / op["gpu_ns_per_pixel_frame"]
    per_kernel = {}
    for r in table:
        k = per_kernel.setdefault(r["kernel"], {"launches": 0, "ms": 0.0, "bytes": 0.0})
        k["launches"] += int(r["launches"])
        k["ms"] += r["ms"]
        k["bytes"] += r["bytes"]
    for k in per_kernel.values():
        k["GB/s"] = k["bytes"] / (k["ms"] / 1e3) / 1e9 if k["ms"] > 0 else None
        k["ms_per_step"] = k["ms"]

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": workload_label(args),
                           "n_frames": n, "shape": list(shape), "levels": L, "tlevels": Q,
                           "mode": args.mode, "image_storage": args.image_dtype, "autotune": bool(args.autotune),
                           "l2": "flushed (256 MB write) before every timed step",
                           "parallelism": f"replicas x{world}"},
                "clocks": clk.summary(), "gpu_launches": launches,
                "e2e": {"value": e2e_value, "unit": "frames/s",
                        "h2d_bytes_per_step": int(R.nbytes), "d2h_bytes_per_step": int(y_host.numel() * 4)},
                "roofline": roof, "cpu_baseline": cpu, "final_J": outJ[0], "kernels": per_kernel,
                "kernel_levels": table, "kernel_table_note": "per-kernel times from one extra untimed "
                "registration with CUDA events around every launch",
                "per_step_ms": ms_steps,
                "gir_stats": [{k: s[k] for k in ("level", "tlevel", "n_frames", "gn_iters", "cg_iters",
                                                 "ls_trials", "stopped_early")} for s in stats],
                "spml": spml, "batch": batch, "learned": learned, "affine": affine, "volume": volume,
                "ugrid": ugrid, "tuning": tuning}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
