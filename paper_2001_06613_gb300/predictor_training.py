"""Training data and training loop of the learned temporal predictor.

The network (include/stml_net.h) learns to propose the field of a frame k
from its registered neighbours l < k < r and the three images.  Its training
pairs come from the registration itself: every sequence is registered (STML,
classical predictors), and at every spatial level the registered fields
y_{l,all} of all frames give inputs (y_l, y_r) and targets y_k for triples
(l, k, r) at the gaps the temporal tree of Sec. 3 makes (r - l = 2, 4, 8 with
k in the middle) and at uneven gaps (1-3 frames on either side of k).

Everything here is host bookkeeping (which frames, which crop); the network's
forward and backward passes and Adam run in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from . import binding as B


@dataclass
class LevelData:
    y: object          # torch CUDA tensor (n, 2, H, W): registered fields y_{l,all}
    T: object          # torch CUDA tensor (n, H, W): images of the level
    h: float


def collect(S, sequences: Sequence[np.ndarray], params, mode: int = B.MODE_STML, stream=None,
            min_size: int = 16) -> List[LevelData]:
    """Registers each (n, H, W) float32 sequence and keeps, per spatial level of
    at least min_size pixels a side, the fields of all frames and the images."""
    import torch
    out = []
    for R in sequences:
        ctx = S.Context(params, stream)
        try:
            S.stml_load_sequence(ctx.ptr, torch.from_numpy(np.ascontiguousarray(R, np.float32)).cuda())
            S.stml_build_pyramid(ctx.ptr)
            S.stml_register(ctx.ptr, mode)
            n = R.shape[0]
            for lvl in range(params.n_levels):
                shape3, h = S.stml_level_info(ctx.ptr, lvl)
                H, W = int(shape3[1]), int(shape3[2])
                if min(H, W) < min_size:
                    continue
                y = torch.empty((n, 2, H, W), device="cuda")
                T = torch.empty((n, H, W), device="cuda")
                S.stml_get_field(ctx.ptr, lvl, y)
                S.stml_get_images(ctx.ptr, lvl, T)
                out.append(LevelData(y, T, float(h)))
        finally:
            ctx.close()
    return out


def _triple(rng, n: int):
    """(l, k, r): symmetric gaps 1, 2, 4 (k mid-way) or uneven ones."""
    if rng.random() < 0.75:
        s = int(rng.choice([1, 2, 4], p=[0.6, 0.3, 0.1]))
        s = min(s, (n - 1) // 2)
        k = int(rng.integers(s, n - s))
        return k - s, k, k + s
    a, b = (int(v) for v in rng.integers(1, 4, size=2))
    if a + b > n - 1:
        a, b = 1, 1
    k = int(rng.integers(a, n - b))
    return k - a, k, k + b


def sample_batch(data: List[LevelData], rng: np.random.Generator, batch: int, crop: int):
    """A batch of `batch` crops from one level (picked in proportion to its
    pixels): (NetSample array, H, W)."""
    sizes = np.array([d.T.shape[1] * d.T.shape[2] * d.T.shape[0] for d in data], dtype=np.float64)
    # crops share one shape: pick a level size first, then sequences of that size
    i0 = int(rng.choice(len(data), p=sizes / sizes.sum()))
    H0, W0 = data[i0].T.shape[1:]
    same = [i for i, d in enumerate(data) if d.T.shape[1:] == (H0, W0)]
    ch, cw = min(crop, H0), min(crop, W0)
    arr = (B.NetSample * batch)()
    for b in range(batch):
        d = data[int(rng.choice(same))]
        n = d.T.shape[0]
        l, k, r = _triple(rng, n)
        y0 = int(rng.integers(0, H0 - ch + 1))
        x0 = int(rng.integers(0, W0 - cw + 1))
        off = y0 * W0 + x0
        fb, ib = 2 * H0 * W0, H0 * W0
        yp, tp = d.y.data_ptr(), d.T.data_ptr()
        s = arr[b]
        s.y_l = yp + 4 * (l * fb + off)
        s.y_r = yp + 4 * (r * fb + off)
        s.target = yp + 4 * (k * fb + off)
        s.T_l = tp + 4 * (l * ib + off)
        s.T_k = tp + 4 * (k * ib + off)
        s.T_r = tp + 4 * (r * ib + off)
        s.out = None
        s.plane, s.ld, s.ld_img = H0 * W0, W0, W0
        s.w_l = (r - k) / (r - l)
        s.h = d.h
    return arr, ch, cw


def train(S, net, data: List[LevelData], steps: int, batch: int = 16, crop: int = 64, lr: float = 1e-3,
          seed: int = 0, log_every: int = 0) -> List[float]:
    """Adam steps on random batches; returns the loss of every logged step."""
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(steps):
        smp, H, W = sample_batch(data, rng, batch, crop)
        want = log_every > 0 and (it % log_every == 0 or it == steps - 1)
        L = S.stml_net_train_step(net, smp, H, W, lr=lr, want_loss=want)
        if want:
            losses.append(float(L))
    return losses


def mean_loss(S, net, data: List[LevelData], batches: int = 8, batch: int = 16, crop: int = 64,
              seed: int = 1) -> float:
    """Mean loss (cells^2) over a fixed set of random batches."""
    rng = np.random.default_rng(seed)
    tot = 0.0
    for _ in range(batches):
        smp, H, W = sample_batch(data, rng, batch, crop)
        L, _ = S.stml_net_loss_grad(net, smp, H, W, want_grad=False)
        tot += L
    return tot / batches


# ------------------------------------------------------------------ recipe
def training_spec(seed: int, frames: int = 100, size: int = 256):
    """Training sequences: size x size OCT-like frames whose motion has the
    kind of the 16-frame evaluation sequences (4 spatial modes, 2 px at most,
    period 16 frames, noise 0.01)."""
    from . import synthetic
    return synthetic.SequenceSpec(n=frames, shape=(size, size), n_modes=4, amp=2.0, periods=[(16.0, 0.0)],
                                  noise_sd=0.01, seed=seed)


def _register_timed(S, R, params, net=None, repeats: int = 3):
    """STML registration of R (n, H, W): best wall time of `repeats`, the
    statistics and the final objective over all frames on the finest level."""
    import time
    import torch
    ctx = S.Context(params)
    try:
        S.stml_load_sequence(ctx.ptr, torch.from_numpy(np.ascontiguousarray(R, np.float32)).cuda())
        S.stml_build_pyramid(ctx.ptr)
        if net is not None:
            S.stml_set_predictor_net(ctx, net)
        best, stats = float("inf"), None
        for _ in range(repeats):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            stats = S.stml_register(ctx.ptr, B.MODE_STML)
            best = min(best, time.perf_counter() - t0)
        n = R.shape[0]
        top = params.n_levels - 1
        y = torch.empty((n, 2) + tuple(R.shape[1:]), device="cuda")
        S.stml_get_field(ctx.ptr, top, y)
        J = float(S.stml_eval(ctx.ptr, top, list(range(n)), y)[0])
    finally:
        ctx.close()
    return best, stats, J


def _with_target(S, params, target: float):
    import ctypes
    p = type(params)()
    ctypes.memmove(ctypes.byref(p), ctypes.byref(params), ctypes.sizeof(params))
    p.target_J = target
    return p


def compare(S, net, sequences, params, repeats: int = 3, equal_objective: bool = True) -> dict:
    """Registration of each sequence with and without the network: frames/s,
    PCG and Gauss-Newton iterations, learned proposals kept, final objective;
    with equal_objective also both runs to a common target per sequence (the
    higher of the two natural final objectives, which each reaches on its own
    path; the last GIR lands on it by regula falsi): frames/s at equal final
    objective."""
    rows = []
    for R in sequences:
        t1, st1, J1 = _register_timed(S, R, params, net, repeats)
        t0, st0, J0 = _register_timed(S, R, params, None, repeats)
        eq = None
        if equal_objective:
            target = max(J0, J1)
            u1, s1, K1 = _register_timed(S, R, _with_target(S, params, target), net, repeats)
            u0, s0, K0 = _register_timed(S, R, _with_target(S, params, target), None, repeats)
            eq = dict(target=target, seconds_learned=u1, seconds_classic=u0, J_learned=K1, J_classic=K0,
                      cg_learned=sum(s["cg_iters"] for s in s1), cg_classic=sum(s["cg_iters"] for s in s0))
        rows.append(dict(eq=eq,
            frames=int(R.shape[0]), seconds_learned=t1, seconds_classic=t0, J_learned=J1, J_classic=J0,
            cg_learned=sum(s["cg_iters"] for s in st1), cg_classic=sum(s["cg_iters"] for s in st0),
            gn_learned=sum(s["gn_iters"] for s in st1), gn_classic=sum(s["gn_iters"] for s in st0),
            kept=sum(1 for s in st1 if s["pred_learned"] == 1) + sum(1 for s in st1 if s["fill_learned"] == 1),
            judged=sum(1 for s in st1 if s["pred_learned"] >= 0) + sum(1 for s in st1 if s["fill_learned"] >= 0),
            decisions=[(s["level"], s["tlevel"], s["pred_learned"]) for s in st1 if s["pred_learned"] >= 0]))
    frames = sum(r["frames"] for r in rows)
    return dict(
        frames_per_s_learned=frames / sum(r["seconds_learned"] for r in rows),
        frames_per_s_classic=frames / sum(r["seconds_classic"] for r in rows),
        cg_learned=sum(r["cg_learned"] for r in rows), cg_classic=sum(r["cg_classic"] for r in rows),
        gn_learned=sum(r["gn_learned"] for r in rows), gn_classic=sum(r["gn_classic"] for r in rows),
        kept=sum(r["kept"] for r in rows), judged=sum(r["judged"] for r in rows),
        decisions_by_level={str(lv): [sum(1 for r in rows for (l, _, d) in r["decisions"] if l == lv and d == 1),
                                      sum(1 for r in rows for (l, _, d) in r["decisions"] if l == lv)]
                            for lv in sorted({l for r in rows for (l, _, _) in r["decisions"]})},
        max_rel_J_change=max(abs(r["J_learned"] - r["J_classic"]) / abs(r["J_classic"]) for r in rows),
        mean_rel_J_change=float(np.mean([(r["J_learned"] - r["J_classic"]) / abs(r["J_classic"]) for r in rows])),
        equal_objective=None if not equal_objective else dict(
            frames_per_s_learned=frames / sum(r["eq"]["seconds_learned"] for r in rows),
            frames_per_s_classic=frames / sum(r["eq"]["seconds_classic"] for r in rows),
            cg_learned=sum(r["eq"]["cg_learned"] for r in rows), cg_classic=sum(r["eq"]["cg_classic"] for r in rows),
            max_rel_J_diff=max(abs(r["eq"]["J_learned"] / r["eq"]["J_classic"] - 1.0) for r in rows),
            how="both runs to a common target per sequence: the higher of the two natural final objectives"))


def main(argv=None):
    """Trains the predictor on fields the registration produces and reports what
    it gains on held-out sequences; writes the parameters (float32) to --out."""
    import argparse
    import json
    import time
    from . import synthetic
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--sequences", type=int, default=500)
    ap.add_argument("--frames", type=int, default=100)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--tlevels", type=int, default=3)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--crop", type=int, default=64)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--held-out", type=int, default=4)
    ap.add_argument("--eval-seqs", type=int, default=8)
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)
    import paper_2001_06613_gb300 as S
    S.load()
    prm = S.stml_default_params(n_levels=a.levels, n_tlevels=a.tlevels)
    t0 = time.perf_counter()
    data = []
    for i in range(a.sequences):
        R = synthetic.make_sequence(training_spec(a.seed + i, a.frames, a.size), device="cuda")
        data += collect(S, [R], prm)
    t_data = time.perf_counter() - t0
    held = []
    for i in range(a.held_out):
        R = synthetic.make_sequence(training_spec(a.seed + 100000 + i, a.frames, a.size), device="cuda")
        held += collect(S, [R], prm)
    net = S.Net(synthetic.net_init_params(a.seed), max_batch=max(a.batch, 64), max_h=a.size, max_w=a.size)
    before = mean_loss(S, net, held, batch=a.batch, crop=a.crop)
    t0 = time.perf_counter()
    losses = train(S, net, data, a.steps, batch=a.batch, crop=a.crop, lr=a.lr, seed=a.seed,
                   log_every=max(1, a.steps // 10))
    import torch
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    after = mean_loss(S, net, held, batch=a.batch, crop=a.crop)
    if a.out:
        S.stml_net_get_params(net).tofile(a.out)
    tiny = [synthetic.make_sequence(synthetic.spec_tiny(seed=a.seed + 200000 + i)) for i in range(a.eval_seqs)]
    res_tiny = compare(S, net, tiny, S.stml_default_params(n_levels=2, n_tlevels=2))
    report = dict(sequences=a.sequences, frames=a.frames, size=a.size, samples_levels=len(data),
                  data_seconds=round(t_data, 1), train_steps=a.steps, train_seconds=round(t_train, 2),
                  train_loss=losses, held_out_loss_interpolation=before, held_out_loss_trained=after,
                  eval_16x64x64=res_tiny)
    print(json.dumps(report))
    net.close()
    return report


if __name__ == "__main__":
    main()
