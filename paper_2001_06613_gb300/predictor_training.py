"""Training data and training loop of the learned temporal predictor.

The network (include/stml_net.h) learns to propose the field of a frame k
from its registered neighbours l < k < r and the three images.  Its training
pairs come from the registration itself: every sequence is registered (STML,
classical predictors), and at every spatial level the registered fields
y_{l,all} of all frames give inputs (y_l, y_r) and targets y_k for triples
(l, k, r) at the gaps the temporal tree of Sec. 3 makes (r - l = 2, 4, 8 with
k in the middle) and at uneven gaps (k one frame from l or r).

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
        s = int(rng.choice([1, 2, 4], p=[0.5, 0.3, 0.2]))
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
