"""Learned temporal predictor: FP64 reference of the convolutional
encoder-decoder, its loss, its gradient and the Adam update.

TEST INFRASTRUCTURE ONLY (like the rest of this package).

What the network does.  The predictors of Sec. 3 (linear interpolation on the
coarsest level, the least-squares predictor of eq. (2) on finer ones) propose
the field of a frame k that the next temporal level adds, from the fields
registered on K_q.  The learned predictor proposes it from the two registered
neighbours l < k < r of k and the three images:

    z_k = h * (base + delta),   base = (w_l y_l + (1 - w_l) y_r) / h,
    delta = N_theta(x0),        x0 = [y_l / h, y_r / h, T_l, T_k, T_r]

with w_l = (r - k) / (r - l) the linear-interpolation weight of the left
neighbour and h the cell width of the level (fields in cells inside the
network, so one network serves every level).  With the head's weights zero
the network returns linear interpolation exactly.  The registration keeps the
proposal only where the objective of eq. (1) at the proposal is lower than at
the classical predictor's (the objective decides).

Architecture (2-D, channels-first arrays (B, C, H, W) here):

    level 0  e0a: conv 7->32,   e0b: conv 32->32          (H,   W)
    level 1  e1a: conv 32->64,  e1b: conv 64->64          (H/2, W/2)  after avg-pool
    level 2  e2a: conv 64->96,  e2b: conv 96->96          (H/4, W/4)
    level 3  ba:  conv 96->128, bb:  conv 128->128        (H/8, W/8)
    decoder  d2a: conv [up(bb), e2b] 224->96, d2b: 96->96
             d1a: conv [up(d2b), e1b] 160->64, d1b: 64->64
             d0a: conv [up(d1b), e0b] 96->32,  d0b: 32->32
    head     1x1 conv 32->2 (no activation)

Every "conv" is a 3x3 cross-correlation with zero padding (same size), bias,
then leaky ReLU with slope 0.1; "avg-pool" is the mean of 2x2 blocks; "up" is
nearest-neighbour upsampling by 2; [a, b] stacks channels.  The network runs
on the image zero-padded to multiples of 8 (H8, W8) and its output is cropped.

Mixed precision.  The GPU network multiplies BF16 operands and accumulates in
FP32.  ``forward``/``loss_grad`` take a rounding function ``q`` applied at the
same operand points: the conv weights, x0, every post-activation output and
pooled map, and every gradient with respect to a conv's pre-activation (the
operand of the weight- and input-gradient products).  With ``q`` the identity
(default) everything is plain FP64.

Parameter vector (the layout of the C interface): for each conv layer in the
order above its weights W[ky][kx][ci][co] (C order) then its bias[co]; then
the head's W[ci][co] (32 x 2) and bias[2].
"""
from __future__ import annotations

from typing import Callable, Dict, List, Sequence, Tuple

import numpy as np

SLOPE = 0.1
IN_CH = 7
OUT_CH = 2
CONVS: List[Tuple[str, int, int]] = [
    ("e0a", 7, 32), ("e0b", 32, 32),
    ("e1a", 32, 64), ("e1b", 64, 64),
    ("e2a", 64, 96), ("e2b", 96, 96),
    ("ba", 96, 128), ("bb", 128, 128),
    ("d2a", 224, 96), ("d2b", 96, 96),
    ("d1a", 160, 64), ("d1b", 64, 64),
    ("d0a", 96, 32), ("d0b", 32, 32),
]
HEAD = ("head", 32, 2)


def _ident(a):
    return a


# ---------------------------------------------------------------------------
# parameter vector
# ---------------------------------------------------------------------------
def param_shapes() -> List[Tuple[str, Tuple[int, ...]]]:
    out = []
    for name, ci, co in CONVS:
        out.append((name + ".W", (3, 3, ci, co)))
        out.append((name + ".b", (co,)))
    out.append(("head.W", (HEAD[1], HEAD[2])))
    out.append(("head.b", (HEAD[2],)))
    return out


def param_count() -> int:
    return int(sum(np.prod(s) for _, s in param_shapes()))


def unflatten(theta: np.ndarray) -> Dict[str, np.ndarray]:
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == param_count()
    out, o = {}, 0
    for name, shape in param_shapes():
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def flatten(p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in param_shapes()])


# ---------------------------------------------------------------------------
# layers and their adjoints
# ---------------------------------------------------------------------------
def leaky(z: np.ndarray) -> np.ndarray:
    return np.where(z > 0, z, SLOPE * z)


def leaky_slope(y: np.ndarray) -> np.ndarray:
    """Derivative of the leaky ReLU, read from its output (same sign as input)."""
    return np.where(y > 0, 1.0, SLOPE)


def conv3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[n, o, y, x] = b[o] + sum_{ky, kx, c} W[ky, kx, c, o] x[n, c, y+ky-1, x+kx-1]
    (zero outside the image)."""
    B, C, H, Wd = x.shape
    xp = np.zeros((B, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((B, W.shape[3], H, Wd)) + b.reshape(1, -1, 1, 1)
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("nchw,co->nohw", xp[:, :, ky:ky + H, kx:kx + Wd], W[ky, kx])
    return out


def conv3_backward(x: np.ndarray, W: np.ndarray, g: np.ndarray):
    """Gradients of <g, conv3(x, W, b)> with respect to x, W and b."""
    B, C, H, Wd = x.shape
    xp = np.zeros((B, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            gW[ky, kx] = np.einsum("nchw,nohw->co", xp[:, :, ky:ky + H, kx:kx + Wd], g)
            gxp[:, :, ky:ky + H, kx:kx + Wd] += np.einsum("nohw,co->nchw", g, W[ky, kx])
    return gxp[:, :, 1:-1, 1:-1], gW, g.sum(axis=(0, 2, 3))


def pool2(x: np.ndarray) -> np.ndarray:
    B, C, H, W = x.shape
    return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def pool2_backward(g: np.ndarray) -> np.ndarray:
    return 0.25 * np.repeat(np.repeat(g, 2, axis=2), 2, axis=3)


def up2(x: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up2_backward(g: np.ndarray) -> np.ndarray:
    B, C, H, W = g.shape
    return g.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def pad8(n: int) -> int:
    return (n + 7) // 8 * 8


def features(y_l, y_r, T_l, T_k, T_r, h, w_l):
    """x0 (B, 7, H8, W8) and base (B, 2, H8, W8), zero outside (H, W).

    y_l, y_r: (B, 2, H, W) fields in the level's physical units; T_*: (B, H, W);
    h, w_l: (B,) cell width and left interpolation weight per sample."""
    y_l = np.asarray(y_l, np.float64)
    B, _, H, W = y_l.shape
    H8, W8 = pad8(H), pad8(W)
    h = np.asarray(h, np.float64).reshape(B, 1, 1, 1)
    w = np.asarray(w_l, np.float64).reshape(B, 1, 1, 1)
    x0 = np.zeros((B, IN_CH, H8, W8))
    base = np.zeros((B, 2, H8, W8))
    x0[:, 0:2, :H, :W] = y_l / h
    x0[:, 2:4, :H, :W] = np.asarray(y_r, np.float64) / h
    x0[:, 4, :H, :W] = T_l
    x0[:, 5, :H, :W] = T_k
    x0[:, 6, :H, :W] = T_r
    base[:, :, :H, :W] = (w * y_l + (1.0 - w) * np.asarray(y_r, np.float64)) / h
    return x0, base


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
_ENC = [("e0a", "e0b"), ("e1a", "e1b"), ("e2a", "e2b"), ("ba", "bb")]
_DEC = [("d2a", "d2b", "e2b"), ("d1a", "d1b", "e1b"), ("d0a", "d0b", "e0b")]


def forward(theta: np.ndarray, x0: np.ndarray, q: Callable = _ident):
    """delta (B, 2, H8, W8) and the activations needed by the backward pass."""
    P = unflatten(theta)
    Wq = {n: q(P[n + ".W"]) for n, _, _ in CONVS}
    act = {}
    inp = {}
    x = q(x0)
    for lvl, (a, b) in enumerate(_ENC):
        if lvl > 0:
            x = q(pool2(x))
        inp[a] = x
        x = q(leaky(conv3(x, Wq[a], P[a + ".b"])))
        act[a] = x
        inp[b] = x
        x = q(leaky(conv3(x, Wq[b], P[b + ".b"])))
        act[b] = x
    for a, b, skip in _DEC:
        x = np.concatenate([up2(x), act[skip]], axis=1)
        inp[a] = x
        x = q(leaky(conv3(x, Wq[a], P[a + ".b"])))
        act[a] = x
        inp[b] = x
        x = q(leaky(conv3(x, Wq[b], P[b + ".b"])))
        act[b] = x
    delta = np.einsum("nchw,co->nohw", x, P["head.W"]) + P["head.b"].reshape(1, -1, 1, 1)
    return delta, dict(act=act, inp=inp, W=Wq, P=P)


def predict(theta: np.ndarray, y_l, y_r, T_l, T_k, T_r, h, w_l, q: Callable = _ident) -> np.ndarray:
    """Proposed fields z (B, 2, H, W) in the level's physical units."""
    x0, base = features(y_l, y_r, T_l, T_k, T_r, h, w_l)
    delta, _ = forward(theta, x0, q)
    H, W = np.asarray(y_l).shape[2:]
    return np.asarray(h, np.float64).reshape(-1, 1, 1, 1) * (base + delta)[:, :, :H, :W]


def loss_grad(theta: np.ndarray, y_l, y_r, T_l, T_k, T_r, h, w_l, target,
              q: Callable = _ident, want_grad: bool = True):
    """Mean squared error in cells over the B x 2 x H x W outputs,
    L = mean((base + delta - target / h)^2), and dL/dtheta (flat)."""
    x0, base = features(y_l, y_r, T_l, T_k, T_r, h, w_l)
    delta, c = forward(theta, x0, q)
    B, _, H, W = np.asarray(target).shape
    hh = np.asarray(h, np.float64).reshape(B, 1, 1, 1)
    e = np.zeros_like(delta)
    e[:, :, :H, :W] = (base + delta)[:, :, :H, :W] - np.asarray(target, np.float64) / hh
    count = B * 2 * H * W
    L = float(np.sum(e * e)) / count
    if not want_grad:
        return L, None
    P, act, inp, Wq = c["P"], c["act"], c["inp"], c["W"]
    G = {}
    gdelta = 2.0 * e / count
    x = act["d0b"]
    G["head.W"] = np.einsum("nchw,nohw->co", x, gdelta)
    G["head.b"] = gdelta.sum(axis=(0, 2, 3))
    gx = np.einsum("nohw,co->nchw", gdelta, P["head.W"])      # dL/d(act d0b)
    pend: Dict[str, np.ndarray] = {}                            # skip gradients waiting

    def conv_back(name, g_out):
        gz = q(g_out * leaky_slope(act[name]))                  # dL/d(pre-activation)
        gi, G[name + ".W"], G[name + ".b"] = conv3_backward(inp[name], Wq[name], gz)
        return gi

    for a, b, skip in reversed(_DEC):
        gx = conv_back(b, gx)
        gx = conv_back(a, gx)
        cu = gx.shape[1] - act[skip].shape[1]
        pend[skip] = gx[:, cu:]
        gx = up2_backward(gx[:, :cu])
    for lvl in reversed(range(len(_ENC))):
        a, b = _ENC[lvl]
        if b in pend:
            gx = gx + pend.pop(b)
        gx = conv_back(b, gx)
        gx = conv_back(a, gx)
        if lvl > 0:
            gx = pool2_backward(gx)
    return L, flatten(G)


# ---------------------------------------------------------------------------
# optimiser
# ---------------------------------------------------------------------------
def adam_step(theta, m, v, g, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) at step t >= 1; returns
    (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
