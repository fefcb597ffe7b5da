"""Learned temporal predictor on the GPU against the FP64 oracle (oracle/net.py).

The GPU network multiplies BF16 operands with FP32 accumulation.  Each result
is compared with the oracle applying the same BF16 rounding to the convolution
operands and with the plain FP64 oracle.  Through 14 layers the two BF16
networks do not stay bit-close: a rounding that FP32 and FP64 accumulation
take differently changes a value by one BF16 unit, which moves the next
layer's sums across further rounding boundaries, so after a few layers both
differ from each other by about as much as from FP64 (about 1e-2 of the
output's scale).  The tolerances below are set at that level; single layers,
where no such cascade starts, are compared tightly in test_gpu_net_layers.py.
"""
import numpy as np
import pytest

from _util import cuda_lib
from oracle import net as onet
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _params(seed, head_scale=1.0, bias_sd=0.05):
    th = synthetic.net_init_params(seed, head_scale=head_scale)
    rng = np.random.default_rng(seed + 100)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in onet.param_shapes()])
    for (name, _), lo, hi in zip(onet.param_shapes(), offs[:-1], offs[1:]):
        if name.endswith(".b"):                       # non-zero biases exercise the bias paths
            th[lo:hi] = rng.normal(scale=bias_sd, size=hi - lo)
    return th.astype(np.float32)


def _batch(rng, B, H, W, amp=1.5):
    """Smooth-ish fields and OCT-like images; targets near the interpolation."""
    spec = synthetic.spec_custom(B + 2, (H, W), seed=int(rng.integers(1 << 30)), amp=amp)
    R = synthetic.make_sequence(spec)
    f = synthetic.random_field(rng, B + 2, 2, (H, W), amp=amp, rough=0.05)
    yl, yr = f[:B], f[2:B + 2]
    tgt = 0.5 * (yl + yr) + synthetic.random_field(rng, B, 2, (H, W), amp=0.3)
    h = rng.choice([1.0, 2.0, 4.0], size=B)
    wl = rng.choice([0.5, 0.25, 0.75], size=B)
    return dict(y_l=yl, y_r=yr, T_l=R[:B], T_k=R[1:B + 1], T_r=R[2:B + 2], h=h, w_l=wl, target=tgt.astype(np.float32))


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _gpu_samples(S, b, out=None):
    t = {k: _dev(b[k]) for k in ("y_l", "y_r", "T_l", "T_k", "T_r", "target")}
    smp = S.net_samples(t["y_l"], t["y_r"], t["T_l"], t["T_k"], t["T_r"], b["h"], b["w_l"],
                        target=t["target"], out=out)
    return smp, t


def _oracle_args(b):
    return (b["y_l"].astype(np.float64), b["y_r"].astype(np.float64), b["T_l"], b["T_k"], b["T_r"],
            b["h"], b["w_l"])


SHAPES = [(3, 21, 27), (2, 64, 48), (1, 8, 8)]


@pytest.mark.parametrize("B,H,W", SHAPES)
def test_forward_parity(S, B, H, W):
    import torch
    rng = np.random.default_rng(11 + H)
    th = _params(3)
    b = _batch(rng, B, H, W)
    net = S.Net(th, max_batch=4, max_h=64, max_w=64)
    try:
        out = torch.full((B, 2, H, W), float("nan"), device="cuda")
        smp, keep = _gpu_samples(S, b, out=out)
        S.stml_net_forward(net, smp, H, W)
        torch.cuda.synchronize()
        z = out.cpu().numpy().astype(np.float64)
    finally:
        net.close()
    th64 = th.astype(np.float64)
    zq = onet.predict(th64, *_oracle_args(b), q=onet.bf16)
    z64 = onet.predict(th64, *_oracle_args(b))
    base = onet.predict(np.where(np.arange(th.size) >= th.size - 66, 0.0, th64), *_oracle_args(b))
    scale = float(np.abs(z64 - base).max())                 # size of h * delta
    err_q = float(np.abs(z - zq).max()) / scale
    err_64 = float(np.abs(z - z64).max()) / scale
    print(f"\nforward {B}x{H}x{W}: max err / max|h delta|: vs BF16-operand oracle {err_q:.2e}, "
          f"vs FP64 {err_64:.2e}")
    assert np.all(np.isfinite(z))
    assert err_q <= 1e-2
    assert err_64 <= 6e-2


def test_zero_head_is_linear_interpolation(S):
    import torch
    rng = np.random.default_rng(12)
    b = _batch(rng, 3, 24, 40)
    net = S.Net(synthetic.net_init_params(4), max_batch=3, max_h=24, max_w=40)
    try:
        out = torch.empty((3, 2, 24, 40), device="cuda")
        smp, keep = _gpu_samples(S, b, out=out)
        S.stml_net_forward(net, smp, 24, 40)
        z = out.cpu().numpy().astype(np.float64)
    finally:
        net.close()
    w = b["w_l"].reshape(3, 1, 1, 1)
    ref = w * b["y_l"].astype(np.float64) + (1 - w) * b["y_r"].astype(np.float64)
    assert np.abs(z - ref).max() <= 2e-6 * np.abs(ref).max()


@pytest.mark.parametrize("B,H,W", [(2, 21, 27), (2, 32, 32)])
def test_loss_and_gradient_parity(S, B, H, W):
    rng = np.random.default_rng(13 + H)
    th = _params(5)
    b = _batch(rng, B, H, W)
    net = S.Net(th, max_batch=2, max_h=32, max_w=32)
    try:
        smp, keep = _gpu_samples(S, b)
        L, g = S.stml_net_loss_grad(net, smp, H, W)
    finally:
        net.close()
    th64 = th.astype(np.float64)
    Lq, gq = onet.loss_grad(th64, *_oracle_args(b), b["target"], q=onet.bf16)
    L64, g64 = onet.loss_grad(th64, *_oracle_args(b), b["target"])
    assert abs(L - Lq) <= 2e-2 * Lq, (L, Lq)
    assert abs(L - L64) <= 2e-2 * L64, (L, L64)
    g = g.astype(np.float64)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in onet.param_shapes()])
    errs = []
    for (name, _), lo, hi in zip(onet.param_shapes(), offs[:-1], offs[1:]):
        eq = np.linalg.norm(g[lo:hi] - gq[lo:hi]) / np.linalg.norm(gq[lo:hi])
        e64 = np.linalg.norm(g[lo:hi] - g64[lo:hi]) / np.linalg.norm(g64[lo:hi])
        errs.append((name, eq, e64))
    cos = float(g @ g64 / (np.linalg.norm(g) * np.linalg.norm(g64)))
    print(f"\ngradient {B}x{H}x{W}: loss rel err vs BF16-operand oracle {abs(L - Lq) / Lq:.2e}, vs FP64 "
          f"{abs(L - L64) / L64:.2e}; cos vs FP64 {cos:.6f}; per tensor rel L2 err (BF16-operand, FP64): " +
          ", ".join(f"{n} {a:.1e}/{b:.1e}" for n, a, b in errs))
    for name, eq, e64 in errs:
        assert eq <= 6e-2 and e64 <= 1e-1, (name, eq, e64)
    assert cos >= 0.998


def test_adam_step_parity(S):
    """One training step: the update equals the oracle's Adam step taken with the
    oracle's gradient, wherever the gradient's sign is not in doubt."""
    rng = np.random.default_rng(14)
    th = _params(6)
    b = _batch(rng, 2, 16, 24)
    lr = 1e-3
    net = S.Net(th, max_batch=2, max_h=16, max_w=24)
    try:
        smp, keep = _gpu_samples(S, b)
        L = S.stml_net_train_step(net, smp, 16, 24, lr=lr)
        th1 = S.stml_net_get_params(net).astype(np.float64)
    finally:
        net.close()
    th64 = th.astype(np.float64)
    Lq, gq = onet.loss_grad(th64, *_oracle_args(b), b["target"], q=onet.bf16)
    ref, _, _ = onet.adam_step(th64, np.zeros_like(th64), np.zeros_like(th64), gq, 1, lr)
    assert abs(L - Lq) <= 2e-2 * Lq
    d_gpu, d_ref = th1 - th64, ref - th64
    # entries whose gradient is well above the per-tensor BF16 noise (a few
    # percent of the tensor's RMS) have a certain sign: there the step is -lr sign(g)
    sure = np.zeros(th.size, bool)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in onet.param_shapes()])
    for lo, hi in zip(offs[:-1], offs[1:]):
        sure[lo:hi] = np.abs(gq[lo:hi]) > 0.3 * np.sqrt(np.mean(gq[lo:hi] ** 2))
    assert np.abs(d_gpu - d_ref)[sure].max() <= 1e-3 * lr + 1e-7
    assert np.mean(np.abs(d_gpu - d_ref) > 0.1 * lr) < 0.02


def test_training_reduces_the_loss(S):
    rng = np.random.default_rng(15)
    b = _batch(rng, 4, 32, 32)
    net = S.Net(synthetic.net_init_params(7, head_scale=0.1), max_batch=4, max_h=32, max_w=32)
    try:
        smp, keep = _gpu_samples(S, b)
        losses = [S.stml_net_train_step(net, smp, 32, 32, lr=1e-3) for _ in range(40)]
    finally:
        net.close()
    print(f"\ntraining on one batch: loss {losses[0]:.4g} -> {losses[-1]:.4g}")
    assert losses[-1] < 0.5 * losses[0]


def test_bad_batches_are_refused(S):
    import torch
    rng = np.random.default_rng(16)
    b = _batch(rng, 2, 16, 16)
    net = S.Net(synthetic.net_init_params(8), max_batch=2, max_h=16, max_w=16)
    try:
        smp, keep = _gpu_samples(S, b)
        with pytest.raises(S.StmlError):
            S.stml_net_forward(net, smp, 16, 16)          # no `out`
        with pytest.raises(S.StmlError):
            S.stml_net_loss_grad(net, smp, 24, 16)         # larger than the canvas
        smp[0].w_l = 1.5
        with pytest.raises(S.StmlError):
            S.stml_net_loss_grad(net, smp, 16, 16)
    finally:
        net.close()
    with pytest.raises((S.StmlError, ValueError)):
        S.Net(np.zeros(10, np.float32), 1, 8, 8)
    with pytest.raises(S.StmlError):
        S.Net(synthetic.net_init_params(8), 0, 8, 8)
    del torch
