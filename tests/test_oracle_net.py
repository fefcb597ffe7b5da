"""Pins of the learned predictor's FP64 reference (oracle/net.py) against
things fixed outside it: a textbook cross-correlation, adjoint identities of
every layer, central finite differences of the whole network's loss, the
linear-interpolation predictor (zero head), Adam's closed-form steps and the
BF16 rounding rule."""
import numpy as np
import pytest

from oracle import net, predictor
from paper_2001_06613_gb300 import synthetic


def _batch(rng, B, H, W, amp=1.0):
    yl = amp * rng.normal(size=(B, 2, H, W))
    yr = amp * rng.normal(size=(B, 2, H, W))
    T = rng.random((3, B, H, W))
    return yl, yr, T[0], T[1], T[2]


def test_param_count_is_about_one_million():
    assert net.param_count() == 906274
    assert synthetic.net_init_params(0).size == net.param_count()


def test_conv3_is_the_textbook_cross_correlation():
    from scipy.signal import correlate2d
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 7, 5))
    W = rng.normal(size=(3, 3, 3, 4))
    b = rng.normal(size=4)
    out = net.conv3(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, c], W[:, :, c, o], mode="same") for c in range(3))
            np.testing.assert_allclose(out[n, o], ref, rtol=1e-12, atol=1e-12)


def test_layer_adjoints():
    """<L x, g> = <x, L^T g> for the linear part of every layer."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 3, 8, 6))
    W = rng.normal(size=(3, 3, 3, 5))
    g = rng.normal(size=(2, 5, 8, 6))
    gx, gW, gb = net.conv3_backward(x, W, g)
    lin = float(np.sum(net.conv3(x, W, np.zeros(5)) * g))
    assert abs(lin - float(np.sum(x * gx))) <= 1e-10 * abs(lin)
    assert abs(lin - float(np.sum(W * gW))) <= 1e-10 * abs(lin)
    np.testing.assert_allclose(gb, g.sum(axis=(0, 2, 3)))
    a = rng.normal(size=(2, 3, 4, 3))
    c = rng.normal(size=(2, 3, 8, 6))
    assert np.isclose(np.sum(net.up2(a) * c), np.sum(a * net.up2_backward(c)))
    assert np.isclose(np.sum(net.pool2(c) * a), np.sum(c * net.pool2_backward(a)))
    np.testing.assert_array_equal(net.pool2(net.up2(a)), a)          # pool o up = identity
    np.testing.assert_allclose(net.pool2(np.full((1, 1, 4, 4), 3.0)), 3.0)


def test_leaky_relu_and_its_slope():
    z = np.array([-2.0, -0.5, 0.0, 0.25, 3.0])
    np.testing.assert_array_equal(net.leaky(z), [-0.2, -0.05, 0.0, 0.25, 3.0])
    np.testing.assert_array_equal(net.leaky_slope(net.leaky(z)), [0.1, 0.1, 0.1, 1.0, 1.0])


@pytest.mark.parametrize("shape", [(8, 8), (13, 11)])
def test_gradient_matches_central_differences(shape):
    """Sampled entries of every layer's weights and biases and of the head."""
    rng = np.random.default_rng(3)
    th = synthetic.net_init_params(5, head_scale=1.0).astype(np.float64)
    th += 0.01 * rng.normal(size=th.size)           # non-zero biases too
    B = 2
    H, W = shape
    args = _batch(rng, B, H, W) + ([1.0, 2.0], [0.5, 0.75], rng.normal(size=(B, 2, H, W)))
    L, g = net.loss_grad(th, *args)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in net.param_shapes()])
    for lo, hi in zip(offs[:-1], offs[1:]):
        for i in rng.choice(np.arange(lo, hi), size=min(2, hi - lo), replace=False):
            e = 1e-6 * max(1.0, abs(th[i]))   # small enough to cross no ReLU kink
            tp, tm = th.copy(), th.copy()
            tp[i] += e
            tm[i] -= e
            fd = (net.loss_grad(tp, *args, want_grad=False)[0] -
                  net.loss_grad(tm, *args, want_grad=False)[0]) / (2 * e)
            assert abs(g[i] - fd) <= 1e-5 * abs(fd) + 1e-8 * np.abs(g).max(), (i, g[i], fd)


def test_zero_head_reproduces_linear_interpolation():
    """The untrained network (zero head) proposes exactly the linear predictor of
    Sec. 3 between the two neighbours, at the midpoint and at uneven gaps."""
    rng = np.random.default_rng(4)
    th = synthetic.net_init_params(6).astype(np.float64)
    yl, yr, Tl, Tk, Tr = _batch(rng, 2, 10, 12, amp=2.0)
    K = [0, 4]
    for k in (2, 1, 3):
        wl = (K[1] - k) / (K[1] - K[0])
        z = net.predict(th, yl, yr, Tl, Tk, Tr, [1.0, 4.0], [wl, wl])
        for b in range(2):
            ref = predictor.predict_linear(np.stack([yl[b], yr[b]]), K, [k])[0]
            np.testing.assert_allclose(z[b], ref, rtol=1e-13, atol=1e-13)


def test_adam_closed_forms():
    rng = np.random.default_rng(5)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr = 1e-3
    # step 1: the bias-corrected moments are g and g^2
    t1, m, v = net.adam_step(th, m, v, g, 1, lr)
    np.testing.assert_allclose(t1, th - lr * g / (np.abs(g) + 1e-8), rtol=1e-14)
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
    cur = t1
    for t in range(2, 6):
        nxt, m, v = net.adam_step(cur, m, v, g, t, lr)
        np.testing.assert_allclose(nxt - cur, -lr * g / (np.abs(g) + 1e-8), rtol=1e-10)
        cur = nxt


def test_bf16_round_to_nearest_even():
    e = 2.0 ** -8
    x = np.array([1.0, 1.0 + e, 1.0 + 3 * e, 1.0 + 1.5 * e, -(1.0 + e), 3.0, 2.0 ** -130])
    ref = np.array([1.0, 1.0, 1.0 + 4 * e, 1.0 + 2 * e, -1.0, 3.0, 2.0 ** -130])
    np.testing.assert_array_equal(net.bf16(x), ref)


def test_bf16_operands_change_the_output_by_rounding_only():
    """The BF16-operand network differs from FP64 by a few units of BF16 rounding."""
    rng = np.random.default_rng(6)
    th = synthetic.net_init_params(7, head_scale=1.0).astype(np.float64)
    x0, _ = net.features(*_batch(rng, 1, 16, 16), [1.0], [0.5])
    d64, _ = net.forward(th, x0)
    d16, _ = net.forward(th, x0, q=net.bf16)
    rel = np.abs(d16 - d64).max() / np.abs(d64).max()
    assert 1e-5 < rel < 5e-2
