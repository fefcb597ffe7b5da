"""Single convolutions of the learned predictor's network (stml_net_conv3_block)
against the FP64 oracle's layer functions on the same BF16-rounded operands:
forward (bias, leaky ReLU, BF16 output), input gradient and weight/bias
gradient (FP32 outputs).  One layer starts no rounding cascade, so the only
differences are FP32 against FP64 accumulation (and, forward, the final BF16
rounding): tight tolerances.  Shapes cover every channel count of the network,
ragged pixel tiles, every output-channel tile width, and CTAs that run
several tiles."""
import numpy as np
import pytest

from _util import cuda_lib
from oracle import net as onet

pytestmark = pytest.mark.gpu

CASES = [  # B, H, W, Cin, Cout
    (2, 13, 21, 32, 32),
    (1, 24, 40, 64, 96),
    (3, 9, 7, 96, 128),
    (2, 16, 12, 224, 96),
    (2, 11, 17, 96, 224),
    (1, 8, 8, 160, 64),
    (2, 5, 6, 128, 32),
]


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _nchw(a):
    return np.ascontiguousarray(np.transpose(a, (0, 3, 1, 2)))


def _nhwc(a):
    return np.ascontiguousarray(np.transpose(a, (0, 2, 3, 1)))


def _operands(seed, B, H, W, Cin, Cout):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, H, W, Cin)).astype(np.float32)
    g = rng.normal(size=(B, H, W, Cout)).astype(np.float32)
    Wt = (rng.normal(size=(3, 3, Cin, Cout)) * np.sqrt(2.0 / (9 * Cin))).astype(np.float32)
    b = rng.normal(scale=0.1, size=Cout).astype(np.float32)
    return x, g, Wt, b


# more 16 x 8 tiles than the kernel launches CTAs: each CTA runs a sequence of
# tiles (double-buffered TMEM accumulator, epilogue under the next tile's MMAs;
# resident weights for a single 32-channel chunk, reloaded per chunk otherwise)
BIG = [(8, 128, 128, 32, 32), (8, 128, 124, 96, 64)]


@pytest.mark.parametrize("B,H,W,Cin,Cout", CASES + BIG)
def test_forward(S, B, H, W, Cin, Cout):
    import torch
    x, _, Wt, b = _operands(1, B, H, W, Cin, Cout)
    y = torch.empty((B, H, W, Cout), device="cuda")
    S.stml_net_conv3_block(0, _dev(x), None, _dev(Wt), _dev(b), y)
    got = y.cpu().numpy().astype(np.float64)
    ref = _nhwc(onet.leaky(onet.conv3(_nchw(onet.bf16(x)), onet.bf16(Wt), b.astype(np.float64))))
    # the GPU output is the BF16 rounding of a value within FP32 accumulation error of ref
    err = np.abs(got - ref)
    assert np.all(err <= 2.0 ** -8 * np.abs(ref) + 1e-5 * np.abs(ref).max())
    assert np.mean(got != onet.bf16(ref)) < 2e-3


@pytest.mark.parametrize("B,H,W,Cin,Cout", CASES + BIG)
def test_input_gradient(S, B, H, W, Cin, Cout):
    import torch
    x, g, Wt, b = _operands(2, B, H, W, Cin, Cout)
    y = torch.empty((B, H, W, Cin), device="cuda")
    S.stml_net_conv3_block(1, _dev(g), None, _dev(Wt), _dev(b), y)
    got = y.cpu().numpy().astype(np.float64)
    gx, _, _ = onet.conv3_backward(_nchw(x), onet.bf16(Wt), _nchw(onet.bf16(g)))
    ref = _nhwc(gx)
    assert np.abs(got - ref).max() <= 5e-5 * np.abs(ref).max()


@pytest.mark.parametrize("B,H,W,Cin,Cout", CASES)
def test_weight_gradient(S, B, H, W, Cin, Cout):
    import torch
    x, g, Wt, b = _operands(3, B, H, W, Cin, Cout)
    y = torch.empty(9 * Cin * Cout + Cout, device="cuda")
    S.stml_net_conv3_block(2, _dev(g), _dev(x), _dev(Wt), _dev(b), y)
    got = y.cpu().numpy().astype(np.float64)
    _, gW, gb = onet.conv3_backward(_nchw(onet.bf16(x)), onet.bf16(Wt), _nchw(onet.bf16(g)))
    assert np.abs(got[:-Cout] - gW.ravel()).max() <= 5e-5 * np.abs(gW).max()
    assert np.abs(got[-Cout:] - gb).max() <= 5e-5 * np.abs(gb).max()


def test_bad_arguments_are_refused(S):
    import torch
    x = torch.zeros((1, 4, 4, 48), device="cuda")
    Wt = torch.zeros((3, 3, 48, 32), device="cuda")
    b = torch.zeros(32, device="cuda")
    y = torch.zeros((1, 4, 4, 32), device="cuda")
    with pytest.raises(S.StmlError):
        S.stml_net_conv3_block(0, x, None, Wt, b, y)          # 48 channels: not a multiple of 32
