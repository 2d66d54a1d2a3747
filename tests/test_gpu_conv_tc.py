"""The learned stage's tensor-core convolutions (tcgen05, bfloat16 operands,
float32 accumulation in tensor memory) one at a time, through the C ABI
(mxp_cnn_conv3x3), against the fp64 oracle fed the same bfloat16-rounded
operands: forward (stride 1 and 2, upsampled input, relu, bias), input
gradient and weight gradient, for every layer shape of the network and for
pixel counts that leave a ragged last tile of 128.  With identical operands the
only difference is float32 accumulation: element-wise within 1e-5 of max|ref|.
(A whole-network comparison cannot be this tight: a float32 activation and
its float64 counterpart occasionally round to different bfloat16 neighbours,
and such flips multiply from layer to layer.)"""
import numpy as np
import pytest

from oracle import cnn as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03617_gb300 import native as N
    N.load()
    return N


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# (Cin, Cout, stride, upsample, N, H, W): the network's six layers on a 40 x 48
# image pair, and ragged shapes (pixel counts not multiples of 128)
SHAPES = [(3, 32, 1, 0, 2, 40, 48), (32, 64, 2, 0, 2, 40, 48), (64, 64, 1, 0, 2, 20, 24),
          (64, 32, 1, 1, 2, 20, 24), (32, 2, 1, 0, 2, 40, 48), (5, 17, 1, 0, 1, 7, 9),
          (9, 24, 2, 0, 3, 14, 10)]


def _data(Cin, Cout, N, H, W, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((N, Cin, H, W)).astype(np.float32)
    Wt = torch.from_numpy((rng.standard_normal((Cout, Cin, 3, 3)) / np.sqrt(9 * Cin)).astype(np.float32))
    wb = Wt.to(torch.bfloat16)
    bias = rng.standard_normal(Cout).astype(np.float32)
    return x, wb, wb.to(torch.float64).numpy(), bias


@pytest.mark.parametrize("shape", SHAPES, ids=[str(s) for s in SHAPES])
def test_forward(native, shape):
    Cin, Cout, S, U, N, H, W = shape
    x, wb, W64, bias = _data(Cin, Cout, N, H, W, 1)
    y = native.conv3x3(0, torch.from_numpy(x).cuda(), wb.cuda(), bias=torch.from_numpy(bias).cuda(),
                       stride=S, upsample=U, relu=True).cpu().numpy()
    xin = C.up2(x.astype(np.float64)) if U else x.astype(np.float64)
    ref = np.maximum(C.conv(C.round_bf16(xin), W64, bias.astype(np.float64), stride=S), 0)
    assert y.shape == ref.shape
    assert _maxrel(y, ref) < TOL, _maxrel(y, ref)


@pytest.mark.parametrize("shape", [s for s in SHAPES if not s[3]], ids=[str(s) for s in SHAPES if not s[3]])
def test_input_gradient(native, shape):
    Cin, Cout, S, _, N, H, W = shape
    x, wb, W64, _ = _data(Cin, Cout, N, H, W, 2)
    rng = np.random.default_rng(3)
    g = rng.standard_normal((N, Cout, (H + S - 1) // S, (W + S - 1) // S)).astype(np.float32)
    gin = native.conv3x3(1, torch.from_numpy(g).cuda(), wb.cuda(), stride=S, in_hw=(H, W)).cpu().numpy()
    ref, _, _ = C.conv_backward(x.astype(np.float64), W64, g.astype(np.float64), stride=S,
                                round_operands=True)
    assert gin.shape == ref.shape
    assert _maxrel(gin, ref) < TOL, _maxrel(gin, ref)


@pytest.mark.parametrize("shape", SHAPES, ids=[str(s) for s in SHAPES])
def test_weight_gradient(native, shape):
    Cin, Cout, S, U, N, H, W = shape
    x, wb, W64, _ = _data(Cin, Cout, N, H, W, 4)
    Hl, Wl = (2 * H, 2 * W) if U else (H, W)
    rng = np.random.default_rng(5)
    g = rng.standard_normal((N, Cout, (Hl + S - 1) // S, (Wl + S - 1) // S)).astype(np.float32)
    gw = native.conv3x3(2, torch.from_numpy(x).cuda(), b=torch.from_numpy(g).cuda(), stride=S, upsample=U,
                        cout=Cout).cpu().numpy()
    xin = C.up2(x.astype(np.float64)) if U else x.astype(np.float64)
    _, ref, _ = C.conv_backward(xin, W64, g.astype(np.float64), stride=S, round_operands=True)
    ref = ref.reshape(Cout, Cin * 9)
    assert _maxrel(gw, ref) < TOL, _maxrel(gw, ref)


def test_sizes_are_checked(native):
    x = torch.zeros((1, 3, 8, 8), dtype=torch.float32, device="cuda")
    w = torch.zeros((70, 3, 3, 3), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(native.MxpError):
        native.conv3x3(0, x, w)                                   # Cout > 64
    with pytest.raises(native.MxpError):
        native.conv3x3(1, x, w[:4], stride=3)                     # stride 3
