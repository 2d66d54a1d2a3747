"""Pins for the CNN oracle of the learned stage: library correlation,
stride-2 subsampling, adjoint identities and finite-difference gradients."""
import numpy as np
import scipy.signal as ss

from oracle import cnn as C
from paper_2506_03617_gb300 import inputs as I


def test_stride1_conv_is_channel_summed_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 7, 9))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = C.conv(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(ss.correlate2d(x[n, c], W[o, c], mode="same") for c in range(3))
            assert np.allclose(y[n, o], ref, atol=1e-12)


def test_stride2_conv_subsamples_the_stride1_conv():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 2, 8, 10))
    W = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    assert np.allclose(C.conv(x, W, b, stride=2), C.conv(x, W, b)[:, :, ::2, ::2])


def test_adjoint_identities():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, 3, 4, 5))
    g = rng.standard_normal((2, 3, 8, 10))
    assert np.isclose(np.sum(C.up2(a) * g), np.sum(a * C.up2_backward(g)))
    for stride in (1, 2):
        x = rng.standard_normal((2, 3, 8, 6))
        W = rng.standard_normal((4, 3, 3, 3))
        y = C.conv(x, W, np.zeros(4), stride)
        gy = rng.standard_normal(y.shape)
        gx, gW, gb = C.conv_backward(x, W, gy, stride)
        assert np.isclose(np.sum(y * gy), np.sum(x * gx))
        assert np.isclose(np.sum(y * gy), np.sum(W * gW))


def test_network_gradients_match_central_differences():
    rng = np.random.default_rng(4)
    theta = I.cnn_initial_params(5).astype(np.float64) + 0.01 * rng.standard_normal(C.num_params())
    x = rng.standard_normal((2, 3, 8, 8))
    y, cache = C.forward(theta, x)
    gy = rng.standard_normal(y.shape)
    g_theta, g_x = C.backward(theta, cache, gy)
    f = lambda th, xx: float(np.sum(C.forward(th, xx)[0] * gy))
    eps = 1e-6
    for k in rng.choice(theta.size, 25, replace=False):
        e = np.zeros_like(theta)
        e[k] = eps
        fd = (f(theta + e, x) - f(theta - e, x)) / (2 * eps)
        assert abs(fd - g_theta[k]) <= 1e-6 * (1 + abs(fd)), (k, fd, g_theta[k])
    for idx in [(0, 0, 3, 4), (1, 2, 7, 0), (0, 1, 0, 0)]:
        e = np.zeros_like(x)
        e[idx] = eps
        fd = (f(theta, x + e) - f(theta, x - e)) / (2 * eps)
        assert abs(fd - g_x[idx]) <= 1e-6 * (1 + abs(fd))


def test_parameter_count_and_layer_list_agree_with_the_input_module():
    assert C.num_params() == I.cnn_initial_params(0).size
    assert [tuple(l) for l in C.LAYERS] == [tuple(l) for l in I.CNN_LAYERS]


def test_bf16_rounding_matches_torch_and_ties_to_even():
    """The oracle's bfloat16 operand rounding equals torch's float32 -> bfloat16
    conversion (round to nearest, ties to even) on random values, and resolves
    the exact halfway cases to the even neighbour."""
    import torch
    rng = np.random.default_rng(9)
    v = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        [0.0, -0.0, 1.0, -3.5]])
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(C.round_bf16(v), ref)
    one = np.float32(1.0).view(np.uint32)
    half_up = np.array([one + 0x8000], dtype=np.uint32).view(np.float32)     # 1 + 2^-8: tie, even is 1
    half_up2 = np.array([one + 0x18000], dtype=np.uint32).view(np.float32)   # tie whose even neighbour is above
    assert C.round_bf16(half_up)[0] == 1.0
    assert C.round_bf16(half_up2)[0] == np.array([one + 0x20000], dtype=np.uint32).view(np.float32)[0]


def test_rounded_operands_change_the_output_by_bf16_rounding_only():
    rng = np.random.default_rng(10)
    theta = rng.standard_normal(C.num_params()) * 0.1
    x = rng.standard_normal((1, 3, 8, 8))
    y, _ = C.forward(theta, x)
    yq, cache = C.forward(theta, x, round_operands=True)
    rel = np.linalg.norm(y - yq) / np.linalg.norm(y)
    assert 0 < rel < 2e-2
    _, c0 = C.forward(theta, x)
    for k in c0:                                      # cached activations differ only through the rounding
        assert c0[k].shape == cache[k].shape
