"""CNN oracle for the learned preconditioning stage -- TEST INFRASTRUCTURE ONLY.

Plain float64 numpy forward and backward passes of the six-layer U-Net-style
network that the learned FGMRES stage uses (the paper has no learned stage;
the network is this project's).  Only the tests may use it.  It shares nothing
with the CUDA kernels: the layer list below is restated here, and weights are
always passed in.

Network (NCHW, 3x3 kernels, zero padding 1):
  a1 = relu(conv(x,  W1, b1))                3 -> 32, stride 1
  a2 = relu(conv(a1, W2, b2, stride 2))     32 -> 64, stride 2
  a3 = relu(conv(a2, W3, b3))               64 -> 64
  a4 = relu(conv(a3, W4, b4))               64 -> 64
  a5 = relu(conv(up2(a4), W5, b5)) + a1     64 -> 32, nearest upsample x2, skip
  y  = conv(a5, W6, b6)                     32 -> 2
conv(x, W, b, s)[n, o, i, j] = b[o] + sum_{c, ky, kx} W[o, c, ky, kx] x[n, c, s i + ky - 1, s j + kx - 1]
Flat parameter order: W1, b1, W2, b2, ..., W6, b6.
Loss: mean squared error over all output elements.
"""
from __future__ import annotations

import numpy as np

LAYERS = [  # (c_in, c_out, stride, upsample_input, relu)
    (3, 32, 1, False, True),
    (32, 64, 2, False, True),
    (64, 64, 1, False, True),
    (64, 64, 1, False, True),
    (64, 32, 1, True, True),
    (32, 2, 1, False, False),
]


def num_params() -> int:
    return sum(ci * co * 9 + co for ci, co, _, _, _ in LAYERS)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, k = [], 0
    for ci, co, _, _, _ in LAYERS:
        W = theta[k:k + co * ci * 9].reshape(co, ci, 3, 3)
        k += co * ci * 9
        b = theta[k:k + co]
        k += co
        out.append((W, b))
    assert k == theta.size
    return out


def conv(x, W, b, stride=1):
    n, c, h, w = x.shape
    ho, wo = h // stride, w // stride
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((n, W.shape[0], ho, wo)) + b[None, :, None, None]
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + stride * ho:stride, kx:kx + stride * wo:stride]
            y += np.einsum("oc,nchw->nohw", W[:, :, ky, kx], patch)
    return y


def conv_backward(x, W, gy, stride=1, round_operands=False):
    """Gradients of sum(gy * conv(x, W, b, stride)) w.r.t. x, W and b.
    round_operands: the input and weight gradients take gy and x rounded to
    bfloat16 (the operand precision of tensor-core contractions); b uses gy
    as is."""
    n, c, h, w = x.shape
    ho, wo = gy.shape[2], gy.shape[3]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    gq = round_bf16(gy) if round_operands else gy
    xq = round_bf16(xp) if round_operands else xp
    for ky in range(3):
        for kx in range(3):
            sl = (slice(None), slice(None), slice(ky, ky + stride * ho, stride),
                  slice(kx, kx + stride * wo, stride))
            gW[:, :, ky, kx] = np.einsum("nohw,nchw->oc", gq, xq[sl])
            gxp[sl] += np.einsum("oc,nohw->nchw", W[:, :, ky, kx], gq)
    return gxp[:, :, 1:-1, 1:-1], gW, gy.sum(axis=(0, 2, 3))


def up2(x):
    return x.repeat(2, axis=2).repeat(2, axis=3)


def up2_backward(g):
    n, c, h, w = g.shape
    return g.reshape(n, c, h // 2, 2, w // 2, 2).sum(axis=(3, 5))


def round_bf16(a):
    """Round to bfloat16 the way a float32 value is (float64 -> float32 -> the
    nearest bfloat16, ties to even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    bits = a32.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, x, round_operands=False):
    """Returns (y, cache).  round_operands: every convolution sees its input
    rounded to bfloat16 (the operand precision of tensor-core convolutions with
    bfloat16 operands and wide accumulation); the cache keeps the unrounded
    activations, which the backward pass uses."""
    P = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    q = round_bf16 if round_operands else (lambda v: v)
    a1 = np.maximum(conv(q(x), *P[0]), 0)
    a2 = np.maximum(conv(q(a1), *P[1], stride=2), 0)
    a3 = np.maximum(conv(q(a2), *P[2]), 0)
    a4 = np.maximum(conv(q(a3), *P[3]), 0)
    u4 = up2(a4)
    r5 = np.maximum(conv(q(u4), *P[4]), 0)
    a5 = r5 + a1
    y = conv(q(a5), *P[5])
    return y, dict(x=x, a1=a1, a2=a2, a3=a3, a4=a4, u4=u4, r5=r5, a5=a5)


def backward(theta, cache, gy, round_operands=False):
    """Gradient of sum(gy * y) w.r.t. the flat parameters and the input.
    round_operands: every input gradient rounds its incoming gradient to
    bfloat16 (see conv_backward)."""
    P = unpack(theta)
    c = cache
    ro = round_operands
    grads = [None] * 6
    g5, gW, gb = conv_backward(c["a5"], P[5][0], gy, round_operands=ro)
    grads[5] = (gW, gb)
    g1_skip = g5
    g = g5 * (c["r5"] > 0)
    gu4, gW, gb = conv_backward(c["u4"], P[4][0], g, round_operands=ro)
    grads[4] = (gW, gb)
    g = up2_backward(gu4) * (c["a4"] > 0)
    g, gW, gb = conv_backward(c["a3"], P[3][0], g, round_operands=ro)
    grads[3] = (gW, gb)
    g = g * (c["a3"] > 0)
    g, gW, gb = conv_backward(c["a2"], P[2][0], g, round_operands=ro)
    grads[2] = (gW, gb)
    g = g * (c["a2"] > 0)
    g, gW, gb = conv_backward(c["a1"], P[1][0], g, stride=2, round_operands=ro)
    grads[1] = (gW, gb)
    g = (g + g1_skip) * (c["a1"] > 0)
    gx, gW, gb = conv_backward(c["x"], P[0][0], g, round_operands=ro)
    grads[0] = (gW, gb)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return flat, gx


def mse(y, target):
    d = y - target
    return float(np.mean(d * d)), 2.0 * d / d.size
