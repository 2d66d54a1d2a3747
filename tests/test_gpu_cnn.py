"""Learned stage on the GPU: the tensor-core (tcgen05) forward convolutions and
input gradients and the weight-gradient kernels against the fp64 CNN oracle
(same bfloat16-rounded weights; the oracle rounds every tensor-core operand to
bfloat16 as the kernels do: the convolution inputs in the forward pass and
the incoming gradients of the input gradients), training reduces the loss,
and the learned FGMRES stage keeps the solve correct with MatExPre as
fallback."""
import numpy as np
import pytest

from oracle import cnn as C
import oracle
from paper_2506_03617_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03617_gb300 import native as N
    N.load()
    return N


def _bf16(theta):
    """Weights as the kernels see them (bfloat16), biases kept in float32."""
    out = np.array(theta, dtype=np.float64)
    k = 0
    for ci, co, _, _, _ in C.LAYERS:
        nw = ci * co * 9
        out[k:k + nw] = torch.from_numpy(np.asarray(theta[k:k + nw], np.float32)).to(
            torch.bfloat16).to(torch.float64).numpy()
        k += nw + co
    return out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _log(what, a, b):
    """Measured errors behind the bounds (appended to MXP_PARITY_LOG when set)."""
    import json
    import os
    path = os.environ.get("MXP_PARITY_LOG")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps({"what": what, "l2_or_weight": float(a), "max_or_bias": float(b)}) + "\n")


def test_forward_and_backward_match_the_oracle(native):
    rng = np.random.default_rng(1)
    theta = I.cnn_initial_params(3) + (0.02 * rng.standard_normal(C.num_params())).astype(np.float32)
    # biases nonzero so they are exercised
    net = native.Cnn(2, 40, 48)
    net.set_params(theta)
    x = rng.standard_normal((2, 3, 40, 48)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    y = net.forward(xd).cpu().numpy()
    th = _bf16(theta)
    y_ref, cache = C.forward(th, x.astype(np.float64), round_operands=True)
    # Same bfloat16 operands on both sides, but a float32 activation and its
    # float64 counterpart now and then round to different bfloat16 neighbours;
    # each such flip perturbs the next layer's sums enough to cause more flips, so
    # over six layers the network outputs differ by far more than float32
    # accumulation (each convolution alone agrees within 1e-5: test_gpu_conv_tc).
    # Measured on GB300: 4.8e-4 (l2), 2.1e-3 (max).
    e_fwd = (_rel(y, y_ref), np.max(np.abs(y - y_ref)) / np.max(np.abs(y_ref)))
    _log("cnn forward", *e_fwd)
    assert e_fwd[0] < 2e-3 and e_fwd[1] < 1e-2, e_fwd
    gy = rng.standard_normal(y.shape).astype(np.float32)
    g = net.backward(xd, torch.from_numpy(gy).cuda()).cpu().numpy()
    g_ref, _ = C.backward(th, cache, gy.astype(np.float64), round_operands=True)
    # per layer (weights and biases separately)
    k = 0
    for li, (ci, co, _, _, _) in enumerate(C.LAYERS):
        nw = ci * co * 9
        ew, eb = _rel(g[k:k + nw], g_ref[k:k + nw]), _rel(g[k + nw:k + nw + co], g_ref[k + nw:k + nw + co])
        _log(f"cnn layer {li + 1} weight / bias gradient", ew, eb)
        # the same flips run back through the five input gradients (measured on
        # GB300: at most 1.3e-2 for a weight and 1.5e-2 for a bias gradient)
        assert ew < 4e-2 and eb < 4e-2, (li, ew, eb)
        k += nw + co


def test_training_reduces_the_loss_on_a_fixed_batch(native):
    rng = np.random.default_rng(2)
    net = native.Cnn(8, 32, 32)
    net.set_params(I.cnn_initial_params(4))
    x = torch.from_numpy(rng.standard_normal((8, 3, 32, 32)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((8, 2, 32, 32)).astype(np.float32)).cuda()
    losses = [net.train_step(x, t, 1e-3) for _ in range(60)]
    assert losses[-1] < 0.7 * losses[0]


def test_learned_stage_in_fgmres_keeps_the_solve_correct(native):
    from paper_2506_03617_gb300 import learned as L
    X, T = L.generate_pairs(n_interior=112, npml=8, media_seeds=(0,), sources=2, iterates=3)
    assert X.shape[1:] == (3, 64, 64) and len(X) > 0
    tr = native.Cnn(16, 64, 64)
    tr.set_params(I.cnn_initial_params(5))
    hist = L.train(tr, X, T, epochs=3, batch=4)
    assert np.isfinite(hist).all()
    g = I.Grid(2, (112, 112), 8)
    c = I.layered_grf(g, I.SEED_BASE + 6001)
    p = I.paper_params(g, c, ppw=8.0)
    G = native.Problem.from_grid(g, c, p)
    G.set_params(prec="c64", exp_tol=1e-6)
    inf = native.Cnn(1, 128, 128)
    inf.set_params(tr.get_params())
    b = I.rhs_from_source(I.gaussian_source(g)).ravel()
    _, st0 = G.solve(torch.from_numpy(b).cuda(), rtol=1e-6)
    # accept every learned direction: every outer step uses the network and the
    # FGMRES residual can only decrease (it may stall without the fallback)
    native.attach_cnn(G, inf, 1.0)
    x1, st1 = G.solve(torch.from_numpy(b).cuda(), rtol=1e-6, maxit=40, check=False)
    assert st1["nn_accepted"] == st1["outer_iters"] == 40 and st1["nn_rejected"] == 0
    assert st1["true_relres"] <= 1.0
    # default threshold: a learned direction is kept only if it reduces the
    # residual enough, MatExPre otherwise; the solve reaches the tolerance
    native.attach_cnn(G, inf, 0.5)
    x2, st2 = G.solve(torch.from_numpy(b).cuda(), rtol=1e-6)
    assert st2["nn_accepted"] + st2["nn_rejected"] == st2["outer_iters"]
    assert st2["converged"]
    P = oracle.Problem.from_grid(g, c, p)
    xs = x2.cpu().numpy()
    assert np.linalg.norm(b - P.apply(xs)) / np.linalg.norm(b) <= 1.000001e-6
