"""Learned FGMRES stage: data generation with MatExPre, GPU training, evaluation.

The network and its kernels live in the CUDA library (mxp_cnn_*); this module
only drives them:

* pairs: residuals r_k = b - A x_k of the first FGMRES iterates (x_0 = 0) on
  seeded 2D media, and their MatExPre corrections z_k = MatExPre(r_k) computed
  by the library, both scaled to unit root-mean-square;
* crops: 64 x 64 windows of (Re r, Im r, c / c_max) -> (Re z, Im z);
* training: Adam on the mean squared error, on the GPU (mxp_cnn_train_step);
* checkpoint: flat float32 weights (.bin) plus a JSON manifest;
* evaluation: FGMRES with the learned stage (MatExPre as fallback) against plain
  MatExPre on held-out media: outer iterations, inner iterations, wall time,
  true residual.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import inputs as I
from . import native as N

CROP = 64


def _problem(n_interior, npml, seed, prec="c64", ppw=8.0):
    g = I.Grid(2, (n_interior, n_interior), npml)
    c = I.layered_grf(g, seed)
    p = I.paper_params(g, c, ppw=ppw)
    G = N.Problem.from_grid(g, c, p)
    G.set_params(prec=prec, exp_tol=1e-6)
    return g, c, p, G


def generate_pairs(n_interior=512, npml=16, media_seeds=(0, 1, 2, 3), sources=4, iterates=5,
                   seed_base=I.SEED_BASE + 5000):
    """Crops (X [M,3,64,64], T [M,2,64,64]) as float32 numpy arrays."""
    import torch
    xs, ts = [], []
    for ms in media_seeds:
        g, c, p, G = _problem(n_interior, npml, seed_base + ms)
        ny, nx = g.shape
        cmax = float(c.max())
        cfield = (c / cmax).astype(np.float32)
        for ctr in I.random_centers(g, sources, seed=seed_base + 100 + ms):
            b = torch.from_numpy(I.rhs_from_source(I.gaussian_source(g, center=ctr)).ravel()).cuda()
            for k in range(iterates):
                if k == 0:
                    r = b.clone()
                else:
                    x, _ = G.solve(b, rtol=1e-12, maxit=k, check=False)
                    r = b - G.apply_operator(x)
                z, _ = G.apply_matexpre(r)
                rn = (r / r.abs().pow(2).mean().sqrt()).cpu().numpy().reshape(ny, nx)
                zn = (z / z.abs().pow(2).mean().sqrt()).cpu().numpy().reshape(ny, nx)
                for y0 in range(0, ny - CROP + 1, CROP):
                    for x0 in range(0, nx - CROP + 1, CROP):
                        sl = (slice(y0, y0 + CROP), slice(x0, x0 + CROP))
                        xs.append(np.stack([rn[sl].real, rn[sl].imag, cfield[sl]]))
                        ts.append(np.stack([zn[sl].real, zn[sl].imag]))
        G.close()
    return np.asarray(xs, dtype=np.float32), np.asarray(ts, dtype=np.float32)


def train(net, X, T, epochs=4, batch=32, lr=1e-3, seed=0, time_budget_s=None):
    """Adam on the GPU; returns the per-epoch mean losses."""
    import torch
    rng = np.random.default_rng(seed)
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    hist = []
    t0 = time.time()
    for ep in range(epochs):
        perm = rng.permutation(len(X))
        losses = []
        for i in range(0, len(perm) - batch + 1, batch):
            idx = torch.from_numpy(perm[i:i + batch]).cuda()
            losses.append(net.train_step(Xd[idx].contiguous(), Td[idx].contiguous(), lr))
        hist.append(float(np.mean(losses)) if losses else float("nan"))
        if time_budget_s is not None and time.time() - t0 > time_budget_s:
            break
    return hist


def save(net, path, info=None):
    theta = net.get_params()
    theta.tofile(path + ".bin")
    manifest = dict(format="float32 flat, layer order W1,b1..W6,b6, W [c_out][c_in][3][3]",
                    layers=[list(l) for l in I.CNN_LAYERS], num_params=int(theta.size),
                    info=info or {})
    with open(path + ".json", "w") as fh:
        json.dump(manifest, fh, indent=1)


def load(net, path):
    theta = np.fromfile(path + ".bin", dtype=np.float32)
    net.set_params(theta)
    return theta


_FP64_SOLUTIONS = {}


def evaluate(net, n_interior=1024, npml=32, seeds=(0,), accept_tol=0.5,
             seed_base=I.SEED_BASE + 6000, rtol=1e-6):
    """FGMRES with and without the learned stage on held-out media, each
    solution's error against the solve with FP64 actions."""
    import torch
    rows = []
    for s in seeds:
        g, c, p, G = _problem(n_interior, npml, seed_base + s)
        b = torch.from_numpy(I.rhs_from_source(I.gaussian_source(g)).ravel()).cuda()
        torch.cuda.synchronize()
        x0, st0 = G.solve(b, rtol=rtol, maxit=200)
        N.attach_cnn(G, net, accept_tol)
        x1, st1 = G.solve(b, rtol=rtol, maxit=200)
        N.attach_cnn(G, None)
        key = (n_interior, npml, seed_base + s, rtol)
        if key not in _FP64_SOLUTIONS:          # one FP64 solve per held-out medium
            prm = G.get_params()
            G.set_params(prec="c128")
            _FP64_SOLUTIONS[key] = G.solve(b, rtol=rtol, maxit=200)[0].cpu()
            G.set_params(prec=prm["prec"])
        x64 = _FP64_SOLUTIONS[key].cuda()
        nrm = float(torch.linalg.vector_norm(x64))
        st0["solution_rel_err_vs_fp64"] = float(torch.linalg.vector_norm(x0 - x64)) / nrm
        st1["solution_rel_err_vs_fp64"] = float(torch.linalg.vector_norm(x1 - x64)) / nrm
        rows.append(dict(seed=s, plain=st0, learned=st1))
        G.close()
    return rows


def _rho(G, v, z):
    """Acceptance ratio of a direction: min_a ||v - a A z|| / ||v||."""
    import torch
    az = G.apply_operator(z)
    vv = float(torch.vdot(v, v).real)
    aa = float(torch.vdot(az, az).real)
    va = torch.vdot(az, v)
    if aa <= 0 or vv <= 0:
        return 1.0
    return float(max(0.0, 1.0 - abs(complex(va)) ** 2 / (aa * vv)) ** 0.5)


def direction_study(net, n_interior=1024, npml=32, seed=0, iterates=5, seed_base=I.SEED_BASE + 6000):
    """The acceptance ratio rho = min_a ||v - a A z|| / ||v|| of MatExPre's
    direction z = MatExPre(v) and of the network's z = net(v), for the first
    FGMRES residual directions v of a held-out problem.  A learned direction is
    kept when rho <= accept_tol; this tells which thresholds MatExPre's own
    directions would pass."""
    import torch
    g, c, p, G = _problem(n_interior, npml, seed_base + seed)
    b = torch.from_numpy(I.rhs_from_source(I.gaussian_source(g)).ravel()).cuda()
    ny, nx = g.shape
    cmax = float(c.max())
    cf = torch.from_numpy((c / cmax).astype(np.float32).reshape(ny, nx)).cuda()
    rows = []
    for k in range(iterates):
        if k == 0:
            r = b.clone()
        else:
            x, _ = G.solve(b, rtol=1e-12, maxit=k, check=False)
            r = b - G.apply_operator(x)
        v = r / torch.linalg.vector_norm(r)
        zm, st = G.apply_matexpre(v)
        vs = v * (v.numel() ** 0.5)                    # unit root-mean-square, as the stage feeds the network
        xin = torch.stack([vs.real.reshape(ny, nx).float(), vs.imag.reshape(ny, nx).float(), cf])[None]
        y = net.forward(xin.contiguous())
        zn = torch.complex(y[0, 0].double(), y[0, 1].double()).reshape(-1).contiguous()
        rows.append(dict(iterate=k, rho_matexpre=_rho(G, v, zm), rho_network=_rho(G, v, zn),
                         matexpre_inner=st["inner_iters"]))
    G.close()
    return rows


def main():
    import argparse
    import torch
    ap = argparse.ArgumentParser(description="train and evaluate the learned FGMRES stage")
    ap.add_argument("--train-size", type=int, default=512)
    ap.add_argument("--media", type=int, default=4)
    ap.add_argument("--sources", type=int, default=4)
    ap.add_argument("--iterates", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--eval-size", type=int, default=1024)
    ap.add_argument("--accept-tol", type=float, nargs="+", default=[0.5])
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default="learned_stage")
    a = ap.parse_args()
    t0 = time.time()
    X, T = generate_pairs(a.train_size, 16, tuple(range(a.media)), a.sources, a.iterates)
    t_gen = time.time() - t0
    print(json.dumps(dict(stage="pairs", crops=int(len(X)), gen_s=t_gen)), flush=True)
    net = N.Cnn(a.batch, CROP, CROP)                  # training instance (batches of crops)
    net.set_params(I.cnn_initial_params(I.SEED_BASE + 7000))
    t0 = time.time()
    hist = train(net, X, T, epochs=a.epochs, batch=a.batch, lr=a.lr)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    print(json.dumps(dict(stage="train", epochs=len(hist), train_s=t_train, loss=hist)), flush=True)
    save(net, a.out, dict(crops=int(len(X)), epochs=len(hist), loss=hist))
    side = a.eval_size + 64
    inf = N.Cnn(1, side, side)                         # inference instance (one full grid)
    inf.set_params(net.get_params())
    print(json.dumps(dict(stage="directions", rows=direction_study(inf, a.eval_size, 32))), flush=True)
    for tol in a.accept_tol:
        rows = evaluate(inf, a.eval_size, 32, (0,), tol)
        print(json.dumps(dict(stage="eval", accept_tol=tol, crops=int(len(X)), eval=rows)), flush=True)


if __name__ == "__main__":
    main()
