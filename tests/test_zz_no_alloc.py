"""The allocation-free action mxp_apply_phi_noalloc, for callers that cannot
allocate device memory when they need an exp / psi_1 action (under a host
application's own memory pool, or in loops that cannot afford a synchronising
cudaMalloc).  Called through the C ABI and checked against the problem-handle
entry point mxp_apply_phi (complex128) on two calls in a row, to the 1e-10
relative tolerance of the complex128 parity tests, on a 2D and a 3D grid; the
second call also shows that the shared workspace left by the first does not
leak into the next result."""
import ctypes as ct

import numpy as np
import pytest

from paper_2506_03617_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _noalloc(lib, N, grid_struct, params, c_dev, which, x):
    y = torch.empty_like(x)
    passes = ct.c_int64(0)
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = lib.mxp_apply_phi_noalloc(ct.byref(grid_struct), ct.byref(params),
                                  ct.c_void_p(c_dev.data_ptr()), which,
                                  ct.c_void_p(x.data_ptr()), ct.c_void_p(y.data_ptr()),
                                  stream, ct.byref(passes))
    return s, y, passes.value


@pytest.mark.parametrize("grid", [I.Grid(2, (150, 120), 10), I.Grid(3, (32, 32, 32), 8)],
                         ids=["2d", "3d"])
def test_noalloc_action_matches_problem_entry_point_on_two_calls(grid):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03617_gb300 import native as N
    lib = N.load()
    c = I.layered_grf(grid, seed=I.SEED_BASE + 7, corr_cells=4.0)
    p = I.paper_params(grid, c, ppw=10.0)
    G = N.Problem.from_grid(grid, c, p)
    G.set_params(prec="c128", exp_tol=1e-12)
    params = N.Params()
    assert lib.mxp_get_params(G._h, ct.byref(params)) == 0
    c_dev = torch.from_numpy(np.ascontiguousarray(c.ravel())).cuda()
    for which, seed in [(0, 101), (1, 102)]:
        x = torch.from_numpy(I.random_complex(grid.n_total, seed)).cuda()
        s, y, passes = _noalloc(lib, N, G._grid, params, c_dev, which, x)
        assert s == 0, lib.mxp_last_error()
        assert passes > 0
        ref, ref_passes = G.apply_phi(which, x)
        torch.cuda.synchronize()
        assert passes == ref_passes
        assert _rel(y.cpu().numpy(), ref.cpu().numpy()) < 1e-10


def test_noalloc_rejects_a_non_finite_medium():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03617_gb300 import native as N
    lib = N.load()
    grid = I.Grid(2, (40, 36), 6)
    c = I.homogeneous(grid)
    p = I.paper_params(grid, c, ppw=10.0)
    G = N.Problem.from_grid(grid, c, p)
    params = N.Params()
    assert lib.mxp_get_params(G._h, ct.byref(params)) == 0
    x = torch.from_numpy(I.random_complex(grid.n_total, 5)).cuda()
    for bad in (float("nan"), 0.0, -1.0):
        cb = c.ravel().copy()
        cb[123] = bad
        c_dev = torch.from_numpy(cb).cuda()
        s, _, _ = _noalloc(lib, N, G._grid, params, c_dev, 0, x)
        assert s == 1, bad
        assert b"wave speed" in lib.mxp_last_error()


def test_noalloc_rejects_grids_beyond_its_workspace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03617_gb300 import native as N
    lib = N.load()
    g = N.Grid()
    g.dim = 2
    g.n_interior[0] = 600
    g.n_interior[1] = 600
    g.npml = 8
    g.h = 1.0 / 600
    prm = N.Params()
    assert lib.mxp_default_params(ct.byref(g), 1.0, 10.0, ct.byref(prm)) == 0
    x = torch.zeros(616 * 616, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    c_dev = torch.ones(616 * 616, dtype=torch.float64, device="cuda")
    s = lib.mxp_apply_phi_noalloc(ct.byref(g), ct.byref(prm), ct.c_void_p(c_dev.data_ptr()), 0,
                                  ct.c_void_p(x.data_ptr()), ct.c_void_p(y.data_ptr()), None, None)
    assert s == 1
    assert b"262144" in lib.mxp_last_error()
