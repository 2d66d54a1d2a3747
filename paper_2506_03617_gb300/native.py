"""ctypes binding of libmatexpre (C ABI in ``include/matexpre.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Vectors are torch complex128 CUDA tensors (one value per unknown,
x fastest); torch supplies device memory and the current stream.  There is no
CPU fallback: if the library cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

MXP_C128, MXP_C64, MXP_BF16S = 0, 1, 2
PRECISIONS = {"c128": MXP_C128, "c64": MXP_C64, "bf16s": MXP_BF16S}
STATUS = {0: "MXP_OK", 1: "MXP_EINVAL", 2: "MXP_ENOMEM", 3: "MXP_ECUDA", 4: "MXP_ENOCONV",
          5: "MXP_EBREAKDOWN", 6: "MXP_ENAN", 7: "MXP_ETIMEOUT"}


class MxpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("n_interior", ct.c_int64 * 3), ("npml", ct.c_int),
                ("h", ct.c_double)]


class Params(ct.Structure):
    _fields_ = [("omega", ct.c_double), ("c_pml", ct.c_double), ("shift_s", ct.c_double),
                ("t", ct.c_double), ("fprtol", ct.c_double), ("exp_tol", ct.c_double),
                ("inner_restart", ct.c_int), ("inner_maxit", ct.c_int),
                ("inner_fixed", ct.c_int), ("prec", ct.c_int), ("theta_max", ct.c_double),
                ("fuse_k", ct.c_int), ("tile_cfg", ct.c_int), ("persist_cfg", ct.c_int),
                ("precond", ct.c_int), ("neumann_n", ct.c_int)]


class ApplyStats(ct.Structure):
    _fields_ = [("inner_iters", ct.c_int), ("converged", ct.c_int),
                ("inner_relres", ct.c_double), ("stencil_passes", ct.c_int64),
                ("pt_updates", ct.c_int64)]


class SolveOpts(ct.Structure):
    _fields_ = [("rtol", ct.c_double), ("restart", ct.c_int), ("maxit", ct.c_int),
                ("x0_given", ct.c_int)]


class SolveStats(ct.Structure):
    _fields_ = [("outer_iters", ct.c_int), ("inner_iters_total", ct.c_int),
                ("converged", ct.c_int), ("true_relres", ct.c_double),
                ("est_relres", ct.c_double), ("stencil_passes", ct.c_int64),
                ("pt_updates", ct.c_int64), ("seconds", ct.c_double),
                ("nn_accepted", ct.c_int), ("nn_rejected", ct.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# name -> (restype, argtypes); every symbol declared in include/matexpre.h
SIGNATURES = {
    "mxp_create": (ct.c_int, [ct.POINTER(Grid), ct.POINTER(ct.c_double), ct.c_int, ct.c_void_p,
                              ct.POINTER(ct.c_void_p)]),
    "mxp_default_params": (ct.c_int, [ct.POINTER(Grid), ct.c_double, ct.c_double,
                                      ct.POINTER(Params)]),
    "mxp_create_slab": (ct.c_int, [ct.POINTER(Grid), ct.c_int64, ct.c_int64, ct.POINTER(ct.c_double),
                                   ct.POINTER(ct.c_double), ct.c_int, ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "mxp_horner_step": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                   ct.POINTER(ct.c_double), ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                   ct.c_void_p]),
    "mxp_get_plan": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int),
                                ct.POINTER(ct.c_int)]),
    "mxp_vec_mdot": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_int, ct.c_void_p, ct.c_int64,
                                ct.c_int64, ct.POINTER(ct.c_double)]),
    "mxp_vec_combine": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_double), ct.c_void_p, ct.c_int64,
                                   ct.c_int, ct.POINTER(ct.c_double)]),
    "mxp_set_params": (ct.c_int, [ct.c_void_p, ct.POINTER(Params)]),
    "mxp_get_params": (ct.c_int, [ct.c_void_p, ct.POINTER(Params)]),
    "mxp_apply_operator": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p]),
    "mxp_apply_phi": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p,
                                 ct.POINTER(ct.c_int64)]),
    "mxp_apply_matexpre": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                      ct.POINTER(ApplyStats)]),
    "mxp_solve": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.POINTER(SolveOpts),
                             ct.POINTER(SolveStats)]),
    "mxp_solve_host": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.POINTER(SolveOpts),
                                  ct.POINTER(SolveStats)]),
    "mxp_solve_batch": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, ct.c_int,
                                   ct.POINTER(ct.c_int), ct.POINTER(ct.c_void_p),
                                   ct.POINTER(ct.c_void_p), ct.POINTER(SolveOpts),
                                   ct.POINTER(SolveStats)]),
    "mxp_apply_phi_noalloc": (ct.c_int, [ct.POINTER(Grid), ct.POINTER(Params),
                                         ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p,
                                         ct.c_void_p, ct.POINTER(ct.c_int64)]),
    "mxp_num_unknowns": (ct.c_int64, [ct.c_void_p]),
    "mxp_measure_fma_peak": (ct.c_int, [ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]),
    "mxp_cnn_num_params": (ct.c_int64, []),
    "mxp_cnn_create": (ct.c_int, [ct.c_int, ct.c_void_p, ct.c_int, ct.c_int, ct.c_int,
                                  ct.POINTER(ct.c_void_p)]),
    "mxp_cnn_set_params": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_float)]),
    "mxp_cnn_get_params": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_float)]),
    "mxp_cnn_forward": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p,
                                   ct.c_void_p]),
    "mxp_cnn_backward": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "mxp_cnn_train_step": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p,
                                      ct.c_void_p, ct.c_float, ct.POINTER(ct.c_float)]),
    "mxp_cnn_destroy": (None, [ct.c_void_p]),
    "mxp_attach_cnn": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_double]),
    "mxp_cnn_conv3x3": (ct.c_int, [ct.c_int] * 10 + [ct.c_void_p] * 4 + [ct.c_int, ct.c_void_p, ct.c_void_p]),
    "mxp_selftest_barrier_timeout": (ct.c_int, [ct.c_void_p]),
    "mxp_kernel_launch_count": (ct.c_int64, []),
    "mxp_num_tile_configs": (ct.c_int, []),
    "mxp_num_persist_configs": (ct.c_int, []),
    "mxp_tile_config": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int)]),
    "mxp_persist_config": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int)]),
    "mxp_persist_geometry": (ct.c_int, [ct.c_void_p] + [ct.POINTER(ct.c_int)] * 5),
    "mxp_set_boundary": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int)]),
    "mxp_get_boundary": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int)]),
    "mxp_sweep_kernel": (ct.c_int, [ct.c_void_p]),
    "mxp_taylor_plan": (ct.c_int, [ct.c_double, ct.c_double, ct.c_double, ct.c_int,
                                   ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "mxp_persist_tile_plan": (ct.c_int, [ct.c_int] * 6 + [ct.POINTER(ct.c_int)] * 4),
    "mxp_destroy": (None, [ct.c_void_p]),
    "mxp_status_string": (ct.c_char_p, [ct.c_int]),
    "mxp_last_error": (ct.c_char_p, []),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmatexpre (building it first if absent).  Raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libmatexpre not found at {path}; run build() first")
            lib = ct.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status):
    if status != 0:
        msg = load().mxp_last_error()
        raise MxpError(status, msg.decode() if msg else "")


def _ptr(t):
    import torch
    if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
        raise ValueError("vectors must be contiguous complex128 CUDA tensors")
    return ct.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ct.c_void_p(stream.cuda_stream)


class Problem:
    """A Helmholtz problem on one GPU: grid, medium c(x) and method parameters."""

    def __init__(self, dim, n_interior, npml, c, h=None, device=0, stream=None, params=None):
        import torch
        self._lib = load()
        self.dim = int(dim)
        ni = [int(v) for v in n_interior]
        self.n_interior = tuple(ni)
        self.npml = int(npml)
        self.h = float(h) if h is not None else 1.0 / max(ni)
        self.n = tuple(m + 2 * self.npml for m in ni)
        self.n_total = int(np.prod(self.n))
        self.device = int(device)
        g = Grid()
        g.dim = self.dim
        for d in range(3):
            g.n_interior[d] = ni[d] if d < self.dim else 1
        g.npml = self.npml
        g.h = self.h
        self._grid = g
        c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1))
        if c.size != self.n_total:
            raise ValueError(f"medium has {c.size} values, grid has {self.n_total}")
        self.cmin = float(c.min())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h_out = ct.c_void_p()
        _check(self._lib.mxp_create(ct.byref(g), c.ctypes.data_as(ct.POINTER(ct.c_double)),
                                    self.device, _stream_handle(self.stream), ct.byref(h_out)))
        self._h = h_out
        if params is not None:
            self.set_params(**params)

    @classmethod
    def slab(cls, grid, row0, nrows, c_slab, c_range, params=None, device=0, stream=None):
        """The problem on rows [row0, row0 + nrows) of the last axis of `grid`
        (mxp_create_slab); c_slab: the wave speed of those rows; c_range: (min,
        max) of c over the whole grid."""
        import torch
        self = cls.__new__(cls)
        self._lib = load()
        self.dim = grid.dim
        self.n_interior = tuple(grid.ni)
        self.npml = grid.npml
        self.h = grid.h
        n = list(grid.n)
        n[-1] = int(nrows)
        self.n = tuple(n)
        self.n_total = int(np.prod(self.n))
        self.device = int(device)
        g = Grid()
        g.dim = grid.dim
        for d in range(3):
            g.n_interior[d] = grid.ni[d] if d < grid.dim else 1
        g.npml = grid.npml
        g.h = grid.h
        self._grid = g
        c = np.ascontiguousarray(np.asarray(c_slab, dtype=np.float64).reshape(-1))
        if c.size != self.n_total:
            raise ValueError(f"slab medium has {c.size} values, the slab has {self.n_total}")
        self.cmin = float(c_range[0])
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        rng = (ct.c_double * 2)(float(c_range[0]), float(c_range[1]))
        h_out = ct.c_void_p()
        _check(self._lib.mxp_create_slab(ct.byref(g), int(row0), int(nrows),
                                         c.ctypes.data_as(ct.POINTER(ct.c_double)), rng, self.device,
                                         _stream_handle(self.stream), ct.byref(h_out)))
        self._h = h_out
        if params is not None:
            self.set_params(omega=params.omega, shift_s=params.shift, t=params.t, c_pml=params.cpml,
                            fprtol=params.fprtol)
        return self

    def horner_step(self, sigma, p, y=None, v=None, gamma=0j, rho=1 + 0j, out=None):
        """out = rho (y + sigma (A_s - mu) p + gamma v) (mxp_horner_step)."""
        o = self.empty() if out is None else out
        c2 = lambda z: (ct.c_double * 2)(complex(z).real, complex(z).imag)
        _check(self._lib.mxp_horner_step(self._h, c2(sigma), c2(gamma), c2(rho), _ptr(p),
                                         _ptr(y) if y is not None else None,
                                         _ptr(v) if v is not None else None, _ptr(o)))
        return o

    def _rows(self, V):
        """(pointer, leading dimension) of a vector or of a 2D tensor of vectors."""
        import torch
        if V.dim() == 1:
            return _ptr(V), self.n_total
        if not (V.is_cuda and V.dtype == torch.complex128 and V.stride(1) == 1 and V.shape[1] == self.n_total):
            raise ValueError("V must hold complex128 CUDA rows of the problem's size")
        return ct.c_void_p(V.data_ptr()), V.stride(0)

    def vec_mdot(self, V, k, w, row_lo, row_hi):
        """[sum over rows [row_lo, row_hi) of conj(V[i]) w for i < k] (mxp_vec_mdot);
        V a 2D complex128 CUDA tensor (one vector per row) or one vector."""
        out = (ct.c_double * (2 * k))()
        vp, ld = self._rows(V)
        _check(self._lib.mxp_vec_mdot(self._h, vp, int(ld), int(k), _ptr(w), int(row_lo), int(row_hi), out))
        a = np.frombuffer(out, dtype=np.float64)
        return a[0::2] + 1j * a[1::2]

    def vec_combine(self, y, beta, V=None, coefs=()):
        """y = beta y + sum_i coefs[i] V[i] (mxp_vec_combine); V as for vec_mdot."""
        k = len(coefs)
        b = (ct.c_double * 2)(complex(beta).real, complex(beta).imag)
        cf = (ct.c_double * max(1, 2 * k))()
        for i, z in enumerate(coefs):
            cf[2 * i], cf[2 * i + 1] = complex(z).real, complex(z).imag
        vp, ld = self._rows(V) if k else (None, self.n_total)
        _check(self._lib.mxp_vec_combine(self._h, _ptr(y), b, vp, int(ld), int(k), cf))
        return y

    def plan(self, which=0):
        """(mu, S, m) of action `which` (mxp_get_plan)."""
        mu, S, m = ct.c_double(0), ct.c_int(0), ct.c_int(0)
        _check(self._lib.mxp_get_plan(self._h, int(which), ct.byref(mu), ct.byref(S), ct.byref(m)))
        return float(mu.value), int(S.value), int(m.value)

    @classmethod
    def from_grid(cls, grid, c, params=None, **kw):
        p = None
        if params is not None:
            p = dict(omega=params.omega, shift_s=params.shift, t=params.t, c_pml=params.cpml,
                     fprtol=params.fprtol)
        return cls(grid.dim, grid.ni, grid.npml, c, grid.h, params=p, **kw)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mxp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters
    def get_params(self) -> dict:
        p = Params()
        _check(self._lib.mxp_get_params(self._h, ct.byref(p)))
        return {k: getattr(p, k) for k, _ in Params._fields_}

    def set_params(self, **kw):
        p = Params()
        _check(self._lib.mxp_get_params(self._h, ct.byref(p)))
        for k, v in kw.items():
            if k == "prec" and isinstance(v, str):
                v = PRECISIONS[v]
            setattr(p, k, v)
        _check(self._lib.mxp_set_params(self._h, ct.byref(p)))

    BC = {"dirichlet": 0, "sound_hard": 1, "absorbing": 2}

    def set_boundary(self, bc=None):
        """Face conditions (x-, x+, y-, y+, z-, z+) as names of BC or codes;
        None = zero Dirichlet everywhere."""
        codes = [self.BC[v] if isinstance(v, str) else int(v) for v in (bc or [])]
        codes += [0] * (6 - len(codes))
        arr = (ct.c_int * 6)(*codes[:6])
        _check(self._lib.mxp_set_boundary(self._h, arr))

    def boundary(self):
        arr = (ct.c_int * 6)()
        _check(self._lib.mxp_get_boundary(self._h, arr))
        return tuple(arr)

    def tile_config(self):
        """(configuration index or -1 for the unfused sweep, fused step count)."""
        k = ct.c_int(0)
        cfg = self._lib.mxp_tile_config(self._h, ct.byref(k))
        return int(cfg), int(k.value)

    SWEEP_KINDS = ("pointwise", "fused_2d", "persistent_2d", "fused_3d", "zmarch_3d", "zmarch_tma_3d")

    def sweep_kernel(self):
        """Name of the kernel that runs this problem's exp-action sweeps."""
        k = self._lib.mxp_sweep_kernel(self._h)
        if k < 0:
            _check(1)
        return self.SWEEP_KINDS[k]

    def persist_config(self):
        """(persistent exp kernel configuration or -1, number of tiles)."""
        k = ct.c_int(0)
        cfg = self._lib.mxp_persist_config(self._h, ct.byref(k))
        return int(cfg), int(k.value)

    def persist_geometry(self):
        """(txo, tyo, ntx, nty, K) of the persistent kernel's tiles, or None."""
        v = [ct.c_int(0) for _ in range(5)]
        cfg = self._lib.mxp_persist_geometry(self._h, *[ct.byref(x) for x in v])
        return tuple(int(x.value) for x in v) if cfg >= 0 else None

    # -- operations (all on the problem's stream)
    def empty(self):
        import torch
        return torch.empty(self.n_total, dtype=torch.complex128, device=f"cuda:{self.device}")

    def apply_operator(self, x, shifted=False, out=None):
        y = self.empty() if out is None else out
        _check(self._lib.mxp_apply_operator(self._h, int(bool(shifted)), _ptr(x), _ptr(y)))
        return y

    def apply_phi(self, which, x, out=None):
        y = self.empty() if out is None else out
        ps = ct.c_int64(0)
        _check(self._lib.mxp_apply_phi(self._h, int(which), _ptr(x), _ptr(y), ct.byref(ps)))
        return y, int(ps.value)

    def apply_matexpre(self, r, out=None):
        w = self.empty() if out is None else out
        st = ApplyStats()
        _check(self._lib.mxp_apply_matexpre(self._h, _ptr(r), _ptr(w), ct.byref(st)))
        return w, {k: getattr(st, k) for k, _ in ApplyStats._fields_}

    def solve(self, b, x=None, rtol=1e-6, restart=30, maxit=500, x0_given=False, check=True):
        xo = self.empty() if x is None else x
        o = SolveOpts(rtol, restart, maxit, int(bool(x0_given)))
        st = SolveStats()
        s = self._lib.mxp_solve(self._h, _ptr(b), _ptr(xo), ct.byref(o), ct.byref(st))
        if s != 4 or check:
            _check(s)
        return xo, st.as_dict()

    def solve_host(self, b_host: np.ndarray, x_host: np.ndarray, rtol=1e-6, restart=30,
                   maxit=500, x0_given=False):
        """Solve with host (numpy complex128) buffers through the host entry point."""
        assert b_host.dtype == np.complex128 and x_host.dtype == np.complex128
        assert b_host.flags.c_contiguous and x_host.flags.c_contiguous
        o = SolveOpts(rtol, restart, maxit, int(bool(x0_given)))
        st = SolveStats()
        _check(self._lib.mxp_solve_host(self._h, ct.c_void_p(b_host.ctypes.data),
                                        ct.c_void_p(x_host.ctypes.data), ct.byref(o),
                                        ct.byref(st)))
        return st.as_dict()


class Cnn:
    """The learned-stage network on one GPU (see include/matexpre.h)."""

    def __init__(self, max_batch, max_h, max_w, device=0, stream=None):
        import torch
        self._lib = load()
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ct.c_void_p()
        _check(self._lib.mxp_cnn_create(self.device, _stream_handle(self.stream), int(max_batch),
                                        int(max_h), int(max_w), ct.byref(h)))
        self._h = h
        self.num_params = int(self._lib.mxp_cnn_num_params())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mxp_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _fptr(t):
        import torch
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("tensors must be contiguous float32 CUDA tensors")
        return ct.c_void_p(t.data_ptr())

    def set_params(self, theta: np.ndarray):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        assert theta.size == self.num_params
        _check(self._lib.mxp_cnn_set_params(self._h, theta.ctypes.data_as(ct.POINTER(ct.c_float))))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        _check(self._lib.mxp_cnn_get_params(self._h, out.ctypes.data_as(ct.POINTER(ct.c_float))))
        return out

    def forward(self, x):
        import torch
        n, c, h, w = x.shape
        y = torch.empty((n, 2, h, w), dtype=torch.float32, device=x.device)
        _check(self._lib.mxp_cnn_forward(self._h, n, h, w, self._fptr(x), self._fptr(y)))
        return y

    def backward(self, x, gy):
        import torch
        g = torch.empty(self.num_params, dtype=torch.float32, device=x.device)
        _check(self._lib.mxp_cnn_backward(self._h, self._fptr(x), self._fptr(gy), self._fptr(g)))
        return g

    def train_step(self, x, target, lr):
        n, c, h, w = x.shape
        loss = ct.c_float(0)
        _check(self._lib.mxp_cnn_train_step(self._h, n, h, w, self._fptr(x), self._fptr(target),
                                            float(lr), ct.byref(loss)))
        return float(loss.value)


def conv3x3(mode, a, w_bf16=None, b=None, bias=None, stride=1, upsample=False, relu=False, cout=None,
            in_hw=None):
    """One tensor-core 3x3 convolution (mxp_cnn_conv3x3).  a: float32 CUDA tensor
    [N, C, H, W] (mode 0, 2: the input x; mode 1: the output gradient g);
    w_bf16: torch.bfloat16 CUDA tensor [Cout, Cin, 3, 3] (modes 0, 1); b: the
    output gradient g (mode 2); cout: output channels (mode 2 only); in_hw: the
    input's (H, W) for mode 1 (default: the gradient's size times the stride)."""
    import torch
    N = int(a.shape[0])
    if mode == 1:
        Cout, Ho, Wo = int(a.shape[1]), int(a.shape[2]), int(a.shape[3])
        Cin = int(w_bf16.shape[1])
        Hs, Ws = (int(in_hw[0]), int(in_hw[1])) if in_hw else (Ho * stride, Wo * stride)
        out = torch.empty((N, Cin, Hs, Ws), dtype=torch.float32, device=a.device)
    else:
        Cin, Hs, Ws = int(a.shape[1]), int(a.shape[2]), int(a.shape[3])
        Hl, Wl = (2 * Hs, 2 * Ws) if upsample else (Hs, Ws)
        Ho, Wo = (Hl + stride - 1) // stride, (Wl + stride - 1) // stride
        Cout = int(w_bf16.shape[0]) if mode == 0 else int(cout)
        out = (torch.empty((N, Cout, Ho, Wo), dtype=torch.float32, device=a.device) if mode == 0
               else torch.empty((Cout, Cin * 9), dtype=torch.float32, device=a.device))
    ptr = lambda t: ct.c_void_p(t.data_ptr()) if t is not None else None
    _check(load().mxp_cnn_conv3x3(int(mode), int(stride), int(bool(upsample)), N, Cin, Hs, Ws, Cout, Ho, Wo,
                                  ptr(a), ptr(b), ptr(w_bf16), ptr(bias), int(bool(relu)), ptr(out),
                                  _stream_handle(None)))
    return out


def attach_cnn(problem, net, accept_tol=0.5):
    _check(load().mxp_attach_cnn(problem._h, net._h if net is not None else None,
                                 float(accept_tol)))


def taylor_plan(nu, tol, theta_max, kmult=1):
    """(sub-steps S, degree m) of the library's Taylor plan, or None."""
    S, m = ct.c_int(0), ct.c_int(0)
    ok = load().mxp_taylor_plan(float(nu), float(tol), float(theta_max), int(kmult), ct.byref(S), ct.byref(m))
    return (int(S.value), int(m.value)) if ok else None


def persist_tile_plan(n0, n1, slots, k, txmax, tymax):
    """Tile plan of the persistent exp kernel: (txo, tyo, ntx, nty) or None."""
    out = [ct.c_int(0) for _ in range(4)]
    ok = load().mxp_persist_tile_plan(int(n0), int(n1), int(slots), int(k), int(txmax), int(tymax),
                                      *[ct.byref(v) for v in out])
    return tuple(int(v.value) for v in out) if ok else None


def measure_fma_peak(device=0):
    """(FP32, FP64) fused multiply-add throughput of the device in flop/s."""
    f32, f64 = ct.c_double(0), ct.c_double(0)
    _check(load().mxp_measure_fma_peak(int(device), ct.byref(f32), ct.byref(f64)))
    return float(f32.value), float(f64.value)


def kernel_launch_count() -> int:
    return int(load().mxp_kernel_launch_count())


def solve_batch(problems, prob_of_rhs, bs, xs, rtol=1e-6, restart=30, maxit=500):
    lib = load()
    nprob, nrhs = len(problems), len(bs)
    hp = (ct.c_void_p * nprob)(*[p._h for p in problems])
    po = (ct.c_int * nrhs)(*prob_of_rhs)
    bp = (ct.c_void_p * nrhs)(*[_ptr(b).value for b in bs])
    xp = (ct.c_void_p * nrhs)(*[_ptr(x).value for x in xs])
    o = SolveOpts(rtol, restart, maxit, 0)
    st = (SolveStats * max(nrhs, 1))()
    s = lib.mxp_solve_batch(hp, nprob, nrhs, po, bp, xp, ct.byref(o), st)
    if s not in (0, 4):
        _check(s)
    return [st[i].as_dict() for i in range(nrhs)]
