"""MatExPre CPU oracle (test infrastructure only).

A plain double-precision restatement of the method written from the paper
(arXiv 2506.03617), in C (``mxp_oracle.c``) with this thin ctypes wrapper.  Only
``tests/``, the smoke check and the benchmark's CPU-baseline leg may import it;
the product path never does, and the oracle shares no code with the CUDA path.

Pinned functions (the pins live in ``tests/test_oracle_*.py``):
  apply      operator A / A_s         -- sine-mode closed form, PML manufactured
                                          solution, symmetry of diag(prod s_d) A
  phi        exp / psi_1 actions       -- scalar closed form on sine modes, dense
                                          expm of the operator matrix, semigroup
  matexpre   Algorithm 1               -- converged apply = (i/t) A_s^{-1} r
  fgmres     outer FGMRES              -- converged solution = direct solve
  neumann    P_N of Sec. 3.2           -- eigenvalues of P_N A (Thm. 3.1)
  apply with sound-hard / absorbing faces  -- cosine-mode eigenpairs, plane-wave
                                          consistency at second order, Im(lambda) >= 0
  phi(2), matexpre(variant=1)         -- psi_2 scalar closed form, dense expm of
             second inverse formula       the augmented matrix, converged apply =
                                          (i/t) A_s^{-1} r
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mxp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmxp_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-fcx-fortran-rules",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("ni", ct.c_int * 3), ("npml", ct.c_int),
                ("h", ct.c_double), ("omega", ct.c_double), ("cpml", ct.c_double),
                ("shift", ct.c_double), ("t", ct.c_double),
                ("c", ct.POINTER(ct.c_double)), ("bc", ct.c_int * 6)]


class _SolveStats(ct.Structure):
    _fields_ = [("outer_iters", ct.c_int), ("converged", ct.c_int),
                ("true_relres", ct.c_double), ("est_relres", ct.c_double),
                ("spmv", ct.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ct.CDLL(build())
            P = ct.POINTER(_Problem)
            cd = ct.POINTER(ct.c_double)
            lib.orc_apply.argtypes = [P, ct.c_int, cd, cd]
            lib.orc_apply.restype = None
            lib.orc_phi.argtypes = [P, ct.c_int, ct.c_int, cd, cd]
            lib.orc_phi.restype = ct.c_int64
            lib.orc_norm_inf_tA.argtypes = [P, ct.c_int]
            lib.orc_norm_inf_tA.restype = ct.c_double
            lib.orc_matexpre.argtypes = [P, cd, cd, ct.c_double, ct.c_int, ct.c_int,
                                         ct.c_int, ct.POINTER(ct.c_int64)]
            lib.orc_matexpre.restype = ct.c_int
            lib.orc_matexpre_v.argtypes = [P, ct.c_int, cd, cd, ct.c_double, ct.c_int, ct.c_int,
                                           ct.c_int, ct.POINTER(ct.c_int64)]
            lib.orc_matexpre_v.restype = ct.c_int
            lib.orc_fgmres_v.argtypes = [P, ct.c_int, cd, cd, ct.c_double, ct.c_int, ct.c_int,
                                         ct.c_double, ct.c_int, ct.c_int, ct.c_int,
                                         ct.POINTER(ct.c_int), ct.c_int, cd,
                                         ct.POINTER(_SolveStats)]
            lib.orc_fgmres_v.restype = None
            lib.orc_fgmres.argtypes = [P, cd, cd, ct.c_double, ct.c_int, ct.c_int,
                                       ct.c_double, ct.c_int, ct.c_int, ct.c_int,
                                       ct.POINTER(ct.c_int), ct.c_int, cd,
                                       ct.POINTER(_SolveStats)]
            lib.orc_fgmres.restype = None
            lib.orc_gmres_plain.argtypes = [P, ct.c_int, cd, cd, ct.c_double, ct.c_int,
                                            ct.c_int]
            lib.orc_neumann.argtypes = [P, ct.c_int, ct.c_int, cd, cd]
            lib.orc_neumann.restype = ct.c_int64
            lib.orc_gmres_plain.restype = ct.c_int
            lib.orc_set_threads.argtypes = [ct.c_int]
            lib.orc_set_threads.restype = None
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle's loops use (for timing runs)."""
    _load().orc_set_threads(int(n))


class Problem:
    """Discrete Helmholtz problem: grid (dim, interior cells, PML cells), medium
    c (numpy array of the full grid, x fastest), omega, C_pml, shift s and t."""

    BC = {"dirichlet": 0, "sound_hard": 1, "absorbing": 2}

    def __init__(self, dim, ni, npml, c, omega, shift, t, cpml=20.0, h=None, bc=None):
        ni = tuple(int(v) for v in ni)
        self.dim = int(dim)
        self.ni = ni
        self.npml = int(npml)
        self.h = float(h) if h is not None else 1.0 / max(ni)
        self.n = tuple(m + 2 * self.npml for m in ni)
        self.n_total = int(np.prod(self.n))
        self.c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1))
        assert self.c.size == self.n_total
        self.omega, self.shift, self.t, self.cpml = float(omega), float(shift), float(t), float(cpml)
        self._s = _Problem()
        self._s.dim = self.dim
        for d in range(3):
            self._s.ni[d] = ni[d] if d < self.dim else 1
        self._s.npml = self.npml
        self._s.h = self.h
        self._s.omega = self.omega
        self._s.cpml = self.cpml
        self._s.shift = self.shift
        self._s.t = self.t
        self._s.c = self.c.ctypes.data_as(ct.POINTER(ct.c_double))
        self.set_bc(bc)

    def set_bc(self, bc=None):
        """Face conditions (x-, x+, y-, y+, z-, z+): names of BC or 0/1/2;
        None = zero Dirichlet everywhere."""
        bc = list(bc) if bc is not None else [0] * 6
        bc = [self.BC[v] if isinstance(v, str) else int(v) for v in bc] + [0] * (6 - len(bc))
        for f in range(6):
            self._s.bc[f] = bc[f]
        self.bc = tuple(bc[:6])

    @classmethod
    def from_grid(cls, grid, c, params, bc=None):
        return cls(grid.dim, grid.ni, grid.npml, c, params.omega, params.shift, params.t,
                   params.cpml, grid.h, bc)

    def _vec(self, x):
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128).reshape(-1))
        assert x.size == self.n_total
        return x

    @staticmethod
    def _ptr(a):
        return a.ctypes.data_as(ct.POINTER(ct.c_double))

    def apply(self, x, shifted=False):
        """y = A x, or A_s x when shifted."""
        x = self._vec(x)
        y = np.empty_like(x)
        _load().orc_apply(ct.byref(self._s), int(bool(shifted)), self._ptr(x), self._ptr(y))
        return y

    def phi(self, which, x, shifted=True):
        """which=0: exp(i t A_s) x; 1: psi_1(i t A_s) x; 2: psi_2(i t A_s) x.
        Returns (y, spmv)."""
        x = self._vec(x)
        y = np.empty_like(x)
        sp = _load().orc_phi(ct.byref(self._s), int(which), int(bool(shifted)),
                             self._ptr(x), self._ptr(y))
        return y, int(sp)

    def expv(self, x, shifted=True):
        return self.phi(0, x, shifted)[0]

    def psi1v(self, x, shifted=True):
        return self.phi(1, x, shifted)[0]

    def norm_inf_tA(self, shifted=True):
        return float(_load().orc_norm_inf_tA(ct.byref(self._s), int(bool(shifted))))

    def matexpre(self, r, fprtol=0.08, restart=30, maxit=1000, fixed=0, variant=0):
        """Algorithm 1 (variant 0) or its form on the second inverse formula,
        psi_2 right-hand side and I - psi_1 operator (variant 1).
        Returns (w, inner_iterations, spmv)."""
        r = self._vec(r)
        w = np.empty_like(r)
        sp = ct.c_int64(0)
        it = _load().orc_matexpre_v(ct.byref(self._s), int(variant), self._ptr(r), self._ptr(w),
                                    float(fprtol), int(restart), int(maxit), int(fixed),
                                    ct.byref(sp))
        return w, int(it), int(sp.value)

    def fgmres(self, b, rtol=1e-6, restart=30, maxit=200, fprtol=0.08, inner_restart=30,
               inner_maxit=1000, inner_fixed=0, x0=None, variant=0):
        """Outer FGMRES with Algorithm 1 (or its variant, see matexpre) as right
        preconditioner.  Returns (u, info dict)."""
        b = self._vec(b)
        u = np.zeros_like(b) if x0 is None else self._vec(x0).copy()
        log_cap = 4096
        inner_log = (ct.c_int * log_cap)()
        res_log = np.zeros(max(maxit, 1), dtype=np.float64)
        st = _SolveStats()
        _load().orc_fgmres_v(ct.byref(self._s), int(variant), self._ptr(b), self._ptr(u),
                             float(rtol), int(restart), int(maxit), float(fprtol),
                             int(inner_restart), int(inner_maxit), int(inner_fixed), inner_log,
                             log_cap, res_log.ctypes.data_as(ct.POINTER(ct.c_double)),
                             ct.byref(st))
        it = st.outer_iters
        info = dict(outer_iters=it, converged=bool(st.converged),
                    true_relres=st.true_relres, est_relres=st.est_relres, spmv=int(st.spmv),
                    inner=[inner_log[i] for i in range(min(it, log_cap))],
                    res_hist=res_log[:it].copy())
        return u, info

    def neumann(self, r, nterms, shifted=True):
        """w = (sum_{n=0}^{N} exp(i t A_s)^n) psi_1(i t A_s) r (P_N of Sec. 3.2 without -i t)."""
        r = self._vec(r)
        w = np.empty_like(r)
        _load().orc_neumann(ct.byref(self._s), int(bool(shifted)), int(nterms), self._ptr(r),
                            self._ptr(w))
        return w

    def gmres_plain(self, b, shifted=False, rtol=1e-10, restart=30, maxit=10000):
        b = self._vec(b)
        x = np.zeros_like(b)
        it = _load().orc_gmres_plain(ct.byref(self._s), int(bool(shifted)), self._ptr(b),
                                     self._ptr(x), float(rtol), int(restart), int(maxit))
        return x, int(it)

    def dense(self, shifted=False):
        """The operator as a dense matrix, column by column (tiny grids only)."""
        n = self.n_total
        M = np.empty((n, n), dtype=np.complex128)
        e = np.zeros(n, dtype=np.complex128)
        for j in range(n):
            e[j] = 1.0
            M[:, j] = self.apply(e, shifted)
            e[j] = 0.0
        return M
