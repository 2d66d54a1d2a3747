"""Sparse matrix of a 5/7-point operator obtained by probing it with coloured
unit-vector sums (test helper; works for any linear stencil of radius 1)."""
import itertools

import numpy as np
import scipy.sparse as sp


def probe_sparse(apply, shape_xyz):
    """apply: function on flat complex vectors (x fastest); shape_xyz = (n0, n1[, n2])."""
    dim = len(shape_xyz)
    n = int(np.prod(shape_xyz))
    idx = np.arange(n)
    coords = []
    rem = idx.copy()
    for d in range(dim):
        coords.append(rem % shape_xyz[d])
        rem //= shape_xyz[d]
    rows, cols, vals = [], [], []
    for color in itertools.product(range(3), repeat=dim):
        mask = np.ones(n, dtype=bool)
        for d in range(dim):
            mask &= coords[d] % 3 == color[d]
        e = mask.astype(np.complex128)
        y = apply(e)
        # column j's entries live at rows within distance 1 of j
        js = np.nonzero(mask)[0]
        for off in itertools.product((-1, 0, 1), repeat=dim):
            if sum(abs(o) for o in off) > 1:
                continue
            ok = np.ones(js.size, dtype=bool)
            r = js.copy()
            stride = 1
            for d in range(dim):
                cd = coords[d][js] + off[d]
                ok &= (cd >= 0) & (cd < shape_xyz[d])
                r = r + off[d] * stride
                stride *= shape_xyz[d]
            rows.append(r[ok]); cols.append(js[ok]); vals.append(y[r[ok]])
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
