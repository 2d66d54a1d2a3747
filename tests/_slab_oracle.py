"""A slab "device" on the CPU for the slab-decomposed solver: the oracle's
operator on the whole grid restricted to the slab's rows, with zero values
beyond them (what a slab problem's kernels compute), on torch CPU vectors.
Test infrastructure: it stands in for mxp_create_slab's problem so that the
distributed driver runs over gloo ranks without a GPU."""
import numpy as np
import torch


class OracleSlab:
    def __init__(self, P, grid, e0, e1, params, plans):
        self.P, self.N = P, grid.n_total
        self.row = int(np.prod(grid.n[:-1]))
        self.e0, self.e1 = int(e0), int(e1)
        self.n_total = (self.e1 - self.e0) * self.row
        self._params, self._plans = dict(params), list(plans)

    def get_params(self):
        return dict(self._params)

    def plan(self, which=0):
        return self._plans[which]

    def empty(self):
        return torch.empty(self.n_total, dtype=torch.complex128)

    def _A(self, x, shifted):
        full = np.zeros(self.N, dtype=np.complex128)
        full[self.e0 * self.row:self.e1 * self.row] = x.numpy()
        return self.P.apply(full, shifted=shifted)[self.e0 * self.row:self.e1 * self.row]

    def horner_step(self, sigma, p, y=None, v=None, gamma=0j, rho=1 + 0j, out=None):
        mu = self._plans[0][0]
        r = sigma * (self._A(p, True) - mu * p.numpy())
        if y is not None:
            r = r + y.numpy()
        if v is not None:
            r = r + gamma * v.numpy()
        out.copy_(torch.from_numpy(rho * r))
        return out

    def apply_operator(self, x, shifted=False, out=None):
        out.copy_(torch.from_numpy(self._A(x, shifted)))
        return out

    def vec_mdot(self, V, k, w, row_lo, row_hi):
        Vn = V.numpy() if V.dim() == 2 else V.numpy()[None]
        sl = slice(row_lo * self.row, row_hi * self.row)
        wn = w.numpy()[sl]
        return np.array([np.vdot(Vn[i][sl], wn) for i in range(k)])

    def vec_combine(self, y, beta, V=None, coefs=()):
        yn = beta * y.numpy()
        if len(coefs):
            Vn = V.numpy() if V.dim() == 2 else V.numpy()[None]
            for i, c in enumerate(coefs):
                yn = yn + c * Vn[i]
        y.copy_(torch.from_numpy(yn))
        return y
