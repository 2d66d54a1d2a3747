"""Multi-process helpers (one process per GPU).

Two ways to spread the MatExPre path over GPUs:

* Independent units (solve_sharded): the medium is replicated on every rank
  and the sources (right-hand sides) are split among the ranks, each of which
  solves its share with the batched solver on its own GPU.  Nothing is
  exchanged on the data path; the only collectives are the final gather of the
  per-source results and the combination of the timings (the job's time is the
  slowest rank's, its work the sum).
* One grid in slabs (SlabSolver): the rows of the last axis are split among
  the ranks, each holding its rows plus K halo rows of each neighbour; the
  Taylor-Horner steps exchange halos every K steps, and every Krylov dot
  product is summed over the ranks (the paper's distributed layout, Sec. 4).
"""
from __future__ import annotations

import os

import numpy as np


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank, world):
    """The units this rank owns: round-robin, every unit exactly once."""
    return list(items)[rank::world]


def _distributed():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def reduce_job(seconds: float, units: float, device=None):
    """(max over ranks of seconds, sum over ranks of units); identity when not
    distributed.  Uses the default process group (gloo on CPU, nccl on GPU)."""
    import torch
    import torch.distributed as dist
    if not _distributed():
        return float(seconds), float(units)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def gather_by_index(local: dict, total: int):
    """Merge {unit index: result} from every rank into a list ordered by unit
    index (one all_gather of host objects); identity when not distributed.
    Raises if some unit has no result or two ranks report the same unit."""
    import torch.distributed as dist
    parts = [local]
    if _distributed():
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, local)
    out = [None] * total
    seen = set()
    for part in parts:
        for k, v in part.items():
            if k in seen or not 0 <= k < total:
                raise RuntimeError(f"unit {k} reported twice or out of range")
            seen.add(k)
            out[k] = v
    if len(seen) != total:
        raise RuntimeError(f"units without a result: {sorted(set(range(total)) - seen)}")
    return out


def solve_sharded(sources, solve_share, rank=None, world=None):
    """Solve many sources split across the ranks.

    sources     the job's right-hand sides, in a fixed order every rank agrees on
    solve_share callable(list of (index, source)) -> list of per-source results,
                run by each rank on its own share (on the GPU: the batched C-ABI
                solver on the rank's device, the medium replicated per rank)
    Returns every source's result, in source order, on every rank.
    """
    r0, w0, _ = env()
    rank = r0 if rank is None else rank
    world = w0 if world is None else world
    mine = shard(range(len(sources)), rank, world)
    results = solve_share([(i, sources[i]) for i in mine]) if mine else []
    if len(results) != len(mine):
        raise RuntimeError("solve_share returned a result count different from its share")
    return gather_by_index(dict(zip(mine, results)), len(sources))


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ------------------------------------------------------------- slab decomposition
# One grid split into slabs of rows of its last axis (y in 2D, z in 3D), one per
# rank, as in the paper's distributed runs (Sec. 4).  Each rank keeps its owned
# rows plus `halo` rows of each neighbour.  A Taylor-Horner step on the extended
# slab is exact on every row at least one row away from the slab's outer edge;
# after K <= halo steps the owned rows are still exact, so the ranks exchange
# their edge rows every `halo` steps (and at every sub-step end, where y is
# taken from p).  The Krylov dot products need one sum over the ranks.


def slab_bounds(n_rows: int, world: int):
    """Owned rows [r0, r1) of every rank: a balanced split of n_rows."""
    base, extra = divmod(int(n_rows), int(world))
    out, r = [], 0
    for k in range(world):
        m = base + (1 if k < extra else 0)
        out.append((r, r + m))
        r += m
    return out


def slab_extended(bounds, rank: int, halo: int, n_rows: int):
    """Rows [e0, e1) a rank holds: its owned rows plus `halo` rows of each neighbour."""
    r0, r1 = bounds[rank]
    return max(0, r0 - halo), min(int(n_rows), r1 + halo)


class SlabExchange:
    """Exchange of `halo` edge rows between neighbouring slabs over
    torch.distributed point-to-point operations (gloo for CPU tensors, nccl for
    CUDA tensors), one slab per rank.  Vectors hold the extended slab, x
    fastest, `row_len` values per row; called with the list of this rank's
    vectors (one)."""

    def __init__(self, bounds, rank: int, halo: int, row_len: int, n_rows: int):
        self.bounds, self.rank, self.halo, self.row_len = bounds, int(rank), int(halo), int(row_len)
        self.world = len(bounds)
        for r0, r1 in bounds:
            if r1 - r0 < halo:
                raise ValueError("every slab must own at least `halo` rows")
        self.e0, self.e1 = slab_extended(bounds, rank, halo, n_rows)
        self.r0, self.r1 = bounds[rank]

    def _rows(self, v, a, b):
        """The rows [a, b) (global indices) of the extended-slab vector v."""
        return v[(a - self.e0) * self.row_len:(b - self.e0) * self.row_len]

    def __call__(self, vs):
        import torch.distributed as dist
        v = vs[0]
        reqs = []
        lo, hi = self.rank - 1, self.rank + 1
        if lo >= 0:
            reqs.append(dist.isend(self._rows(v, self.r0, self.r0 + self.halo).contiguous(), lo))
            reqs.append(dist.irecv(self._rows(v, self.e0, self.r0), lo))
        if hi < self.world:
            reqs.append(dist.isend(self._rows(v, self.r1 - self.halo, self.r1).contiguous(), hi))
            reqs.append(dist.irecv(self._rows(v, self.r1, self.e1), hi))
        for r in reqs:
            r.wait()


class LocalSlabExchange:
    """The same exchange for all slabs of a grid held by one process (the
    vectors of every slab, in slab order): halo rows are copied from the
    neighbouring slab's owned rows."""

    def __init__(self, bounds, halo: int, row_len: int, n_rows: int):
        self.bounds, self.halo, self.row_len = bounds, int(halo), int(row_len)
        for r0, r1 in bounds:
            if r1 - r0 < halo:
                raise ValueError("every slab must own at least `halo` rows")
        self.ext = [slab_extended(bounds, k, halo, n_rows) for k in range(len(bounds))]

    def _rows(self, k, v, a, b):
        e0 = self.ext[k][0]
        return v[(a - e0) * self.row_len:(b - e0) * self.row_len]

    def __call__(self, vs):
        for k in range(len(vs) - 1):
            r1 = self.bounds[k][1]                     # boundary between slab k and k + 1
            e1 = self.ext[k][1]
            e0n = self.ext[k + 1][0]
            self._rows(k, vs[k], r1, e1).copy_(self._rows(k + 1, vs[k + 1], r1, e1))
            self._rows(k + 1, vs[k + 1], e0n, r1).copy_(self._rows(k, vs[k], e0n, r1))


def slab_exp_action(steps, plan, t, p0s, bufs, exchange, halo):
    """exp(i t A_s) x on extended slabs by the sub-stepped Taylor-Horner
    recurrence (Def. psi; the plan (mu, S, m) of the whole grid):
      per sub-step, y = p at its start, then p <- y + i t / (S k) (A_s - mu) p for
      k = m .. 1, the last step of the last sub-step multiplied by e^{i t mu}.
    For every slab this process holds: steps[i](sigma, p, y, rho, out) computes
    out = rho (y + sigma (A_s - mu) p) on the extended slab (mxp_horner_step of a
    slab problem), p0s[i] holds x on the extended slab (halo rows are filled by
    the first exchange), bufs[i] two more vectors of the same size.
    exchange(list of vectors) refreshes the halo rows.  Returns, per slab, the
    vector that holds the result (its owned rows are exact)."""
    import cmath
    mu, S, m = plan
    rho_end = cmath.exp(1j * t * mu)
    ns = len(p0s)
    vecs = [[p0s[i], bufs[i][0], bufs[i][1]] for i in range(ns)]
    exchange([v[0] for v in vecs])
    iy = 0                                      # index of y (the sub-step start)
    for sub in range(S):
        cur, since = iy, 0
        for k in range(m, 0, -1):
            if since == halo:
                exchange([v[cur] for v in vecs])
                since = 0
            out = (iy + 1) % 3 if cur == iy else 3 - iy - cur
            rho = rho_end if (sub == S - 1 and k == 1) else 1.0
            for i in range(ns):
                steps[i](1j * t / (S * k), vecs[i][cur], vecs[i][iy], rho, vecs[i][out])
            cur = out
            since += 1
        if sub < S - 1:
            exchange([v[cur] for v in vecs])    # the next y needs exact halo rows
        iy = cur
    return [v[iy] for v in vecs]


def slab_dot(a, b, owned):
    """sum over the whole grid of conj(a) b for vectors split into slabs: the
    local sum over this rank's owned rows (`owned`, a slice of the extended
    slab) and one all_reduce (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    loc = torch.vdot(a[owned], b[owned])
    if not _distributed():
        return complex(loc)
    t = torch.stack([loc.real, loc.imag]).to(torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return complex(float(t[0]), float(t[1]))


# -------------------------------------------------- slab-decomposed Algorithm 1 / FGMRES

class _AugScalars:
    """Scalar rows of the augmented matrix of a psi action (Def. psi): psi_1 adds
    one scalar whose state feeds v into the grid block, psi_2 a 2x2 Jordan
    block; both advance by the Horner recursion of the grid block, shifted by
    -i t mu (rot = -i t mu / S per sub-step of length 1/S)."""

    def __init__(self, which, rot, nsub):
        self.which, self.rot, self.invS, self.S = which, rot, 1.0 / nsub, float(nsub)
        self.z1 = 1.0 + 0j if which == 1 else 0j
        self.z2 = 1.0 + 0j if which == 2 else 0j
        self.g1, self.g2 = self.z1, self.z2

    def begin(self):
        self.g1, self.g2 = self.z1, self.z2

    def gamma(self, k):
        """Coefficient of v in the grid-block update of Horner step k."""
        return self.g1 / (self.S * k) if self.which else 0j

    def step(self, k):
        n1 = self.z1 + (self.rot * self.g1 + self.invS * self.g2) / k
        n2 = self.z2 + self.rot * self.g2 / k
        self.g1, self.g2 = n1, n2

    def end(self):
        self.z1, self.z2 = self.g1, self.g2


def _givens(a, b):
    """c (real), s (complex) with [c s; -conj(s) c] (a, b) = (r, 0)."""
    if b == 0:
        return 1.0, 0j
    if a == 0:
        return 0.0, complex(np.conj(b)) / abs(b)
    na = abs(a)
    nrm = float(np.hypot(na, abs(b)))
    return na / nrm, (a / na) * np.conj(b) / nrm


class _Lsq:
    """Incremental least squares of GMRES: Givens rotations of the Hessenberg
    columns, residual estimate |g[j + 1]|, back substitution."""

    def __init__(self, R, beta):
        self.H = np.zeros((R + 1, R), dtype=np.complex128)
        self.g = np.zeros(R + 1, dtype=np.complex128)
        self.g[0] = beta
        self.cs, self.sn = [], []

    def add(self, j, h, hn):
        col = np.zeros(j + 2, dtype=np.complex128)
        col[:j + 1] = h
        col[j + 1] = hn
        for i in range(j):
            c, s = self.cs[i], self.sn[i]
            col[i], col[i + 1] = c * col[i] + s * col[i + 1], -np.conj(s) * col[i] + c * col[i + 1]
        c, s = _givens(col[j], col[j + 1])
        self.cs.append(c)
        self.sn.append(s)
        col[j] = c * col[j] + s * col[j + 1]
        col[j + 1] = 0.0
        self.H[:j + 2, j] = col
        self.g[j + 1] = -np.conj(s) * self.g[j]
        self.g[j] = c * self.g[j]
        return abs(self.g[j + 1])

    def solve(self, k):
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (self.g[i] - self.H[i, i + 1:k] @ y[i + 1:k]) / self.H[i, i]
        return y


def torch_allreduce(a):
    """Sum of a complex numpy array over the ranks of torch.distributed
    (identity when not distributed)."""
    if not _distributed():
        return a
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(np.stack([a.real, a.imag]).astype(np.float64)))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    t = t.numpy()
    return t[0] + 1j * t[1]


class SlabSolver:
    """Algorithm 1 inside FGMRES on one grid split into slabs of rows of its
    last axis (the distributed scheme of Sec. 4: halo rows exchanged between
    neighbouring slabs, every dot product summed over the ranks).

    slabs: the slab problems this process holds (mxp_create_slab, or any
      object with the same methods), all with the same parameters;
    owned: per slab, the local rows [lo, hi) it owns;
    exchange(vectors): refreshes the halo rows of one vector per slab
      (SlabExchange across ranks, LocalSlabExchange within a process);
    allreduce(array): sums a complex array over the ranks (torch_allreduce;
      the identity when all slabs are in this process);
    halo: rows held of each neighbour (K >= 1): the Horner steps exchange
      every K steps and at every sub-step end, the operator after one.
    Vectors are lists with one extended-slab vector per slab.  Every stencil
    step, dot product and linear combination runs in the slab problem's
    kernels (mxp_horner_step, mxp_apply_operator, mxp_vec_mdot,
    mxp_vec_combine); the host keeps the (R + 1) x R Hessenberg matrices."""

    def __init__(self, slabs, owned, exchange, allreduce=None, halo=1):
        self.slabs, self.owned = list(slabs), [tuple(o) for o in owned]
        self.exchange, self.halo = exchange, int(halo)
        if self.halo < 1:
            raise ValueError("halo must be at least one row")
        self.allreduce = allreduce or (lambda a: a)
        prm = self.slabs[0].get_params()
        self.t, self.fprtol = float(prm["t"]), float(prm["fprtol"])
        self.R_in = int(prm["inner_restart"])
        self.inner_maxit, self.inner_fixed = int(prm["inner_maxit"]), int(prm["inner_fixed"])
        self.precond, self.neumann_n = int(prm["precond"]), int(prm["neumann_n"])
        self.plans = [self.slabs[0].plan(w) for w in range(3)]
        for s in self.slabs[1:]:
            if [s.plan(w) for w in range(3)] != self.plans:
                raise ValueError("every slab of a grid must have the same shift and Taylor plans")
        self.work = [[self._zeros(s) for _ in range(4)] for s in self.slabs]
        self.rt = [self._zeros(s) for s in self.slabs]
        self.tmp = [self._zeros(s) for s in self.slabs]
        self._inner_V = None
        self.passes = 0

    @staticmethod
    def _zeros(s, rows=None):
        v = s.empty()
        if rows is not None:
            v = v.new_zeros((rows, v.shape[0]))
        else:
            v.zero_()
        return v

    # -- distributed vector operations
    def dot(self, xs, ys):
        acc = np.zeros(1, dtype=np.complex128)
        for s, x, y, (lo, hi) in zip(self.slabs, xs, ys, self.owned):
            acc += s.vec_mdot(x, 1, y, lo, hi)
        return complex(self.allreduce(acc)[0])

    def norm(self, xs):
        return float(np.sqrt(max(0.0, self.dot(xs, xs).real)))

    def mdot(self, Vs, k, ws):
        acc = np.zeros(k, dtype=np.complex128)
        for s, V, w, (lo, hi) in zip(self.slabs, Vs, ws, self.owned):
            acc += s.vec_mdot(V, k, w, lo, hi)
        return self.allreduce(acc)

    def combine(self, ys, beta, Vs=None, coefs=()):
        for i, (s, y) in enumerate(zip(self.slabs, ys)):
            s.vec_combine(y, beta, Vs[i] if len(coefs) else None, coefs)

    def copy(self, dst, src):
        self.combine(dst, 0.0, src, [1.0])

    # -- stencil work
    def op(self, xs, outs):
        """outs = A xs (unshifted operator): one halo exchange, one step."""
        self.exchange(xs)
        for s, x, o in zip(self.slabs, xs, outs):
            s.apply_operator(x, shifted=False, out=o)
        self.passes += 1

    def phi(self, which, xs, outs, out_mode=0):
        """outs = phi_which(i t A_s) xs (0 exp, 1 psi_1, 2 psi_2), or xs minus it
        (out_mode 1): the sub-stepped Taylor-Horner recurrence of the whole
        grid's plan, the augmented scalars carrying v for the psi actions."""
        import cmath
        mu, S, m = self.plans[which]
        t = self.t
        aug = _AugScalars(which, complex(0.0, -t * mu / S), S)
        rho_end = cmath.exp(1j * t * mu)
        vecs = [w[:3] for w in self.work]
        vs = [w[3] for w in self.work]
        if which == 0:
            self.copy([v[0] for v in vecs], xs)
        else:
            self.copy(vs, xs)
            self.combine([v[0] for v in vecs], 0.0)
            self.exchange(vs)
        self.exchange([v[0] for v in vecs])
        iy = 0
        for sub in range(S):
            cur, since = iy, 0
            aug.begin()
            for k in range(m, 0, -1):
                if since == self.halo:
                    self.exchange([v[cur] for v in vecs])
                    since = 0
                out = (iy + 1) % 3 if cur == iy else 3 - iy - cur
                rho = rho_end if (sub == S - 1 and k == 1) else 1.0
                gam = aug.gamma(k)
                for i, s in enumerate(self.slabs):
                    s.horner_step(1j * t / (S * k), vecs[i][cur], vecs[i][iy], vs[i] if which else None,
                                  gamma=gam, rho=rho, out=vecs[i][out])
                aug.step(k)
                cur = out
                since += 1
                self.passes += 1
            if sub < S - 1:
                self.exchange([v[cur] for v in vecs])
            iy = cur
            aug.end()
        res = [v[iy] for v in vecs]
        if out_mode == 0:
            self.copy(outs, res)
        else:
            self.copy(outs, xs)
            self.combine(outs, 1.0, res, [-1.0])

    # -- Krylov
    def _arnoldi(self, Vs, j):
        """Orthonormalise Vs[.][j + 1] against Vs[.][:j + 1] (classical
        Gram-Schmidt, twice); returns the column h and the new norm."""
        w = [V[j + 1] for V in Vs]
        h = self.mdot(Vs, j + 1, w)
        self.combine(w, 1.0, Vs, -h)
        h2 = self.mdot(Vs, j + 1, w)
        self.combine(w, 1.0, Vs, -h2)
        h = h + h2
        hn = self.norm(w)
        if hn > 0:
            self.combine(w, 1.0 / hn)
        return h, hn

    def matexpre(self, rs, ws):
        """ws = MatExPre(rs) (Algorithm 1: r~ = psi_1 r, GMRES on (I - exp) w = r~
        from w = 0 to fprtol; the second inverse formula uses psi_2 and
        I - psi_1; precond 1 the truncated Neumann series).  Returns the inner
        iteration count."""
        if self.precond == 1:
            self.phi(1, rs, ws)
            z = self.rt
            self.copy(z, ws)
            for _ in range(self.neumann_n):
                self.phi(0, z, self.tmp)
                self.combine(ws, 1.0, self.tmp, [1.0])
                self.copy(z, self.tmp)
            return self.neumann_n
        R = self.R_in
        if self._inner_V is None:
            self._inner_V = [self._zeros(s, R + 1) for s in self.slabs]
        V = self._inner_V
        rhs_which, op_which = (2, 1) if self.precond == 2 else (1, 0)
        self.phi(rhs_which, rs, self.rt)
        self.combine(ws, 0.0)
        zeta = self.norm(self.rt)
        tol = self.fprtol * zeta
        target = self.inner_fixed if self.inner_fixed > 0 else self.inner_maxit
        total, est = 0, zeta
        converged = zeta == 0.0
        beta, start = zeta, self.rt
        while not converged and total < target:
            self.combine([v[0] for v in V], 0.0, start, [1.0 / beta])
            lsq = _Lsq(R, beta)
            j, stop = 0, False
            while j < R and total < target:
                self.phi(op_which, [v[j] for v in V], [v[j + 1] for v in V], out_mode=1)
                h, hn = self._arnoldi(V, j)
                est = lsq.add(j, h, hn)
                total += 1
                j += 1
                if hn == 0.0 or (self.inner_fixed <= 0 and est <= tol):
                    stop = converged = True
                    break
            self.combine(ws, 1.0, V, lsq.solve(j))
            if stop or total >= target:
                break
            # restart from the true inner residual r~ - (I - exp) w
            self.phi(op_which, ws, self.tmp, out_mode=1)
            self.combine(self.tmp, -1.0, self.rt, [1.0])
            beta = est = self.norm(self.tmp)
            start = self.tmp
            if self.inner_fixed <= 0 and est <= tol:
                converged = True
            if beta == 0.0:
                break
        return total

    def solve(self, bs, xs, rtol=1e-6, restart=30, maxit=300):
        """FGMRES(restart) on A x = b, right-preconditioned by matexpre; the true
        residual is computed at every restart.  Returns a stats dict."""
        R = int(restart)
        V = [self._zeros(s, R + 1) for s in self.slabs]
        Z = [self._zeros(s, R) for s in self.slabs]
        r = [self._zeros(s) for s in self.slabs]
        bnorm = self.norm(bs)
        self.combine(xs, 0.0)
        self.copy(r, bs)
        total = inner_total = 0
        converged, relres = bnorm == 0.0, 0.0 if bnorm == 0.0 else 1.0
        passes0 = self.passes
        while not converged and total < maxit:
            beta = self.norm(r)
            relres = beta / bnorm
            if beta <= rtol * bnorm:
                converged = True
                break
            self.combine([v[0] for v in V], 0.0, r, [1.0 / beta])
            lsq = _Lsq(R, beta)
            j = 0
            while j < R and total < maxit:
                inner_total += self.matexpre([v[j] for v in V], [z[j] for z in Z])
                self.op([z[j] for z in Z], [v[j + 1] for v in V])
                h, hn = self._arnoldi(V, j)
                est = lsq.add(j, h, hn)
                total += 1
                j += 1
                if hn == 0.0 or est <= rtol * bnorm:
                    break
            self.combine(xs, 1.0, Z, lsq.solve(j))
            self.op(xs, r)                              # true residual r = b - A x
            self.combine(r, -1.0, bs, [1.0])
            relres = self.norm(r) / bnorm
            if relres <= rtol:
                converged = True
        return {"outer_iters": total, "inner_iters_total": inner_total, "converged": bool(converged),
                "true_relres": relres, "stencil_passes": self.passes - passes0}
