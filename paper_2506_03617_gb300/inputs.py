"""Seeded synthetic inputs: grids, media c(x), sources and the paper's parameter rules.

This module holds no arithmetic of the method itself (no operator, no matrix
function, no Krylov step).  It produces the data that both the CUDA path and
the CPU oracle consume, so that the two sides see identical inputs.

Grid reading used throughout: axis d has ``N_d`` interior cells plus ``npml``
PML cells on each side, unknown ``j`` sits at ``x_j = (j - npml + 1/2) h`` and
``h = 1 / max_d N_d`` (the paper scales the largest interior dimension to 1,
Sec. 4).  Arrays are C-ordered as ``[z][y][x]`` (x fastest).

Parameter rules (Sec. 4): ``omega = 2 pi c_min / (ppw h)`` so that the slowest
wave has ``ppw`` points per wavelength; in the paper's scaled units (domain 1,
``c_min = 1``) ``freq = 1/(ppw h)``; the shift is ``s = 1/freq``; the time length
follows ``t = 0.4/freq^2`` at ppw 10 and ``t = 0.1/freq^2`` at ppw 20, i.e.
``t = 40 h^2`` in both cases, which is the rule used here for every grid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2506036170


@dataclass(frozen=True)
class Grid:
    dim: int
    ni: tuple            # interior cells per axis (x, y[, z])
    npml: int

    @property
    def h(self) -> float:
        return 1.0 / max(self.ni)

    @property
    def n(self) -> tuple:
        """Unknowns per axis, x first."""
        return tuple(m + 2 * self.npml for m in self.ni)

    @property
    def shape(self) -> tuple:
        """numpy shape, slowest axis first ([z][y][x])."""
        return tuple(reversed(self.n))

    @property
    def n_total(self) -> int:
        return int(np.prod(self.n))

    def node_coords(self, d: int) -> np.ndarray:
        j = np.arange(self.n[d], dtype=np.float64)
        return (j - self.npml + 0.5) * self.h


@dataclass
class Params:
    omega: float
    shift: float
    t: float
    cpml: float = 20.0
    fprtol: float = 0.08
    freq: float = 0.0
    extra: dict = field(default_factory=dict)


def paper_params(grid: Grid, c: np.ndarray, ppw: float = 10.0, cpml: float = 20.0,
                 fprtol: float = 0.08, t_over_h2: float = 40.0,
                 shift_mult: float = 1.0) -> Params:
    """omega from ppw w.r.t. c_min, s = shift_mult/freq, t = 40 h^2 (Sec. 4)."""
    h = grid.h
    cmin = float(np.min(c))
    omega = 2.0 * math.pi * cmin / (ppw * h)
    freq = 1.0 / (ppw * h)          # scaled units: unit domain, c_min = 1
    return Params(omega=omega, shift=shift_mult / freq, t=t_over_h2 * h * h, cpml=cpml,
                  fprtol=fprtol, freq=freq)


def _clamp_into_pml(grid: Grid, interior: np.ndarray) -> np.ndarray:
    """Extend an interior field into the PML by repeating the nearest interior value."""
    pad = [(grid.npml, grid.npml)] * grid.dim
    return np.pad(interior, pad, mode="edge")


def homogeneous(grid: Grid, value: float = 1.0) -> np.ndarray:
    return np.full(grid.shape, value, dtype=np.float64)


def lens(grid: Grid, center=(0.5, 0.25, 0.5), sigma: float = 1.0 / 32.0) -> np.ndarray:
    """Converging-lens medium c = 1 - exp(-|x-x0|^2 / (2 sigma^2)) / 2 (Sec. 4.4)."""
    axes = [grid.node_coords(d) for d in range(grid.dim)]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")      # slowest axis first
    r2 = np.zeros(grid.shape)
    for d in range(grid.dim):
        r2 += (mesh[grid.dim - 1 - d] - center[d]) ** 2
    c = 1.0 - 0.5 * np.exp(-r2 / (2.0 * sigma * sigma))
    # the medium inside the PML repeats the nearest interior value
    sl = tuple(slice(grid.npml, grid.npml + m) for m in reversed(grid.ni))
    return _clamp_into_pml(grid, c[sl])


def gaussian_random_field(shape, corr_cells: float, rng: np.random.Generator) -> np.ndarray:
    """White noise smoothed by a separable Gaussian of std ``corr_cells`` cells,
    periodic boundary, normalised to max |g| = 1."""
    g = rng.standard_normal(shape)
    for ax in range(len(shape)):
        n = shape[ax]
        k = np.fft.fftfreq(n)
        filt = np.exp(-0.5 * (2.0 * math.pi * k * corr_cells) ** 2)
        g = np.real(np.fft.ifft(np.fft.fft(g, axis=ax) * filt.reshape(
            [-1 if a == ax else 1 for a in range(len(shape))]), axis=ax))
    return g / np.max(np.abs(g))


def layered_grf(grid: Grid, seed: int, vmin: float = 1.5, vmax: float = 4.5,
                grf_amp: float = 0.15, corr_cells: float = 20.0) -> np.ndarray:
    """Layered background (6-10 horizontal layers, velocity increasing with depth
    from vmin to vmax) times (1 + grf_amp * g) with g a Gaussian random field of
    correlation length ``corr_cells``; depth is the last spatial axis."""
    rng = np.random.default_rng(seed)
    nlayers = int(rng.integers(6, 11))
    depth_cells = grid.ni[-1]
    nlayers = min(nlayers, depth_cells)          # tiny grids: at most one layer per cell
    cuts = np.sort(rng.choice(np.arange(1, depth_cells), size=nlayers - 1, replace=False))
    vel = np.sort(rng.uniform(vmin, vmax, size=nlayers))
    vel[0], vel[-1] = vmin, vmax
    layer_of_depth = np.searchsorted(cuts, np.arange(depth_cells), side="right")
    background = vel[layer_of_depth]                       # along depth
    ishape = tuple(reversed(grid.ni))                        # slowest = depth
    bshape = [depth_cells] + [1] * (grid.dim - 1)
    c = np.broadcast_to(background.reshape(bshape), ishape).copy()
    c *= 1.0 + grf_amp * gaussian_random_field(ishape, corr_cells, rng)
    return _clamp_into_pml(grid, c)


def gaussian_source(grid: Grid, center=None, sigma_cells: float = 1.0) -> np.ndarray:
    """Normalised Gaussian f = exp(-|x-x0|^2/(2 sigma^2)) / (2 pi sigma^2)^(d/2),
    sampled at the nodes (sigma in cells)."""
    if center is None:
        center = tuple(0.5 * m * grid.h for m in grid.ni)
    sigma = sigma_cells * grid.h
    axes = [grid.node_coords(d) for d in range(grid.dim)]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    r2 = np.zeros(grid.shape)
    for d in range(grid.dim):
        r2 += (mesh[grid.dim - 1 - d] - center[d]) ** 2
    return np.exp(-r2 / (2 * sigma * sigma)) / (2 * math.pi * sigma * sigma) ** (grid.dim / 2)


def rhs_from_source(f: np.ndarray) -> np.ndarray:
    """b = -f (Eq. helmholtz written as A u = -f), complex128."""
    return (-f).astype(np.complex128)


def random_centers(grid: Grid, count: int, seed: int, margin_cells: int = 4):
    """Seeded source positions inside the interior, away from its edge."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append(tuple(float((rng.integers(margin_cells, m - margin_cells) + 0.5) * grid.h)
                         for m in grid.ni))
    return out


def random_complex(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


# ---- named workloads (sizes of the paper-shaped configurations) ----

def config_2d_homogeneous():
    """128^2 interior + 16-cell PML, c = 1, ppw 10 (freq 12.8), Gaussian source at centre."""
    g = Grid(2, (128, 128), 16)
    c = homogeneous(g)
    return g, c, paper_params(g, c, ppw=10.0)


# Face conditions (x-, x+, y-, y+) of the Marmousi-II case of Sec. 4: a
# sound-hard water surface on top (the y- face; depth is the last axis) and
# first-order absorbing conditions on the other faces.
MARMOUSI_BC = ("absorbing", "absorbing", "sound_hard", "absorbing")
BC_CODES = {"dirichlet": 0, "sound_hard": 1, "absorbing": 2}


def marmousi_like(grid: Grid, seed: int, water_frac: float = 0.13, vwater: float = 1.5,
                  vmin: float = 1.6, vmax: float = 4.7, grf_amp: float = 0.1,
                  corr_cells: float = 20.0) -> np.ndarray:
    """A seeded stand-in for the Marmousi-II velocity model (not available
    here): a water layer of velocity ``vwater`` over the top ``water_frac`` of
    the depth, above a layered sediment column (velocity increasing with depth
    from vmin to vmax) times (1 + grf_amp g).  No PML is expected (npml = 0)."""
    c = layered_grf(grid, seed, vmin=vmin, vmax=vmax, grf_amp=grf_amp, corr_cells=corr_cells)
    rows = max(1, int(round(water_frac * grid.ni[-1])))
    c[:grid.npml + rows] = vwater           # with a PML, its top cells repeat the water value
    return c


def config_2d_marmousi_like(nx: int = 1700, seed: int = SEED_BASE + 8000, ppw: float = 10.0):
    """Marmousi-shaped 2D case: nx x round(nx * 1400 / 6800) cells (the
    aspect ratio of the model in Sec. 4), no PML, ppw 10 w.r.t. the water
    velocity, t = 40 h^2, s = 1/freq; use with MARMOUSI_BC and a source near the
    surface, centred in x."""
    ny = int(round(nx * 1400 / 6800))
    g = Grid(2, (nx, ny), 0)
    c = marmousi_like(g, seed)
    return g, c, paper_params(g, c, ppw=ppw)


def config_2d_layered(n_interior: int = 1024, npml: int = 32, seed: int = SEED_BASE + 1000):
    """1024^2 interior + 32-cell PML, layered 1.5-4.5 background with a +-15%
    Gaussian random field (correlation 20 cells), ppw 8 w.r.t. c_min."""
    g = Grid(2, (n_interior, n_interior), npml)
    c = layered_grf(g, seed)
    return g, c, paper_params(g, c, ppw=8.0)


def config_3d_homogeneous(n_interior: int = 256, npml: int = 16):
    g = Grid(3, (n_interior,) * 3, npml)
    c = homogeneous(g)
    return g, c, paper_params(g, c, ppw=10.0)


def config_3d_lens(n_interior: int = 256, npml: int = 16):
    g = Grid(3, (n_interior,) * 3, npml)
    c = lens(g)
    return g, c, paper_params(g, c, ppw=10.0)


def config_batched_2d(sources_per_medium: int = 8):
    """The multi-source batch on mixed 2D grids: eight seeded layered + GRF media
    (as the 2D layered workload, ppw 8), three of 256^2 and three of 512^2
    interior cells with a 16-cell PML and two of 1024^2 with a 32-cell PML, each
    with `sources_per_medium` Gaussian sources at seeded interior positions (64
    sources in all).  Returns a list of (grid, c, params, centres)."""
    sizes = [(256, 16)] * 3 + [(512, 16)] * 3 + [(1024, 32)] * 2
    out = []
    for i, (n, p) in enumerate(sizes):
        g = Grid(2, (n, n), p)
        c = layered_grf(g, SEED_BASE + 3000 + i)
        out.append((g, c, paper_params(g, c, ppw=8.0),
                    random_centers(g, sources_per_medium, seed=SEED_BASE + 3100 + i)))
    return out


def config_batched_3d(n_interior: int = 400, npml: int = 16, sources: int = 8):
    """The 3D part of the multi-source batch: a seeded layered + GRF medium on
    400^3 interior cells with a 16-cell PML (432^3 unknowns), ppw 8, with
    `sources` Gaussian sources at seeded interior positions."""
    g = Grid(3, (n_interior,) * 3, npml)
    c = layered_grf(g, SEED_BASE + 3200)
    return g, c, paper_params(g, c, ppw=8.0), random_centers(g, sources, seed=SEED_BASE + 3300)


# ---- learned preconditioning stage: seeded initial weights ----

CNN_LAYERS = [  # (c_in, c_out, stride, upsample_input, relu), input order of the flat vector
    (3, 32, 1, False, True),
    (32, 64, 2, False, True),
    (64, 64, 1, False, True),
    (64, 64, 1, False, True),
    (64, 32, 1, True, True),
    (32, 2, 1, False, False),
]


def cnn_initial_params(seed: int) -> np.ndarray:
    """He-normal initial weights (std sqrt(2 / fan_in)), zero biases, flat float32
    vector in layer order W1, b1, ..., W6, b6 (W as [c_out][c_in][3][3])."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co, _, _, _ in CNN_LAYERS:
        parts.append(rng.standard_normal(co * ci * 9) * math.sqrt(2.0 / (ci * 9)))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)
