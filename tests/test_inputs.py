"""The seeded input recipe (no GPU, no oracle arithmetic): the media, sources
and parameter rules that both the oracle and the CUDA path consume."""
import math

import numpy as np

from paper_2506_03617_gb300 import inputs as I


def test_media_are_seeded_and_in_range():
    g = I.Grid(2, (200, 120), 8)
    a = I.layered_grf(g, seed=5)
    b = I.layered_grf(g, seed=5)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, I.layered_grf(g, seed=6))
    assert a.shape == g.shape
    assert a.min() >= 1.5 * (1 - 0.15) - 1e-12 and a.max() <= 4.5 * (1 + 0.15) + 1e-12
    # the PML repeats the nearest interior value
    assert np.array_equal(a[:8], np.broadcast_to(a[8], a[:8].shape))
    assert np.array_equal(a[:, -8:], np.broadcast_to(a[:, -9:-8], a[:, -8:].shape))


def test_marmousi_like_water_layer_and_aspect():
    g, c, p = I.config_2d_marmousi_like(nx=680)
    assert g.ni == (680, 140) and g.npml == 0
    rows = int(round(0.13 * 140))
    assert np.all(c[:rows] == 1.5) and np.all(c[rows:] > 1.5 * 0.9)
    gp = I.Grid(2, (680, 140), 10)
    cp = I.marmousi_like(gp, I.SEED_BASE + 8000)
    assert np.all(cp[:10 + rows] == 1.5)               # the top PML holds water too
    assert I.MARMOUSI_BC[2] == "sound_hard" and set(I.MARMOUSI_BC) - {"sound_hard"} == {"absorbing"}


def test_paper_parameter_rules():
    g = I.Grid(2, (1024, 1024), 32)
    c = I.layered_grf(g, seed=I.SEED_BASE + 1000)
    p = I.paper_params(g, c, ppw=8.0)
    h = 1.0 / 1024
    assert math.isclose(p.omega, 2 * math.pi * c.min() / (8 * h))
    assert math.isclose(p.t, 40 * h * h)
    assert math.isclose(p.shift, 8 * h)                 # s = 1 / freq, freq = 1 / (ppw h)
    assert p.cpml == 20.0 and p.fprtol == 0.08


def test_gaussian_source_is_normalised_and_centred():
    g = I.Grid(2, (64, 48), 6)
    f = I.gaussian_source(g)
    assert math.isclose(f.sum() * g.h ** 2, 1.0, rel_tol=1e-6)
    j, i = np.unravel_index(np.argmax(f), f.shape)
    assert abs(g.node_coords(0)[i] - 0.5 * 64 * g.h) <= g.h and abs(g.node_coords(1)[j] - 0.5 * 48 * g.h) <= g.h
    b = I.rhs_from_source(f)
    assert b.dtype == np.complex128 and np.array_equal(b, -f)
