"""CPU checks of the element-wise comparison used by every GPU parity test: the
PML and face masks select the right cells, and an error planted in a single
PML corner cell, a single interior cell or a single boundary row shows up in
the matching maximum at its own size, where the l2 norm dilutes it."""
import numpy as np

from paper_2506_03617_gb300 import inputs as I

from _parity import errors, face_mask, pml_mask


def test_pml_mask_counts_and_layout():
    for g in (I.Grid(2, (30, 20), 4), I.Grid(3, (7, 6, 5), 2), I.Grid(2, (10, 10), 0)):
        m = pml_mask(g)
        assert m.size == g.n_total
        assert int((~m).sum()) == int(np.prod(g.ni))
    g = I.Grid(2, (30, 20), 4)
    m = pml_mask(g).reshape(g.shape)          # [y][x]
    assert m[0, 10] and m[10, 0] and m[-1, 10] and m[10, -1]
    assert not m[4, 4] and not m[g.n[1] - 5, g.n[0] - 5] and m[3, 4] and m[4, 3]


def test_face_mask_is_the_boundary_rows():
    g = I.Grid(3, (5, 4, 3), 0)
    m = face_mask(g).reshape(g.shape)
    inner = m[1:-1, 1:-1, 1:-1]
    assert not inner.any()
    assert int(m.sum()) == g.n_total - int(np.prod([n - 2 for n in g.n]))


def test_single_wrong_cell_is_seen_at_its_own_size():
    g = I.Grid(2, (200, 150), 16)
    rng = np.random.default_rng(0)
    ref = rng.standard_normal(g.n_total) + 1j * rng.standard_normal(g.n_total)
    scale = np.max(np.abs(ref))
    corner = 0                                   # (x, y) = (0, 0): a PML corner cell
    inner = (g.n[1] // 2) * g.n[0] + g.n[0] // 2
    for cell, key in ((corner, "max_pml"), (inner, "max_int")):
        got = ref.copy()
        got[cell] += 1e-3 * scale
        e = errors(got, ref, g)
        assert abs(e[key] - 1e-3) < 1e-9
        other = "max_int" if key == "max_pml" else "max_pml"
        assert e[other] == 0.0
        assert e["l2"] < 5e-5                    # the norm alone would pass it at a 1e-4 bound
    e = errors(ref, ref, g)
    assert e == {"max_int": 0.0, "max_pml": 0.0, "l2": 0.0}
