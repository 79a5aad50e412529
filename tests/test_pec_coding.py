"""PEC faces as materials, on the CPU: the coded material ids and table that the two-step kernels read.

Tangential E vanishes on the PEC walls (Sec. 2; the edge steps of Listing 1). The library writes that
condition into the material table:
- a cell on the walls i = 0, j = 0 or k = 0 takes an entry whose E coefficients are zero for the
  components lying in those walls;
- a cell outside the cavity reads id 0, whose entry has ce = 0.

Here the rule is restated from geometry, independently of the library's code: a component lies in a wall
when its axis differs from the wall's normal. Every entry is checked against it. The GPU tests
(`test_gpu_pec_materials.py`) check that the kernels then give the masked results bit for bit.
"""
import itertools

import numpy as np
import pytest

from paper_2504_09118_gb300 import binding as B

AWAY = (5, 9, 13)   # a cell index on no wall, per axis


def walls(i, j, k):
    """Normal axes (0 = x, 1 = y, 2 = z) of the PEC walls the cell (i, j, k) lies on."""
    return [a for a, c in enumerate((i, j, k)) if c == 0]


def expected(tab, m, normals):
    e = tab[m].copy()
    for comp in range(3):
        if any(comp != n for n in normals):   # Ex, Ey or Ez lies in a wall whose normal is another axis
            e[comp] = 0.0
    return e


def random_table(ntab, seed):
    rng = np.random.default_rng(seed)
    t = np.zeros((ntab, 8), np.float32)
    t[:, 0:3] = rng.uniform(0.05, 0.6, (ntab, 3))
    t[:, 4:7] = rng.uniform(0.05, 0.6, (ntab, 3))
    return t


@pytest.mark.parametrize("ntab", [1, 2, 3, 17, 31])
def test_entries_follow_the_wall_geometry(ntab):
    tab = random_table(ntab, ntab)
    coded = B.fdtd_debug_pec_table(tab)
    assert coded.shape == (1 + 8 * ntab, 8)
    seen = {0}
    for m in range(ntab):
        for on in itertools.product((False, True), repeat=3):   # on the x, y, z wall or not
            cell = [0 if on[a] else AWAY[a] for a in range(3)]
            code = B.fdtd_debug_pec_code(ntab, m, *cell)
            assert 1 <= code <= 8 * ntab and code not in seen
            seen.add(code)
            want = expected(tab, m, walls(*cell))
            assert np.array_equal(coded[code][[0, 1, 2, 4, 5, 6]], want[[0, 1, 2, 4, 5, 6]]), (m, on)
    assert seen == set(range(1 + 8 * ntab))   # every entry is reached by exactly one (material, walls)
    # outside the cavity: E stays the zero its box read, H takes material 0's coefficients
    assert np.array_equal(coded[0][0:3], np.zeros(3, np.float32))
    assert np.array_equal(coded[0][4:7], tab[0][4:7])


def test_code_depends_only_on_the_walls():
    for ntab, m in ((4, 0), (4, 3), (31, 30)):
        base = B.fdtd_debug_pec_code(ntab, m, *AWAY)
        assert B.fdtd_debug_pec_code(ntab, m, 100, 7, 2) == base
        assert B.fdtd_debug_pec_code(ntab, m, 0, 7, 2) == B.fdtd_debug_pec_code(ntab, m, 0, 1, 300)
        assert B.fdtd_debug_pec_code(ntab, m, 0, 0, 0) != base


def test_masks_applied_again_change_nothing():
    """Kernels that still apply their PEC masks (batches, the first planes of a tile) multiply the same
    zero: masking a coded entry once more leaves it as it is."""
    ntab = 5
    tab = random_table(ntab, 1)
    coded = B.fdtd_debug_pec_table(tab)
    for m in range(ntab):
        for cell in itertools.product((0, 3), repeat=3):
            e = coded[B.fdtd_debug_pec_code(ntab, m, *cell)]
            again = expected(coded, B.fdtd_debug_pec_code(ntab, m, *cell), walls(*cell))
            assert np.array_equal(e, again)


@pytest.mark.parametrize("args", [(0, 0, 1, 1, 1), (32, 0, 1, 1, 1), (4, 4, 1, 1, 1), (4, -1, 1, 1, 1),
                                  (4, 0, -1, 1, 1), (4, 0, 1, -1, 1), (4, 0, 1, 1, -1)])
def test_code_rejects_bad_arguments(args):
    with pytest.raises(B.FdtdError):
        B.fdtd_debug_pec_code(*args)


@pytest.mark.parametrize("ntab", [32, 40])
def test_table_only_up_to_31_materials(ntab):
    with pytest.raises(B.FdtdError):
        B.fdtd_debug_pec_table(random_table(ntab, 2))
