"""Pins of the oracle's fourth-order scheme (staggered (2,4) differences, image-closed PEC walls).

Sec. 6 of the paper names higher-order schemes without fixing one, so the oracle's
reading is pinned by what that reading implies mathematically: it reduces to Eq. 2
when (c1, c2) = (1, 0); its one-step matrix equals one assembled from grid
positions alone; its spectrum is the fourth-order dispersion relation of the
cavity's standing waves; closed-form eigenmodes evolve exactly; the discrete
energy and divergences are invariant; the step is time reversible; and its
frequencies approach the continuum far faster than the second-order scheme's.
"""
import math

import numpy as np
import pytest

import cavity_inputs as ci
from tests import yee_closed_forms as cf
from tests.test_oracle_pins import DT, rand_coefs, state
from tests.yee_matrix import YeeSpace, mode_frequencies, one_step_matrix


def test_second_order_coefficients_give_eq2_bitwise(oracle_mod):
    """(c1, c2) = (1, 0) must be the second-order step exactly: same extents, signs and indices."""
    for dims in ((7, 6, 5), (3, 4, 9), (1, 2, 3)):
        nx, ny, nz = dims
        ce, ch = rand_coefs(80, nx, ny, nz)
        f = state(81, nx, ny, nz)
        g = [a.copy() for a in f]
        oracle_mod.step(f, ce, ch, 6)
        oracle_mod.step4(g, ce, ch, 6, c1=1.0, c2=0.0)
        for c in range(6):
            assert np.array_equal(f[c], g[c]), (dims, ci.COMPONENTS[c])
        w2 = oracle_mod.energy(f, ce, ch, 1.0)
        w4 = oracle_mod.energy4(f, ce, ch, 1.0, c1=1.0, c2=0.0)
        assert abs(w2 - w4) <= 1e-14 * abs(w2)
        d2, h2 = oracle_mod.divergence(f, ce, ch)
        d4, h4 = oracle_mod.divergence4(f, ce, ch, c1=1.0, c2=0.0)
        assert np.max(np.abs(d2 - d4)) <= 1e-12 and np.max(np.abs(h2 - h4)) <= 1e-12


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 4, 5), (2, 5, 3)])
def test_bruteforce_matrix_matches_oracle(oracle_mod, dims):
    nx, ny, nz = dims
    sp = YeeSpace(nx, ny, nz, order=4)
    ce, ch = rand_coefs(82, nx, ny, nz)
    M, CE, CH = one_step_matrix(sp, ce, ch)
    f = state(83, nx, ny, nz)
    x = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    oracle_mod.step4(f, ce, ch, 1)
    y = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    assert np.max(np.abs(M @ x - y)) <= 1e-14
    for c, name in enumerate(("Ex", "Ey", "Ez")):
        assert np.all(f[c][ci.tangential_e_mask(name, nx, ny, nz)] == 0.0)


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 4, 5)])
def test_bruteforce_operator_structure(dims):
    """Under the image closure the two curls are adjoint and div curl = 0, as for Eq. 2."""
    nx, ny, nz = dims
    sp = YeeSpace(nx, ny, nz, order=4)
    CE, CH = sp.curl_e(), sp.curl_h()
    assert np.array_equal(CH, CE.T)
    assert np.abs(sp.div_nodes() @ CH).max() <= 1e-15
    assert np.abs(sp.div_cells() @ CE).max() <= 1e-15


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 4, 5), (5, 3, 6)])
def test_spectrum_matches_fourth_order_dispersion(oracle_mod, dims):
    """The one-step matrix built column by column from the ORACLE has |lambda| = 1 and the angles
    2 asin(sqrt(ce ch sum sigma^2)) with sigma = c1 sin(pi m/2n) + c2 sin(3 pi m/2n), every mode with
    TE/TM multiplicity; everything else is the static subspace (lambda = 1)."""
    nx, ny, nz = dims
    sp = YeeSpace(nx, ny, nz)
    sh = (nz + 1, ny + 1, nx + 1)
    nh, ne = len(sp.h_pts), len(sp.e_pts)
    M = np.zeros((nh + ne, nh + ne))
    for col in range(nh + ne):
        x = np.zeros(nh + ne); x[col] = 1.0
        f = [np.zeros(sh) for _ in range(6)]
        sp.scatter(x[:nh], f, sp.h_pts, 3)
        sp.scatter(x[nh:], f, sp.e_pts, 0)
        oracle_mod.step4(f, DT, DT, 1)
        M[:, col] = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    lam = np.linalg.eigvals(M)
    assert np.max(np.abs(np.abs(lam) - 1.0)) < 1e-9
    ang = np.sort(np.angle(lam[lam.imag > 1e-9]))
    expect = mode_frequencies(nx, ny, nz, DT, DT, DT, order=4)
    assert ang.shape == expect.shape
    assert np.max(np.abs(ang - expect)) < 1e-9
    assert int(np.sum(np.abs(lam - 1.0) < 1e-9)) == nh + ne - 2 * len(expect)


@pytest.mark.parametrize("dims,steps", [((32, 32, 32), 100), ((12, 10, 7), 60), ((5, 9, 3), 41)])
def test_tm110_closed_form(oracle_mod, dims, steps):
    nx, ny, nz = dims
    f, w = cf.tm110(nx, ny, nz, DT, 0, order=4)
    oracle_mod.step4(f, DT, DT, steps)
    g, _ = cf.tm110(nx, ny, nz, DT, steps, order=4)
    for c in range(6):
        assert np.max(np.abs(f[c] - g[c])) <= 1e-12, ci.COMPONENTS[c]


@pytest.mark.parametrize("dims,steps", [((10, 7, 12), 77), ((32, 4, 16), 50)])
def test_te101_closed_form(oracle_mod, dims, steps):
    nx, ny, nz = dims
    f, _ = cf.te101(nx, ny, nz, DT, 0, order=4)
    oracle_mod.step4(f, DT, DT, steps)
    g, _ = cf.te101(nx, ny, nz, DT, steps, order=4)
    for c in range(6):
        assert np.max(np.abs(f[c] - g[c])) <= 1e-12, ci.COMPONENTS[c]


def test_dispersion_error_is_fourth_order():
    """The scheme's point: on a 16-cell cavity the TM110 spatial error of the (2,4) symbol is far below
    the second-order one, and halving the cell shrinks it ~16x (against ~4x for Eq. 2)."""
    from tests.yee_matrix import sigma
    def err(n, order):   # relative error of the spatial symbol of sin(pi x / n), dx = 1
        exact = math.pi / (2 * n)
        return abs(float(sigma(1, n, order)) - exact) / exact
    assert err(16, 4) < err(16, 2) / 50
    assert 14.0 < err(16, 4) / err(32, 4) < 17.0
    assert 3.5 < err(16, 2) / err(32, 2) < 4.5


def test_energy_conserved_per_position_coefficients(oracle_mod):
    nx, ny, nz = 11, 9, 8
    ce, ch = rand_coefs(84, nx, ny, nz)
    f = state(85, nx, ny, nz)
    w0 = oracle_mod.energy4(f, ce, ch, 1.0)
    for _ in range(5):
        oracle_mod.step4(f, ce, ch, 20)
        w = oracle_mod.energy4(f, ce, ch, 1.0)
        assert abs(w - w0) <= 1e-12 * abs(w0)
    # the second-order energy is not the invariant of this scheme
    assert abs(oracle_mod.energy(f, ce, ch, 1.0) - w0) > 1e-6 * abs(w0)


def test_energy_conserved_sphere_workload(oracle_mod):
    dims = (24, 20, 18)
    sph = ci.sphere_list(86, 4, dims, 3.0, 8.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    ce = [c.astype(np.float64) for c in ce]
    f = state(87, *dims)
    w0 = oracle_mod.energy4(f, ce, ch, 1.0)
    oracle_mod.step4(f, ce, ch, 100)
    assert abs(oracle_mod.energy4(f, ce, ch, 1.0) - w0) <= 1e-12 * abs(w0)


def test_divergence_invariant(oracle_mod):
    nx, ny, nz = 9, 10, 7
    ce, ch = rand_coefs(88, nx, ny, nz)
    f = state(89, nx, ny, nz)
    de0, dh0 = oracle_mod.divergence4(f, ce, ch)
    assert np.max(np.abs(de0)) > 0.1 and np.max(np.abs(dh0)) > 0.1   # random init is not divergence free
    oracle_mod.step4(f, ce, ch, 50)
    de, dh = oracle_mod.divergence4(f, ce, ch)
    assert np.max(np.abs(de - de0)) <= 1e-12 * np.max(np.abs(de0))
    assert np.max(np.abs(dh - dh0)) <= 1e-12 * np.max(np.abs(dh0))


def test_pec_tangential_zero_and_normal_h_constant(oracle_mod):
    nx, ny, nz = 8, 7, 6
    ce, ch = rand_coefs(90, nx, ny, nz)
    f = state(91, nx, ny, nz)
    f0 = [a.copy() for a in f]
    oracle_mod.step4(f, ce, ch, 25)
    for c, name in enumerate(("Ex", "Ey", "Ez")):
        assert np.all(f[c][ci.tangential_e_mask(name, nx, ny, nz)] == 0.0)
    assert np.array_equal(f[3][:, :, 0], f0[3][:, :, 0]) and np.array_equal(f[3][:, :, nx], f0[3][:, :, nx])
    assert np.array_equal(f[4][:, 0, :], f0[4][:, 0, :]) and np.array_equal(f[4][:, ny, :], f0[4][:, ny, :])
    assert np.array_equal(f[5][0], f0[5][0]) and np.array_equal(f[5][nz], f0[5][nz])


def test_time_reversible(oracle_mod):
    """Stepping back with -dt, E first then H, retraces the run to roundoff."""
    nx, ny, nz = 7, 8, 6
    ce, ch = rand_coefs(92, nx, ny, nz)
    f = state(93, nx, ny, nz)
    f0 = [a.copy() for a in f]
    n = 30
    oracle_mod.step4(f, ce, ch, n)
    mce, mch = [-c for c in ce], [-c for c in ch]
    for _ in range(n):
        oracle_mod.update_e4(f, mce)
        oracle_mod.pec_e(f)
        oracle_mod.update_h4(f, mch)
    for c in range(6):
        assert np.max(np.abs(f[c] - f0[c])) <= 1e-12


def test_currents_enter_as_in_second_order(oracle_mod):
    """A point current adds -ce dx J after the E update, whatever the difference order: the driven run
    minus the undriven run is the response of the linear step to that injection alone."""
    nx, ny, nz = 6, 5, 7
    ce, ch = rand_coefs(94, nx, ny, nz)
    src = [(2, 3, 2, 4), (0, 2, 3, 3)]
    wave = np.random.default_rng(95).uniform(-1, 1, (2, 5))
    f = state(96, nx, ny, nz)
    g = [a.copy() for a in f]
    oracle_mod.step4(f, ce, ch, 5, sources=src, wave=wave, dx=0.5)
    oracle_mod.step4(g, ce, ch, 5)
    z = [np.zeros_like(a) for a in f]          # zero initial state, driven
    oracle_mod.step4(z, ce, ch, 5, sources=src, wave=wave, dx=0.5)
    for c in range(6):
        assert np.max(np.abs((f[c] - g[c]) - z[c])) <= 1e-13
    # one step from zero: only the source entries move, by -ce dx J
    y = [np.zeros_like(a) for a in f]
    oracle_mod.step4(y, ce, ch, 1, sources=src, wave=wave, dx=0.5)
    for s, (c, i, j, k) in enumerate(src):
        assert y[c][k, j, i] == -ce[c][k, j, i] * 0.5 * wave[s, 0]
