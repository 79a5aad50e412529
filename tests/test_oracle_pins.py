"""Pins of the FP64 oracle to facts the Yee scheme fixes (CPU only).

Each test checks the oracle against something other than itself: closed-form
eigenmodes, exact invariants, brute force from a position-based operator
constructor, reversibility, symmetry, locality, and an independent NumPy
restatement in the slicing style of the paper's Listing 3.
"""
import math

import numpy as np
import pytest

import cavity_inputs as ci
from tests import yee_closed_forms as cf
from tests.yee_matrix import YeeSpace, mode_frequencies, one_step_matrix

DT = ci.COURANT_HALF_DT


def rand_coefs(seed, nx, ny, nz, lo=0.5, hi=1.0):
    """Per-position positive coefficients (scaled by dt), distinct per component."""
    rng = np.random.default_rng(seed)
    sh = (nz + 1, ny + 1, nx + 1)
    ce = [DT * rng.uniform(lo, hi, sh) for _ in range(3)]
    ch = [DT * rng.uniform(lo, hi, sh) for _ in range(3)]
    return ce, ch


def state(seed, nx, ny, nz):
    import oracle
    return oracle.as_f64(ci.random_fields(seed, nx, ny, nz))


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ---------------------------------------------------------------- eigenmodes
@pytest.mark.parametrize("dims,steps", [((32, 32, 32), 100), ((12, 10, 7), 60), ((5, 9, 3), 41)])
def test_tm110_closed_form(oracle_mod, dims, steps):
    nx, ny, nz = dims
    f, w = cf.tm110(nx, ny, nz, DT, 0)
    oracle_mod.step(f, DT, DT, steps)
    g, _ = cf.tm110(nx, ny, nz, DT, steps)
    for c in range(6):
        assert np.max(np.abs(f[c] - g[c])) <= 1e-12, ci.COMPONENTS[c]
    if dims == (32, 32, 32):
        # discrete omega vs continuum pi*sqrt(2)/32 at 32^3, dt = 0.5/sqrt(3)
        assert abs(w - 0.138794) < 5e-6 and abs(w - math.pi * math.sqrt(2) / 32) < 1e-4


@pytest.mark.parametrize("dims,steps", [((10, 7, 12), 77), ((32, 4, 16), 50)])
def test_te101_closed_form(oracle_mod, dims, steps):
    nx, ny, nz = dims
    f, _ = cf.te101(nx, ny, nz, DT, 0)
    oracle_mod.step(f, DT, DT, steps)
    g, _ = cf.te101(nx, ny, nz, DT, steps)
    for c in range(6):
        assert np.max(np.abs(f[c] - g[c])) <= 1e-12, ci.COMPONENTS[c]


def test_mode_with_scaled_coefficients(oracle_mod):
    # dielectric-filled cavity: ce = dt/(eps dx) scalar, eps = 2.25 -> lower frequency
    nx, ny, nz = 9, 11, 4
    ce, ch = DT / 2.25, DT
    f, w = cf.tm110(nx, ny, nz, DT, 0, ce=ce, ch=ch)
    oracle_mod.step(f, ce, ch, 30)
    g, w2 = cf.tm110(nx, ny, nz, DT, 30, ce=ce, ch=ch)
    for c in range(6):
        assert np.max(np.abs(f[c] - g[c])) <= 1e-12


# ---------------------------------------------------------------- invariants
def test_energy_conserved_random_init_spheres(oracle_mod):
    nx, ny, nz = 32, 32, 32
    sph = ci.sphere_list(1, 4, (nx, ny, nz), 3.0, 9.0)
    ce, ch = ci.sphere_coefficients(sph, nx, ny, nz, DT)
    ce = [c.astype(np.float64) for c in ce]
    f = state(0, nx, ny, nz)
    w0 = oracle_mod.energy(f, ce, ch, DT)
    for _ in range(4):
        oracle_mod.step(f, ce, ch, 25)
        w = oracle_mod.energy(f, ce, ch, DT)
        assert abs(w - w0) / w0 <= 1e-12
    assert w0 > 0


def test_energy_conserved_per_position_h_coefficients(oracle_mod):
    nx, ny, nz = 7, 6, 9
    ce, ch = rand_coefs(3, nx, ny, nz)
    f = state(4, nx, ny, nz)
    w0 = oracle_mod.energy(f, ce, ch, DT)
    oracle_mod.step(f, ce, ch, 200)
    assert abs(oracle_mod.energy(f, ce, ch, DT) - w0) / w0 <= 1e-12


def test_plain_field_energy_not_conserved(oracle_mod):
    # the naive 1/2 sum(eps E^2 + mu H^2) oscillates; the Yee invariant above does not
    nx, ny, nz = 8, 8, 8
    f = state(5, nx, ny, nz)
    naive = lambda g: 0.5 * sum(float(np.sum(a * a)) for a in g)
    n0 = naive(f)
    oracle_mod.step(f, DT, DT, 10)
    assert abs(naive(f) - n0) / n0 > 1e-6


def test_divergence_invariant(oracle_mod):
    nx, ny, nz = 9, 8, 7
    ce, ch = rand_coefs(6, nx, ny, nz)
    f = state(7, nx, ny, nz)
    de0, dh0 = oracle_mod.divergence(f, ce, ch)
    assert np.abs(de0).max() > 0.1 and np.abs(dh0).max() > 0.1   # random init is not divergence-free
    oracle_mod.step(f, ce, ch, 100)
    de, dh = oracle_mod.divergence(f, ce, ch)
    assert np.abs(de - de0).max() <= 1e-12 * np.abs(de0).max() * 100
    assert np.abs(dh - dh0).max() <= 1e-12 * np.abs(dh0).max() * 100


def test_pec_tangential_zero_and_normal_h_constant(oracle_mod):
    nx, ny, nz = 6, 5, 7
    ce, ch = rand_coefs(8, nx, ny, nz)
    f = state(9, nx, ny, nz)
    faces0 = (f[3][:, :, [0, nx]].copy(), f[4][:, [0, ny], :].copy(), f[5][[0, nz], :, :].copy())
    for _ in range(20):
        oracle_mod.step(f, ce, ch, 1)
        for c, name in enumerate(("Ex", "Ey", "Ez")):
            t = ci.tangential_e_mask(name, nx, ny, nz)
            assert np.all(f[c][t] == 0.0)
        # normal H on faces is bit-constant
        assert np.array_equal(f[3][:nz, :ny, [0, nx]], faces0[0][:nz, :ny])
        assert np.array_equal(f[4][:nz, [0, ny], :nx], faces0[1][:nz, :, :nx])
        assert np.array_equal(f[5][[0, nz], :ny, :nx], faces0[2][:, :ny, :nx])


def test_time_reversible(oracle_mod):
    nx, ny, nz = 8, 7, 6
    ce, ch = rand_coefs(10, nx, ny, nz)
    f = state(11, nx, ny, nz)
    f0 = [a.copy() for a in f]
    oracle_mod.step(f, ce, ch, 50)
    for _ in range(50):   # inverse of one step: E -= ce curl H, then H += ch curl E
        oracle_mod.update_e(f, [-c for c in ce])
        oracle_mod.update_h(f, [-c for c in ch])
    for c in range(6):
        assert np.max(np.abs(f[c] - f0[c])) <= 1e-11


def test_cyclic_axis_symmetry(oracle_mod):
    n = 7
    ce, ch = rand_coefs(12, n, n, n)
    f = state(13, n, n, n)
    rot = lambda a: np.ascontiguousarray(np.transpose(a, (1, 2, 0)))
    # x -> y -> z -> x : new_y = rot(old_x), new_z = rot(old_y), new_x = rot(old_z)
    rot3 = lambda v: [rot(v[2]), rot(v[0]), rot(v[1])]
    g = rot3(f[:3]) + rot3(f[3:])
    ceg, chg = rot3(ce), rot3(ch)
    oracle_mod.step(f, ce, ch, 13)
    oracle_mod.step(g, ceg, chg, 13)
    fr = rot3(f[:3]) + rot3(f[3:])
    for c in range(6):
        assert np.array_equal(fr[c], g[c]), ci.COMPONENTS[c]


def test_locality_subbox_core_matches(oracle_mod):
    """After s steps a value depends only on inputs within s+1 cells (light cone).

    A sub-box run with its own PEC walls matches the full run away from the cut faces;
    the full-size GPU parity tests rely on this to check sampled outputs.
    """
    nx, ny, nz = 20, 18, 16
    ce, ch = rand_coefs(14, nx, ny, nz)
    f = state(15, nx, ny, nz)
    a, b = (4, 3, 2), (16, 15, 14)          # sub-box cells [a, b)
    s = 3
    sl = (slice(a[2], b[2] + 1), slice(a[1], b[1] + 1), slice(a[0], b[0] + 1))
    g = [np.ascontiguousarray(x[sl]) for x in f]
    ceg = [np.ascontiguousarray(x[sl]) for x in ce]
    chg = [np.ascontiguousarray(x[sl]) for x in ch]
    oracle_mod.pec_e(g)
    oracle_mod.step(f, ce, ch, s)
    oracle_mod.step(g, ceg, chg, s)
    m = s + 2
    core = (slice(m, -m), slice(m, -m), slice(m, -m))
    for c in range(6):
        assert np.array_equal(g[c][core], f[c][sl][core])


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 4, 5)])
def test_bruteforce_matrix_matches_oracle(oracle_mod, dims):
    nx, ny, nz = dims
    sp = YeeSpace(nx, ny, nz)
    ce, ch = rand_coefs(20, nx, ny, nz)
    M, CE, CH = one_step_matrix(sp, ce, ch)
    f = state(21, nx, ny, nz)
    x = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    oracle_mod.step(f, ce, ch, 1)
    y = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    assert np.max(np.abs(M @ x - y)) <= 1e-14
    # every canonical entry the unknowns do not cover is untouched/zero in E
    for c, name in enumerate(("Ex", "Ey", "Ez")):
        assert np.all(f[c][ci.tangential_e_mask(name, nx, ny, nz)] == 0.0)


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 4, 5)])
def test_bruteforce_operator_structure(dims):
    nx, ny, nz = dims
    sp = YeeSpace(nx, ny, nz)
    CE, CH = sp.curl_e(), sp.curl_h()
    assert np.array_equal(CH, CE.T)                       # discrete curls are adjoint under PEC
    assert np.abs(sp.div_nodes() @ CH).max() == 0.0        # div curl H = 0 at interior nodes
    assert np.abs(sp.div_cells() @ CE).max() == 0.0        # div curl E = 0 in every cell


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 4, 5)])
def test_bruteforce_spectrum_matches_dispersion(oracle_mod, dims):
    nx, ny, nz = dims
    sp = YeeSpace(nx, ny, nz)
    sh = (nz + 1, ny + 1, nx + 1)
    ce = [np.full(sh, DT)] * 3
    ch = [np.full(sh, DT)] * 3
    # build M column by column from the ORACLE (not from the constructor) and check its spectrum
    nh, ne = len(sp.h_pts), len(sp.e_pts)
    M = np.zeros((nh + ne, nh + ne))
    for col in range(nh + ne):
        x = np.zeros(nh + ne); x[col] = 1.0
        f = [np.zeros(sh) for _ in range(6)]
        sp.scatter(x[:nh], f, sp.h_pts, 3)
        sp.scatter(x[nh:], f, sp.e_pts, 0)
        oracle_mod.step(f, ce, ch, 1)
        M[:, col] = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    lam = np.linalg.eigvals(M)
    assert np.max(np.abs(np.abs(lam) - 1.0)) < 1e-9
    ang = np.sort(np.angle(lam[lam.imag > 1e-9]))
    expect = mode_frequencies(nx, ny, nz, DT, DT, DT)
    assert ang.shape == expect.shape
    assert np.max(np.abs(ang - expect)) < 1e-9
    n_static = int(np.sum(np.abs(lam - 1.0) < 1e-9))
    assert n_static == nh + ne - 2 * len(expect)


# ---------------------------------------------------------------- NumPy restatement
def numpy_step(f, ce, ch):
    """Whole-array slicing restatement of Eq. 2 in the style of Listing 3 (arrays are [k, j, i])."""
    Ex, Ey, Ez, Hx, Hy, Hz = f
    cex, cey, cez = ce
    chx, chy, chz = ch
    nz, ny, nx = Ex.shape[0] - 1, Ex.shape[1] - 1, Ex.shape[2] - 1
    s = np.s_
    Hx[s[:nz, :ny, :]] -= chx[s[:nz, :ny, :]] * ((Ez[s[:nz, 1:, :]] - Ez[s[:nz, :ny, :]])
                                                 - (Ey[s[1:, :ny, :]] - Ey[s[:nz, :ny, :]]))
    Hy[s[:nz, :, :nx]] -= chy[s[:nz, :, :nx]] * ((Ex[s[1:, :, :nx]] - Ex[s[:nz, :, :nx]])
                                                 - (Ez[s[:nz, :, 1:]] - Ez[s[:nz, :, :nx]]))
    Hz[s[:, :ny, :nx]] -= chz[s[:, :ny, :nx]] * ((Ey[s[:, :ny, 1:]] - Ey[s[:, :ny, :nx]])
                                                 - (Ex[s[:, 1:, :nx]] - Ex[s[:, :ny, :nx]]))
    Ex[s[1:nz, 1:ny, :nx]] += cex[s[1:nz, 1:ny, :nx]] * (
        (Hz[s[1:nz, 1:ny, :nx]] - Hz[s[1:nz, :ny - 1, :nx]]) - (Hy[s[1:nz, 1:ny, :nx]] - Hy[s[:nz - 1, 1:ny, :nx]]))
    Ey[s[1:nz, :ny, 1:nx]] += cey[s[1:nz, :ny, 1:nx]] * (
        (Hx[s[1:nz, :ny, 1:nx]] - Hx[s[:nz - 1, :ny, 1:nx]]) - (Hz[s[1:nz, :ny, 1:nx]] - Hz[s[1:nz, :ny, :nx - 1]]))
    Ez[s[:nz, 1:ny, 1:nx]] += cez[s[:nz, 1:ny, 1:nx]] * (
        (Hy[s[:nz, 1:ny, 1:nx]] - Hy[s[:nz, 1:ny, :nx - 1]]) - (Hx[s[:nz, 1:ny, 1:nx]] - Hx[s[:nz, :ny - 1, 1:nx]]))


def test_numpy_restatement_agrees(oracle_mod):
    nx, ny, nz = 13, 9, 11
    ce, ch = rand_coefs(30, nx, ny, nz)
    f = state(31, nx, ny, nz)
    g = [a.copy() for a in f]
    oracle_mod.step(f, ce, ch, 17)
    for _ in range(17):
        numpy_step(g, ce, ch)
    for c in range(6):
        m = ci.extent_mask(ci.COMPONENTS[c], nx, ny, nz)
        assert np.max(np.abs(f[c][m] - g[c][m])) <= 1e-14 * 17


def test_omp_build_bitwise_equal(oracle_mod):
    nx, ny, nz = 24, 20, 18
    ce, ch = rand_coefs(40, nx, ny, nz)
    f = state(41, nx, ny, nz)
    g = [a.copy() for a in f]
    oracle_mod.step(f, ce, ch, 9, omp=False)
    oracle_mod.step(g, ce, ch, 9, omp=True)
    for c in range(6):
        assert np.array_equal(f[c], g[c])
