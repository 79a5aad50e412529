"""Pins of the oracle's point currents (Eq. 1 with J != 0): the brute-force step matrix, and cavity
resonances read from a probed time series against the discrete dispersion relation."""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.test_oracle_pins import DT, rand_coefs, state
from tests.yee_matrix import YeeSpace, mode_frequencies, one_step_matrix

# half-cell coordinates of (comp, i, j, k): Ex (2i+1, 2j, 2k), Ey (2i, 2j+1, 2k), Ez (2i, 2j, 2k+1)
def half(comp, i, j, k):
    q = [2 * i, 2 * j, 2 * k]
    q[comp] += 1
    return tuple(q)


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 4, 5)])
def test_sources_follow_matrix_recursion(dims):
    """x_{n+1} = M x_n + J^{n+1/2} b with b = -ce dx at the source's E unknown (assembled from Yee
    positions, not from the oracle's loops)."""
    import oracle
    nx, ny, nz = dims
    sp = YeeSpace(nx, ny, nz)
    ce, ch = rand_coefs(60, nx, ny, nz)
    M, _, _ = one_step_matrix(sp, ce, ch)
    nh = len(sp.h_pts)
    sources = [(2, 1, 2, 1), (0, 1, 1, 2), (1, 2, 1, 1)]     # an interior Ez, Ex, Ey
    dx = 0.75
    rng = np.random.default_rng(61)
    wave = rng.uniform(-1, 1, (len(sources), 6))
    f = state(62, nx, ny, nz)
    x = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    n0, nsteps = 2, 7                                          # waveform indices 2..8; zero from 6 on
    oracle.step_sources(f, ce, ch, nsteps, sources, wave, n0=n0, dx=dx)
    for n in range(nsteps):
        x = M @ x
        t = n0 + n
        for s, (c, i, j, k) in enumerate(sources):
            if t < wave.shape[1]:
                x[nh + sp.e_idx[half(c, i, j, k)]] -= ce[c][k, j, i] * dx * wave[s, t]
    y = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    assert np.max(np.abs(x - y)) <= 1e-13


def test_zero_current_is_the_plain_step():
    import oracle
    nx, ny, nz = 7, 6, 5
    ce, ch = rand_coefs(70, nx, ny, nz)
    f = state(71, nx, ny, nz)
    g = [a.copy() for a in f]
    oracle.step(f, ce, ch, 5)
    oracle.step_sources(g, ce, ch, 5, [(2, 3, 3, 2)], np.zeros((1, 5)))
    for a, b in zip(f, g):
        assert np.array_equal(a, b)


def pulse(n_len, width, delay):
    """Derivative of a Gaussian (zero mean: no static charge is left behind), unit peak."""
    t = np.arange(n_len, dtype=np.float64)
    g = -(t - delay) / width * np.exp(-0.5 * ((t - delay) / width) ** 2)
    return g / np.max(np.abs(g))


def spectrum_peaks(trace, count, w_max):
    """omega*dt of the `count` strongest local maxima of the Hann-windowed spectrum below w_max."""
    w = np.hanning(len(trace))
    p = np.abs(np.fft.rfft(trace * w))
    top = int(w_max * len(trace) / (2 * np.pi))
    peaks = [n for n in range(2, min(top, len(p) - 1)) if p[n] > p[n - 1] and p[n] >= p[n + 1]]
    peaks.sort(key=lambda n: -p[n])
    return [2 * np.pi * n / len(trace) for n in peaks[:count]], 2 * np.pi / len(trace)


def test_driven_cavity_resonances_match_dispersion():
    """A short pulse of Ez current in a vacuum cavity rings at the cavity's discrete modes: the strongest
    peaks of a probed Ez trace sit on frequencies of the Yee dispersion relation, and once the current is
    off the discrete energy stays constant."""
    import oracle
    nx, ny, nz = 12, 10, 8
    f = [np.zeros((nz + 1, ny + 1, nx + 1)) for _ in range(6)]
    src = [(2, 3, 4, 2)]
    wave = pulse(200, 12.0, 50.0)[None, :]   # spectrum mostly below omega*dt = 0.2
    trace, energy = [], []
    N = 4096
    for n in range(N):
        oracle.step_sources(f, DT, DT, 1, src, wave, n0=n)
        trace.append(f[2][5, 6, 8])
        if n >= 200 and n % 128 == 0:
            energy.append(oracle.energy(f, DT, DT, DT))
    # below 0.21 the modes of this cavity are >= 4 FFT bins apart (0.1177 = TM110, 0.1356, 0.1445, ...)
    modes = mode_frequencies(nx, ny, nz, DT, DT, DT)
    peaks, bin_w = spectrum_peaks(np.array(trace), 3, 0.21)
    assert len(peaks) == 3
    for w in peaks:
        assert np.min(np.abs(modes - w)) <= bin_w, (w, modes[np.argmin(np.abs(modes - w))])
    e = np.array(energy)
    assert e[0] > 0 and np.max(np.abs(e - e[0])) <= 1e-12 * e[0]
