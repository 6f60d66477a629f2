"""Pins for the oracle's resampling steps (iii)-(vii) (CPU only).

The resampling method approximates the demodulation integrals of Sec. 2, so
the oracle is pinned by the exact definition (brute-force eqs. Fa_DET,
Fb_DET on tiny inputs), by closed forms (matched noise-free template gives
2F = rho^2, interpolation of band-limited tones, integer-shift special
cases) and by direct DFT sums for the FFT bin convention.
"""

import math

import numpy as np
import pytest

from oracle import demod, geometry, metrics, resamp, synth
from workloads import small_target


def _in_band(t):
    half = t.n_fft // 2
    lim = int(0.4 * t.n_fft)
    return np.arange(half - lim, half + lim)


def test_timing_inversion_residual_and_monotonic():
    t = small_target(n_samples=20000, dt=1.0, n_det=2, seed=1)
    a, d = t.skies[0]
    t_b = resamp.ssb_times(t, a, d)
    for det in t.detectors:
        T = resamp.step_iv(t, t_b, det, a, d)
        res = T + geometry.roemer_delay(T, det, a, d, t.ephemeris) - t_b
        assert np.max(np.abs(res)) < 1e-9
        assert np.all(np.diff(T) > 0)


def test_dirichlet_weight_cardinal_even_and_sinc_limit():
    m = np.arange(-8, 9, dtype=np.float64)
    w = resamp.dirichlet_weight(m, 4096, 8)
    assert np.allclose(w, (m == 0).astype(float), atol=1e-13)
    x = np.linspace(-8.5, 8.5, 341)
    assert np.allclose(resamp.dirichlet_weight(x, 4096, 8), resamp.dirichlet_weight(-x, 4096, 8),
                       atol=1e-15)
    # N -> infinity and D -> infinity (taper -> 1): the kernel tends to sinc.
    assert np.allclose(resamp.dirichlet_weight(x, 10**12, 10**9), np.sinc(x), atol=1e-9)


@pytest.mark.parametrize("nu", [0.05, 0.2, 0.35, 0.4, -0.4])
def test_tone_interpolation_error(nu):
    # A complex tone well inside the band is reproduced to <= 5e-3.
    n = 2048
    rng = np.random.default_rng(3)
    z = np.exp(2j * np.pi * nu * np.arange(n))
    u = rng.uniform(100, n - 100, 4000)
    zi, valid = resamp.step_v(z, u, 8)
    assert valid.all()
    assert np.max(np.abs(zi - np.exp(2j * np.pi * nu * u))) < 5e-3


def test_step_v_integer_positions_and_validity():
    rng = np.random.default_rng(4)
    z = rng.standard_normal(100) + 1j * rng.standard_normal(100)
    u = np.array([-0.6, -0.4, 0.0, 17.0, 99.0, 99.4, 99.6])
    zi, valid = resamp.step_v(z, u, 8)
    assert list(valid) == [False, True, True, True, True, True, False]
    assert zi[0] == 0 and zi[-1] == 0
    assert zi[2] == z[0] and zi[3] == z[17] and zi[4] == z[99]


def test_resampled_white_noise_spectrum_is_flat_in_band():
    # Resampled unit white noise keeps unit power in |nu| < 0.4 (to 1%).
    rng = np.random.default_rng(8)
    n = 1 << 14
    acc = np.zeros(n)
    for _ in range(16):
        z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2)
        u = np.arange(n) + rng.uniform(-0.5, 0.5) + 0.37 * np.sin(np.arange(n) / 700.0)
        zi, valid = resamp.step_v(z, u, 8)
        acc += np.abs(np.fft.fft(zi[64:-64], n=n)) ** 2 / (n - 128)
    spec = np.fft.fftshift(acc / 16)
    nu = (np.arange(n) - n // 2) / n
    # bands of width 0.05 in |nu| hold ~26k periodogram samples: sd ~ 0.006
    for lo in np.arange(0.0, 0.4, 0.05):
        sel = (np.abs(nu) >= lo) & (np.abs(nu) < lo + 0.05)
        assert abs(spec[sel].mean() - 1.0) < 0.02
    assert abs(spec[np.abs(nu) < 0.4].mean() - 1.0) < 0.01


def test_fft_bin_convention_matches_direct_dft():
    t = small_target(n_samples=3001, dt=2.0, n_fft=1 << 13, n_det=2, seed=2,
                     f1dots=(-2e-10,), f2dots=(1e-15,))
    x = synth.make_data(t)
    a, d = t.skies[0]
    prep = resamp.sky_prep(t, x, a, d)
    full = resamp.twoF(t, prep, -2e-10, 1e-15)
    bins = np.array([0, 1, 17, t.n_fft // 2 - 1, t.n_fft // 2, t.n_fft // 2 + 5, t.n_fft - 1])
    spot = resamp.twoF_at_bins(t, prep, -2e-10, 1e-15, bins)
    assert np.allclose(full[bins], spot, rtol=1e-9, atol=1e-9)


def test_zero_input_gives_zero():
    t = small_target(n_samples=500, n_fft=1 << 10, seed=3)
    x = [np.zeros(t.n_samples, dtype=np.complex128) for _ in t.detectors]
    prep = resamp.sky_prep(t, x, *t.skies[0])
    assert np.all(resamp.twoF(t, prep, 0.0, 0.0) == 0.0)


@pytest.mark.parametrize("seed,f1,f2", [(3, 0.0, 0.0), (5, -3e-9, 0.0), (6, -1e-9, 3e-13)])
def test_bruteforce_matched_template_gives_rho2(seed, f1, f2):
    # Noise-free data and the matched template: Fa = e^{i phi0}(A Aa + C Ab),
    # Fb = e^{i phi0}(C Aa + B Ab), hence 2F = 2 A^dag M A = rho^2 exactly.
    t = small_target(n_samples=4096, dt=1.0, n_fft=1 << 13, n_det=2, n_inj=1,
                     rho2_range=(100.0, 100.0), seed=seed, f1dots=(f1,), f2dots=(f2,))
    inj = t.injections[0]
    x = synth.make_data(t, noise=False)
    a, d = t.skies[0]
    bf = demod.demod_twoF(t, x, a, d, inj.f1dot, inj.f2dot, [inj.f0])
    assert abs(bf[0] - inj.rho2) < 1e-8 * inj.rho2


@pytest.mark.parametrize("seed,f1,f2", [(3, 0.0, 0.0), (5, -3e-9, 0.0), (6, -1e-9, 3e-13)])
def test_resampling_recovers_rho2_noise_free(seed, f1, f2):
    # On-bin, in-band injection: resampling loses at most 1% of rho^2, and the
    # peak sits on the injected bin.  (It can exceed rho^2 by a few 1e-4: the
    # valid SSB samples and the detector samples differ at the span edges.)
    t = small_target(n_samples=4096, dt=1.0, n_fft=1 << 13, n_det=2, n_inj=1,
                     rho2_range=(100.0, 100.0), seed=seed, f1dots=(f1,), f2dots=(f2,))
    inj = t.injections[0]
    x = synth.make_data(t, noise=False)
    a, d = t.skies[0]
    prep = resamp.sky_prep(t, x, a, d)
    tf = resamp.twoF(t, prep, inj.f1dot, inj.f2dot)
    assert int(np.argmax(tf)) == inj.bin_index
    assert 0.99 <= tf[inj.bin_index] / inj.rho2 <= 1.005


def test_resampling_agrees_with_bruteforce_demodulation():
    # Noisy data, spindown template, 2 detectors: the resampled 2F follows
    # the exact definition within the interpolation loss at in-band bins.
    t = small_target(n_samples=4096, dt=1.0, n_fft=1 << 13, n_det=2, n_inj=1,
                     rho2_range=(60.0, 60.0), seed=4, f1dots=(-3e-9,), f2dots=(2e-13,))
    inj = t.injections[0]
    x = synth.make_data(t, noise=True)
    a, d = t.skies[0]
    prep = resamp.sky_prep(t, x, a, d)
    tf = resamp.twoF(t, prep, inj.f1dot, inj.f2dot)
    rng = np.random.default_rng(0)
    bins = np.concatenate([np.sort(rng.choice(_in_band(t), 200, replace=False)), [inj.bin_index]])
    bf = demod.demod_twoF(t, x, a, d, inj.f1dot, inj.f2dot, t.freq(bins))
    rs = tf[bins]
    assert np.all(np.abs(rs - bf) <= 0.02 * bf + 0.05)
    assert metrics.r1(rs, bf) < 5e-3
    assert metrics.r2(rs, bf) < 5e-3
    assert metrics.theta(rs, bf) < 5e-3


def test_spindown_template_selects_injection():
    # The injection's own f1dot gives the largest 2F among neighbouring templates.
    t = small_target(n_samples=8192, dt=1.0, n_fft=1 << 14, n_det=1, n_inj=1,
                     rho2_range=(200.0, 200.0), seed=12, f1dots=(-2e-8,), f2dots=(0.0,))
    inj = t.injections[0]
    x = synth.make_data(t, noise=False)
    prep = resamp.sky_prep(t, x, *t.skies[0])
    step = 1.0 / (4.0 * t.t_span ** 2)
    peaks = [resamp.twoF(t, prep, inj.f1dot + k * step * 8, 0.0).max() for k in (-2, -1, 0, 1, 2)]
    assert int(np.argmax(peaks)) == 2
    assert peaks[2] > 0.99 * inj.rho2
