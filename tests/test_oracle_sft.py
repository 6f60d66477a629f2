"""Pins for the oracle's step (ii) from SFTs (CPU only).

* a real on-bin tone inside the band comes out as the analytic heterodyned
  complex tone (half amplitude: its negative-frequency image is outside the
  band), sample by sample;
* an on-bin tone outside the band vanishes (the low-pass);
* a mixture of in-band on-bin complex tones is reproduced exactly at every
  sample, segment after segment (the band-limited reconstruction);
* the f_h grid requirement is enforced.
"""

import numpy as np
import pytest

from oracle import sft

T_SFT, M, NB = 8.0, 512, 32          # raw rate 64 Hz, band 4 Hz, dt = 0.25 s
F_H = 10.0                           # q_h = 80


def _xh(x, t_start=3.0):
    sf = sft.sfts_from_series(x, M)
    q_h = int(F_H * T_SFT)
    return sft.xh_from_band(sft.band(sf, q_h - NB // 2, NB), q_h - NB // 2, t_start, T_SFT, M, F_H)


def _t_raw(n_sft, t_start=3.0):
    return t_start + np.arange(n_sft * M) * (T_SFT / M)


def _t_out(n_sft, t_start=3.0):
    return t_start + np.arange(n_sft * NB) * (T_SFT / NB)


def test_in_band_real_tone_becomes_the_heterodyned_tone():
    f = F_H + 5 / T_SFT                  # 5 bins above f_h
    tr = _t_raw(6)
    xh = _xh(np.cos(2 * np.pi * f * tr + 0.3))
    to = _t_out(6)
    # the raw tone's positive-frequency half, heterodyned by exp(-2 pi i f_h t)
    want = 0.5 * np.exp(1j * (2 * np.pi * f * to + 0.3)) * np.exp(-2j * np.pi * F_H * to)
    assert np.max(np.abs(xh - want)) < 1e-12


def test_out_of_band_tone_is_removed():
    f = F_H + 40 / T_SFT                 # 40 bins above f_h, band is +-16
    xh = _xh(np.cos(2 * np.pi * f * _t_raw(4)))
    assert np.max(np.abs(xh)) < 1e-12


def test_in_band_mixture_is_reconstructed_exactly():
    rng = np.random.default_rng(3)
    tr = _t_raw(5)
    to = _t_out(5)
    ks = rng.choice(np.arange(-NB // 2, NB // 2), 7, replace=False)
    amps = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    x = sum(a * np.exp(2j * np.pi * (F_H + k / T_SFT) * tr) for a, k in zip(amps, ks))
    want = sum(a * np.exp(2j * np.pi * (k / T_SFT) * to) for a, k in zip(amps, ks))
    assert np.max(np.abs(_xh(x) - want)) < 1e-11


def test_band_must_sit_on_the_sft_grid():
    sf = np.zeros((2, M), dtype=complex)
    with pytest.raises(ValueError):
        sft.xh_from_band(sft.band(sf, 60, NB), 60, 0.0, T_SFT, M, F_H)
    with pytest.raises(ValueError):
        sft.xh_from_band(sft.band(sf, 64, NB), 64, 0.0, T_SFT, M, F_H + 0.01)
