"""Pins for the oracle's 2F post-processing (CPU only).

* hand-built rows whose crossings and band maxima are written out by hand
  (strict threshold, ties resolved to the smallest bin, negative values);
* a brute-force double loop over random rows with planted ties;
* the limiting cases n_bands = 1 (global maximum) and n_bands = n_fft
  (every bin its own band);
* the paper's statistics: in noise 2F ~ chi^2_4 (Sec. 5.4), so the number of
  in-band crossings of a threshold x is Poisson-close to K exp(-x/2)(1+x/2).
"""

import math

import numpy as np
import pytest

from oracle import peaks, resamp, synth
from workloads import small_target


def test_hand_built_rows():
    tf = np.array([[0.0, 5.0, 5.0, 1.0, 3.0, 9.0, 2.0, 9.0],
                   [-1.0, -0.5, -2.0, -0.5, 70.0, 70.5, 69.9, 80.0]])
    vmax, vbin = peaks.band_maxima(tf, 2)
    assert vmax.tolist() == [[5.0, 9.0], [-0.5, 80.0]]
    assert vbin.tolist() == [[1, 5], [1, 7]]
    vmax, vbin = peaks.band_maxima(tf, 4)
    assert vmax.tolist() == [[5.0, 5.0, 9.0, 9.0], [-0.5, -0.5, 70.5, 80.0]]
    assert vbin.tolist() == [[1, 2, 5, 7], [1, 3, 5, 7]]
    assert peaks.crossings(tf, 5.0) == [(0, 5, 9.0), (0, 7, 9.0), (1, 4, 70.0), (1, 5, 70.5),
                                        (1, 6, 69.9), (1, 7, 80.0)]
    assert peaks.crossings(tf, 70.0, tmpl_offset=10) == [(11, 5, 70.5), (11, 7, 80.0)]


def test_brute_force_loops_with_ties():
    rng = np.random.default_rng(5)
    for n_bands in (1, 2, 8, 64):
        tf = rng.integers(0, 6, size=(3, 64)).astype(np.float64)  # many ties
        vmax, vbin = peaks.band_maxima(tf, n_bands)
        w = 64 // n_bands
        for i in range(3):
            for b in range(n_bands):
                best, arg = -np.inf, -1
                for m in range(b * w, (b + 1) * w):
                    if tf[i, m] > best:
                        best, arg = tf[i, m], m
                assert vmax[i, b] == best and vbin[i, b] == arg
        want = [(i, m, tf[i, m]) for i in range(3) for m in range(64) if tf[i, m] > 3.5]
        assert peaks.crossings(tf, 3.5) == want


def test_limiting_band_counts():
    rng = np.random.default_rng(6)
    tf = rng.standard_normal((4, 128))
    vmax, vbin = peaks.band_maxima(tf, 1)
    assert np.array_equal(vmax[:, 0], tf.max(axis=1))
    assert np.array_equal(vbin[:, 0], tf.argmax(axis=1))
    vmax, vbin = peaks.band_maxima(tf, 128)
    assert np.array_equal(vmax, tf)
    assert np.array_equal(vbin, np.broadcast_to(np.arange(128), (4, 128)))
    with pytest.raises(ValueError):
        peaks.band_maxima(tf, 3)


def test_noise_crossings_follow_chi2_4_tail():
    t = small_target(n_samples=1 << 15, dt=1.0, n_fft=1 << 16, n_det=2, seed=23)
    x = synth.make_data(t)
    prep = resamp.sky_prep(t, x, *t.skies[0])
    half, lim = t.n_fft // 2, int(0.4 * t.n_fft)
    rows = [resamp.twoF(t, prep, f1, 0.0)[half - lim: half + lim][::2] for f1 in (0.0, -1e-9)]
    tf = np.stack(rows)
    thr = 12.0
    k = tf.size
    want = k * math.exp(-thr / 2.0) * (1.0 + thr / 2.0)
    got = len(peaks.crossings(tf, thr))
    assert abs(got - want) < 4.0 * math.sqrt(want), (got, want)
    # every band maximum is one of the values and no value of its band exceeds it
    sub = tf[:, :16384]
    vmax, vbin = peaks.band_maxima(sub, 16)
    assert np.all(sub[np.arange(2)[:, None], vbin] == vmax)
    assert np.all(vmax >= sub.reshape(2, 16, -1).max(axis=2))
