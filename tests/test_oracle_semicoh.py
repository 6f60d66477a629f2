"""Pins for the oracle's semi-coherent sum (CPU only).

* one segment spanning the data is the coherent 2F (shift 0);
* in noise the sum over S segments is chi^2 with 4S degrees of freedom
  (mean 4S, variance 8S), each segment's 2F being chi^2_4 (Sec. 5.4);
* a noise-free injection whose frequency at every segment's reference time
  falls on a bin: the sum at the injected global bin equals the total
  rho^2 within the resampling loss (1%), and is the maximum over bins; this
  fixes the direction of the sliding (with the wrong sign the segments'
  peaks would not line up and the sum would fall to about rho^2 / S).
"""

import math

import numpy as np

from oracle import resamp, semicoh, synth
from workloads import segment_slices, small_target, split_segments
from workloads.gen import template_grid


def _segments(t, n_seg, x):
    segs = split_segments(t, n_seg)
    data = [[xx[a:a + n] for xx in x] for a, n in segment_slices(t, n_seg)]
    return segs, data


def test_single_segment_is_the_coherent_statistic():
    t = small_target(n_samples=3001, dt=2.0, n_fft=1 << 13, n_det=2, n_inj=1, seed=81,
                     f1dots=(-3e-10, 0.0), f2dots=(0.0, 1e-16))
    x = synth.make_data(t)
    segs, data = _segments(t, 1, x)
    tm = t.templates()
    got = semicoh.semicoherent(segs, data, tm, t.t_reference)
    assert np.allclose(got, resamp.fstat(t, x, tm), rtol=1e-12, atol=1e-12)


def test_noise_sum_is_chi2_with_4S_degrees_of_freedom():
    S = 4
    t = small_target(n_samples=S << 14, dt=1.0, n_fft=1 << 15, n_det=2, seed=82,
                     f1dots=(0.0,), f2dots=(0.0,))
    x = synth.make_data(t)
    segs, data = _segments(t, S, x)
    tf = semicoh.semicoherent(segs, data, t.templates(), t.t_reference)[0]
    half, lim = t.n_fft // 2, int(0.4 * t.n_fft)
    v = tf[half - lim: half + lim][::2]
    n = len(v)
    assert abs(v.mean() - 4 * S) < 3.0 * math.sqrt(8 * S / n)
    # Var of chi^2_k sample variance: (mu4 - sigma^4)/n, mu4 = 12k(k+4) for k = 4S
    k = 4 * S
    assert abs(v.var() - 2 * k) < 3.0 * math.sqrt((12 * k * (k + 4) - 4 * k * k) / n)


def test_injection_lines_up_across_segments():
    S = 3
    n_seg = 6000
    dt = 1.0
    n_fft = 1 << 14
    df = 1.0 / (n_fft * dt)
    t_seg = n_seg * dt
    q, p = 3, 1
    f1 = q * df / t_seg                 # f1dot * T_seg = q bins
    f2 = 2.0 * p * df / t_seg ** 2      # f2dot * T_seg^2 / 2 = p bins
    t = small_target(n_samples=S * n_seg, dt=dt, n_fft=n_fft, n_det=2, n_inj=1,
                     rho2_range=(300.0, 300.0), seed=83, f1dots=(f1,), f2dots=(f2,))
    inj = t.injections[0]
    assert inj.f1dot == f1 and inj.f2dot == f2
    x = synth.make_data(t, noise=False)
    segs, data = _segments(t, S, x)
    tm = template_grid(((inj.alpha, inj.delta),), np.array([f1]), np.array([f2]))
    tf = semicoh.semicoherent(segs, data, tm, t.t_reference)[0]
    shifts = [semicoh.segment_shift(df, s.t_reference - t.t_reference, f1, f2) for s in segs]
    assert shifts == [-q + p, 0, q + p]
    m = inj.bin_index
    assert abs(tf[m] / inj.rho2 - 1.0) < 0.02, tf[m] / inj.rho2
    assert int(np.argmax(tf)) == m
    # sliding the other way does not line the segments up
    bad = np.zeros(n_fft)
    for s, d, k in zip(segs, data, shifts):
        row = resamp.fstat(s, d, semicoh.segment_template(tm, s.t_reference - t.t_reference))[0]
        bad += np.roll(row, k)          # bad[m] = row[m - k]: the opposite sliding
    assert bad.max() < 0.75 * inj.rho2
