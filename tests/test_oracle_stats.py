"""Statistical pins for the oracle (CPU only).

Sec. 5.4: in Gaussian noise 2F follows chi^2 with 4 degrees of freedom; with
a signal of optimal SNR^2 rho^2 the expectation is 4 + rho^2 (non-central
chi^2_4).  Checked on in-band bins (|f - f_h| <= 0.4/dt) where the
interpolation keeps the noise spectrum flat.
"""

import json
import math
import os

import numpy as np
from scipy import stats

from oracle import resamp, synth
from workloads import small_target

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _chi2_4_sf(x):
    # closed form of the chi^2_4 survival function: exp(-x/2) (1 + x/2)
    return math.exp(-x / 2.0) * (1.0 + x / 2.0)


def test_paper_false_alarm_number_pins_chi2_4_tail():
    g = json.load(open(GOLDEN))["chi2_false_alarm"]
    p = _chi2_4_sf(g["threshold"])
    fa = -math.expm1(g["n_values"] * math.log1p(-p))
    assert abs(fa - g["false_alarm_probability"]) < 0.02
    assert abs(stats.chi2(4).sf(g["threshold"]) - p) < 1e-20


def test_paper_template_arithmetic():
    g = json.load(open(GOLDEN))
    pc = g["pilot_template_count"]
    assert abs(pc["n_templates"] * pc["n_freqs"] / pc["n_values"] - 1.0) < 2e-3
    fs = g["pilot_frequency_spacing"]
    t_obs = fs["gps_end"] - fs["gps_start"]
    assert abs(1.0 / (2.0 * t_obs) / fs["spacing_hz"] - 1.0) < 0.02


def test_noise_only_twoF_is_chi2_4():
    t = small_target(n_samples=1 << 16, dt=1.0, n_fft=1 << 17, n_det=2, seed=21)
    x = synth.make_data(t)
    prep = resamp.sky_prep(t, x, *t.skies[0])
    tf = resamp.twoF(t, prep, 0.0, 0.0)
    half, lim = t.n_fft // 2, int(0.4 * t.n_fft)
    band = tf[half - lim: half + lim]
    # zero padding by 2 correlates neighbours: keep every 2nd bin
    s = band[::2]
    n_eff = len(s)
    assert n_eff > 50000
    assert abs(s.mean() - 4.0) < 3.0 * math.sqrt(8.0 / n_eff)
    # sample variance of chi^2_4: Var ~ (mu4 - sigma^4)/n, mu4 = 12 k (k + 4) = 384
    var_sd = math.sqrt((384.0 - 64.0) / n_eff)
    assert abs(s.var() - 8.0) < 3.0 * var_sd
    assert stats.kstest(s[::4], stats.chi2(4).cdf).pvalue > 1e-3


def test_injection_mean_is_4_plus_rho2():
    rho2 = 20.0
    vals = []
    for r in range(64):
        t = small_target(n_samples=2048, dt=1.0, n_fft=1 << 12, n_det=2, n_inj=1,
                         rho2_range=(rho2, rho2), seed=500 + r)
        inj = t.injections[0]
        x = synth.make_data(t)
        prep = resamp.sky_prep(t, x, *t.skies[0])
        vals.append(resamp.twoF_at_bins(t, prep, 0.0, 0.0, [inj.bin_index])[0])
    vals = np.array(vals)
    sd = math.sqrt(2.0 * (4.0 + 2.0 * rho2) / len(vals))
    # resampling loses <= 1% of rho^2 (pinned separately)
    assert abs(vals.mean() - (4.0 + rho2)) < 3.0 * sd + 0.01 * rho2
