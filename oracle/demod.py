"""Brute-force demodulation: eqs. (Fa_DET), (Fb_DET) of Sec. 2, discretised.

    Fa(f) = sum_X w_X sum_k x_h,X[k] a_X(t_k)
            exp(-i 2 pi [(f - f_h) tau_k + f_h t_m,X(t_k) + f1dot tau_k^2/2
                         + f2dot tau_k^3/6])
    tau_k = t_k + t_m,X(t_k) - t_ref

(x_h is the data heterodyned by exp(-i 2 pi f_h t); the constant
exp(-i 2 pi (f - f_h) t_ref) per bin is common to Fa and Fb and cancels in
2F.)  A, B, C are sums of w_X a^2, w_X b^2, w_X a b over detector samples.
O(N x bins): tiny inputs only.  This is the exact definition the resampling
steps approximate (Sec. 2 makes dt/dt_b ~ 1 and t_b(T/2) ~ T/2).
"""

from __future__ import annotations

import numpy as np

from . import geometry as geo
from .resamp import detector_times, frac, reference_time, twoF_from_fafb


def demod(target, xh_list, alpha, delta, f1dot, f2dot, freqs, sample_mask=None):
    """Returns (Fa, Fb, prep) with prep holding A, B, C, D.

    ``sample_mask`` (optional, per detector boolean arrays) restricts the sums
    to a subset of detector samples."""
    freqs = np.atleast_1d(np.asarray(freqs, dtype=np.float64))
    t = detector_times(target)
    t_ref = reference_time(target)
    fa = np.zeros(len(freqs), dtype=np.complex128)
    fb = np.zeros(len(freqs), dtype=np.complex128)
    A = B = C = 0.0
    for X, det in enumerate(target.detectors):
        w = 1.0 / (2.0 * target.sigmas[X] ** 2)
        tm = geo.roemer_delay(t, det, alpha, delta, target.ephemeris)
        tau = t + tm - t_ref
        a, b = geo.antenna_ab(t, det, alpha, delta, target.ephemeris)
        x = np.asarray(xh_list[X], dtype=np.complex128)
        if sample_mask is not None:
            msk = sample_mask[X]
            a, b, x, tau, tm = a[msk], b[msk], x[msk], tau[msk], tm[msk]
        base = frac(target.f_het * tm) + frac(f1dot * tau * tau / 2.0) + frac(f2dot * tau ** 3 / 6.0)
        for i, f in enumerate(freqs):
            e = np.exp(-2j * np.pi * (frac((f - target.f_het) * tau) + base))
            fa[i] += w * np.sum(x * a * e)
            fb[i] += w * np.sum(x * b * e)
        A += w * float(np.sum(a * a))
        B += w * float(np.sum(b * b))
        C += w * float(np.sum(a * b))
    prep = {"A": A, "B": B, "C": C, "D": A * B - C * C}
    return fa, fb, prep


def demod_twoF(target, xh_list, alpha, delta, f1dot, f2dot, freqs, sample_mask=None):
    fa, fb, prep = demod(target, xh_list, alpha, delta, f1dot, f2dot, freqs, sample_mask)
    return twoF_from_fafb(prep, fa, fb)
