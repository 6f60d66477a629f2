"""2F and its gradient at arbitrary (off-grid) parameters (oracle, FP64).

The statistic refined here is eq. (Fstat) evaluated with the demodulation
integrals of eqs. (Fa_DET)/(Fb_DET) (Sec. 2) summed directly over detector
samples at a single frequency f, for theta = (f, f1dot, alpha, delta) with
f2dot held fixed:

    Phi_k   = (f - f_h) tau_k + f_h t_m(t_k) + f1dot tau_k^2/2 + f2dot tau_k^3/6   [cycles]
    tau_k   = t_k + t_m(t_k) - t_ref
    Fa      = sum_X w_X sum_k x_h,X[k] a_X(t_k) exp(-i 2 pi Phi_k),  Fb likewise with b
    2F      = 2 (B |Fa|^2 + A |Fb|^2 - 2 C Re(Fa Fb*)) / D

Derivatives in f and f1dot are analytic (A, B, C do not depend on them):
    dFa/df     = sum w x a e^{-i 2 pi Phi} (-i 2 pi tau_k)
    dFa/df1dot = sum w x a e^{-i 2 pi Phi} (-i 2 pi tau_k^2 / 2)
Derivatives in alpha and delta (through t_m, a, b, A, B, C) are central
differences of 2F with a small step in radians.
"""

from __future__ import annotations

import numpy as np

from . import geometry as geo
from .demod import demod
from .resamp import detector_times, frac, reference_time


def twoF_abc(prep, fa, fb):
    A, B, C, D = prep["A"], prep["B"], prep["C"], prep["D"]
    return 2.0 * (B * abs(fa) ** 2 + A * abs(fb) ** 2 - 2.0 * C * (fa * np.conj(fb)).real) / D


def twoF_at(target, xh_list, theta, f2dot=0.0):
    """2F at theta = (f, f1dot, alpha, delta)."""
    f, f1, a, d = (float(v) for v in theta)
    fa, fb, prep = demod(target, xh_list, a, d, f1, f2dot, [f])
    return float(twoF_abc(prep, fa[0], fb[0]))


def _fa_fb_and_derivs(target, xh_list, theta, f2dot):
    f, f1, alpha, delta = (float(v) for v in theta)
    t = detector_times(target)
    t_ref = reference_time(target)
    out = np.zeros((3, 2), dtype=np.complex128)   # rows: value, d/df, d/df1dot; cols: a, b
    A = B = C = 0.0
    for X, det in enumerate(target.detectors):
        w = 1.0 / (2.0 * target.sigmas[X] ** 2)
        tm = geo.roemer_delay(t, det, alpha, delta, target.ephemeris)
        tau = t + tm - t_ref
        a, b = geo.antenna_ab(t, det, alpha, delta, target.ephemeris)
        x = np.asarray(xh_list[X], dtype=np.complex128)
        cyc = (frac((f - target.f_het) * tau) + frac(target.f_het * tm)
               + frac(f1 * tau * tau / 2.0) + frac(f2dot * tau ** 3 / 6.0))
        e = x * np.exp(-2j * np.pi * cyc) * w
        for col, pat in enumerate((a, b)):
            out[0, col] += np.sum(e * pat)
            out[1, col] += np.sum(e * pat * (-2j * np.pi * tau))
            out[2, col] += np.sum(e * pat * (-2j * np.pi * tau * tau / 2.0))
        A += w * float(np.sum(a * a))
        B += w * float(np.sum(b * b))
        C += w * float(np.sum(a * b))
    return out, {"A": A, "B": B, "C": C, "D": A * B - C * C}


def grad(target, xh_list, theta, f2dot=0.0, h_sky=1e-7):
    """(2F, [d2F/df, d2F/df1dot, d2F/dalpha, d2F/ddelta]) at theta."""
    v, prep = _fa_fb_and_derivs(target, xh_list, theta, f2dot)
    A, B, C, D = prep["A"], prep["B"], prep["C"], prep["D"]
    fa, fb = v[0]
    two_f = float(twoF_abc(prep, fa, fb))
    g = np.zeros(4)
    for i in (1, 2):
        dfa, dfb = v[i]
        g[i - 1] = 2.0 * (2.0 * B * (np.conj(fa) * dfa).real + 2.0 * A * (np.conj(fb) * dfb).real
                          - 2.0 * C * (dfa * np.conj(fb) + fa * np.conj(dfb)).real) / D
    th = np.asarray(theta, dtype=np.float64)
    for i in (2, 3):
        tp, tm_ = th.copy(), th.copy()
        tp[i] += h_sky
        tm_[i] -= h_sky
        g[i] = (twoF_at(target, xh_list, tp, f2dot) - twoF_at(target, xh_list, tm_, f2dot)) / (2 * h_sky)
    return two_f, g
