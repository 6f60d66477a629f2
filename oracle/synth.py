"""CW signal injection (oracle-side; uses the oracle's timing/antenna model).

Signal model (Sec. 2 phase model; JKS amplitude parameters):
    s_X[k] = (Aa a_X(t_k) + Ab b_X(t_k)) exp(i Psi_k)
    Psi_k  = 2 pi [(f0 - f_h) tau_k + f_h t_m,X(t_k) + f1 tau_k^2/2 + f2 tau_k^3/6] + phi0
    tau_k  = t_k + t_m,X(t_k) - t_ref
with A+ = h0 (1 + cos^2 i)/2, Ax = h0 cos i, Aa = (A+ cos 2psi + i Ax sin 2psi)/2,
Ab = (A+ sin 2psi - i Ax cos 2psi)/2 (the positive-frequency part of
F+ h+ + Fx hx with F+ = a cos 2psi + b sin 2psi, Fx = b cos 2psi - a sin 2psi).
h0 is set so that rho^2 = 2 sum_X w_X sum_k |s_X[k]|^2 hits the requested value.
"""

from __future__ import annotations

import numpy as np

from workloads.gen import make_noise

from . import geometry as geo
from .resamp import detector_times, frac, reference_time


def amplitudes(h0, cosi, psi):
    ap = h0 * (1.0 + cosi * cosi) / 2.0
    ax = h0 * cosi
    aa = (ap * np.cos(2 * psi) + 1j * ax * np.sin(2 * psi)) / 2.0
    ab = (ap * np.sin(2 * psi) - 1j * ax * np.cos(2 * psi)) / 2.0
    return aa, ab


def signal(target, inj, X, h0=1.0):
    det = target.detectors[X]
    t = detector_times(target)
    tm = geo.roemer_delay(t, det, inj.alpha, inj.delta, target.ephemeris)
    tau = t + tm - reference_time(target)
    a, b = geo.antenna_ab(t, det, inj.alpha, inj.delta, target.ephemeris)
    aa, ab = amplitudes(h0, inj.cosi, inj.psi)
    cyc = (frac((inj.f0 - target.f_het) * tau) + frac(target.f_het * tm)
           + frac(inj.f1dot * tau * tau / 2.0) + frac(inj.f2dot * tau ** 3 / 6.0))
    return (aa * a + ab * b) * np.exp(1j * (2.0 * np.pi * frac(cyc) + inj.phi0))


def rho2_of(target, sigs):
    return float(sum(2.0 / (2.0 * target.sigmas[X] ** 2) * np.sum(np.abs(s) ** 2)
                     for X, s in enumerate(sigs)))


def injected_signals(target, inj):
    """Per-detector signal arrays of one injection scaled to its rho^2."""
    sigs = [signal(target, inj, X) for X in range(len(target.detectors))]
    scale = np.sqrt(inj.rho2 / rho2_of(target, sigs))
    return [s * scale for s in sigs]


def make_data(target, noise=True, injections=None):
    """x_h per detector: seeded noise (sigma_X per quadrature) plus every
    injection of the target, stored in the target's dtype."""
    injections = target.injections if injections is None else injections
    ctype = np.complex128 if target.dtype == "c128" else np.complex64
    out = []
    for X in range(len(target.detectors)):
        if noise:
            x = make_noise(target.seed, X, target.n_samples, target.sigmas[X], "c128"
                           if target.dtype == "c128" else "c64").astype(np.complex128)
        else:
            x = np.zeros(target.n_samples, dtype=np.complex128)
        out.append(x)
    for inj in injections:
        for X, s in enumerate(injected_signals(target, inj)):
            out[X] += s
    return [x.astype(ctype) for x in out]
