"""Accuracy of the step-(v) interpolator variants (oracle, test infrastructure).

For each kernel (tapered, untapered, periodic Dirichlet) and half-width D,
with the oracle's FP64 resampling path:

* loss: 1 - 2F / rho^2 for a noise-free injection on an FFT bin, at several
  offsets nu = (f - f_h) dt inside the band (the exact brute-force value is
  rho^2, so the loss is the interpolation's);
* edge: the power of resampled unit white noise in the outer band
  0.45 <= |nu| < 0.5 (1 = flat).

Run as ``python -m oracle.interp_study``; prints one line per kernel and D.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import resamp, synth

NAMES = {resamp.TAPERED: "tapered", resamp.UNTAPERED: "untapered", resamp.PERIODIC: "periodic"}


def injection_loss(kind: int, dterms: int, nus=(0.05, 0.2, 0.3, 0.4), seed=70):
    from workloads import small_target

    out = []
    for nu in nus:
        t = small_target(n_samples=4096, dt=1.0, n_fft=1 << 13, n_det=2, n_inj=1,
                         rho2_range=(100.0, 100.0), seed=seed, f1dots=(0.0,), f2dots=(0.0,),
                         dterms=dterms, interp=kind)
        m = t.n_fft // 2 + int(round(nu * t.n_fft))
        inj = dataclasses.replace(t.injections[0], bin_index=m,
                                  f0=t.f_het + (m - t.n_fft // 2) / (t.n_fft * t.dt))
        x = synth.make_data(t, noise=False, injections=[inj])
        prep = resamp.sky_prep(t, x, inj.alpha, inj.delta)
        tf = resamp.twoF_at_bins(t, prep, inj.f1dot, inj.f2dot, [m])[0]
        out.append(1.0 - tf / inj.rho2)
    return out


def edge_power(kind: int, dterms: int, n=1 << 14, reps=8, seed=9):
    rng = np.random.default_rng(seed)
    acc = np.zeros(n)
    for _ in range(reps):
        z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2)
        u = np.arange(n) + rng.uniform(-0.5, 0.5) + 0.37 * np.sin(np.arange(n) / 700.0)
        zi, _ = resamp.step_v(z, u, dterms, kind)
        acc += np.abs(np.fft.fft(zi[64:-64], n=n)) ** 2 / (n - 128)
    spec = np.fft.fftshift(acc / reps)
    nu = np.abs((np.arange(n) - n // 2) / n)
    return float(spec[(nu >= 0.45) & (nu < 0.5)].mean()), float(spec[nu < 0.4].mean())


def main():
    for kind in (resamp.TAPERED, resamp.UNTAPERED, resamp.PERIODIC):
        for d in (4, 8, 16, 32):
            loss = injection_loss(kind, d)
            edge, inner = edge_power(kind, d)
            print(f"{NAMES[kind]:9s} D={d:2d}  loss(nu=.05,.2,.3,.4) = "
                  + " ".join(f"{v:+.2e}" for v in loss)
                  + f"  noise power inner {inner:.3f} edge {edge:.3f}")


if __name__ == "__main__":
    main()
