"""Seeded random draws: noise, noise levels, template grids, injection parameters.

Streams: numpy ``Generator(PCG64(SeedSequence([seed, stream])))`` so that the
noise of each detector and the injection draws are independent and stable.
"""

from __future__ import annotations

import math

import numpy as np

TEMPLATE_DTYPE = np.dtype([("alpha", "<f8"), ("delta", "<f8"),
                           ("f1dot", "<f8"), ("f2dot", "<f8")])

_STREAM_NOISE = 11
_STREAM_SIGMA = 12
_STREAM_INJ = 13


def _rng(seed: int, stream: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), stream, sub])))


def make_noise(seed: int, det: int, n: int, sigma: float, dtype: str = "c64") -> np.ndarray:
    """White complex Gaussian noise: real and imaginary parts independent
    N(0, sigma^2), i.e. E|n|^2 = 2 sigma^2."""
    rng = _rng(seed, _STREAM_NOISE, det)
    ctype = np.complex128 if dtype == "c128" else np.complex64
    out = np.empty(n, dtype=ctype)
    rtype = np.float64 if dtype == "c128" else np.float32
    chunk = 1 << 22
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        re = rng.standard_normal(e - s, dtype=np.float64) * sigma
        im = rng.standard_normal(e - s, dtype=np.float64) * sigma
        out.real[s:e] = re.astype(rtype)
        out.imag[s:e] = im.astype(rtype)
    return out


def draw_sigmas(seed: int, n_det: int, lo: float, hi: float) -> tuple:
    rng = _rng(seed, _STREAM_SIGMA)
    return tuple(float(x) for x in rng.uniform(lo, hi, size=n_det))


def template_grid(skies, f1dots, f2dots) -> np.ndarray:
    """Cartesian template bank, sky-major, then f2dot, then f1dot (fastest)."""
    f1 = np.asarray(f1dots, dtype=np.float64)
    f2 = np.asarray(f2dots, dtype=np.float64)
    n = len(skies) * len(f1) * len(f2)
    out = np.empty(n, dtype=TEMPLATE_DTYPE)
    i = 0
    for (a, d) in skies:
        for v2 in f2:
            out["alpha"][i:i + len(f1)] = a
            out["delta"][i:i + len(f1)] = d
            out["f1dot"][i:i + len(f1)] = f1
            out["f2dot"][i:i + len(f1)] = v2
            i += len(f1)
    return out


def draw_injections(target, n_inj: int, rho2_range, min_sep_bins: int, seed: int) -> tuple:
    """Injection parameters: on an FFT bin inside the inner 80% of the band
    (|f0 - f_h| <= 0.4/dt), at least ``min_sep_bins`` apart, spindowns and sky
    on template-grid points, rho^2 uniform, cos(iota) ~ U[-1,1],
    psi ~ U[-pi/4, pi/4], phi0 ~ U[0, 2pi)."""
    from .configs import Injection

    rng = _rng(seed, _STREAM_INJ)
    half = target.n_fft // 2
    lim = int(math.floor(0.4 * target.n_fft))
    bins = []
    tries = 0
    while len(bins) < n_inj:
        tries += 1
        if tries > 100000:
            raise RuntimeError("cannot place injections with the requested separation")
        m = int(rng.integers(half - lim, half + lim + 1))
        if all(abs(m - b) >= min_sep_bins for b in bins):
            bins.append(m)
    out = []
    for m in bins:
        a, d = target.skies[int(rng.integers(0, len(target.skies)))]
        f1 = float(target.f1dots[int(rng.integers(0, len(target.f1dots)))])
        f2 = float(target.f2dots[int(rng.integers(0, len(target.f2dots)))])
        rho2 = float(rng.uniform(rho2_range[0], rho2_range[1]))
        out.append(Injection(
            f0=float(target.f_het + (m - half) / (target.n_fft * target.dt)),
            f1dot=f1, f2dot=f2, alpha=float(a), delta=float(d), rho2=rho2,
            cosi=float(rng.uniform(-1.0, 1.0)),
            psi=float(rng.uniform(-math.pi / 4, math.pi / 4)),
            phi0=float(rng.uniform(0.0, 2.0 * math.pi)),
            bin_index=m,
        ))
    return tuple(out)
