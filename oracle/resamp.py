"""Resampling F-statistic, steps (iii)-(vii) of Sec. 3, in FP64 (oracle).

One template at a time, in the order the paper lists the steps:

(iii) z_X(t_k) = x_h,X(t_k) exp(-i 2 pi f_h t_m,X(t_k))          [phase mod 1]
(iv)  regular SSB epochs t_b^j = t_b^0 + j dt; detector epochs T_X^j with
      T + t_m,X(T) = t_b^j by three fixed-point iterations
(v)   z_X(T_X^j) by a truncated, Hamming-tapered Dirichlet-kernel
      interpolator over the 2 Dterms + 1 nearest samples
(vi)  Fa, Fb = FFT of sum_X w_X a_X z_X exp(-i Phi_s) and the b_X analogue,
      zero-padded to n_fft (eqs. Fa, Fb of Sec. 2)
(vii) 2F = 2 (B |Fa|^2 + A |Fb|^2 - 2 C Re(Fa Fb*)) / D        (eq. Fstat)

Readings of points the paper leaves open:

* sign of step (iii): with the phase model Phi = 2 pi f0 [t + t_m] of Sec. 2,
  demodulation by exp(-i Phi) in eqs. (Fa_DET)/(Fb_DET) and heterodyning by
  exp(-i 2 pi f_h t), the factor that leaves z a function of t_b alone is
  exp(-i 2 pi f_h t_m); Sec. 3 prints the opposite sign, which belongs to the
  mirror-image heterodyne convention.  The brute-force pin decides.
* SSB grid: t_b^0 = t_0 + (orbital Roemer delay at the data midpoint), the
  same n_samples and dt as the detector grid, so the grid covers the data.
* interpolation kernel (Sec. 3 says only "interpolating"), by default
      W(x) = sin(pi x) / (N sin(pi x / N)) * (0.54 + 0.46 cos(pi x / (D + 1)))
  (untapered and periodic variants in dirichlet_weight),
  with N the detector sample count, W(0) = 1, taps k0 - D .. k0 + D with
  k0 = rint(u) (half to even), samples outside [0, N) count as zero, and the
  SSB point is valid for detector X iff 0 <= k0 <= N - 1.
* noise weights w_X = 1 / (2 sigma_X^2) with sigma_X the per-quadrature
  standard deviation, so that 2F ~ chi^2_4 in Gaussian noise (Sec. 5.4);
  A, B, C = sum over valid (X, j) of w_X a^2, w_X b^2, w_X a b.
* reference time t_ref = t_0 + floor(N/2) dt unless given; the spindown phase
  is Phi_s = 2 pi (f1dot tau^2 / 2 + f2dot tau^3 / 6), tau = t_b - t_ref.
* output bins in ascending frequency: bin m <-> f_h + (m - n_fft/2) / (n_fft dt).
"""

from __future__ import annotations

import numpy as np

from . import geometry as geo


def frac(x):
    """x - floor(x), the phase in cycles reduced to [0, 1)."""
    return x - np.floor(x)


def reference_time(target) -> float:
    return target.t_reference


def ssb_start(target, alpha: float, delta: float) -> float:
    """t_b^0: start of the regular SSB grid for this sky position."""
    t_mid = target.t0 + 0.5 * target.n_samples * target.dt
    return target.t0 + float(geo.roemer_orbit(t_mid, alpha, delta, target.ephemeris))


def ssb_times(target, alpha, delta) -> np.ndarray:
    return ssb_start(target, alpha, delta) + np.arange(target.n_samples, dtype=np.float64) * target.dt


def detector_times(target) -> np.ndarray:
    return target.t0 + np.arange(target.n_samples, dtype=np.float64) * target.dt


def step_iii(target, xh, det, alpha, delta):
    """z(t_k) = x_h(t_k) exp(-i 2 pi frac(f_h t_m(t_k)))."""
    tm = geo.roemer_delay(detector_times(target), det, alpha, delta, target.ephemeris)
    return np.asarray(xh, dtype=np.complex128) * np.exp(-2j * np.pi * frac(target.f_het * tm))


def step_iv(target, t_b, det, alpha, delta, iters: int = 3):
    """Detector epochs T with T + t_m(T) = t_b: start at t_b - t_m(t_b), then
    iterate T <- t_b - t_m(T) ``iters`` times."""
    eph = target.ephemeris
    T = t_b - geo.roemer_delay(t_b, det, alpha, delta, eph)
    for _ in range(iters):
        T = t_b - geo.roemer_delay(T, det, alpha, delta, eph)
    return T


TAPERED, UNTAPERED, PERIODIC = 0, 1, 2


def dirichlet_weight(x, n: int, dterms: int, kind: int = TAPERED):
    """Interpolation weight W(x), W(0) = 1, for the kernels the step-(v)
    interpolator can use (the paper names none; see the readings):

    TAPERED    sin(pi x) / (n sin(pi x / n)) * (0.54 + 0.46 cos(pi x / (D + 1)))
               (Dirichlet kernel of the full n-sample series, truncated to
               2D + 1 taps, Hamming taper)
    UNTAPERED  sin(pi x) / (n sin(pi x / n))            (truncated, no taper)
    PERIODIC   sin(pi x) / (M sin(pi x / M)), M = 2D + 1 (Dirichlet kernel of
               the 2D + 1 taps themselves)
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x != 0.0
    xs = x[nz]
    if kind == PERIODIC:
        m = 2 * dterms + 1
        out[nz] = np.sin(np.pi * xs) / (m * np.sin(np.pi * xs / m))
    elif kind == UNTAPERED:
        out[nz] = np.sin(np.pi * xs) / (n * np.sin(np.pi * xs / n))
    elif kind == TAPERED:
        out[nz] = (np.sin(np.pi * xs) / (n * np.sin(np.pi * xs / n))
                   * (0.54 + 0.46 * np.cos(np.pi * xs / (dterms + 1))))
    else:
        raise ValueError(f"unknown interpolation kernel {kind}")
    return out


def step_v(z, u, dterms: int, kind: int = TAPERED):
    """Interpolate z at fractional sample positions u (units of dt from t_0).

    Returns (values, valid).  k0 = rint(u); taps k0-D..k0+D; out-of-range
    taps are zero; points with k0 outside [0, N) are invalid (value 0)."""
    n = len(z)
    k0 = np.rint(u).astype(np.int64)
    dlt = u - k0
    valid = (k0 >= 0) & (k0 <= n - 1)
    out = np.zeros(len(u), dtype=np.complex128)
    for m in range(-dterms, dterms + 1):
        k = k0 + m
        ok = valid & (k >= 0) & (k < n)
        w = dirichlet_weight(dlt - m, n, dterms, kind)
        out[ok] += z[k[ok]] * w[ok]
    exact = valid & (dlt == 0.0)
    out[exact] = z[k0[exact]]
    return out, valid


def sky_prep(target, xh_list, alpha: float, delta: float) -> dict:
    """Per-sky work: steps (iii)-(v) for every detector, antenna weighting
    and the detector sum.  Returns G_a, G_b (complex128, length N) and the
    antenna-pattern integrals A, B, C, D."""
    n = target.n_samples
    t_b = ssb_times(target, alpha, delta)
    ga = np.zeros(n, dtype=np.complex128)
    gb = np.zeros(n, dtype=np.complex128)
    A = B = C = 0.0
    for X, det in enumerate(target.detectors):
        w = 1.0 / (2.0 * target.sigmas[X] ** 2)
        z = step_iii(target, xh_list[X], det, alpha, delta)
        T = step_iv(target, t_b, det, alpha, delta)
        u = (T - target.t0) / target.dt
        zi, valid = step_v(z, u, target.dterms, getattr(target, "interp", TAPERED))
        a, b = geo.antenna_ab(T, det, alpha, delta, target.ephemeris)
        a = np.where(valid, a, 0.0)
        b = np.where(valid, b, 0.0)
        ga += w * a * zi
        gb += w * b * zi
        A += w * float(np.sum(a * a))
        B += w * float(np.sum(b * b))
        C += w * float(np.sum(a * b))
    return {"Ga": ga, "Gb": gb, "A": A, "B": B, "C": C, "D": A * B - C * C,
            "t_b0": float(t_b[0]), "alpha": alpha, "delta": delta}


def spindown_phase(target, prep, f1dot: float, f2dot: float):
    """Phi_s / (2 pi) mod 1 at the SSB grid, tau = t_b - t_ref."""
    tau = (prep["t_b0"] + np.arange(target.n_samples, dtype=np.float64) * target.dt
           - reference_time(target))
    return frac(f1dot * tau * tau / 2.0 + f2dot * tau * tau * tau / 6.0)


def spindown_corrected(target, prep, f1dot: float, f2dot: float):
    """y_a, y_b: G_a, G_b times exp(-i Phi_s) (length N, before zero padding)."""
    rot = np.exp(-2j * np.pi * spindown_phase(target, prep, f1dot, f2dot))
    return prep["Ga"] * rot, prep["Gb"] * rot


def twoF_from_fafb(prep, fa, fb):
    """Eq. (Fstat) with the chi^2_4 normalisation: 2 (B|Fa|^2 + A|Fb|^2 -
    2 C Re(Fa Fb*)) / D (E = 0: no Im(Fa Fb*) term, Fig. 1)."""
    A, B, C, D = prep["A"], prep["B"], prep["C"], prep["D"]
    return 2.0 * (B * np.abs(fa) ** 2 + A * np.abs(fb) ** 2
                  - 2.0 * C * np.real(fa * np.conj(fb))) / D


def fafb(target, prep, f1dot: float, f2dot: float):
    """Step (vi): zero-padded FFTs of y_a, y_b, reordered to ascending
    frequency (bin m <-> f_h + (m - n_fft/2) df)."""
    ya, yb = spindown_corrected(target, prep, f1dot, f2dot)
    fa = np.fft.fftshift(np.fft.fft(ya, n=target.n_fft))
    fb = np.fft.fftshift(np.fft.fft(yb, n=target.n_fft))
    return fa, fb


def twoF(target, prep, f1dot: float, f2dot: float):
    """Steps (vi)-(vii) for one template: 2F over all n_fft bins, ascending."""
    fa, fb = fafb(target, prep, f1dot, f2dot)
    return twoF_from_fafb(prep, fa, fb)


def fafb_at_bins(target, prep, f1dot: float, f2dot: float, bins):
    """Fa, Fb at selected ascending bins by direct DFT sums (no FFT), for
    spot checks at sizes where a full FFT per template is too slow."""
    ya, yb = spindown_corrected(target, prep, f1dot, f2dot)
    j = np.arange(target.n_samples, dtype=np.float64)
    bins = np.asarray(bins, dtype=np.int64)
    k = (bins - target.n_fft // 2) % target.n_fft
    fa = np.empty(len(bins), dtype=np.complex128)
    fb = np.empty(len(bins), dtype=np.complex128)
    for i, kk in enumerate(k):
        e = np.exp(-2j * np.pi * frac(kk * j / target.n_fft))
        fa[i] = np.sum(ya * e)
        fb[i] = np.sum(yb * e)
    return fa, fb


def twoF_at_bins(target, prep, f1dot, f2dot, bins):
    fa, fb = fafb_at_bins(target, prep, f1dot, f2dot, bins)
    return twoF_from_fafb(prep, fa, fb)


def fstat(target, xh_list, templates):
    """2F[n_templates, n_fft] for a structured template array
    (fields alpha, delta, f1dot, f2dot), one template at a time."""
    out = np.empty((len(templates), target.n_fft), dtype=np.float64)
    cache = {}
    for i, t in enumerate(templates):
        key = (float(t["alpha"]), float(t["delta"]))
        if key not in cache:
            cache.clear()
            cache[key] = sky_prep(target, xh_list, *key)
        out[i] = twoF(target, cache[key], float(t["f1dot"]), float(t["f2dot"]))
    return out
