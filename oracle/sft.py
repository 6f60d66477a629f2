"""Step (ii) of Sec. 3 from short Fourier transforms (oracle, test infrastructure).

Sec. 3 starts from SFTs: discrete Fourier transforms of the detector output
over consecutive segments short enough (T_sft, ~1800 s) that the Doppler and
spindown modulations are small within one.  Steps (i)-(ii) combine them,
heterodyne at f_h, low-pass and downsample in the frequency domain, and
inverse-FFT to the series x_h(t_k).  Stated here per SFT:

An SFT of segment s (start t_s = t_start + s T_sft, M raw samples at
dt_raw = T_sft / M) holds X_s[q] = sum_n x(t_s + n dt_raw) exp(-2 pi i q n / M).
With f_h on the SFT grid (q_h = f_h T_sft an integer) and a band of B bins,
q = q_h - B/2 .. q_h + B/2 - 1, the heterodyned, band-limited series at
dt = T_sft / B over segment s is

    x_h(t_s + m dt) = exp(-2 pi i f_h t_s) / M * sum_{k=-B/2}^{B/2-1} X_s[q_h + k] exp(2 pi i k m / B),

m = 0 .. B - 1: the inverse DFT of the band, shifted to f_h.  Consecutive
SFTs give consecutive blocks of x_h.  It is exact for a signal whose
components in each segment are SFT-bin tones inside the band.
"""

from __future__ import annotations

import numpy as np

from .resamp import frac


def sfts_from_series(x, m_raw: int):
    """SFTs of consecutive segments of m_raw raw samples (numpy's forward DFT,
    exp(-2 pi i q n / M), unnormalised): [n_sft, m_raw] complex."""
    x = np.asarray(x)
    n_sft = len(x) // m_raw
    return np.fft.fft(x[: n_sft * m_raw].reshape(n_sft, m_raw), axis=1)


def band(sfts, q0: int, n_bins: int):
    """Bins q0 .. q0 + n_bins - 1 of every SFT."""
    return np.asarray(sfts)[:, q0: q0 + n_bins]


def xh_from_band(bins, q0: int, t_start: float, t_sft: float, m_raw: int, f_het: float):
    """x_h from the band bins [n_sft][B] (bin q0 + i in column i); requires
    q0 = q_h - B/2 with q_h = f_het t_sft an integer.  Returns n_sft * B
    complex samples at dt = t_sft / B starting at t_start."""
    bins = np.asarray(bins, dtype=np.complex128)
    n_sft, nb = bins.shape
    q_h = f_het * t_sft
    if abs(q_h - round(q_h)) > 1e-9 or int(round(q_h)) - nb // 2 != q0:
        raise ValueError("band must be the bins q_h - B/2 .. q_h + B/2 - 1 with q_h = f_het t_sft integral")
    k = np.arange(nb) - nb // 2                    # column i holds k = i - B/2
    m = np.arange(nb)
    kernel = np.exp(2j * np.pi * frac(np.outer(k, m) / nb))   # [k][m], exp(2 pi i k m / B)
    out = np.empty((n_sft, nb), dtype=np.complex128)
    for s in range(n_sft):
        t_s = t_start + s * t_sft
        rot = np.exp(-2j * np.pi * frac(f_het * t_s))
        out[s] = rot / m_raw * (bins[s] @ kernel)
    return out.reshape(-1)
