"""On-device post-processing of 2F, stated plainly (oracle, test infrastructure).

Sec. 5.4 keeps only the bins with 2F > 70 and performs that retention next
to the computation so the full band never has to leave the device; Sec. 4.1
names the maximum of 2F over a frequency band as the simplest such
reduction.  For a block of 2F rows (one per template, bins in ascending
frequency) this module computes both by definition:

* crossings: every (template, bin) with 2F strictly above the threshold;
* band maxima: bins split into n_bands equal consecutive bands of W bins;
  per template and band the largest 2F and the smallest bin holding it.
"""

from __future__ import annotations

import numpy as np


def crossings(twoF: np.ndarray, threshold: float, tmpl_offset: int = 0):
    """Sorted (template, bin, 2F) triples with 2F > threshold."""
    twoF = np.atleast_2d(np.asarray(twoF))
    ti, mi = np.nonzero(twoF > threshold)
    return [(int(t) + tmpl_offset, int(m), float(twoF[t, m])) for t, m in zip(ti, mi)]


def band_maxima(twoF: np.ndarray, n_bands: int):
    """(max [n, n_bands], bin [n, n_bands]) over bands of n_fft / n_bands bins."""
    twoF = np.atleast_2d(np.asarray(twoF))
    n, n_fft = twoF.shape
    if n_bands < 1 or n_fft % n_bands:
        raise ValueError("n_bands must divide the number of bins")
    w = n_fft // n_bands
    blocks = twoF.reshape(n, n_bands, w)
    first = np.argmax(blocks, axis=2)                 # first occurrence: smallest bin on ties
    vmax = np.take_along_axis(blocks, first[..., None], axis=2)[..., 0]
    return vmax, first + w * np.arange(n_bands)[None, :]
