"""Seeded synthetic workloads for the resampling F-statistic.

This package holds *inputs only*: detector sites, sample grids, template
grids, per-detector noise levels, random draws of injection parameters and
seeded complex Gaussian noise.  It contains none of the method's arithmetic
(no timing model, no antenna patterns, no resampling, no FFT), so the CPU
oracle and the CUDA library can both consume it without sharing any of the
computation they are compared on.

Signal waveforms for injections need the timing and antenna model and are
therefore synthesised by whoever owns that model (the oracle, in the tests).
"""

from .configs import (  # noqa: F401
    Detector,
    Injection,
    Target,
    DETECTORS,
    EPHEMERIS,
    config1,
    config2,
    config3,
    config5,
    segment_slices,
    small_target,
    split_segments,
)
from .gen import make_noise, template_grid  # noqa: F401
