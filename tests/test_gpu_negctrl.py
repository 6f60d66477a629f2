"""Negative control: the parity test must be able to see precision loss.

The paper's Resamp needs the detector-to-SSB timing in double precision:
f_h t_m reaches ~5e4 cycles and the sample position u = (T - t0)/dt
~1.7e6 samples, where single precision keeps ~4e-3 cycles and ~0.1 sample.
A second build of the library forms exactly those two quantities in FP32
(FSTAT_NEGCTRL_FP32_TIMING, compiled only here).  On the 10-day
two-detector workload with its injections, the regular build meets
|d2F| <= 1e-3 2F + 0.02 on whole rows, and the degraded build must fail it.
"""

import numpy as np
import pytest

import paper_2201_00451_gb300 as pkg
from oracle import resamp, synth
from workloads import config2

pytestmark = pytest.mark.gpu

REL, ABS = 1e-3, 0.02


def _rows(lib, t, x, rows):
    with pkg.FstatPlan.from_target(t, lib=lib) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.set_split(1024)
        got = plan.compute(rows).cpu().numpy()
        plan.sync()
    return got


def test_fp32_timing_fails_the_tolerance_the_fp64_timing_meets():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    regular = pkg.load()
    degraded = pkg.open_library(fbuild.build_variant("negctrl", ["FSTAT_NEGCTRL_FP32_TIMING"]))
    t = config2()
    x = synth.make_data(t)
    injs = sorted(t.injections, key=lambda i: -i.rho2)[:2]
    rows = np.empty(len(injs), dtype=pkg.TEMPLATE_DTYPE)
    for k, inj in enumerate(injs):
        rows[k] = (inj.alpha, inj.delta, inj.f1dot, inj.f2dot)
    prep = resamp.sky_prep(t, x, *t.skies[0])
    ref = np.stack([resamp.twoF(t, prep, float(r["f1dot"]), float(r["f2dot"])) for r in rows])
    tol = REL * np.abs(ref) + ABS

    good = _rows(regular, t, x, rows)
    assert not (np.abs(good - ref) > tol).any()

    bad = _rows(degraded, t, x, rows)
    excess = np.abs(bad - ref) - tol
    assert (excess > 0).sum() > 100, int((excess > 0).sum())
    # the loss shows at the injections themselves
    m = [inj.bin_index for inj in injs]
    assert np.any(np.abs(bad[np.arange(len(injs)), m] - ref[np.arange(len(injs)), m]) > tol[np.arange(len(injs)), m])
