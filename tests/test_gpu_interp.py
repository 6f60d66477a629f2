"""GPU parity of the step-(v) interpolator variants and half-widths.

Every kernel (tapered, untapered and periodic Dirichlet) at D = 4, 8, 16,
32 against the oracle: the per-sky resampled, weighted series G_a, G_b
(relative 2e-5 of their largest element, as for the default kernel) and
2F at |d2F| <= 1e-3 2F + 0.02 on a ragged two-detector case.
"""

import numpy as np
import pytest

import paper_2201_00451_gb300 as pkg
from oracle import resamp, synth
from workloads import small_target

pytestmark = pytest.mark.gpu

REL, ABS = 1e-3, 0.02


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


@pytest.mark.parametrize("interp", [pkg.INTERP_TAPERED, pkg.INTERP_UNTAPERED, pkg.INTERP_PERIODIC])
@pytest.mark.parametrize("dterms", [4, 8, 16, 32])
def test_interpolator_variants_match_oracle(interp, dterms):
    t = small_target(n_samples=5003, dt=2.0, n_fft=1 << 14, n_det=2, n_inj=1, rho2_range=(150.0, 150.0),
                     seed=60 + dterms, f1dots=(-3e-10, 0.0), f2dots=(0.0,), dtype="c64", dterms=dterms,
                     interp=interp)
    x = synth.make_data(t)
    a, d = t.skies[0]
    ref = resamp.sky_prep(t, x, a, d)
    tm = t.templates()
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        ga, gb, abcd = plan.export_sky(a, d)
        got = plan.compute(tm)
        plan.sync()
        got = got.cpu().numpy()
    scale = max(np.abs(ref["Ga"]).max(), np.abs(ref["Gb"]).max())
    assert np.abs(ga - ref["Ga"]).max() <= 2e-5 * scale
    assert np.abs(gb - ref["Gb"]).max() <= 2e-5 * scale
    for k, v in zip("ABCD", abcd):
        assert abs(v - ref[k]) <= 1e-10 * abs(ref[k]) + 1e-12
    want = resamp.fstat(t, x, tm)
    excess = np.abs(got - want) - (REL * np.abs(want) + ABS)
    assert excess.max() <= 0, excess.max()
