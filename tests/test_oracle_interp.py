"""Pins for the step-(v) interpolation kernel variants (CPU only).

The paper names no interpolator (Sec. 3 step v).  Besides the default
(tapered Dirichlet) the oracle offers the untapered truncated Dirichlet
kernel and the Dirichlet kernel of the 2D + 1 taps themselves; each is
pinned by what the mathematics fixes:

* every kernel is cardinal (W(m) = delta_m0) and even;
* the periodic (2D + 1)-point kernel reproduces exactly any tone of
  k / (2D + 1) cycles per sample with |k| <= D (trigonometric interpolation
  of a band-limited periodic sequence);
* the untapered kernel tends to sinc as N grows, for any D;
* tone errors order as tapered < untapered < periodic inside the band, and
  the tapered kernel's error falls as D grows.
"""

import numpy as np
import pytest

from oracle import resamp

KINDS = (resamp.TAPERED, resamp.UNTAPERED, resamp.PERIODIC)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dterms", [1, 4, 8, 32])
def test_cardinal_and_even(kind, dterms):
    m = np.arange(-dterms, dterms + 1, dtype=np.float64)
    w = resamp.dirichlet_weight(m, 4096, dterms, kind)
    assert np.allclose(w, (m == 0).astype(float), atol=1e-13)
    x = np.linspace(-dterms - 0.5, dterms + 0.5, 97)
    assert np.allclose(resamp.dirichlet_weight(x, 4096, dterms, kind),
                       resamp.dirichlet_weight(-x, 4096, dterms, kind), atol=1e-15)


@pytest.mark.parametrize("dterms", [2, 4, 8])
def test_periodic_kernel_is_exact_for_its_tones(dterms):
    m = 2 * dterms + 1
    rng = np.random.default_rng(dterms)
    n = 400
    u = rng.uniform(dterms + 1, n - dterms - 2, 500)
    for k in range(-dterms, dterms + 1):
        z = np.exp(2j * np.pi * k * np.arange(n) / m)
        zi, valid = resamp.step_v(z, u, dterms, resamp.PERIODIC)
        assert valid.all()
        assert np.max(np.abs(zi - np.exp(2j * np.pi * k * u / m))) < 1e-12, k
    # and not for the other kernels
    z = np.exp(2j * np.pi * dterms * np.arange(n) / m)
    zi, _ = resamp.step_v(z, u, dterms, resamp.TAPERED)
    assert np.max(np.abs(zi - np.exp(2j * np.pi * dterms * u / m))) > 1e-3


def test_untapered_kernel_tends_to_sinc():
    x = np.linspace(-8.5, 8.5, 341)
    for d in (4, 8, 32):
        assert np.allclose(resamp.dirichlet_weight(x, 10**12, d, resamp.UNTAPERED), np.sinc(x), atol=1e-9)


def _tone_error(kind, dterms, nus=(0.05, 0.2, 0.3, 0.4)):
    n = 2048
    rng = np.random.default_rng(11)
    u = rng.uniform(100, n - 100, 3000)
    err = 0.0
    for nu in nus:
        z = np.exp(2j * np.pi * nu * np.arange(n))
        zi, _ = resamp.step_v(z, u, dterms, kind)
        err = max(err, float(np.max(np.abs(zi - np.exp(2j * np.pi * nu * u)))))
    return err


def test_tone_errors_order_by_kernel_and_fall_with_dterms():
    e = {k: _tone_error(k, 8) for k in KINDS}
    assert e[resamp.TAPERED] < 5e-3
    assert e[resamp.TAPERED] < e[resamp.UNTAPERED] < e[resamp.PERIODIC]
    assert 1e-2 < e[resamp.UNTAPERED] < 0.1
    assert 2e-2 < e[resamp.PERIODIC] < 0.2
    errs = [_tone_error(resamp.TAPERED, d) for d in (4, 8, 16, 32)]
    assert all(a > b for a, b in zip(errs, errs[1:])), errs


def test_unknown_kernel_rejected():
    with pytest.raises(ValueError):
        resamp.dirichlet_weight(np.array([0.5]), 100, 8, 7)
