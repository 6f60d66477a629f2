"""Pins for the oracle's 2F gradient (CPU only).

* analytic d2F/df and d2F/df1dot equal central finite differences of 2F;
* the noise-free matched template is a stationary point of 2F (a maximum
  with value rho^2, the closed form of the brute-force pin), so every
  component of the gradient vanishes there;
* off the injection, the gradient points towards it.
"""

import numpy as np

from oracle import grad as og
from oracle import synth
from workloads import small_target


def _target(seed, noise):
    t = small_target(n_samples=4096, dt=1.0, n_fft=1 << 13, n_det=2, n_inj=1,
                     rho2_range=(200.0, 200.0), seed=seed, f1dots=(-2e-9,), f2dots=(0.0,))
    return t, synth.make_data(t, noise=noise)


def test_analytic_f_and_f1dot_derivatives_match_finite_differences():
    t, x = _target(31, noise=True)
    inj = t.injections[0]
    theta = np.array([inj.f0 + 0.3 / t.t_span, inj.f1dot + 0.2 / t.t_span ** 2, inj.alpha, inj.delta])
    v, g = og.grad(t, x, theta)
    steps = [1e-3 / t.t_span, 1e-3 / t.t_span ** 2]
    for i, h in enumerate(steps):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (og.twoF_at(t, x, tp) - og.twoF_at(t, x, tm)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-4 * abs(fd) + 1e-6 * abs(v) / h
    assert abs(v - og.twoF_at(t, x, theta)) < 1e-9 * abs(v)


def test_matched_noise_free_template_is_stationary():
    t, x = _target(32, noise=False)
    inj = t.injections[0]
    theta = np.array([inj.f0, inj.f1dot, inj.alpha, inj.delta])
    v, g = og.grad(t, x, theta)
    assert abs(v - inj.rho2) < 1e-8 * inj.rho2
    # gradient times a parameter scale over which 2F changes by O(rho^2)
    scale = np.array([1.0 / t.t_span, 1.0 / t.t_span ** 2, 1e-3, 1e-3])
    assert np.all(np.abs(g * scale) < 1e-4 * inj.rho2)


def test_gradient_points_uphill_towards_the_injection():
    t, x = _target(33, noise=False)
    inj = t.injections[0]
    df = 0.25 / t.t_span
    for sgn in (-1.0, 1.0):
        theta = np.array([inj.f0 + sgn * df, inj.f1dot, inj.alpha, inj.delta])
        v, g = og.grad(t, x, theta)
        assert v < inj.rho2
        assert np.sign(g[0]) == -sgn
