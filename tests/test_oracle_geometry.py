"""Pins for the oracle's timing model and antenna patterns (CPU only).

Each check compares the oracle with something other than itself: a closed
form of the circular-orbit / rigid-rotation geometry, the Jaranowski-Krolak-
Schutz closed-form antenna patterns (written out here independently of the
oracle's tensor contraction), or a special case with a known answer.
"""

import math

import numpy as np

from oracle import geometry as geo
from workloads import DETECTORS, EPHEMERIS
from workloads.configs import Detector

YEAR = 365.25636 * 86400.0
SIDEREAL_DAY = 86164.0905


def _eph(**kw):
    e = dict(EPHEMERIS)
    e.update(kw)
    return e


def test_ecliptic_pole_has_no_orbital_delay():
    # The orbit lies in the ecliptic plane, whose normal in equatorial
    # coordinates is (0, -sin eps, cos eps): alpha = 270 deg, delta = 90 - eps.
    eps = EPHEMERIS["obliquity"]
    alpha, delta = 1.5 * math.pi, 0.5 * math.pi - eps
    t = np.linspace(0.0, YEAR, 20001)
    tm = geo.roemer_orbit(t, alpha, delta, EPHEMERIS)
    assert np.max(np.abs(tm)) < 1e-6


def test_ecliptic_source_orbital_range_is_two_au_over_c():
    # A source in the ecliptic plane (the equinox direction alpha = delta = 0)
    # sees the full orbital diameter over one year: max - min = 2 AU / c.
    t = np.linspace(0.0, YEAR, 400001)
    tm = geo.roemer_orbit(t, 0.0, 0.0, EPHEMERIS)
    expect = 2.0 * EPHEMERIS["au"] / EPHEMERIS["c"]
    assert abs(expect - 998.0095) < 1e-3
    assert abs((tm.max() - tm.min()) - expect) < 1e-6


def test_t_m_at_origin_closed_form():
    # t = 0: orbital phase 0 -> Earth at (AU, 0, 0); sidereal angle = lon.
    det = DETECTORS["H1"]
    alpha, delta = 0.3, -0.7
    tm = float(geo.roemer_delay(0.0, det, alpha, delta, EPHEMERIS))
    c, au, re = EPHEMERIS["c"], EPHEMERIS["au"], EPHEMERIS["r_earth"]
    # spherical law of cosines for the site/source angle
    cos_ang = (math.sin(det.lat) * math.sin(delta)
               + math.cos(det.lat) * math.cos(delta) * math.cos(det.lon - alpha))
    expect = (au * math.cos(delta) * math.cos(alpha) + re * cos_ang) / c
    assert abs(tm - expect) < 1e-12


def test_rotation_term_daily_amplitude():
    # With no orbit, t_m oscillates once per sidereal day with peak-to-peak
    # 2 R_E cos(lat) cos(delta) / c about R_E sin(lat) sin(delta) / c.
    eph = _eph(au=0.0)
    det = DETECTORS["L1"]
    delta = 0.4
    t = np.linspace(0.0, SIDEREAL_DAY, 200001)
    tm = geo.roemer_delay(t, det, 1.1, delta, eph)
    re, c = eph["r_earth"], eph["c"]
    assert abs((tm.max() - tm.min()) - 2 * re * math.cos(det.lat) * math.cos(delta) / c) < 1e-9
    assert abs(0.5 * (tm.max() + tm.min()) - re * math.sin(det.lat) * math.sin(delta) / c) < 1e-9


def _jks_ab(t, det, alpha, delta, eph):
    """Jaranowski, Krolak & Schutz (1998) eqs. (12)-(13), arms at 90 deg."""
    lam, gam = det.lat, det.gamma
    h = alpha - (det.lon + eph["sidereal_phase0"] + eph["omega_rot"] * t)
    s2g, c2g = math.sin(2 * gam), math.cos(2 * gam)
    a = (s2g * (3 - math.cos(2 * lam)) * (3 - math.cos(2 * delta)) * np.cos(2 * h) / 16
         - c2g * math.sin(lam) * (3 - math.cos(2 * delta)) * np.sin(2 * h) / 4
         + s2g * math.sin(2 * lam) * math.sin(2 * delta) * np.cos(h) / 4
         - c2g * math.cos(lam) * math.sin(2 * delta) * np.sin(h) / 2
         + 3 * s2g * math.cos(lam) ** 2 * math.cos(delta) ** 2 / 4)
    b = (c2g * math.sin(lam) * math.sin(delta) * np.cos(2 * h)
         + s2g * (3 - math.cos(2 * lam)) * math.sin(delta) * np.sin(2 * h) / 4
         + c2g * math.cos(lam) * math.cos(delta) * np.cos(h)
         + s2g * math.sin(2 * lam) * math.cos(delta) * np.sin(h) / 2)
    return a, b


def test_antenna_patterns_match_jks_closed_form():
    rng = np.random.default_rng(5)
    dets = list(DETECTORS.values()) + [Detector("X", -33.0, 150.0, 17.0)]
    for det in dets:
        for _ in range(4):
            alpha = rng.uniform(0, 2 * math.pi)
            delta = math.asin(rng.uniform(-1, 1))
            t = rng.uniform(0, 3e7, 64)
            a, b = geo.antenna_ab(t, det, alpha, delta, EPHEMERIS)
            aj, bj = _jks_ab(t, det, alpha, delta, EPHEMERIS)
            assert np.max(np.abs(a - aj)) < 1e-12
            assert np.max(np.abs(b - bj)) < 1e-12


def test_zenith_source_has_full_response():
    # A source straight overhead sees the wave in the detector plane:
    # F+^2 + Fx^2 = a^2 + b^2 = 1 for perpendicular arms.
    for det in DETECTORS.values():
        t = 12345.0
        phi = det.lon + EPHEMERIS["sidereal_phase0"] + EPHEMERIS["omega_rot"] * t
        a, b = geo.antenna_ab(np.array([t]), det, phi, det.lat, EPHEMERIS)
        assert abs(a[0] ** 2 + b[0] ** 2 - 1.0) < 1e-12


def test_antenna_only_sidereal_harmonics_0_1_2():
    det = DETECTORS["H1"]
    n = 1024
    t = np.arange(n) * SIDEREAL_DAY / n
    a, b = geo.antenna_ab(t, det, 2.0, -0.3, EPHEMERIS)
    for x in (a, b):
        spec = np.abs(np.fft.rfft(x)) / n
        assert np.max(spec[3:]) < 1e-12
        assert np.max(spec[:3]) > 1e-3


def test_abc_positive_definite_over_a_day():
    rng = np.random.default_rng(9)
    t = np.linspace(0, 86400.0, 2001)
    for _ in range(8):
        alpha = rng.uniform(0, 2 * math.pi)
        delta = math.asin(rng.uniform(-1, 1))
        a, b = geo.antenna_ab(t, DETECTORS["L1"], alpha, delta, EPHEMERIS)
        A, B, C = np.sum(a * a), np.sum(b * b), np.sum(a * b)
        assert A * B - C * C > 1e-6 * A * B
