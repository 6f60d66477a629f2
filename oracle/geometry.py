"""Roemer delay and antenna patterns (oracle, FP64).

Phase model (Sec. 2): Phi(t) = 2 pi f0 [t + t_m(t; alpha, delta)] + Phi_s,
with t_m the offset between detector time and Solar-System-barycentre (SSB)
time, t_b = t + t_m.  The paper takes t_m from LALSuite's ephemerides; here
t_m is the Roemer delay under a simplified ephemeris:

    r_orb(t)   = AU (cos th, cos eps sin th, sin eps sin th),  th = th0 + W_orb t
    r_rot,X(t) = R_E (cos lat cos ph, cos lat sin ph, sin lat), ph = lon + ph0 + W_rot t
    n          = (cos delta cos alpha, cos delta sin alpha, sin delta)
    t_m(t)     = (r_orb(t) + r_rot,X(t)) . n / c

Antenna patterns (Sec. 2 cites Jaranowski, Krolak & Schutz 1998, eqs. 12-13,
without printing them).  The oracle contracts tensors instead of using the
closed form: detector tensor d = (u u^T - v v^T)/2 with arms u, v at angles
gamma -/+ 45 deg from local East towards North, and polarisation tensors
e+ = x x^T - y y^T, ex = x y^T + y x^T built on the sky basis
x = (sin alpha, -cos alpha, 0), y = (-sin delta cos alpha, -sin delta sin alpha,
cos delta) -- the basis under which a = d:e+ and b = d:ex equal the JKS
closed forms (checked in the tests).
"""

from __future__ import annotations

import numpy as np


def sky_vector(alpha: float, delta: float) -> np.ndarray:
    return np.array([np.cos(delta) * np.cos(alpha), np.cos(delta) * np.sin(alpha), np.sin(delta)])


def orbit_position(t, eph) -> np.ndarray:
    """Earth-centre position relative to the SSB, metres, shape (..., 3)."""
    t = np.asarray(t, dtype=np.float64)
    th = eph["orb_phase0"] + eph["omega_orb"] * t
    eps = eph["obliquity"]
    c, s = np.cos(th), np.sin(th)
    return eph["au"] * np.stack([c, np.cos(eps) * s, np.sin(eps) * s], axis=-1)


def sidereal_angle(t, det, eph):
    """Longitude of the detector measured from the inertial x axis."""
    return det.lon + eph["sidereal_phase0"] + eph["omega_rot"] * np.asarray(t, dtype=np.float64)


def rotation_position(t, det, eph) -> np.ndarray:
    """Detector position relative to the Earth centre, metres, shape (..., 3)."""
    ph = sidereal_angle(t, det, eph)
    cl, sl = np.cos(det.lat), np.sin(det.lat)
    return eph["r_earth"] * np.stack([cl * np.cos(ph), cl * np.sin(ph), sl * np.ones_like(ph)], axis=-1)


def roemer_orbit(t, alpha, delta, eph):
    """Orbital part of t_m (shared by all detectors), seconds."""
    return orbit_position(t, eph) @ sky_vector(alpha, delta) / eph["c"]


def roemer_delay(t, det, alpha, delta, eph):
    """t_m(t) for detector ``det``: (r_orb + r_rot) . n / c, seconds."""
    n = sky_vector(alpha, delta)
    r = orbit_position(t, eph) + rotation_position(t, det, eph)
    return r @ n / eph["c"]


def detector_tensor(t, det, eph) -> np.ndarray:
    """d(t) = (u u^T - v v^T) / 2, shape (..., 3, 3)."""
    ph = sidereal_angle(t, det, eph)
    lat = det.lat
    east = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=-1)
    north = np.stack([-np.sin(lat) * np.cos(ph), -np.sin(lat) * np.sin(ph),
                      np.cos(lat) * np.ones_like(ph)], axis=-1)
    g1 = det.gamma - np.pi / 4.0
    g2 = det.gamma + np.pi / 4.0
    u = np.cos(g1) * east + np.sin(g1) * north
    v = np.cos(g2) * east + np.sin(g2) * north
    return 0.5 * (u[..., :, None] * u[..., None, :] - v[..., :, None] * v[..., None, :])


def polarisation_tensors(alpha: float, delta: float):
    x = np.array([np.sin(alpha), -np.cos(alpha), 0.0])
    y = np.array([-np.sin(delta) * np.cos(alpha), -np.sin(delta) * np.sin(alpha), np.cos(delta)])
    ep = np.outer(x, x) - np.outer(y, y)
    ex = np.outer(x, y) + np.outer(y, x)
    return ep, ex


def antenna_ab(t, det, alpha, delta, eph):
    """Antenna patterns a(t), b(t) (psi = 0 responses), each shape t.shape."""
    d = detector_tensor(t, det, eph)
    ep, ex = polarisation_tensors(alpha, delta)
    a = np.einsum("...ij,ij->...", d, ep)
    b = np.einsum("...ij,ij->...", d, ex)
    return a, b
