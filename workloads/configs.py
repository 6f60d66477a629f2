"""Workload definitions: detector sites, sample grids, template banks, seeds.

Everything here is configuration data or a seeded random draw.  The sizes and
shapes follow the narrowband searches the paper benchmarks and runs: 10-day
spans at sub-Hz to few-Hz bands (Sec. 4, "Performance"), and the 100-day,
1 Hz-band pilot search towards Omega Centauri (Sec. 5, Table 3).  The paper's
own data (Makefakedata_v4 output, LIGO O2 strain) are not available here; the
seeded Gaussian noise plus injected signals stand in for them.
"""

from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

from .gen import draw_injections, draw_sigmas, template_grid

DAY = 86400.0


@dataclass(frozen=True)
class Detector:
    """An interferometer site: geodetic latitude and longitude, and the angle
    gamma of the arm bisector measured counter-clockwise from local East."""

    name: str
    lat_deg: float
    lon_deg: float
    gamma_deg: float

    @property
    def lat(self) -> float:
        return math.radians(self.lat_deg)

    @property
    def lon(self) -> float:
        return math.radians(self.lon_deg)

    @property
    def gamma(self) -> float:
        return math.radians(self.gamma_deg)


# Site latitudes/longitudes are the ones the workloads specify; the arm
# orientations are the LIGO Hanford / Livingston values of Jaranowski,
# Krolak & Schutz (1998), the antenna-pattern reference the paper cites in
# Sec. 2.
DETECTORS = {
    "H1": Detector("H1", 46.455, -119.408, 171.8),
    "L1": Detector("L1", 30.563, -90.774, 243.0),
}

# Simplified ephemeris: circular Earth orbit of radius 1 AU in the ecliptic,
# uniform sidereal rotation, orbital phase and Greenwich sidereal angle zero
# at t = 0.  Roemer delay only.
EPHEMERIS = {
    "c": 299792458.0,                       # m/s
    "au": 1.495978707e11,                   # m
    "r_earth": 6.371e6,                     # m (spherical Earth)
    "omega_rot": 2.0 * math.pi / 86164.0905,            # rad/s, sidereal day
    "omega_orb": 2.0 * math.pi / (365.25636 * DAY),     # rad/s, sidereal year
    "obliquity": math.radians(23.4393),     # rad
    "orb_phase0": 0.0,                      # rad
    "sidereal_phase0": 0.0,                 # rad
}


@dataclass(frozen=True)
class Injection:
    """Parameters of one injected CW signal (amplitude set by rho^2)."""

    f0: float        # Hz, frequency at the reference time
    f1dot: float     # Hz/s
    f2dot: float     # Hz/s^2
    alpha: float     # rad
    delta: float     # rad
    rho2: float      # optimal SNR^2 over all detectors
    cosi: float
    psi: float       # rad
    phi0: float      # rad
    bin_index: int   # ascending-frequency bin the injection sits on


@dataclass
class Target:
    """One data set (all detectors share the sample grid) and its template bank."""

    name: str
    detectors: tuple
    t0: float
    dt: float
    n_samples: int
    f_het: float
    n_fft: int
    dterms: int
    sigmas: tuple
    dtype: str                       # "c128" or "c64": storage of x_h
    skies: tuple                     # ((alpha, delta), ...) rad
    f1dots: np.ndarray
    f2dots: np.ndarray
    injections: tuple = ()
    seed: int = 0
    t_ref: float = float("nan")      # NaN -> t0 + (n_samples // 2) * dt
    ephemeris: dict = field(default_factory=lambda: dict(EPHEMERIS))
    interp: int = 0                  # interpolation kernel: 0 tapered Dirichlet, 1 untapered, 2 periodic 2D+1

    @property
    def t_span(self) -> float:
        return self.n_samples * self.dt

    @property
    def t_reference(self) -> float:
        if math.isnan(self.t_ref):
            return self.t0 + (self.n_samples // 2) * self.dt
        return self.t_ref

    @property
    def df(self) -> float:
        return 1.0 / (self.n_fft * self.dt)

    def freq(self, m):
        """Frequency of ascending bin m: f_h + (m - n_fft/2) * df."""
        return self.f_het + (np.asarray(m) - self.n_fft // 2) * self.df

    def templates(self) -> np.ndarray:
        """All templates, sky-major, then f2dot, then f1dot (fastest)."""
        return template_grid(self.skies, self.f1dots, self.f2dots)

    @property
    def n_templates(self) -> int:
        return len(self.skies) * len(self.f1dots) * len(self.f2dots)


def _hms(h, m, s):
    return math.radians(15.0 * (h + m / 60.0 + s / 3600.0))


def _dms(d, m, s):
    sgn = -1.0 if d < 0 or (d == 0 and (m < 0 or s < 0)) else 1.0
    return sgn * math.radians(abs(d) + abs(m) / 60.0 + abs(s) / 3600.0)


def _spindown_steps(t_span):
    # f1dot spacing 1/(4 T^2) and f2dot spacing 1/(8 T^3): fine enough that an
    # on-grid injection is recovered and the range does not change throughput.
    return 1.0 / (4.0 * t_span**2), 1.0 / (8.0 * t_span**3)


def config1(realisation: int = 0) -> Target:
    """Plain method, FP64: 1 detector, 2 days at dt = 2 s (86 400 samples,
    complex128), unit complex variance, one injection at rho^2 ~ 100, one sky
    position, 64 f1dot templates on [-1e-10, 0] Hz/s, Dterms 8, FFT 2^18.
    The sky position is the injection of the paper's Fig. 2 (Sec. 4.2)."""
    seed = 1000 * 1 + realisation
    n, dt = 86400, 2.0
    f1 = np.linspace(-1e-10, 0.0, 64)
    f2 = np.array([0.0])
    sky = (_hms(16, 19, 55.09), _dms(-14, 21, 35.1))
    t = Target(
        name="cfg1", detectors=(DETECTORS["H1"],), t0=0.0, dt=dt, n_samples=n,
        f_het=100.0, n_fft=1 << 18, dterms=8, sigmas=(1.0 / math.sqrt(2.0),),
        dtype="c128", skies=(sky,), f1dots=f1, f2dots=f2, seed=seed,
    )
    t.injections = draw_injections(t, n_inj=1, rho2_range=(100.0, 100.0),
                                   min_sep_bins=200, seed=seed)
    return t


def config2(realisation: int = 0) -> Target:
    """Narrowband single target, mixed precision: H1 + L1, 10 days at
    dt = 0.5 s (1 728 000 complex64 samples per detector), sigma_X ~ U[0.8,
    1.2], 10 injections rho^2 ~ U[40, 400], one sky position,
    8192 f1dot x 4 f2dot templates, Dterms 8, FFT 2^22.  The sky position is
    the injection of the paper's Fig. 3 (Sec. 4.2)."""
    seed = 1000 * 2 + realisation
    n, dt = 1_728_000, 0.5
    t_span = n * dt
    s1, s2 = _spindown_steps(t_span)
    f1 = -s1 * np.arange(8191, -1, -1, dtype=np.float64)       # ends at 0
    f2 = s2 * (np.arange(4, dtype=np.float64) - 1.5)             # centred on 0
    sky = (0.0, _dms(-28, 48, 0.0))
    t = Target(
        name="cfg2", detectors=(DETECTORS["H1"], DETECTORS["L1"]), t0=0.0,
        dt=dt, n_samples=n, f_het=100.0, n_fft=1 << 22, dterms=8,
        sigmas=draw_sigmas(seed, 2, 0.8, 1.2), dtype="c64", skies=(sky,),
        f1dots=f1, f2dots=f2, seed=seed,
    )
    t.injections = draw_injections(t, n_inj=10, rho2_range=(40.0, 400.0),
                                   min_sep_bins=200, seed=seed)
    return t


def config3(realisation: int = 0) -> list:
    """Batched uneven targets: 4 sky positions uniform on the sphere, each
    with band U{0.5, 1, 2, 4} Hz and span U{1, 3, 10, 30} days (dt = 1/band),
    H1 + L1, 2 injections per target, log-uniform 512..16384 f1dot templates,
    N_FFT = clamp(nextpow2(2 N), 2^18, 2^24), f_h ~ U[145, 490] Hz (the pilot
    search's band range, Table 3)."""
    seed = 1000 * 3 + realisation
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(4):
        band = float(rng.choice([0.5, 1.0, 2.0, 4.0]))
        days = float(rng.choice([1.0, 3.0, 10.0, 30.0]))
        dt = 1.0 / band
        n = int(round(band * days * DAY))
        n_fft = int(min(max(1 << int(math.ceil(math.log2(2 * n))), 1 << 18), 1 << 24))
        alpha = float(rng.uniform(0.0, 2.0 * math.pi))
        delta = float(math.asin(rng.uniform(-1.0, 1.0)))
        n_f1 = int(round(math.exp(rng.uniform(math.log(512), math.log(16384)))))
        s1, _ = _spindown_steps(n * dt)
        f1 = -s1 * np.arange(n_f1 - 1, -1, -1, dtype=np.float64)
        tseed = seed * 10 + k
        t = Target(
            name=f"cfg3.{k}", detectors=(DETECTORS["H1"], DETECTORS["L1"]),
            t0=0.0, dt=dt, n_samples=n, f_het=float(rng.uniform(145.0, 490.0)),
            n_fft=n_fft, dterms=8, sigmas=draw_sigmas(tseed, 2, 0.8, 1.2),
            dtype="c64", skies=((alpha, delta),), f1dots=f1,
            f2dots=np.array([0.0]), seed=tseed,
        )
        t.injections = draw_injections(t, n_inj=2, rho2_range=(40.0, 400.0),
                                       min_sep_bins=200, seed=tseed)
        out.append(t)
    return out


def config5(realisation: int = 0) -> Target:
    """Large narrowband search: H1 + L1, 120 days at dt = 1 s (10 368 000
    complex64 samples per detector), 20 injections rho^2 ~ U[30, 300], 64 sky
    positions on an 8 x 8 grid inside a 1' x 1' patch at the Omega Centauri
    pointing of the pilot search (Sec. 5.2), 2048 f1dot x 8 f2dot, FFT 2^24."""
    seed = 1000 * 5 + realisation
    n, dt = 10_368_000, 1.0
    s1, s2 = _spindown_steps(n * dt)
    f1 = -s1 * np.arange(2047, -1, -1, dtype=np.float64)
    f2 = s2 * (np.arange(8, dtype=np.float64) - 3.5)
    a0, d0 = _hms(13, 26, 44.0), _dms(-47, 29, 40.0)
    arcmin = math.radians(1.0 / 60.0)
    skies = tuple(
        (a0 + (i - 3.5) / 8.0 * arcmin / math.cos(d0), d0 + (k - 3.5) / 8.0 * arcmin)
        for k in range(8) for i in range(8)
    )
    t = Target(
        name="cfg5", detectors=(DETECTORS["H1"], DETECTORS["L1"]), t0=0.0,
        dt=dt, n_samples=n, f_het=float(np.round(np.random.Generator(
            np.random.PCG64(seed)).uniform(145.0, 490.0), 3)),
        n_fft=1 << 24, dterms=8, sigmas=draw_sigmas(seed, 2, 0.8, 1.2),
        dtype="c64", skies=skies, f1dots=f1, f2dots=f2, seed=seed,
    )
    t.injections = draw_injections(t, n_inj=20, rho2_range=(30.0, 300.0),
                                   min_sep_bins=200, seed=seed)
    return t


def small_target(n_samples=3001, dt=2.0, n_fft=1 << 13, n_det=1, f_het=100.0,
                 skies=None, f1dots=(0.0,), f2dots=(0.0,), seed=7, dtype="c128",
                 sigmas=None, t0=0.0, dterms=8, n_inj=0, rho2_range=(100.0, 100.0),
                 t_ref=float("nan"), detectors=None, interp=0) -> Target:
    """A small data set for tests: sizes chosen by the caller, defaults give a
    ragged sample count (not a multiple of any tile) padded to 2^13."""
    if detectors is None:
        detectors = (DETECTORS["H1"], DETECTORS["L1"])[:n_det]
    if skies is None:
        rng = np.random.Generator(np.random.PCG64(seed))
        skies = ((float(rng.uniform(0, 2 * math.pi)), float(math.asin(rng.uniform(-1, 1)))),)
    if sigmas is None:
        sigmas = draw_sigmas(seed, len(detectors), 0.8, 1.2)
    t = Target(
        name="small", detectors=tuple(detectors), t0=t0, dt=dt, n_samples=n_samples,
        f_het=f_het, n_fft=n_fft, dterms=dterms, sigmas=tuple(sigmas), dtype=dtype,
        skies=tuple(skies), f1dots=np.asarray(f1dots, dtype=np.float64),
        f2dots=np.asarray(f2dots, dtype=np.float64), seed=seed, t_ref=t_ref, interp=interp,
    )
    if n_inj:
        t.injections = draw_injections(t, n_inj=n_inj, rho2_range=rho2_range,
                                       min_sep_bins=min(200, n_fft // (4 * n_inj)),
                                       seed=seed)
    return t


def split_segments(t: Target, n_seg: int) -> list:
    """Equal consecutive segments of a target's sample grid (the last one
    takes any remainder) for a semi-coherent search: each keeps the target's
    detectors, dt, f_h, n_fft, noise levels, sky and spindown grids, and
    gets its own reference time (its midpoint).  Slice the data with
    ``segment_slices``."""
    n = t.n_samples // n_seg
    out = []
    for k in range(n_seg):
        start = k * n
        cnt = n if k < n_seg - 1 else t.n_samples - start
        out.append(dataclasses.replace(
            t, name=f"{t.name}.seg{k}", t0=t.t0 + start * t.dt, n_samples=cnt, injections=(),
            t_ref=float("nan")))
    return out


def segment_slices(t: Target, n_seg: int) -> list:
    """(start, count) of each segment of ``split_segments``."""
    n = t.n_samples // n_seg
    return [(k * n, n if k < n_seg - 1 else t.n_samples - k * n) for k in range(n_seg)]

