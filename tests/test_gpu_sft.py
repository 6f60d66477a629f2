"""GPU step (ii) from SFTs (fstat_set_sfts) against the oracle.

The oracle (oracle/sft.py) forms x_h per SFT by the defining sum; the GPU's
direct transform is held to FP32 accuracy (1e-5 of the series' largest
value) in mixed plans and to 1e-12 in FP64 plans, sample by sample.  The
whole chain from SFTs to 2F is then held to |d2F| <= 1e-3 2F + 0.02.
"""

import numpy as np
import pytest
import torch

import paper_2201_00451_gb300 as pkg
from oracle import resamp, sft
from workloads import make_noise, small_target

pytestmark = pytest.mark.gpu

T_SFT, M, NB, F_H = 8.0, 512, 32, 10.0   # raw 64 Hz, band 4 Hz, dt = 0.25 s
Q0 = int(F_H * T_SFT) - NB // 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


def _raw(seed, n_sft, tone=True):
    """Raw real series of n_sft SFTs: white noise plus an in-band tone."""
    n = n_sft * M
    rng = np.random.default_rng(seed)
    t = np.arange(n) * (T_SFT / M)
    x = rng.standard_normal(n)
    if tone:
        x = x + 0.5 * np.cos(2 * np.pi * (F_H + 0.37) * t + 1.1)
    return x


def _setup(seed, n_sft, precision=pkg.MIXED, n_det=2):
    t = small_target(n_samples=n_sft * NB, dt=T_SFT / NB, n_fft=1 << 14, n_det=n_det, f_het=F_H, seed=seed,
                     f1dots=(-1e-8, 0.0), f2dots=(0.0,), dtype="c64" if precision == pkg.MIXED else "c128")
    bands = []
    for X in range(n_det):
        sf = sft.sfts_from_series(_raw(seed + X, n_sft), M)
        bands.append(sft.band(sf, Q0, NB))
    xh = [sft.xh_from_band(b, Q0, t.t0, T_SFT, M, F_H) for b in bands]
    return t, bands, xh


@pytest.mark.parametrize("precision,tol", [(pkg.MIXED, 1e-5), (pkg.FP64, 1e-12)])
def test_series_from_sfts_matches_oracle(precision, tol):
    t, bands, xh = _setup(120, 50, precision)
    with pkg.FstatPlan.from_target(t, precision) as plan:
        for X in range(2):
            b = bands[X].astype(np.complex64) if X == 0 else bands[X]   # both input precisions
            plan.set_sfts(X, b, Q0, T_SFT, M, 1.0)
            got = plan.export_data(X)
            ref = xh[X] if X else sft.xh_from_band(b.astype(np.complex128), Q0, t.t0, T_SFT, M, F_H)
            assert got.dtype == (np.complex64 if precision == pkg.MIXED else np.complex128)
            assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_sfts_to_twoF_matches_oracle_chain():
    t, bands, xh = _setup(121, 80)
    sig = [float(np.std(x.real)) for x in xh]
    tm = t.templates()
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_sfts(X, bands[X], Q0, T_SFT, M, sig[X])
        got = plan.compute(tm).cpu().numpy()
        plan.sync()
    t.sigmas = tuple(sig)
    want = resamp.fstat(t, xh, tm)
    excess = np.abs(got - want) - (1e-3 * np.abs(want) + 0.02)
    assert excess.max() <= 0, excess.max()


def test_device_input_equals_host_input():
    t, bands, _ = _setup(122, 20)
    with pkg.FstatPlan.from_target(t) as plan:
        plan.set_sfts(0, bands[0], Q0, T_SFT, M, 1.0)
        host = plan.export_data(0)
        plan.set_sfts(0, torch.from_numpy(bands[0]).cuda(), Q0, T_SFT, M, 1.0)
        assert np.array_equal(plan.export_data(0), host)


def test_non_power_of_two_band_and_odd_sizes():
    # 3600 bins (a 2 Hz band of 1800 s SFTs at dt = 0.5 s), two SFTs
    t = small_target(n_samples=2 * 3600, dt=0.5, n_fft=1 << 14, n_det=1, f_het=100.0, seed=123, dtype="c64")
    q0 = int(100.0 * 1800.0) - 1800
    rng = np.random.default_rng(7)
    b = (rng.standard_normal((2, 3600)) + 1j * rng.standard_normal((2, 3600))).astype(np.complex64)
    ref = sft.xh_from_band(b.astype(np.complex128), q0, t.t0, 1800.0, 7200, 100.0)
    with pkg.FstatPlan.from_target(t) as plan:
        plan.set_sfts(0, b, q0, 1800.0, 7200, 1.0)
        got = plan.export_data(0)
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_argument_checks():
    t, bands, _ = _setup(124, 10, n_det=1)
    with pkg.FstatPlan.from_target(t) as plan:
        for kw in (dict(q0=Q0 + 1), dict(t_sft=T_SFT * 1.5)):
            args = dict(q0=Q0, t_sft=T_SFT)
            args.update(kw)
            with pytest.raises(pkg.FstatError) as e:
                plan.set_sfts(0, bands[0], args["q0"], args["t_sft"], M, 1.0)
            assert e.value.code == -1
        with pytest.raises(pkg.FstatError):           # wrong sample count
            plan.set_sfts(0, bands[0][:5], Q0, T_SFT, M, 1.0)
        with pytest.raises(pkg.FstatError):           # export before data
            plan.export_data(0)
