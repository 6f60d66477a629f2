"""GPU parity: libfstat (through its C ABI) against the FP64 oracle.

Tolerance for the mixed-precision path: |d2F| <= 1e-3 * 2F + 0.02 per
element (the stated target).  The FP64 path is held to 1e-7 relative.
Inputs are the oracle's seeded synthetic data (noise + injections).
"""

import numpy as np
import pytest

import paper_2201_00451_gb300 as pkg
from oracle import resamp, synth
from workloads import config1, small_target

pytestmark = pytest.mark.gpu

REL, ABS = 1e-3, 0.02


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


def run_gpu(t, x, templates, precision=pkg.MIXED, split=None, sigmas=None):
    with pkg.FstatPlan.from_target(t, precision) as plan:
        if split:
            plan.set_split(split)
        for X in range(len(t.detectors)):
            plan.set_data(X, x[X], (sigmas or t.sigmas)[X])
        out = plan.compute(templates)
        plan.sync()
        return out.cpu().numpy()


def assert_parity(gpu, ref, rel=REL, abs_=ABS):
    assert gpu.shape == ref.shape
    assert np.all(np.isfinite(gpu))
    excess = np.abs(gpu - ref) - (rel * np.abs(ref) + abs_)
    i = int(np.argmax(excess))
    assert excess.flat[i] <= 0, (
        f"worst element {np.unravel_index(i, gpu.shape)}: gpu {gpu.flat[i]} oracle {ref.flat[i]}")


def small(seed=3, **kw):
    args = dict(n_samples=3001, dt=2.0, n_fft=1 << 13, n_det=2, n_inj=1, rho2_range=(150.0, 150.0),
                seed=seed, f1dots=(-6e-10, -3e-10, 0.0), f2dots=(-1e-15, 1e-15), dtype="c64")
    args.update(kw)
    return small_target(**args)


def test_small_ragged_two_detectors_mixed():
    t = small()
    x = synth.make_data(t)
    tm = t.templates()
    assert_parity(run_gpu(t, x, tm), resamp.fstat(t, x, tm))


def test_small_fp64_path_matches_oracle_tightly():
    t = small(seed=4, dtype="c128")
    x = synth.make_data(t)
    tm = t.templates()
    assert_parity(run_gpu(t, x, tm, precision=pkg.FP64), resamp.fstat(t, x, tm), rel=1e-7, abs_=1e-7)


# FP64 bound: f_h t_m reaches ~5e4 cycles, so a few ulps of t_m (different
# operation order on the two sides) move the step-(iii) phase by ~1e-10 rad.
@pytest.mark.parametrize("precision,tol", [(pkg.MIXED, 2e-5), (pkg.FP64, 3e-10)])
def test_per_sky_intermediates(precision, tol):
    # G_a, G_b (steps iii-v, antenna weighting, detector sum) and A, B, C, D.
    t = small(seed=5, n_samples=5003, n_fft=1 << 14)
    x = synth.make_data(t)
    a, d = t.skies[0]
    ref = resamp.sky_prep(t, x, a, d)
    with pkg.FstatPlan.from_target(t, precision) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        ga, gb, abcd = plan.export_sky(a, d)
    scale = max(np.abs(ref["Ga"]).max(), np.abs(ref["Gb"]).max())
    assert np.abs(ga - ref["Ga"]).max() <= tol * scale
    assert np.abs(gb - ref["Gb"]).max() <= tol * scale
    for k, v in zip("ABCD", abcd):
        assert abs(v - ref[k]) <= 1e-10 * abs(ref[k]) + 1e-12


@pytest.mark.parametrize("n1", [32, 64, 256, 512])
def test_every_fft_split_agrees(n1):
    t = small(seed=6, n_fft=1 << 14, n_samples=6007)
    x = synth.make_data(t)
    tm = t.templates()[:2]
    assert_parity(run_gpu(t, x, tm, split=n1), resamp.fstat(t, x, tm))


@pytest.mark.parametrize("log2n", [10, 12, 16, 20])
def test_fft_lengths(log2n):
    n = min((1 << log2n) - 7, 200_003)
    t = small(seed=7 + log2n, n_fft=1 << log2n, n_samples=n, dt=1.0, f1dots=(-1e-11,), f2dots=(0.0,))
    x = synth.make_data(t)
    tm = t.templates()
    assert_parity(run_gpu(t, x, tm), resamp.fstat(t, x, tm))


def test_several_skies_in_one_call_keep_row_order():
    t = small(seed=9, n_samples=2001, n_fft=1 << 12,
              skies=((0.3, -0.4), (2.0, 0.9), (4.4, 0.1)), f1dots=(-5e-10, 0.0), f2dots=(0.0,))
    x = synth.make_data(t)
    tm = t.templates()
    rng = np.random.default_rng(0)
    tm = tm[rng.permutation(len(tm))]  # interleave sky positions
    assert_parity(run_gpu(t, x, tm), resamp.fstat(t, x, tm))


def test_no_zero_padding_and_tiny_series():
    t = small(seed=10, n_samples=1024, n_fft=1024, dt=1.0, n_inj=0)
    x = synth.make_data(t)
    tm = t.templates()[:2]
    assert_parity(run_gpu(t, x, tm), resamp.fstat(t, x, tm))
    t = small(seed=11, n_samples=17, n_fft=1024, dt=1.0, n_inj=0)
    x = synth.make_data(t)
    tm = t.templates()[:1]
    assert_parity(run_gpu(t, x, tm), resamp.fstat(t, x, tm))


def test_zero_input_gives_exact_zero():
    t = small(seed=12, n_inj=0)
    x = [np.zeros(t.n_samples, dtype=np.complex64) for _ in range(2)]
    out = run_gpu(t, x, t.templates()[:2])
    assert np.all(out == 0.0)


def test_repeated_calls_are_bitwise_identical():
    t = small(seed=13)
    x = synth.make_data(t)
    tm = t.templates()
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        a = plan.compute(tm).cpu().numpy()
        plan.invalidate_sky()
        b = plan.compute(tm).cpu().numpy()
    assert np.array_equal(a, b)


def test_errors_are_reported():
    t = small(seed=14, n_inj=0)
    x = synth.make_data(t)
    with pkg.FstatPlan.from_target(t) as plan:
        with pytest.raises(pkg.FstatError) as e:
            plan.compute(t.templates()[:1])
        assert e.value.code == -6  # not ready
        bad = x[0].copy()
        bad[100] = np.nan
        with pytest.raises(pkg.FstatError) as e:
            plan.set_data(0, bad, t.sigmas[0])
        assert e.value.code == -5  # non-finite
        with pytest.raises(pkg.FstatError) as e:
            plan.set_data(0, x[0][:-1], t.sigmas[0])
        assert e.value.code == -1
    # a single sample gives A B - C^2 = 0: degenerate
    t1 = small(seed=15, n_samples=1, n_fft=1024, n_det=1, n_inj=0)
    with pkg.FstatPlan.from_target(t1) as plan:
        plan.set_data(0, np.ones(1, dtype=np.complex64), 1.0)
        plan.compute(t1.templates()[:1])
        with pytest.raises(pkg.FstatError) as e:
            plan.sync()
        assert e.value.code == -4


def test_config1_plain_method_both_precisions():
    # 1 detector, 2 days at dt = 2 s (86 400 complex128 samples), FFT 2^18,
    # 64 f1dot templates, one injection at rho^2 ~ 100.
    t = config1()
    x = synth.make_data(t)
    tm = t.templates()
    ref = resamp.fstat(t, x, tm)
    assert_parity(run_gpu(t, x, tm), ref)
    assert_parity(run_gpu(t, x, tm, precision=pkg.FP64), ref, rel=1e-7, abs_=1e-7)
    inj = t.injections[0]
    k = int(np.argmin(np.abs(t.f1dots - inj.f1dot)))
    assert ref[k, inj.bin_index] > 0.9 * inj.rho2


def test_gpu_noise_statistics_chi2_4():
    t = small(seed=16, n_samples=1 << 17, n_fft=1 << 18, dt=1.0, n_inj=0,
              f1dots=(0.0,), f2dots=(0.0,))
    x = synth.make_data(t)
    out = run_gpu(t, x, t.templates())[0]
    half, lim = t.n_fft // 2, int(0.4 * t.n_fft)
    s = out[half - lim: half + lim: 2]
    assert abs(s.mean() - 4.0) < 3 * np.sqrt(8.0 / len(s))


def test_physical_units_give_the_same_2F():
    # 2F is invariant under a common rescaling x_X -> c x_X, sigma_X -> c
    # sigma_X of every detector; strain-scaled data (sigma ~ 1e-23) must not
    # overflow anywhere in FP32.
    t = small(seed=18)
    x = synth.make_data(t)
    tm = t.templates()
    ref = run_gpu(t, x, tm)
    scale = [3e-23, 3e-23]
    xs = [(x[X].astype(np.complex128) * scale[X]).astype(np.complex64) for X in range(2)]
    sig = [t.sigmas[X] * scale[X] for X in range(2)]
    got = run_gpu(t, xs, tm, sigmas=sig)
    assert np.all(np.isfinite(got))
    assert_parity(got, ref, rel=1e-4, abs_=1e-3)


def test_residency_caps_and_single_buffer_schedules_give_identical_2F():
    # The per-SM cap of the persistent passes and the one-buffer schedules
    # change only how tiles are scheduled, never the arithmetic: bitwise.
    t = small(seed=12, n_fft=1 << 18, n_samples=100_003, dt=1.0)
    x = synth.make_data(t)
    tm = t.templates()[:3]
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.set_split(512)            # both passes of length 512: every schedule compiled
        plan.set_cta(2, 2, 0, 0)
        base = plan.compute(tm).cpu().numpy()
        for ra, rb in ((1, 1), (2, 1), (1, 3)):
            plan.set_residency(ra, rb)
            assert np.array_equal(plan.compute(tm).cpu().numpy(), base)
        plan.set_residency(0, 0)
        plan.set_cta(2, 2, 2, 2)
        assert np.array_equal(plan.compute(tm).cpu().numpy(), base)
        with pytest.raises(pkg.FstatError):
            plan.set_residency(-1, 0)
    assert_parity(base, resamp.fstat(t, x, tm))


def test_register_caps_and_tma_loads_give_identical_2F():
    # Radix-16 schedules that differ only in buffering, register cap (two
    # or three CTAs per SM) and how pass B's tiles arrive in shared memory
    # (cp.async or TMA) run the same arithmetic: bitwise equal 2F.
    t = small(seed=13, n_fft=1 << 20, n_samples=400_003, dt=1.0)
    x = synth.make_data(t)
    tm = t.templates()[:3]
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.set_split(1024)           # pass A 1024 points, pass B 1024 points
        plan.set_cta(1, 4, 0, 0)
        base = plan.compute(tm).cpu().numpy()
        # and pass B with half of each next tile staged apart (vb 8)
        for ca, cb, va, vb in ((1, 4, 2, 2), (1, 4, 10, 4), (1, 4, 10, 6), (1, 2, 2, 6), (2, 8, 2, 4),
                               (1, 4, 2, 8), (1, 8, 10, 8), (2, 1, 0, 8)):
            plan.set_cta(ca, cb, va, vb)
            assert plan.cta == (ca, va, cb, vb)
            assert np.array_equal(plan.compute(tm).cpu().numpy(), base), (ca, cb, va, vb)
        for bad in ((1, 4, 4, 0), (1, 4, 11, 0), (1, 4, 0, 9)):
            with pytest.raises(pkg.FstatError):
                plan.set_cta(*bad)
    assert_parity(base, resamp.fstat(t, x, tm))


@pytest.mark.parametrize("n", [300_001, 1_000_003])
def test_staged_4096_point_columns_give_identical_2F(n):
    # Schedule 18: 4096-point columns (256 threads, two CTAs per SM where
    # the staging allows) with the next column staged apart, against
    # schedule 2 (staged in the column buffer): bitwise equal 2F.
    t = small(seed=23, n_fft=1 << 20, n_samples=n, dt=1.0)
    x = synth.make_data(t)
    tm = t.templates()[:3]
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.set_split(256)            # pass A 4096 points, pass B 256
        plan.set_cta(1, 0, 2, 0)
        base = plan.compute(tm).cpu().numpy()
        plan.set_cta(1, 0, 18, 0)
        assert plan.cta[1] == 18
        assert np.array_equal(plan.compute(tm).cpu().numpy(), base)
        plan.sync()
    assert_parity(base, resamp.fstat(t, x, tm))


@pytest.mark.parametrize("n", [600_001, 1_000_003, 1_400_001])
def test_staged_8192_point_columns_give_identical_2F(n):
    # Pass A's schedule 16 stages the next column's samples densely in shared
    # memory of their own (one bulk copy) instead of at padded positions in
    # the column buffer: the same arithmetic, bitwise equal 2F.  600 001
    # samples leave the upper half of every column empty (the half-size
    # first butterflies); 1 400 001 is the most samples per column
    # (5469 of 8192) whose staging still fits beside the column buffer.
    t = small(seed=17, n_fft=1 << 21, n_samples=n, dt=1.0)
    x = synth.make_data(t)
    tm = t.templates()[:3]
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.set_split(256)            # pass A 8192 points, pass B 256
        plan.set_cta(1, 0, 0, 0)
        base = plan.compute(tm).cpu().numpy()
        plan.set_cta(1, 0, 16, 0)
        assert plan.cta[1] == 16
        assert np.array_equal(plan.compute(tm).cpu().numpy(), base)
        plan.sync()
    assert_parity(base, resamp.fstat(t, x, tm))


def test_staged_8192_point_columns_refused_when_the_staging_does_not_fit():
    # 2 000 003 samples over 256 columns: 7813 per column, whose staging
    # (122 KB) does not fit beside the 136 KB column buffer; the launch is
    # refused before anything runs and the plan stays usable.
    t = small(seed=19, n_fft=1 << 21, n_samples=2_000_003, dt=1.0)
    x = synth.make_data(t)
    tm = t.templates()[:2]
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.set_split(256)
        plan.set_cta(1, 0, 16, 0)
        with pytest.raises(pkg.FstatError) as e:
            plan.compute(tm)
        assert e.value.code == -3
        plan.set_cta(1, 0, 0, 0)
        out = plan.compute(tm).cpu().numpy()
        plan.sync()
    assert_parity(out, resamp.fstat(t, x, tm))


@pytest.mark.parametrize("t_ref_days", [-40.0, -450.0, 500.0])
def test_reference_time_far_outside_the_data(t_ref_days):
    # A spindown reference time far from the data (up to ~2.2e7 samples of
    # 2 s away, beyond the 2^24 sample offsets FP32 holds exactly): the phase
    # polynomial is expanded about the data sample nearest t_ref, so the
    # sample offsets stay below the data length and 2F still matches the
    # oracle.
    t = small(seed=31, t_ref=t_ref_days * 86400.0, f1dots=(-3e-13, 0.0, 2e-13), f2dots=(0.0, 2e-21))
    x = synth.make_data(t)
    tm = t.templates()
    assert_parity(run_gpu(t, x, tm), resamp.fstat(t, x, tm))


def test_spindown_phase_excursion_beyond_range_is_rejected():
    # |f1dot| tau^2 over the data above 2^20 cycles cannot be reduced exactly
    # in the FP32 path's phase evaluation: the call is refused, not computed.
    t = small(seed=32, t_ref=-400.0 * 86400.0, f1dots=(1e-9,), f2dots=(0.0,))
    x = synth.make_data(t)
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        with pytest.raises(pkg.FstatError) as e:
            plan.compute(t.templates())
        assert e.value.code == -7
        plan.sync()
