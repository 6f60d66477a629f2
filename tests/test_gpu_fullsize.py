"""GPU parity for every FFT shape the autotuner may pick, and at full size.

* Every compiled (split, pass-A columns per CTA, pass-B rows per CTA) gives
  the oracle's 2F within |d2F| <= 1e-3 2F + 0.02.
* The 10-day two-detector workload at full size (1 728 000 samples,
  FFT 2^22, 10 injections), autotuned exactly as bench.py runs it: 2F at the
  injected bins and at random bins matches the oracle's direct DFT sums,
  two whole rows match the oracle's FFT bin for bin, and each injection is
  recovered near its rho^2.
* The 120-day workload (10 368 000 samples, FFT 2^24): sampled bins of
  several templates and one whole row against the oracle.
"""

import numpy as np
import pytest

import paper_2201_00451_gb300 as pkg
from oracle import resamp, synth
from workloads import config2, small_target

pytestmark = pytest.mark.gpu

REL, ABS = 1e-3, 0.02


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


def _ok(gpu, ref):
    return np.all(np.abs(gpu - ref) <= REL * np.abs(ref) + ABS)


@pytest.mark.parametrize("log2n,n", [(18, 150_001), (19, 200_003), (20, 400_003), (22, 1_000_003),
                                     (24, 1_000_003)])
def test_every_split_and_cta_shape(log2n, n):
    t = small_target(n_samples=n, dt=1.0, n_fft=1 << log2n, n_det=2, n_inj=1,
                     rho2_range=(200.0, 200.0), seed=100 + log2n, f1dots=(0.0, 2e-9),
                     f2dots=(0.0,), dtype="c64")
    x = synth.make_data(t)
    tm = t.templates()
    ref = resamp.fstat(t, x, tm)
    ran = 0
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        # pass A columns up to 8192 points (FP32), pass B rows up to 4096
        for l1 in range(max(5, log2n - 13), min(12, log2n - 5) + 1):
            plan.set_split(1 << l1)
            # radix-8 first (bit 0), one shared buffer (bit 1), pass B tile
            # loads by TMA (bit 2, rows of 1024 points or more), pass A
            # three CTAs per SM (va 10), and columns staged apart (va 16 at
            # 8192 points, 18 at 4096; one column per CTA)
            # and pass B with half of the next tile staged apart (vb 8)
            for v in range(12):
                va, vb = {8: (10, 2), 9: (16, 0), 10: (18, 6), 11: (2, 8)}.get(v, (v & 3, v))
                for ca, cb in [(0, 0), (1, 1), (2, 2), (4, 4), (1, 8), (2, 8)]:
                    plan.set_cta(ca, cb, va, vb)
                    # the two templates swap places from one shape to the
                    # next, so a pass that left its intermediate unwritten
                    # would return the other template's 2F
                    order = [0, 1] if ran % 2 == 0 else [1, 0]
                    try:
                        out = plan.compute(tm[order]).cpu().numpy()
                    except pkg.FstatError as e:
                        assert e.code == -3  # shape not compiled for this length
                        continue
                    for i, k in enumerate(order):
                        assert _ok(out[i], ref[k]), (l1, ca, cb, va, vb, k)
                    ran += 1
        plan.sync()
    assert ran >= 3


def test_autotune_choice_is_correct_and_cached():
    t = small_target(n_samples=200_003, dt=1.0, n_fft=1 << 19, n_det=2, seed=7, f1dots=(0.0,),
                     f2dots=(0.0,), dtype="c64")
    x = synth.make_data(t)
    tm = t.templates()
    ref = resamp.fstat(t, x, tm)
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.autotune()
        first = (plan.split, plan.cta)
        assert _ok(plan.compute(tm).cpu().numpy(), ref)
        plan.set_split(1 << 9)
        plan.set_cta(0, 0, 0, 0)
        plan.autotune()                      # served from the in-process cache
        assert (plan.split, plan.cta) == first
        plan.sync()


def test_full_size_ten_day_two_detector_workload():
    t = config2()
    x = synth.make_data(t)
    a, d = t.skies[0]
    prep = resamp.sky_prep(t, x, a, d)
    rng = np.random.default_rng(2)
    tm_all = t.templates()
    picks = []
    for inj in t.injections:
        k = np.where((tm_all["f1dot"] == inj.f1dot) & (tm_all["f2dot"] == inj.f2dot))[0][0]
        picks.append(int(k))
    picks += [int(v) for v in rng.integers(0, len(tm_all), 2)]
    tm = tm_all[picks]
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.autotune()
        out = plan.compute(tm)
        plan.sync()
        got = out.cpu().numpy()
    half, lim = t.n_fft // 2, int(0.4 * t.n_fft)
    for i, k in enumerate(picks):
        bins = list(rng.integers(0, t.n_fft, 24)) + list(rng.integers(half - lim, half + lim, 24))
        if i < len(t.injections):
            m = t.injections[i].bin_index
            bins += [m - 2, m - 1, m, m + 1, m + 2]
        bins = np.array(bins)
        ref = resamp.twoF_at_bins(t, prep, float(tm_all["f1dot"][k]), float(tm_all["f2dot"][k]), bins)
        assert _ok(got[i, bins], ref), (k, np.max(np.abs(got[i, bins] - ref)))
    for i, inj in enumerate(t.injections):
        v = got[i, inj.bin_index]
        sd = np.sqrt(2.0 * (4.0 + 2.0 * inj.rho2))
        assert abs(v - (4.0 + inj.rho2)) < 5.0 * sd + 0.02 * inj.rho2, (inj.rho2, v)
    # two whole rows (every one of the 2^22 bins) against the oracle's FFT,
    # so that an error confined to one tile or one split position shows
    for i in (0, len(picks) - 1):
        k = picks[i]
        ref = resamp.twoF(t, prep, float(tm_all["f1dot"][k]), float(tm_all["f2dot"][k]))
        bad = np.abs(got[i] - ref) > REL * np.abs(ref) + ABS
        assert not bad.any(), (k, int(bad.sum()), np.flatnonzero(bad)[:8])


def test_full_size_120_day_search_slice():
    # 120 days at dt = 1 s (10 368 000 samples per detector), FFT 2^24, the
    # sky patch of the large search: two sky positions with their injections,
    # 2F at injected and random bins against the oracle's direct DFT sums.
    from workloads import config5

    t = config5()
    skies = []
    for inj in t.injections:
        if (inj.alpha, inj.delta) not in skies:
            skies.append((inj.alpha, inj.delta))
        if len(skies) == 2:
            break
    injs = [i for i in t.injections if (i.alpha, i.delta) in skies][:3]
    x = synth.make_data(t, injections=injs)
    rng = np.random.default_rng(5)
    rows = np.empty(len(injs) + 1, dtype=pkg.TEMPLATE_DTYPE)
    for k, inj in enumerate(injs):
        rows[k] = (inj.alpha, inj.delta, inj.f1dot, inj.f2dot)
    rows[-1] = (skies[0][0], skies[0][1], t.f1dots[100], t.f2dots[3])
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.autotune()
        got = plan.compute(rows).cpu().numpy()
        plan.sync()
    half, lim = t.n_fft // 2, int(0.4 * t.n_fft)
    preps = {}
    for k in range(len(rows)):
        key = (float(rows["alpha"][k]), float(rows["delta"][k]))
        if key not in preps:
            preps[key] = resamp.sky_prep(t, x, *key)
        bins = list(rng.integers(half - lim, half + lim, 12)) + list(rng.integers(0, t.n_fft, 4))
        if k < len(injs):
            m = injs[k].bin_index
            bins += [m - 1, m, m + 1]
        bins = np.array(bins)
        ref = resamp.twoF_at_bins(t, preps[key], float(rows["f1dot"][k]), float(rows["f2dot"][k]), bins)
        assert _ok(got[k, bins], ref), (k, np.max(np.abs(got[k, bins] - ref)))
    for k, inj in enumerate(injs):
        v = got[k, inj.bin_index]
        sd = np.sqrt(2.0 * (4.0 + 2.0 * inj.rho2))
        assert abs(v - (4.0 + inj.rho2)) < 5.0 * sd + 0.02 * inj.rho2, (inj.rho2, v)
    # one whole row (all 2^24 bins) against the oracle's FFT
    key = (float(rows["alpha"][0]), float(rows["delta"][0]))
    ref = resamp.twoF(t, preps[key], float(rows["f1dot"][0]), float(rows["f2dot"][0]))
    bad = np.abs(got[0] - ref) > REL * np.abs(ref) + ABS
    assert not bad.any(), (int(bad.sum()), np.flatnonzero(bad)[:8])


def test_full_size_peaks_and_semicoherent_agree_with_dense_passes():
    # 2^22 bins, the shapes the autotuner picks: compute_peaks against the
    # dense output reduced in numpy (bitwise), and fstat_semicoherent over two
    # 10-day segments against the dense per-segment rows shifted and added
    # in float32 in segment order (bitwise)
    import dataclasses

    from oracle import semicoh
    from workloads import make_noise

    t = config2()
    tm = t.templates()[::4096][:3]
    plans = []
    for k in range(2):
        seg = dataclasses.replace(t, t0=t.t0 + k * t.n_samples * t.dt, injections=(), name=f"seg{k}")
        p = pkg.FstatPlan.from_target(seg)
        for X in range(2):
            p.set_data(X, make_noise(t.seed + 13 * k, X, t.n_samples, t.sigmas[X], "c64"), t.sigmas[X])
        p.autotune()
        plans.append(p)
    dense = [p.compute(tm).cpu().numpy() for p in plans]
    out = plans[0].compute_peaks(tm, threshold=20.0, n_bands=1024, capacity=1 << 16)
    plans[0].sync()
    blocks = dense[0].reshape(len(tm), 1024, -1)
    assert np.array_equal(out["band_max"].cpu().numpy(), blocks.max(axis=2))
    assert int(out["count"].item()) == int((dense[0] > 20.0).sum())
    t_ref = t.t0 + (2 * t.n_samples // 2) * t.dt
    total = pkg.semicoherent(plans, tm, t_ref).cpu().numpy()
    df = 1.0 / (t.n_fft * t.dt)
    want = np.zeros_like(total)
    for k, p in enumerate(plans):
        seg_t_ref = t.t0 + k * t.n_samples * t.dt + (t.n_samples // 2) * t.dt
        d_ref = seg_t_ref - t_ref
        seg_tm = semicoh.segment_template(tm, d_ref)
        rows = p.compute(seg_tm).cpu().numpy()
        for i in range(len(tm)):
            sh = semicoh.segment_shift(df, d_ref, float(tm["f1dot"][i]), float(tm["f2dot"][i]))
            m = np.arange(t.n_fft)
            ok = (m + sh >= 0) & (m + sh < t.n_fft)
            want[i, ok] = want[i, ok] + rows[i, (m + sh)[ok]]
    assert np.array_equal(total, want)
    for p in plans:
        p.close()
