"""GPU post-processing of 2F (fstat_compute_peaks) against the oracle.

The device reduces each template's 2F to the crossings of a threshold and
the maximum of every band of bins (Sec. 5.4 keeps 2F > 70 on the GPU;
Sec. 4.1 names the band maximum).  Parity is with oracle.peaks applied to
the oracle's FP64 2F at |d2F| <= 1e-3 2F + 0.02.  Within that tolerance
several bins of a band can be the maximum and a bin near the threshold can
fall on either side, so the checks are: every band maximum within
tolerance, the returned bin inside its band with an oracle value within
tolerance of the oracle maximum; every clear oracle crossing listed, every
listed entry a crossing with the oracle's value.  Against the dense
fstat_compute of the same plan (the same arithmetic) the reductions agree
exactly.
"""

import numpy as np
import pytest
import torch

import paper_2201_00451_gb300 as pkg
from oracle import peaks, resamp, synth
from workloads import config2, small_target

pytestmark = pytest.mark.gpu

REL, ABS = 1e-3, 0.02


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


def tol(v):
    return REL * np.abs(v) + ABS


def check_bands(gmax, gbin, ref, n_bands, rel=REL, abs_=ABS):
    omax, _ = peaks.band_maxima(ref, n_bands)
    t = rel * np.abs(omax) + abs_
    assert np.all(np.abs(gmax - omax) <= t), np.max(np.abs(gmax - omax) - t)
    w = ref.shape[1] // n_bands
    assert np.array_equal(gbin // w, np.broadcast_to(np.arange(n_bands), gbin.shape))
    vals = np.take_along_axis(ref, gbin.astype(np.int64), axis=1)
    assert np.all(vals >= omax - 2 * t)


def check_list(found, ref, thr, offset=0, rel=REL, abs_=ABS):
    got = {(int(r["tmpl"]), int(r["bin"])): float(r["twoF"]) for r in found}
    assert len(got) == len(found), "duplicate entries"
    for (ti, m), v in got.items():
        want = ref[ti - offset, m]
        assert abs(v - want) <= rel * abs(want) + abs_, (ti, m, v, want)
        assert v > thr
    for ti, m, v in peaks.crossings(ref, thr, tmpl_offset=offset):
        if v - (rel * abs(v) + abs_) > thr:
            assert (ti, m) in got, (ti, m, v)


def setup(seed, precision=pkg.MIXED, dtype="c64", n_fft=1 << 15, n=20000):
    t = small_target(n_samples=n, dt=1.0, n_fft=n_fft, n_det=2, n_inj=2, rho2_range=(120.0, 240.0),
                     seed=seed, f1dots=(-2e-10, -1e-10, 0.0), f2dots=(0.0,), dtype=dtype)
    x = synth.make_data(t)
    plan = pkg.FstatPlan.from_target(t, precision)
    for X in range(2):
        plan.set_data(X, x[X], t.sigmas[X])
    return t, x, plan


# W = n_fft / n_bands from the whole band down to single bins, so the band
# boundaries fall above, inside and below one CTA's rows and columns.
@pytest.mark.parametrize("n_bands", [1, 64, 4096, 1 << 15])
def test_band_maxima_and_crossings_match_oracle(n_bands):
    t, x, plan = setup(51)
    tm = t.templates()
    ref = resamp.fstat(t, x, tm)
    out = plan.compute_peaks(tm, threshold=12.0, n_bands=n_bands, capacity=1 << 16)
    plan.sync()
    assert int(out["count"].item()) <= 1 << 16
    check_bands(out["band_max"].cpu().numpy(), out["band_bin"].cpu().numpy(), ref, n_bands)
    check_list(pkg.peaks_to_numpy(out), ref, 12.0)
    plan.close()


def test_peaks_equal_the_dense_output_reduced():
    t, x, plan = setup(52, n_fft=1 << 16, n=40000)
    tm = t.templates()
    dense = plan.compute(tm).cpu().numpy()
    for n_bands in (2, 256, 1 << 13):
        out = plan.compute_peaks(tm, threshold=10.0, n_bands=n_bands, capacity=1 << 17)
        plan.sync()
        blocks = dense.reshape(len(tm), n_bands, -1)
        arg = blocks.argmax(axis=2)
        assert np.array_equal(out["band_max"].cpu().numpy(), blocks.max(axis=2))
        assert np.array_equal(out["band_bin"].cpu().numpy(), arg + blocks.shape[2] * np.arange(n_bands))
        lst = pkg.peaks_to_numpy(out)
        ti, mi = np.nonzero(dense > 10.0)
        assert int(out["count"].item()) == len(ti)
        assert sorted(zip(lst["tmpl"].tolist(), lst["bin"].tolist())) == sorted(zip(ti.tolist(), mi.tolist()))
        assert np.array_equal(lst["twoF"], dense[lst["tmpl"], lst["bin"]])
    plan.close()


def test_peaks_equal_dense_for_every_pass_b_schedule():
    # 1024-point pass-B rows: two buffers or one (the tile's 2F then in a
    # region of its own so the next tile loads early), cp.async or TMA
    # loads; band keys in shared memory (whole-row bands) or not.  A plan
    # set to schedule 8 (half the next tile staged apart, which the peaks
    # epilogue has no room for) reduces with schedule 0.
    t, x, plan = setup(57, n_fft=1 << 20, n=400_003)
    tm = t.templates()
    plan.set_split(1024)
    for cb, vb in ((4, 0), (4, 2), (4, 4), (4, 6), (2, 2), (8, 6), (4, 8), (8, 8)):
        plan.set_cta(1, cb, 2, vb)
        dense = plan.compute(tm).cpu().numpy()
        # whole-row bands of 512, 16 and 8 rows (reduced in registers when a
        # warp's rows fit one band), 4 rows, and bands inside a row
        for n_bands in (2, 64, 128, 256, 1 << 13):
            out = plan.compute_peaks(tm, threshold=12.0, n_bands=n_bands, capacity=1 << 18)
            plan.sync()
            blocks = dense.reshape(len(tm), n_bands, -1)
            assert np.array_equal(out["band_max"].cpu().numpy(), blocks.max(axis=2)), (cb, vb, n_bands)
            assert np.array_equal(out["band_bin"].cpu().numpy(),
                                  blocks.argmax(axis=2) + blocks.shape[2] * np.arange(n_bands)), (cb, vb, n_bands)
            lst = pkg.peaks_to_numpy(out)
            ti, mi = np.nonzero(dense > 12.0)
            assert int(out["count"].item()) == len(ti)
            assert sorted(zip(lst["tmpl"].tolist(), lst["bin"].tolist())) == sorted(zip(ti.tolist(), mi.tolist()))
    plan.close()


def test_autotuned_peaks_shape_equals_dense():
    # the autotuner picks pass B of the peaks mode apart from the dense
    # pass; its reduction still equals the dense output's, and an explicit
    # shape applies to both modes again
    t, x, plan = setup(58, n_fft=1 << 20, n=400_003)
    tm = t.templates()
    plan.autotune()
    dense = plan.compute(tm).cpu().numpy()
    cb, vb = plan.peaks_cta
    assert cb > 0 and 0 <= vb <= 7
    out = plan.compute_peaks(tm, threshold=12.0, n_bands=256, capacity=1 << 18)
    plan.sync()
    blocks = dense.reshape(len(tm), 256, -1)
    assert np.array_equal(out["band_max"].cpu().numpy(), blocks.max(axis=2))
    assert np.array_equal(out["band_bin"].cpu().numpy(), blocks.argmax(axis=2) + blocks.shape[2] * np.arange(256))
    plan.set_cta(1, 4, 2, 6)
    assert plan.peaks_cta == (4, 6)
    plan.close()


def test_capacity_overflow_and_appending_calls():
    t, x, plan = setup(53)
    tm = t.templates()
    ref = resamp.fstat(t, x, tm)
    full = plan.compute_peaks(tm, threshold=12.0, capacity=1 << 16)
    plan.sync()
    n_all = int(full["count"].item())
    assert n_all > 20
    small = plan.compute_peaks(tm, threshold=12.0, capacity=7)
    plan.sync()
    assert int(small["count"].item()) == n_all
    part = pkg.peaks_to_numpy(small)
    assert len(part) == 7
    allset = {(int(r["tmpl"]), int(r["bin"])) for r in pkg.peaks_to_numpy(full)}
    assert all((int(r["tmpl"]), int(r["bin"])) in allset for r in part)
    # two calls appending to one list, the second offset by the first's size
    h = len(tm) // 2
    acc = plan.compute_peaks(tm[:h], threshold=12.0, capacity=1 << 16)
    plan.compute_peaks(tm[h:], threshold=12.0, tmpl_offset=h, out=acc)
    plan.sync()
    assert int(acc["count"].item()) == n_all
    check_list(pkg.peaks_to_numpy(acc), ref, 12.0)
    plan.close()


def test_fp64_plan_peaks():
    t, x, plan = setup(54, precision=pkg.FP64, dtype="c128")
    tm = t.templates()
    ref = resamp.fstat(t, x, tm)
    out = plan.compute_peaks(tm, threshold=12.0, n_bands=128, capacity=1 << 16)
    plan.sync()
    # FP64 arithmetic, the reduced values stored as float32
    check_bands(out["band_max"].cpu().numpy(), out["band_bin"].cpu().numpy(), ref, 128, rel=1e-6, abs_=1e-6)
    check_list(pkg.peaks_to_numpy(out), ref, 12.0, rel=1e-6, abs_=1e-6)
    plan.close()


def test_invalid_arguments():
    t, x, plan = setup(55, n_fft=1 << 15)
    tm = t.templates()[:1]
    for kw in (dict(n_bands=3), dict(n_bands=1 << 16), dict(threshold=float("nan"))):
        with pytest.raises(pkg.FstatError) as e:
            plan.compute_peaks(tm, **kw)
        assert e.value.code == -1
    with pytest.raises(pkg.FstatError):   # neither a list nor bands
        plan.compute_peaks(tm, out={"count": None, "peaks": None})
    plan.close()


def test_full_size_band_maxima_and_injections():
    # the 10-day two-detector workload at FFT 2^22: the injected templates'
    # band maxima (1024 bands) against the oracle's full FFT 2F, and the
    # injections found among the crossings of 2F > 70
    t = config2()
    x = synth.make_data(t)
    a, d = t.skies[0]
    prep = resamp.sky_prep(t, x, a, d)
    tm_all = t.templates()
    picks = []
    for inj in t.injections[:2]:
        picks.append(int(np.where((tm_all["f1dot"] == inj.f1dot) & (tm_all["f2dot"] == inj.f2dot))[0][0]))
    tm = tm_all[picks]
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.autotune()
        out = plan.compute_peaks(tm, threshold=70.0, n_bands=1024, capacity=4096)
        plan.sync()
        gmax, gbin = out["band_max"].cpu().numpy(), out["band_bin"].cpu().numpy()
        lst = pkg.peaks_to_numpy(out)
    ref = np.stack([resamp.twoF(t, prep, float(tm_all["f1dot"][k]), float(tm_all["f2dot"][k])) for k in picks])
    check_bands(gmax, gbin, ref, 1024)
    check_list(lst, ref, 70.0)
    for i, inj in enumerate(t.injections[:2]):
        if ref[i, inj.bin_index] > 80.0:
            assert (i, inj.bin_index) in {(int(r["tmpl"]), int(r["bin"])) for r in lst}


def test_reduce_peaks_of_dense_rows_equals_compute_peaks():
    t, x, plan = setup(56, n_fft=1 << 16, n=40000)
    tm = t.templates()
    dense = plan.compute(tm)
    for n_bands in (1, 256, 1 << 13):
        a = plan.compute_peaks(tm, threshold=10.0, n_bands=n_bands, capacity=1 << 17)
        b = plan.reduce_peaks(dense, threshold=10.0, n_bands=n_bands, capacity=1 << 17)
        plan.sync()
        assert torch.equal(a["band_max"], b["band_max"]) and torch.equal(a["band_bin"], b["band_bin"])
        assert int(a["count"].item()) == int(b["count"].item())
        la, lb = pkg.peaks_to_numpy(a), pkg.peaks_to_numpy(b)
        assert sorted(zip(la["tmpl"].tolist(), la["bin"].tolist(), la["twoF"].tolist())) == \
            sorted(zip(lb["tmpl"].tolist(), lb["bin"].tolist(), lb["twoF"].tolist()))
    plan.close()


def test_reduce_peaks_of_a_semicoherent_sum_matches_oracle():
    from oracle import semicoh
    from workloads import segment_slices, split_segments

    S = 3
    t = small_target(n_samples=S * 6000, dt=1.0, n_fft=1 << 14, n_det=2, n_inj=1, rho2_range=(300.0, 300.0),
                     seed=57, f1dots=(0.0, -1e-10), f2dots=(0.0,), dtype="c64")
    x = synth.make_data(t)
    segs = split_segments(t, S)
    data = [[xx[a:a + n] for xx in x] for a, n in segment_slices(t, S)]
    plans = []
    for s_, d in zip(segs, data):
        p = pkg.FstatPlan.from_target(s_)
        for X in range(2):
            p.set_data(X, d[X], t.sigmas[X])
        plans.append(p)
    tm = t.templates()
    total = pkg.semicoherent(plans, tm, t.t_reference)
    out = plans[0].reduce_peaks(total, threshold=40.0, n_bands=64, capacity=1 << 16, tmpl_offset=5)
    plans[0].sync()
    ref = semicoh.semicoherent(segs, data, tm, t.t_reference)
    check_bands(out["band_max"].cpu().numpy(), out["band_bin"].cpu().numpy(), ref, 64, abs_=ABS * S)
    check_list(pkg.peaks_to_numpy(out), ref, 40.0, offset=5, abs_=ABS * S)
    for p in plans:
        p.close()


def test_reduce_peaks_argument_checks():
    t, x, plan = setup(58, n_fft=1 << 15)
    rows = plan.compute(t.templates()[:2])
    with pytest.raises(ValueError):
        plan.reduce_peaks(rows[:, :100], n_bands=4)
    with pytest.raises(pkg.FstatError) as e:
        plan.reduce_peaks(rows, n_bands=3)
    assert e.value.code == -1
    plan.close()
    t = small_target(n_samples=1000, dt=1.0, n_fft=1 << 10, n_det=1, seed=59, dtype="c64")
    with pkg.FstatPlan.from_target(t) as small_plan:
        small_plan.set_data(0, synth.make_data(t)[0], t.sigmas[0])
        r = small_plan.compute(t.templates())
        with pytest.raises(pkg.FstatError) as e:
            small_plan.reduce_peaks(r, n_bands=1)
        assert e.value.code == -7


def test_empty_calls_return_without_work():
    t, x, plan = setup(60, n_fft=1 << 14, n=8000)
    empty = t.templates()[:0]
    out = plan.compute_peaks(empty, threshold=10.0, n_bands=4)
    plan.sync()
    assert int(out["count"].item()) == 0 and out["band_max"].shape == (0, 4)
    rows = torch.empty((0, t.n_fft), dtype=torch.float32, device="cuda")
    out = plan.reduce_peaks(rows, threshold=10.0, n_bands=4)
    plan.sync()
    assert int(out["count"].item()) == 0
    assert pkg.semicoherent([plan], empty, t.t_reference).shape == (0, t.n_fft)
    plan.close()
