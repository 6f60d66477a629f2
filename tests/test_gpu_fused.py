"""The persistent launch of both FFT passes over many templates
(fstat_set_fused), against the two-launch path and the FP64 oracle.

The fused kernel runs the same column and row transforms (Sec. 3 steps vi-
vii) as the two-launch path with radix-16-first schedules, so at the same
split its 2F must equal the two-launch path's bit for bit; on ragged sizes
it must also meet |d2F| <= 1e-3 2F + 0.02 against the oracle.  Templates
per launch exceed the three rotating intermediates, several sky groups
share one call, the launch may sit in a CUDA graph, and a dependency or copy wait that runs out reports
FSTAT_ERR_TIMEOUT without hanging.
"""

import numpy as np
import pytest
import torch

import paper_2201_00451_gb300 as pkg
from oracle import resamp, synth
from workloads import make_noise, small_target

pytestmark = pytest.mark.gpu

REL, ABS = 1e-3, 0.02
TIMEOUT = -8

# (log2 n_fft, n1) of every compiled fused split
SPLITS = [(18, 512), (19, 512), (20, 1024), (21, 1024), (22, 1024), (23, 2048), (24, 4096)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


def _ok(gpu, ref):
    return np.all(np.isfinite(gpu)) and np.all(np.abs(gpu - ref) <= REL * np.abs(ref) + ABS)


def _noise_target(log2n, n, seed, n_f1=7):
    t = small_target(n_samples=n, dt=1.0, n_fft=1 << log2n, n_det=2, seed=seed,
                     f1dots=np.linspace(-3e-12, 3e-12, n_f1), f2dots=(0.0,), dtype="c64")
    xs = [make_noise(seed, X, n, t.sigmas[X], "c64") for X in range(2)]
    return t, xs


@pytest.mark.parametrize("log2n,n1", SPLITS)
@pytest.mark.parametrize("fill", ["short", "long"])
def test_fused_equals_two_launch_path_bitwise(log2n, n1, fill):
    # short: data under half the FFT length (the zero-padded upper half of
    # every column is skipped); long: more than half (every butterfly full)
    n = (1 << log2n) // 4 + 1237 if fill == "short" else (1 << log2n) * 5 // 8 + 411
    t, xs = _noise_target(log2n, n, seed=300 + log2n)
    tm = t.templates()
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, xs[X], t.sigmas[X])
        plan.set_split(n1)
        plan.set_cta(0, 0, 0, 0)
        plan.set_fused(False)
        two = plan.compute(tm).cpu().numpy()
        plan.set_fused(True)
        assert plan.fused
        fused = plan.compute(tm).cpu().numpy()
        plan.sync()
    assert np.array_equal(fused, two)


@pytest.mark.parametrize("log2n,n1,n", [(18, 512, 150_001), (20, 1024, 400_003)])
def test_fused_matches_oracle_with_injections(log2n, n1, n):
    t = small_target(n_samples=n, dt=1.0, n_fft=1 << log2n, n_det=2, n_inj=1, rho2_range=(200.0, 200.0),
                     seed=320 + log2n, f1dots=np.linspace(-4e-12, 2e-12, 6), f2dots=(0.0, 1e-18),
                     dtype="c64")
    x = synth.make_data(t)
    tm = t.templates()
    ref = resamp.fstat(t, x, tm)
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.set_split(n1)
        plan.set_fused(True)
        got = plan.compute(tm).cpu().numpy()
        plan.sync()
    assert _ok(got, ref)


def test_fused_several_sky_groups_in_one_call():
    # three sky positions, their templates shuffled together: one fused
    # launch per sky group, each writing its templates' rows of the output
    t, xs = _noise_target(20, 300_007, seed=341, n_f1=5)
    rng = np.random.default_rng(5)
    skies = [(float(a), float(d)) for a, d in zip(rng.uniform(0, 6.28, 3), rng.uniform(-1.2, 1.2, 3))]
    tm = np.concatenate([small_target(n_samples=10, n_fft=1 << 13, skies=(s,), f1dots=t.f1dots,
                                      f2dots=(0.0,)).templates() for s in skies])
    tm = tm[rng.permutation(len(tm))]
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, xs[X], t.sigmas[X])
        plan.set_split(1024)
        plan.set_cta(0, 0, 0, 0)
        plan.set_fused(False)
        two = plan.compute(tm).cpu().numpy()
        plan.set_fused(True)
        fused = plan.compute(tm).cpu().numpy()
        plan.sync()
    assert np.array_equal(fused, two)


def test_fused_plans_in_one_graph():
    specs = [(18, 512, 100_003, 351), (21, 1024, 700_001, 352)]
    plans, outs, refs = [], [], []
    with pkg.FstatBatch() as batch:
        for log2n, n1, n, seed in specs:
            t, xs = _noise_target(log2n, n, seed)
            tm = t.templates()
            plan = pkg.FstatPlan.from_target(t)
            for X in range(2):
                plan.set_data(X, xs[X], t.sigmas[X])
            plan.set_split(n1)
            plan.set_cta(0, 0, 0, 0)
            refs.append(plan.compute(tm).cpu().numpy())
            plan.set_fused(True)
            out = torch.zeros((len(tm), t.n_fft), dtype=torch.float32, device="cuda")
            batch.add(plan, tm, out)
            plans.append(plan)
            outs.append(out)
        batch.instantiate()
        for _ in range(2):
            for o in outs:
                o.zero_()
            batch.launch()
            torch.cuda.synchronize()
            for o, r in zip(outs, refs):
                assert np.array_equal(o.cpu().numpy(), r)
    for p in plans:
        p.close()


def test_fused_wait_that_runs_out_reports_timeout_and_recovers():
    t, xs = _noise_target(20, 300_007, seed=361)
    tm = t.templates()
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, xs[X], t.sigmas[X])
        plan.set_split(1024)
        plan.set_fused(False)
        ref = plan.compute(tm).cpu().numpy()
        plan.set_fused(True)
        plan.set_wait_limit(0)
        plan.compute(tm)
        with pytest.raises(pkg.FstatError) as e:
            plan.sync()
        assert e.value.code == TIMEOUT
        plan.set_wait_limit(-1)
        got = plan.compute(tm).cpu().numpy()
        plan.sync()
    assert np.array_equal(got, ref)


def test_fused_unsupported_split_and_precision_are_refused():
    t, xs = _noise_target(20, 300_007, seed=371, n_f1=1)
    with pkg.FstatPlan.from_target(t) as plan:
        plan.set_split(256)                     # 256 x 4096: no fused shape compiled
        with pytest.raises(pkg.FstatError) as e:
            plan.set_fused(True)
        assert e.value.code == -7
    with pkg.FstatPlan.from_target(t, pkg.FP64) as plan:
        with pytest.raises(pkg.FstatError) as e:
            plan.set_fused(True)
        assert e.value.code == -7
