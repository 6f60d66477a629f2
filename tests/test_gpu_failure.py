"""Failure detection without a GPU fault (Sec. 3 steps vi-vii run as usual).

* Timeout: the first wait of every pass-B tile for its bulk tensor copies
  is given zero polls (fstat_set_wait_limit), so each wait gives up at
  once.  The kernel records FSTAT_ERR_TIMEOUT, lets the copies it issued
  land under the full limit, and returns; fstat_sync reports the code, and
  the same plan then computes correct 2F with the default limit.
* Out of memory: a device-memory cap (FSTAT_DEVICE_BYTES_CAP, read when a
  plan is created) below what a plan needs makes fstat_plan_create return
  FSTAT_ERR_OOM; a cap between the plan's needs and those of more template
  streams makes fstat_set_streams return FSTAT_ERR_OOM and leaves the plan
  working.
"""

import os

import numpy as np
import pytest

import paper_2201_00451_gb300 as pkg
from oracle import resamp, synth
from workloads import small_target

pytestmark = pytest.mark.gpu

TIMEOUT, OOM = -8, -2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


def _target():
    # 2^20 bins split 1024 x 1024: pass B rows of 1024 points, which the TMA
    # schedules cover
    return small_target(n_samples=300_007, dt=1.0, n_fft=1 << 20, n_det=2, n_inj=1,
                        rho2_range=(150.0, 150.0), seed=41, f1dots=(-1e-12, 0.0), f2dots=(0.0,), dtype="c64")


def _ok(gpu, ref):
    return np.all(np.abs(gpu - ref) <= 1e-3 * np.abs(ref) + 0.02)


@pytest.mark.parametrize("vb", [4, 6])
def test_wait_that_runs_out_reports_timeout_and_the_plan_recovers(vb):
    t = _target()
    x = synth.make_data(t)
    tm = t.templates()
    ref = resamp.fstat(t, x, tm)
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.set_split(1024)
        plan.set_cta(0, 0, 0, vb)
        plan.set_wait_limit(0)
        plan.compute(tm)
        with pytest.raises(pkg.FstatError) as e:
            plan.sync()
        assert e.value.code == TIMEOUT
        plan.set_wait_limit(-1)
        out = plan.compute(tm).cpu().numpy()
        plan.sync()
    assert _ok(out, ref)


def test_staged_column_wait_that_runs_out_reports_timeout_and_the_plan_recovers():
    # pass A's schedule 16 (8192-point columns whose samples arrive by one
    # bulk copy each): every CTA's first wait gives up at once, the copy in
    # flight is drained under the full limit, the kernel returns
    t = _target()
    x = synth.make_data(t)
    tm = t.templates()
    ref = resamp.fstat(t, x, tm)
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        plan.set_split(128)            # pass A 8192 points
        plan.set_cta(1, 0, 16, 0)
        plan.set_wait_limit(0)
        plan.compute(tm)
        with pytest.raises(pkg.FstatError) as e:
            plan.sync()
        assert e.value.code == TIMEOUT
        plan.set_wait_limit(-1)
        out = plan.compute(tm).cpu().numpy()
        plan.sync()
    assert _ok(out, ref)


def test_device_memory_cap_gives_oom_and_leaves_plans_usable(monkeypatch):
    t = _target()
    x = synth.make_data(t)
    tm = t.templates()[:1]
    monkeypatch.setenv("FSTAT_DEVICE_BYTES_CAP", str(1 << 20))
    with pytest.raises(pkg.FstatError) as e:
        pkg.FstatPlan.from_target(t)
    assert e.value.code == OOM
    # enough for the plan, its data and its two default template streams
    # (~50 MB), not for eight streams (six more 16.8 MB intermediates)
    z_bytes = t.n_fft * 16
    monkeypatch.setenv("FSTAT_DEVICE_BYTES_CAP", str(4 * z_bytes + (32 << 20)))
    with pkg.FstatPlan.from_target(t) as plan:
        monkeypatch.delenv("FSTAT_DEVICE_BYTES_CAP")
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        with pytest.raises(pkg.FstatError) as e:
            plan.set_streams(8)
        assert e.value.code == OOM
        out = plan.compute(tm).cpu().numpy()
        plan.sync()
    assert _ok(out, resamp.fstat(t, x, tm))
    assert os.environ.get("FSTAT_DEVICE_BYTES_CAP") is None
