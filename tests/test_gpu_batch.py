"""Uneven targets in one CUDA graph (fstat_batch_*), against the oracle.

Targets differ in sample count, span, band, heterodyne frequency, FFT
length and template count, as in the batched multi-target workload; each
target's 2F must match the oracle at |d2F| <= 1e-3 2F + 0.02, on first
launch and on replay.
"""

import numpy as np
import pytest
import torch

import paper_2201_00451_gb300 as pkg
from oracle import resamp, synth
from workloads import small_target

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


def _ok(gpu, ref):
    return np.all(np.abs(gpu - ref) <= 1e-3 * np.abs(ref) + 0.02)


def _targets():
    specs = [  # (n_samples, dt, log2 n_fft, f_het, f1dots, seed)
        (3001, 2.0, 13, 145.3, (-1e-10, 0.0, 1e-10), 61),
        (20011, 1.0, 15, 301.7, (-2e-11, 0.0), 62),
        (7001, 0.5, 14, 487.2, (0.0,), 63),
        (50003, 0.25, 17, 220.9, (-1e-11, 0.0, 1e-11, 2e-11), 64),
    ]
    out = []
    for n, dt, l2, fh, f1, seed in specs:
        t = small_target(n_samples=n, dt=dt, n_fft=1 << l2, n_det=2, f_het=fh, n_inj=1,
                         rho2_range=(120.0, 120.0), seed=seed, f1dots=f1, f2dots=(0.0,), dtype="c64")
        out.append(t)
    return out


def test_uneven_targets_in_one_graph():
    ts = _targets()
    plans, outs, refs = [], [], []
    with pkg.FstatBatch() as batch:
        for t in ts:
            x = synth.make_data(t)
            plan = pkg.FstatPlan.from_target(t)
            for X in range(2):
                plan.set_data(X, x[X], t.sigmas[X])
            tm = t.templates()
            out = torch.zeros((len(tm), t.n_fft), dtype=torch.float32, device="cuda")
            batch.add(plan, tm, out)
            plans.append(plan)
            outs.append(out)
            refs.append(resamp.fstat(t, x, tm))
        batch.instantiate()
        assert batch.nodes > 2 * sum(len(t.templates()) for t in ts)
        for rep in range(2):
            for o in outs:
                o.zero_()
            batch.launch()
            torch.cuda.synchronize()
            for o, r in zip(outs, refs):
                assert _ok(o.cpu().numpy(), r)
            # ordinary calls between replays do not disturb the graph
            plans[0].compute(ts[0].templates()[:1])
            plans[0].sync()
    for p in plans:
        p.close()


def test_output_ring_keeps_the_last_rows():
    t = _targets()[0]
    x = synth.make_data(t)
    tm = small_target(n_samples=t.n_samples, dt=t.dt, n_fft=t.n_fft, n_det=2, f_het=t.f_het, seed=61,
                      f1dots=np.linspace(-2e-10, 2e-10, 6), f2dots=(0.0,)).templates()
    tm["alpha"], tm["delta"] = t.skies[0]
    ref = resamp.fstat(t, x, tm)
    with pkg.FstatPlan.from_target(t) as plan, pkg.FstatBatch() as batch:
        for X in range(2):
            plan.set_data(X, x[X], t.sigmas[X])
        out = torch.zeros((2, t.n_fft), dtype=torch.float32, device="cuda")
        batch.add(plan, tm, out, out_rows=2)
        batch.instantiate()
        batch.launch()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    assert _ok(got[0], ref[4]) and _ok(got[1], ref[5])
