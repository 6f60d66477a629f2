"""The batched uneven-target workload itself (four targets drawn from the
pilot search's band range: spans of 1-30 days, bands of 0.25-4 Hz, f_h
between 145 and 490 Hz, FFT lengths 2^18-2^22), in one CUDA graph through
fstat_batch_*, against the FP64 oracle.

Per target: both injection templates and one more bank template, every bin
of every row compared at |d2F| <= 1e-3 2F + 0.02 (Sec. 3 steps iii-vii),
on the first launch and on a replay.
"""

import numpy as np
import pytest
import torch

import paper_2201_00451_gb300 as pkg
from oracle import resamp, synth
from workloads import config3

pytestmark = pytest.mark.gpu

REL, ABS = 1e-3, 0.02


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


def _rows(t):
    """Both injections' templates and one more from the middle of the bank."""
    rows = np.empty(len(t.injections) + 1, dtype=pkg.TEMPLATE_DTYPE)
    for k, inj in enumerate(t.injections):
        rows[k] = (inj.alpha, inj.delta, inj.f1dot, inj.f2dot)
    a, d = t.skies[0]
    rows[-1] = (a, d, t.f1dots[len(t.f1dots) // 2], t.f2dots[0])
    return rows


def test_config3_targets_in_one_graph_against_oracle():
    targets = config3()
    assert {t.n_fft for t in targets} >= {1 << 18, 1 << 22}
    assert max(t.f_het for t in targets) > 300.0 and max(t.t_span for t in targets) >= 30 * 86400
    plans, outs, refs = [], [], []
    with pkg.FstatBatch() as batch:
        for t in targets:
            assert all((inj.alpha, inj.delta) == t.skies[0] for inj in t.injections)
            x = synth.make_data(t)
            rows = _rows(t)
            plan = pkg.FstatPlan.from_target(t)
            for X in range(2):
                plan.set_data(X, x[X], t.sigmas[X])
            plan.autotune()
            out = torch.zeros((len(rows), t.n_fft), dtype=torch.float32, device="cuda")
            batch.add(plan, rows, out)
            plans.append(plan)
            outs.append(out)
            prep = resamp.sky_prep(t, x, *t.skies[0])
            refs.append(np.stack([resamp.twoF(t, prep, float(r["f1dot"]), float(r["f2dot"])) for r in rows]))
        batch.instantiate()
        for rep in range(2):
            for o in outs:
                o.zero_()
            batch.launch()
            torch.cuda.synchronize()
            for t, o, r in zip(targets, outs, refs):
                got = o.cpu().numpy()
                bad = np.abs(got - r) > REL * np.abs(r) + ABS
                assert not bad.any(), (t.name, rep, int(bad.sum()), np.argwhere(bad)[:4])
        for p in plans:
            assert p.sync() is None
    # the injections are recovered near their rho^2 at their bins
    for t, r in zip(targets, refs):
        for k, inj in enumerate(t.injections):
            sd = np.sqrt(2.0 * (4.0 + 2.0 * inj.rho2))
            assert abs(r[k, inj.bin_index] - (4.0 + inj.rho2)) < 5.0 * sd + 0.02 * inj.rho2
    for p in plans:
        p.close()
