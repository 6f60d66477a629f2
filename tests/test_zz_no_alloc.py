"""fstat_twoF_noalloc through the C ABI (GPU), against the FP64 oracle and
against fstat_compute.

fstat_twoF_noalloc serves callers that may not call cudaMalloc (a plug-in
inside an application whose memory pool owns the device memory, or a
pipeline that must not allocate after start-up): its scratch memory is a
fixed device array inside the library, shared by every call.  The test
feeds it resampled series G_a, G_b and checks, at the tolerance the other
parity tests use (|d2F| <= 1e-3 2F + 0.02):

* two consecutive calls at its largest size (2^18 bins) against the
  oracle's 2F (steps vi-vii on the oracle's own per-sky series) and
  against fstat_compute on the same templates;
* then calls at 2^17 and 2^11 bins with sample counts that are not
  multiples of the FFT split and smaller than the previous call's, so that
  stale data left in the shared scratch must not leak into the result;
* a size beyond the scratch array is refused.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""

import ctypes

import numpy as np
import pytest

import paper_2201_00451_gb300 as pkg
from oracle import resamp, synth
from workloads import config1, small_target

pytestmark = pytest.mark.gpu

REL, ABS = 1e-3, 0.02


def _call(lib, prep, t, f1dot, f2dot, stream, n_fft=None):
    import torch

    pairs = np.stack([prep["Ga"].real, prep["Ga"].imag, prep["Gb"].real, prep["Gb"].imag],
                     axis=1).astype(np.float32)
    # caller-owned buffers (torch's allocator, outside the entry point)
    g_dev = torch.from_numpy(pairs).cuda()
    out = torch.full((n_fft or t.n_fft,), float("nan"), dtype=torch.float32, device="cuda")
    tau0 = prep["t_b0"] - t.t_reference
    rc = lib.fstat_twoF_noalloc(
        ctypes.c_void_p(g_dev.data_ptr()), t.n_samples, n_fft or t.n_fft, t.dt, tau0,
        prep["A"], prep["B"], prep["C"], float(f1dot), float(f2dot), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(stream.cuda_stream))
    return rc, out, g_dev


def _ok(got, ref):
    return np.all(np.isfinite(got)) and np.all(np.abs(got - ref) <= REL * np.abs(ref) + ABS)


def test_noalloc_matches_oracle_and_planned_path():
    import torch

    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    lib = pkg.load()
    stream = torch.cuda.current_stream()

    t = config1()                      # n_fft = 2^18, the entry point's maximum
    x = synth.make_data(t)
    alpha, delta = t.skies[0]
    tm = t.templates()
    picks = [3, 41]
    prep = resamp.sky_prep(t, x, alpha, delta)
    with pkg.FstatPlan.from_target(t) as plan:
        plan.set_data(0, x[0], t.sigmas[0])
        planned = plan.compute(tm[picks]).cpu().numpy()
        plan.sync()
    keep = []
    for i, k in enumerate(picks):      # two calls in a row share the scratch array
        f1, f2 = float(tm["f1dot"][k]), float(tm["f2dot"][k])
        rc, out, g = _call(lib, prep, t, f1, f2, stream)
        assert rc == 0, pkg.ERR.get(rc, rc)
        keep.append((out, g, resamp.twoF(t, prep, f1, f2), planned[i]))
    torch.cuda.synchronize()
    for out, _, ref, planned_row in keep:
        got = out.cpu().numpy()
        assert _ok(got, ref)
        assert _ok(got, planned_row)

    # smaller calls after the larger one: ragged sample counts (not
    # multiples of the split n1 = 256 or 32), unequal passes at 2^17 and 2^11
    for n, log2n, seed in [(100_003, 17, 51), (1_501, 11, 52)]:
        s = small_target(n_samples=n, dt=1.0, n_fft=1 << log2n, n_det=2, n_inj=1, rho2_range=(120.0, 120.0),
                         seed=seed, f1dots=(-1e-11, 0.0), f2dots=(0.0,), dtype="c64")
        xs = synth.make_data(s)
        ps = resamp.sky_prep(s, xs, *s.skies[0])
        for f1 in s.f1dots:
            rc, out, g = _call(lib, ps, s, f1, 0.0, stream)
            assert rc == 0, pkg.ERR.get(rc, rc)
            torch.cuda.synchronize()
            assert _ok(out.cpu().numpy(), resamp.twoF(s, ps, float(f1), 0.0)), (n, f1)

    rc, _, _ = _call(lib, prep, t, 0.0, 0.0, stream, n_fft=1 << 19)
    assert rc == -7  # FSTAT_ERR_UNSUPPORTED: beyond the fixed scratch size
