"""fstat_twoF_noalloc against fstat_compute, through the C ABI (GPU).

fstat_twoF_noalloc serves callers that may not call cudaMalloc (a plug-in
inside an application whose memory pool owns the device memory, or a
pipeline that must not allocate after start-up): its scratch memory is a
fixed device array inside the library.  This test feeds it the per-sky
series the planned path resamples (exported with fstat_export_sky) and
checks two consecutive calls against fstat_compute for the same templates,
at the tolerance the other parity tests use (|d2F| <= 1e-3 2F + 0.02).
The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""

import ctypes

import numpy as np
import pytest

import paper_2201_00451_gb300 as pkg
from oracle import resamp, synth
from workloads import config1

pytestmark = pytest.mark.gpu


def test_noalloc_matches_planned_path_on_two_calls():
    import torch

    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    lib = pkg.load()
    t = config1()                      # n_fft = 2^18, the entry point's maximum
    x = synth.make_data(t)
    alpha, delta = t.skies[0]
    tm = t.templates()
    picks = [3, 41]
    stream = torch.cuda.current_stream()
    with pkg.FstatPlan.from_target(t) as plan:
        plan.set_data(0, x[0], t.sigmas[0])
        ga, gb, abcd = plan.export_sky(alpha, delta)
        ref = plan.compute(tm[picks]).cpu().numpy()
        plan.sync()
    pairs = np.stack([ga.real, ga.imag, gb.real, gb.imag], axis=1).astype(np.float32)
    g_dev = torch.from_numpy(pairs).cuda()
    tau0 = resamp.ssb_start(t, alpha, delta) - t.t_reference
    A, B, C, _ = (float(v) for v in abcd)
    outs = []
    for k in picks:                    # two calls in a row share the scratch array
        out = torch.empty(t.n_fft, dtype=torch.float32, device="cuda")
        rc = lib.fstat_twoF_noalloc(
            ctypes.c_void_p(g_dev.data_ptr()), t.n_samples, t.n_fft, t.dt, tau0, A, B, C,
            float(tm["f1dot"][k]), float(tm["f2dot"][k]), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, pkg.ERR.get(rc, rc)
        outs.append(out)
    torch.cuda.synchronize()
    for i, out in enumerate(outs):
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref[i]) <= 1e-3 * np.abs(ref[i]) + 0.02)

    big = torch.empty(1 << 19, dtype=torch.float32, device="cuda")
    rc = lib.fstat_twoF_noalloc(ctypes.c_void_p(g_dev.data_ptr()), t.n_samples, 1 << 19, t.dt, tau0,
                                A, B, C, 0.0, 0.0, ctypes.c_void_p(big.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream))
    assert rc == -7  # FSTAT_ERR_UNSUPPORTED: beyond the fixed scratch size
