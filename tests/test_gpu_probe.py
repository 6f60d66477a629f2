"""Machine probes used by the benchmark's roofline figures (GPU).

* fstat_probe_fma returns positive FP32 and FP64 FMA rates, FP32 well above
  FP64 on this part.
* fstat_probe_dft16: the radix-16 DFT stage of the FFT passes on the CUDA
  cores and as a TF32 matrix product on the tensor cores (three-term split)
  both match numpy's FP64 16-point DFT to FP32-level accuracy, so their
  timings compare equal work.
"""

import numpy as np
import pytest
import torch

import paper_2201_00451_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


def test_fma_probe_rates():
    f32, _ = pkg.probe_fma(pkg.MIXED, 1 << 12)
    f64, _ = pkg.probe_fma(pkg.FP64, 1 << 10)
    assert f32 > 0 and f64 > 0 and f32 > 4 * f64


def _vectors(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, 16)) + 1j * rng.standard_normal((n, 16))).astype(np.complex128)


@pytest.mark.parametrize("method", [0, 1])
def test_dft16_stage_both_ways_match_fp64(method):
    n = 512 * 6
    x = _vectors(n, 3 + method)
    ref = np.fft.fft(x, axis=1)
    if method == 0:
        # float4 (a.re, a.im, b.re, b.im) [s][256] per block; vector 2v = a of pair v
        blocks = x.reshape(-1, 256, 2, 16)             # [block][pair][a/b][s]
        arr = np.empty((blocks.shape[0], 16, 256, 4), dtype=np.float32)
        arr[..., 0] = blocks[:, :, 0, :].real.transpose(0, 2, 1)
        arr[..., 1] = blocks[:, :, 0, :].imag.transpose(0, 2, 1)
        arr[..., 2] = blocks[:, :, 1, :].real.transpose(0, 2, 1)
        arr[..., 3] = blocks[:, :, 1, :].imag.transpose(0, 2, 1)
        out, ms = pkg.probe_dft16(0, torch.from_numpy(arr).cuda())
        o = out.cpu().numpy().astype(np.float64)
        a = (o[..., 0] + 1j * o[..., 1]).transpose(0, 2, 1)
        b = (o[..., 2] + 1j * o[..., 3]).transpose(0, 2, 1)
        got = np.stack([a, b], axis=2).reshape(n, 16)
    else:
        arr = np.concatenate([x.real, x.imag], axis=1).astype(np.float32)   # [vector][32]
        out, ms = pkg.probe_dft16(1, torch.from_numpy(arr).cuda())
        o = out.cpu().numpy().astype(np.float64)
        got = o[:, :16] + 1j * o[:, 16:]
    assert ms > 0
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err
