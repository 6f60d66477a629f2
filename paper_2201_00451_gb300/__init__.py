"""Python binding of libfstat (GB300 resampling F-statistic).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libfstat.so``.  PyTorch is used for device memory (output
tensors) and stream handles.  The names follow the C ABI in
``include/fstat.h``.

The library is built in-tree by ``paper_2201_00451_gb300.build.build()``.
Importing this package does not load it; the first use does, and raises
``FstatLibraryMissing`` if the shared library has not been built -- there
is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfstat.so")

MAX_DET = 4
OK = 0
ERR = {
    -1: "FSTAT_ERR_INVALID_ARG",
    -2: "FSTAT_ERR_OOM",
    -3: "FSTAT_ERR_CUDA",
    -4: "FSTAT_ERR_DEGENERATE",
    -5: "FSTAT_ERR_NONFINITE",
    -6: "FSTAT_ERR_NOT_READY",
    -7: "FSTAT_ERR_UNSUPPORTED",
    -8: "FSTAT_ERR_TIMEOUT",
}
MIXED, FP64 = 0, 1
C64, C128 = 0, 1
INTERP_TAPERED, INTERP_UNTAPERED, INTERP_PERIODIC = 0, 1, 2

# Every symbol include/fstat.h declares (checked by the tests).
EXPORTS = (
    "fstat_plan_create", "fstat_set_data", "fstat_compute", "fstat_freq_axis",
    "fstat_invalidate_sky", "fstat_export_sky", "fstat_sync", "fstat_set_profiling",
    "fstat_kernel_stats", "fstat_get_split", "fstat_set_split", "fstat_plan_destroy",
    "fstat_strerror", "fstat_twoF_noalloc", "fstat_get_cta", "fstat_set_cta", "fstat_autotune",
    "fstat_grad", "fstat_batch_create", "fstat_batch_add", "fstat_batch_instantiate",
    "fstat_batch_launch", "fstat_batch_nodes", "fstat_batch_destroy", "fstat_set_streams",
    "fstat_compute_peaks", "fstat_semicoherent", "fstat_set_residency", "fstat_get_residency",
    "fstat_set_sfts", "fstat_export_data", "fstat_reduce_peaks", "fstat_set_wait_limit",
    "fstat_probe_fma", "fstat_launch_count", "fstat_set_fused", "fstat_get_fused", "fstat_probe_dft16",
    "fstat_refine", "fstat_get_peaks_cta",
)


class FstatLibraryMissing(ImportError):
    pass


class FstatError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERR.get(code, code)} ({_strerror(code)})")


class Detector(ctypes.Structure):
    _fields_ = [("lat_rad", ctypes.c_double), ("lon_rad", ctypes.c_double),
                ("gamma_rad", ctypes.c_double)]


class Ephemeris(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "c", "au", "r_earth", "omega_rot", "omega_orb", "obliquity", "orb_phase0", "sidereal_phase0")]


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("n_det", ctypes.c_int32), ("dterms", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("interp", ctypes.c_int32), ("det", Detector * MAX_DET), ("t0", ctypes.c_double),
        ("dt", ctypes.c_double), ("n_samples", ctypes.c_int64), ("f_het", ctypes.c_double),
        ("n_fft", ctypes.c_int64), ("t_ref", ctypes.c_double), ("ephem", Ephemeris),
    ]


class Template(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("delta", ctypes.c_double),
                ("f1dot", ctypes.c_double), ("f2dot", ctypes.c_double)]


class PeakOut(ctypes.Structure):
    _fields_ = [
        ("threshold", ctypes.c_float), ("n_bands", ctypes.c_int32), ("tmpl_offset", ctypes.c_int64),
        ("peaks", ctypes.c_void_p), ("capacity", ctypes.c_int64), ("n_peaks", ctypes.c_void_p),
        ("band_max", ctypes.c_void_p), ("band_bin", ctypes.c_void_p),
    ]


# fstat_peak: one threshold crossing (16 bytes)
PEAK_DTYPE = np.dtype([("tmpl", "<i8"), ("bin", "<i4"), ("twoF", "<f4")])

TEMPLATE_DTYPE = np.dtype([("alpha", "<f8"), ("delta", "<f8"), ("f1dot", "<f8"), ("f2dot", "<f8")])
CANDIDATE_DTYPE = np.dtype([("f", "<f8"), ("f1dot", "<f8"), ("alpha", "<f8"), ("delta", "<f8"),
                            ("f2dot", "<f8")])

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libfstat.so (once) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = open_library(path)
    return _lib


def open_library(path: str) -> ctypes.CDLL:
    """Open a build of the library at ``path`` (not cached; ``load`` keeps
    the package's own) with its signatures declared.  Plans take it through
    ``FstatPlan(desc, lib=...)``."""
    if not os.path.exists(path):
        raise FstatLibraryMissing(
            f"{path} is not built; run paper_2201_00451_gb300.build.build() (needs nvcc)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "fstat_plan_create": (i32, [ctypes.POINTER(PlanDesc), ctypes.POINTER(P)]),
        "fstat_set_data": (i32, [P, i32, P, i32, i64, dbl, P]),
        "fstat_compute": (i32, [P, P, i64, P, P]),
        "fstat_freq_axis": (i32, [P, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
        "fstat_invalidate_sky": (i32, [P]),
        "fstat_export_sky": (i32, [P, dbl, dbl, P, P, P, P]),
        "fstat_sync": (i32, [P]),
        "fstat_set_profiling": (i32, [P, i32]),
        "fstat_kernel_stats": (i32, [P, i32, ctypes.POINTER(i64), ctypes.POINTER(dbl)]),
        "fstat_get_split": (i32, [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "fstat_set_split": (i32, [P, i64]),
        "fstat_plan_destroy": (None, [P]),
        "fstat_strerror": (ctypes.c_char_p, [i32]),
        "fstat_twoF_noalloc": (i32, [P, i64, i64, dbl, dbl, dbl, dbl, dbl, dbl, dbl, P, P]),
        "fstat_get_cta": (i32, [P] + [ctypes.POINTER(i32)] * 4),
        "fstat_get_peaks_cta": (i32, [P] + [ctypes.POINTER(i32)] * 2),
        "fstat_set_cta": (i32, [P, i32, i32, i32, i32]),
        "fstat_autotune": (i32, [P, P]),
        "fstat_grad": (i32, [P, P, i64, P, P, P]),
        "fstat_refine": (i32, [P, P, i64, P, i32, dbl, P, P, P]),
        "fstat_batch_create": (i32, [ctypes.POINTER(P)]),
        "fstat_batch_add": (i32, [P, P, P, i64, P, i64]),
        "fstat_batch_instantiate": (i32, [P, P]),
        "fstat_batch_launch": (i32, [P, P]),
        "fstat_batch_nodes": (i32, [P, ctypes.POINTER(i64)]),
        "fstat_batch_destroy": (None, [P]),
        "fstat_set_streams": (i32, [P, i32]),
        "fstat_compute_peaks": (i32, [P, P, i64, ctypes.POINTER(PeakOut), P]),
        "fstat_semicoherent": (i32, [ctypes.POINTER(P), i32, P, i64, dbl, P, P]),
        "fstat_set_residency": (i32, [P, i32, i32]),
        "fstat_set_sfts": (i32, [P, i32, P, i32, i64, i64, i64, dbl, i64, dbl, P]),
        "fstat_export_data": (i32, [P, i32, P, P]),
        "fstat_reduce_peaks": (i32, [P, P, i64, ctypes.POINTER(PeakOut), P]),
        "fstat_get_residency": (i32, [P, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "fstat_set_wait_limit": (i32, [P, i32]),
        "fstat_probe_fma": (i32, [i32, i64, ctypes.POINTER(dbl), ctypes.POINTER(dbl), P]),
        "fstat_launch_count": (i32, [P, ctypes.POINTER(i64)]),
        "fstat_set_fused": (i32, [P, i32]),
        "fstat_get_fused": (i32, [P, ctypes.POINTER(i32)]),
        "fstat_probe_dft16": (i32, [i32, P, P, i64, i32, ctypes.POINTER(dbl), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _strerror(code: int) -> str:
    try:
        return load().fstat_strerror(code).decode()
    except Exception:  # pragma: no cover - only while reporting another error
        return "?"


def _check(rc: int, where: str):
    if rc != OK:
        raise FstatError(rc, where)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_desc(*, detectors, t0, dt, n_samples, f_het, n_fft, dterms=8, precision=MIXED,
              t_ref=float("nan"), ephemeris, interp=INTERP_TAPERED) -> PlanDesc:
    """Fill a PlanDesc.  ``detectors``: objects with lat, lon, gamma (rad);
    ``ephemeris``: mapping with the fstat_ephemeris fields."""
    d = PlanDesc()
    d.n_det = len(detectors)
    d.dterms = int(dterms)
    d.precision = int(precision)
    d.interp = int(interp)
    for X, det in enumerate(detectors):
        d.det[X] = Detector(det.lat, det.lon, det.gamma)
    d.t0, d.dt, d.n_samples = float(t0), float(dt), int(n_samples)
    d.f_het, d.n_fft, d.t_ref = float(f_het), int(n_fft), float(t_ref)
    for k, _ in Ephemeris._fields_:
        setattr(d.ephem, k, float(ephemeris[k]))
    return d


def as_templates(templates) -> np.ndarray:
    """Contiguous structured array of fstat_template records."""
    a = np.asarray(templates)
    if a.dtype.names is None:
        a = np.asarray(a, dtype=np.float64).reshape(-1, 4)
        out = np.empty(len(a), dtype=TEMPLATE_DTYPE)
        for k, name in enumerate(TEMPLATE_DTYPE.names):
            out[name] = a[:, k]
        return out
    out = np.empty(len(a), dtype=TEMPLATE_DTYPE)
    for name in TEMPLATE_DTYPE.names:
        out[name] = a[name]
    return out


class FstatPlan:
    """A plan: sample grid, detectors, FFT length, precision (fstat_plan_*)."""

    def __init__(self, desc: PlanDesc, lib=None):
        self._lib = lib if lib is not None else load()
        self._p = ctypes.c_void_p()
        _check(self._lib.fstat_plan_create(ctypes.byref(desc), ctypes.byref(self._p)), "fstat_plan_create")
        self.desc = desc
        self.n_fft = int(desc.n_fft)
        self.n_samples = int(desc.n_samples)

    @classmethod
    def from_target(cls, target, precision=MIXED, dterms=None, interp=None, lib=None):
        """Plan for an object exposing the workload fields (detectors, t0, dt,
        n_samples, f_het, n_fft, dterms, t_ref, ephemeris; interp optional).
        ``dterms`` / ``interp`` override the target's; ``lib``: a library
        from ``open_library`` instead of the package's own."""
        if interp is None:
            interp = getattr(target, "interp", INTERP_TAPERED)
        return cls(make_desc(detectors=target.detectors, t0=target.t0, dt=target.dt,
                             n_samples=target.n_samples, f_het=target.f_het, n_fft=target.n_fft,
                             dterms=target.dterms if dterms is None else dterms,
                             precision=precision, t_ref=target.t_ref, ephemeris=target.ephemeris,
                             interp=interp), lib=lib)

    # -- lifetime
    def close(self):
        if self._p:
            self._lib.fstat_plan_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- data
    def set_data(self, det: int, xh, sigma: float, stream=None):
        """fstat_set_data: xh is a numpy array (host) or a CUDA torch tensor of
        complex64 / complex128 samples."""
        if isinstance(xh, np.ndarray):
            x = np.ascontiguousarray(xh)
            dtype = {np.dtype(np.complex64): C64, np.dtype(np.complex128): C128}[x.dtype]
            ptr = x.ctypes.data
            keep = x
        else:
            import torch
            x = xh.contiguous()
            dtype = {torch.complex64: C64, torch.complex128: C128}[x.dtype]
            ptr = x.data_ptr()
            keep = x
        rc = self._lib.fstat_set_data(self._p, int(det), ctypes.c_void_p(ptr), dtype, int(len(keep)),
                                      float(sigma), _stream_handle(stream))
        _check(rc, "fstat_set_data")

    def set_sfts(self, det: int, bins, q0: int, t_sft: float, m_raw: int, sigma: float, stream=None):
        """fstat_set_sfts: x_h of detector ``det`` from SFT band bins, a numpy
        array (host) or CUDA tensor [n_sft, n_bins] of complex64/complex128."""
        if isinstance(bins, np.ndarray):
            b = np.ascontiguousarray(bins)
            dtype = {np.dtype(np.complex64): C64, np.dtype(np.complex128): C128}[b.dtype]
            ptr, shape = b.ctypes.data, b.shape
        else:
            import torch
            b = bins.contiguous()
            dtype = {torch.complex64: C64, torch.complex128: C128}[b.dtype]
            ptr, shape = b.data_ptr(), tuple(b.shape)
        rc = self._lib.fstat_set_sfts(self._p, int(det), ctypes.c_void_p(ptr), dtype, int(shape[0]), int(shape[1]),
                                      int(q0), float(t_sft), int(m_raw), float(sigma), _stream_handle(stream))
        _check(rc, "fstat_set_sfts")

    def export_data(self, det: int, stream=None) -> np.ndarray:
        """The stored series of detector ``det`` (complex64 or complex128)."""
        out = np.empty(self.n_samples, dtype=np.complex128)
        rc = self._lib.fstat_export_data(self._p, int(det), ctypes.c_void_p(out.ctypes.data), _stream_handle(stream))
        if rc < 0:
            _check(rc, "fstat_export_data")
        if rc == C64:
            return out.view(np.complex64)[: self.n_samples].copy()
        return out

    def compute(self, templates, out=None, stream=None):
        """fstat_compute: returns a CUDA float32 tensor [n_templates, n_fft] of 2F
        (``out`` may supply it)."""
        import torch
        t = as_templates(templates)
        n = len(t)
        if out is None:
            out = torch.empty((n, self.n_fft), dtype=torch.float32, device="cuda")
        if out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous() or out.numel() < n * self.n_fft:
            raise ValueError("out must be a contiguous CUDA float32 tensor with n_templates*n_fft elements")
        rc = self._lib.fstat_compute(self._p, ctypes.c_void_p(t.ctypes.data), n,
                                     ctypes.c_void_p(out.data_ptr()), _stream_handle(stream))
        _check(rc, "fstat_compute")
        return out

    def compute_ptr(self, templates: np.ndarray, out_ptr: int, stream=None):
        """fstat_compute into a raw device pointer (templates already as TEMPLATE_DTYPE)."""
        rc = self._lib.fstat_compute(self._p, ctypes.c_void_p(templates.ctypes.data), len(templates),
                                     ctypes.c_void_p(out_ptr), _stream_handle(stream))
        _check(rc, "fstat_compute")

    def reduce_peaks(self, twoF, threshold: float = 70.0, n_bands: int = 0, capacity: int = 4096,
                     tmpl_offset: int = 0, out=None, stream=None):
        """fstat_reduce_peaks: the peaks reduction of a CUDA float32 tensor
        [n_rows, n_fft] of 2F already on the device; same result dict as
        compute_peaks."""
        return self._peaks(None, twoF, threshold, n_bands, capacity, tmpl_offset, out, stream)

    def compute_peaks(self, templates, threshold: float = 70.0, n_bands: int = 0, capacity: int = 4096,
                      tmpl_offset: int = 0, out=None, stream=None):
        """fstat_compute_peaks: 2F reduced on the device.  Returns a dict of
        CUDA tensors: ``count`` (int64 [1], every crossing of ``threshold``),
        ``peaks`` (int32 [capacity, 4]: template index lo/hi words, bin, 2F
        bits; see :func:`peaks_to_numpy`), and for ``n_bands > 0``
        ``band_max`` (float32 [n, n_bands]) and ``band_bin`` (int32).
        ``out`` may pass such a dict back in to append to its list (its band
        buffers are reused when their shape fits)."""
        return self._peaks(templates, None, threshold, n_bands, capacity, tmpl_offset, out, stream)

    def _peaks(self, templates, twoF, threshold, n_bands, capacity, tmpl_offset, out, stream):
        import torch
        if templates is not None:
            t = as_templates(templates)
            n = len(t)
        else:
            if twoF.dtype != torch.float32 or not twoF.is_cuda or not twoF.is_contiguous() or \
                    twoF.dim() != 2 or twoF.shape[1] != self.n_fft:
                raise ValueError("twoF must be a contiguous CUDA float32 tensor [n_rows, n_fft]")
            n = twoF.shape[0]
        if out is None:
            out = {"count": torch.zeros(1, dtype=torch.int64, device="cuda"),
                   "peaks": torch.empty((max(capacity, 0), 4), dtype=torch.int32, device="cuda")}
        if n_bands > 0:
            for key, dt in (("band_max", torch.float32), ("band_bin", torch.int32)):
                b = out.get(key)
                if b is None or b.shape != (n, n_bands) or b.dtype != dt or not b.is_cuda:
                    out[key] = torch.empty((n, n_bands), dtype=dt, device="cuda")
        po = PeakOut()
        po.threshold = float(threshold)
        po.n_bands = int(n_bands)
        po.tmpl_offset = int(tmpl_offset)
        cap = out["peaks"].shape[0] if out.get("peaks") is not None else 0
        po.peaks = out["peaks"].data_ptr() if cap else None
        po.capacity = cap
        po.n_peaks = out["count"].data_ptr() if out.get("count") is not None else None
        po.band_max = out["band_max"].data_ptr() if n_bands > 0 else None
        po.band_bin = out["band_bin"].data_ptr() if n_bands > 0 else None
        if templates is not None:
            rc = self._lib.fstat_compute_peaks(self._p, ctypes.c_void_p(t.ctypes.data), n, ctypes.byref(po),
                                               _stream_handle(stream))
            _check(rc, "fstat_compute_peaks")
        else:
            rc = self._lib.fstat_reduce_peaks(self._p, ctypes.c_void_p(twoF.data_ptr()), n, ctypes.byref(po),
                                              _stream_handle(stream))
            _check(rc, "fstat_reduce_peaks")
        return out

    def grad(self, candidates, stream=None):
        """fstat_grad: (2F [n], d2F/d(f, f1dot, alpha, delta) [n, 4]) as CUDA
        float32 tensors for a structured array of CANDIDATE_DTYPE."""
        import torch
        c = np.ascontiguousarray(candidates, dtype=CANDIDATE_DTYPE)
        n = len(c)
        two_f = torch.empty(n, dtype=torch.float32, device="cuda")
        g = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        rc = self._lib.fstat_grad(self._p, ctypes.c_void_p(c.ctypes.data), n, ctypes.c_void_p(two_f.data_ptr()),
                                  ctypes.c_void_p(g.data_ptr()), _stream_handle(stream))
        _check(rc, "fstat_grad")
        return two_f, g

    def refine(self, candidates, scales, steps: int = 20, step0: float = 0.25, stream=None):
        """fstat_refine: gradient ascent on 2F on the device.  Returns (the
        final candidates as a CANDIDATE_DTYPE array, 2F after each step
        [steps + 1, n] float32)."""
        c = np.ascontiguousarray(candidates, dtype=CANDIDATE_DTYPE)
        n = len(c)
        sc = np.ascontiguousarray(scales, dtype=np.float64)
        if sc.shape != (4,):
            raise ValueError("scales: 4 values (f, f1dot, alpha, delta)")
        out = np.empty(n, dtype=CANDIDATE_DTYPE)
        hist = np.empty((int(steps) + 1, n), dtype=np.float32)
        rc = self._lib.fstat_refine(self._p, ctypes.c_void_p(c.ctypes.data), n, ctypes.c_void_p(sc.ctypes.data),
                                    int(steps), float(step0), ctypes.c_void_p(out.ctypes.data),
                                    ctypes.c_void_p(hist.ctypes.data), _stream_handle(stream))
        _check(rc, "fstat_refine")
        return out, hist

    def freq_axis(self):
        f0, df = ctypes.c_double(), ctypes.c_double()
        _check(self._lib.fstat_freq_axis(self._p, ctypes.byref(f0), ctypes.byref(df)), "fstat_freq_axis")
        return f0.value, df.value

    def invalidate_sky(self):
        _check(self._lib.fstat_invalidate_sky(self._p), "fstat_invalidate_sky")

    def export_sky(self, alpha: float, delta: float, stream=None):
        """Per-sky resampled, antenna-weighted series (G_a, G_b) and (A, B, C, D)."""
        ga = np.empty(self.n_samples, dtype=np.complex128)
        gb = np.empty(self.n_samples, dtype=np.complex128)
        abcd = np.empty(4, dtype=np.float64)
        rc = self._lib.fstat_export_sky(self._p, float(alpha), float(delta), ctypes.c_void_p(ga.ctypes.data),
                                        ctypes.c_void_p(gb.ctypes.data), ctypes.c_void_p(abcd.ctypes.data),
                                        _stream_handle(stream))
        _check(rc, "fstat_export_sky")
        return ga, gb, abcd

    def sync(self):
        _check(self._lib.fstat_sync(self._p), "fstat_sync")

    def set_profiling(self, enable: bool):
        _check(self._lib.fstat_set_profiling(self._p, int(bool(enable))), "fstat_set_profiling")

    def kernel_stats(self, kernel: int):
        n, ms = ctypes.c_int64(), ctypes.c_double()
        _check(self._lib.fstat_kernel_stats(self._p, int(kernel), ctypes.byref(n), ctypes.byref(ms)),
               "fstat_kernel_stats")
        return n.value, ms.value

    @property
    def split(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.fstat_get_split(self._p, ctypes.byref(a), ctypes.byref(b)), "fstat_get_split")
        return a.value, b.value

    def set_split(self, n1: int):
        _check(self._lib.fstat_set_split(self._p, int(n1)), "fstat_set_split")

    @property
    def cta(self):
        """(ca, va, cb, vb): pass-A columns/CTA and radix schedule, pass-B rows/CTA and schedule."""
        v = [ctypes.c_int() for _ in range(4)]
        _check(self._lib.fstat_get_cta(self._p, *[ctypes.byref(x) for x in v]), "fstat_get_cta")
        return tuple(x.value for x in v)

    @property
    def peaks_cta(self):
        """(cb, vb): the pass-B shape of compute_peaks (tuned apart by autotune)."""
        v = [ctypes.c_int() for _ in range(2)]
        _check(self._lib.fstat_get_peaks_cta(self._p, *[ctypes.byref(x) for x in v]), "fstat_get_peaks_cta")
        return tuple(x.value for x in v)

    @property
    def residency(self):
        """(ra, rb): persistent CTAs per SM of pass A and pass B (0 = all that fit)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.fstat_get_residency(self._p, ctypes.byref(a), ctypes.byref(b)), "fstat_get_residency")
        return a.value, b.value

    def set_residency(self, ra: int, rb: int):
        """fstat_set_residency: at most ra (pass A) / rb (pass B) persistent
        CTAs per SM, 0 = every CTA that fits."""
        _check(self._lib.fstat_set_residency(self._p, int(ra), int(rb)), "fstat_set_residency")

    def set_cta(self, ca: int, cb: int, va: int = 0, vb: int = 0):
        """fstat_set_cta: columns per CTA of pass A (ca), rows per CTA of pass
        B (cb), 0 = the length's default; schedules va (0..3, 10, 16 or 18)
        and vb (0..8): bit 0 radix-8 first, bit 1 one buffer
        (register-capped for two CTAs per SM), bit 2 pass-B tiles by TMA,
        bit 3 pass A three CTAs per SM, va 16 / 18 columns staged apart, vb
        8 half of the next pass-B tile staged apart."""
        _check(self._lib.fstat_set_cta(self._p, int(ca), int(va), int(cb), int(vb)), "fstat_set_cta")

    def set_streams(self, n: int):
        """fstat_set_streams: templates rotate over n streams (1..8)."""
        _check(self._lib.fstat_set_streams(self._p, int(n)), "fstat_set_streams")

    @property
    def launches(self) -> int:
        """fstat_launch_count: kernel launches enqueued since creation."""
        n = ctypes.c_int64()
        _check(self._lib.fstat_launch_count(self._p, ctypes.byref(n)), "fstat_launch_count")
        return n.value

    @property
    def fused(self) -> bool:
        """fstat_get_fused: whether fstat_compute runs the persistent launch."""
        v = ctypes.c_int()
        _check(self._lib.fstat_get_fused(self._p, ctypes.byref(v)), "fstat_get_fused")
        return bool(v.value)

    def set_fused(self, enable: bool):
        """fstat_set_fused: one persistent launch of both FFT passes per sky
        group (raises FstatError UNSUPPORTED where no shape is compiled)."""
        _check(self._lib.fstat_set_fused(self._p, int(bool(enable))), "fstat_set_fused")

    def set_wait_limit(self, polls: int):
        """fstat_set_wait_limit: polls of pass B's first bulk-copy wait per
        tile (< 0 restores the default)."""
        _check(self._lib.fstat_set_wait_limit(self._p, int(polls)), "fstat_set_wait_limit")

    def autotune(self, stream=None):
        """fstat_autotune: pick the fastest FFT split and CTA shapes."""
        _check(self._lib.fstat_autotune(self._p, _stream_handle(stream)), "fstat_autotune")


def probe_fma(precision=MIXED, iters: int = 1 << 16, stream=None):
    """fstat_probe_fma: measured FMA rate of the CUDA cores, (TFLOP/s, ms)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().fstat_probe_fma(int(precision), int(iters), ctypes.byref(tf), ctypes.byref(ms),
                                  _stream_handle(stream)), "fstat_probe_fma")
    return tf.value, ms.value


def probe_dft16(method: int, x, reps: int = 1, stream=None):
    """fstat_probe_dft16: the radix-16 DFT stage on the CUDA cores (0) or
    the tensor cores (1).  ``x``: CUDA tensor in the method's layout
    (float32, n_vectors * 32 values); returns (output tensor, ms)."""
    import torch
    x = x.contiguous()
    out = torch.empty_like(x)
    ms = ctypes.c_double()
    n_vectors = x.numel() * x.element_size() // 128
    _check(load().fstat_probe_dft16(int(method), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    int(n_vectors), int(reps), ctypes.byref(ms), _stream_handle(stream)),
           "fstat_probe_dft16")
    return out, ms.value


def semicoherent(plans, templates, t_ref: float, out=None, stream=None):
    """fstat_semicoherent: sum over segment plans of 2F with nearest-bin
    sliding, for templates whose spindowns are given at ``t_ref``.  Returns
    a CUDA float32 tensor [n_templates, n_fft] (``out`` may supply it)."""
    import torch
    lib = load()
    t = as_templates(templates)
    n = len(t)
    n_fft = plans[0].n_fft
    if out is None:
        out = torch.empty((n, n_fft), dtype=torch.float32, device="cuda")
    if out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous() or out.numel() < n * n_fft:
        raise ValueError("out must be a contiguous CUDA float32 tensor with n_templates*n_fft elements")
    arr = (ctypes.c_void_p * len(plans))(*[p._p.value for p in plans])
    rc = lib.fstat_semicoherent(arr, len(plans), ctypes.c_void_p(t.ctypes.data), n, float(t_ref),
                                ctypes.c_void_p(out.data_ptr()), _stream_handle(stream))
    _check(rc, "fstat_semicoherent")
    return out


def peaks_to_numpy(out) -> np.ndarray:
    """The filled part of a compute_peaks list as a PEAK_DTYPE array."""
    n = min(int(out["count"].item()), out["peaks"].shape[0])
    return out["peaks"][:n].cpu().numpy().copy().view(PEAK_DTYPE).reshape(n)


class FstatBatch:
    """fstat_batch_*: several plans' template banks replayed as one CUDA graph."""

    def __init__(self):
        self._lib = load()
        self._b = ctypes.c_void_p()
        _check(self._lib.fstat_batch_create(ctypes.byref(self._b)), "fstat_batch_create")
        self._keep = []

    def add(self, plan: FstatPlan, templates, out, out_rows: int = 0):
        t = as_templates(templates)
        rc = self._lib.fstat_batch_add(self._b, plan._p, ctypes.c_void_p(t.ctypes.data), len(t),
                                       ctypes.c_void_p(out.data_ptr()), int(out_rows))
        _check(rc, "fstat_batch_add")
        self._keep.append((plan, out))

    def instantiate(self, stream=None):
        _check(self._lib.fstat_batch_instantiate(self._b, _stream_handle(stream)), "fstat_batch_instantiate")

    def launch(self, stream=None):
        _check(self._lib.fstat_batch_launch(self._b, _stream_handle(stream)), "fstat_batch_launch")

    @property
    def nodes(self) -> int:
        n = ctypes.c_int64()
        _check(self._lib.fstat_batch_nodes(self._b, ctypes.byref(n)), "fstat_batch_nodes")
        return n.value

    def close(self):
        if self._b:
            self._lib.fstat_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
