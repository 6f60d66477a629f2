"""The C-ABI library builds, loads, and exports every declared symbol (CPU).

Argument validation that happens before any CUDA call is checked here too;
no compute call is made without a GPU.
"""

import ctypes
import math
import os
import re

import pytest

import paper_2201_00451_gb300 as pkg
from paper_2201_00451_gb300 import build as fbuild
from workloads import DETECTORS, EPHEMERIS

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "fstat.h")


@pytest.fixture(scope="module")
def lib():
    fbuild.build()
    return pkg.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(fstat_\w+)\s*\(", text, re.M)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(pkg.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {pkg.LIB_PATH}").read()
    for name in declared_functions():
        assert re.search(rf"\bT {name}\b", out), name


def test_strerror_names_every_code(lib):
    for code in [0, -1, -2, -3, -4, -5, -6, -7]:
        s = lib.fstat_strerror(code).decode()
        assert s and s != "unknown error"


def _desc(**over):
    d = pkg.make_desc(detectors=[DETECTORS["H1"]], t0=0.0, dt=1.0, n_samples=1000, f_het=100.0,
                      n_fft=1 << 12, ephemeris=EPHEMERIS)
    for k, v in over.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("field,value,code", [
    ("n_det", 0, -1), ("n_det", 5, -1), ("dterms", 0, -1), ("precision", 7, -1),
    ("dt", 0.0, -1), ("n_samples", 0, -1), ("n_fft", 3000, -1), ("n_samples", 5000, -1),
    ("n_fft", 1 << 25, -7), ("n_fft", 1 << 9, -7), ("interp", 3, -1), ("interp", -1, -1),
])
def test_plan_create_rejects_bad_descriptions(lib, field, value, code):
    d = _desc(**{field: value})
    p = ctypes.c_void_p()
    assert lib.fstat_plan_create(ctypes.byref(d), ctypes.byref(p)) == code
    assert not p.value


def test_null_arguments_are_rejected(lib):
    assert lib.fstat_plan_create(None, None) == -1
    assert lib.fstat_compute(None, None, 0, None, None) == -1
    assert lib.fstat_sync(None) == -1
    f0, df = ctypes.c_double(), ctypes.c_double()
    assert lib.fstat_freq_axis(None, ctypes.byref(f0), ctypes.byref(df)) == -1
    lib.fstat_plan_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(pkg.FstatLibraryMissing):
        saved = pkg._lib
        pkg._lib = None
        try:
            pkg.load(str(tmp_path / "missing.so"))
        finally:
            pkg._lib = saved
