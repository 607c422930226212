"""CPU-side checks of the C ABI: the library loads, exports every symbol the
headers declare, and rejects bad arguments before touching a GPU."""
import ctypes as ct
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(rttda_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import build
    build.build()
    from paper_2601_16949_b300 import binding
    return binding


def test_library_exports_every_declared_symbol(rb):
    names = declared_symbols()
    assert "rttda_create" in names and "rttda_propagate" in names
    missing = [n for n in names if not hasattr(rb.lib, n)]
    assert not missing, missing


def test_abi_version(rb):
    assert rb.rttda_abi_version() == 2


def test_create_rejects_bad_sizes_without_gpu(rb):
    h = ct.c_void_p()
    z = np.zeros(8)
    p = z.ctypes.data_as(ct.POINTER(ct.c_double))
    st = rb.lib.rttda_create(0, 3, 4, p, p, p, p, p, p, p, p, 0.2, 0, ct.byref(h))
    assert st == rb.E_ARG and not h.value
    assert "nocc" in rb.rttda_last_error()
    st = rb.lib.rttda_create(2, 3, 4, p, None, p, p, p, p, p, p, 0.2, 0, ct.byref(h))
    assert st == rb.E_ARG
    st = rb.lib.rttda_create(2, 3, 4, p, p, p, p, p, p, p, p, 0.2, 7, ct.byref(h))
    assert st == rb.E_ARG
    st = rb.lib.rttda_create(2, 3, 4, p, p, p, p, p, p, p, p, 0.2, rb.TF32, ct.byref(h))
    assert st == rb.E_ARG and b"TF32" in rb.lib.rttda_last_error()
    st = rb.lib.rttda_create(513, 3, 4, p, p, p, p, p, p, p, p, 0.2, rb.FP64_OZ, ct.byref(h))
    assert st == rb.E_ARG and b"512" in rb.lib.rttda_last_error()


def test_spectrum_rejects_bad_arguments_without_gpu(rb):
    tr = np.zeros((1, 1))
    with pytest.raises(rb.RTTDAError) as e:
        rb.rttda_spectrum(tr, 0.05, 1e-3, 1e-3, 0.0, 1.0, 5)   # npts < 2
    assert e.value.status == rb.E_ARG
    with pytest.raises(rb.RTTDAError) as e:
        rb.rttda_spectrum(np.zeros((1, 4)), 0.05, 0.0, 1e-3, 0.0, 1.0, 5)   # kappa = 0
    assert e.value.status == rb.E_ARG


def test_null_handle_calls_fail_cleanly(rb):
    assert rb.lib.rttda_set_field(None, None, 1) == rb.E_ARG
    assert rb.lib.rttda_propagate(None, None, 0.05, 1, None, None, None) == rb.E_ARG
    rb.lib.rttda_destroy(None)
