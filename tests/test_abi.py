"""CPU-side checks of the C ABI: the library loads, exports every entry
point include/asolve.h declares, and its structs match the binding."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_11208_gb300 import build
    build.build()
    from paper_2007_11208_gb300 import asolve
    return asolve


def declared_functions():
    src = open(os.path.join(ROOT, "include", "asolve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(asolve_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    L = lib.lib()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(lib.EXPORTS)


def test_version_and_strerror(lib):
    assert b"sm_103a" in lib.lib().asolve_version()
    assert lib.strerror(lib.E_NONFINITE) == "non-finite input"
    assert lib.strerror(12345) == "unknown status"


def test_default_config(lib):
    import numpy as np
    c = lib.default_config()
    eps = np.finfo(np.float64).eps
    assert c.rcond_threshold == 0.5 * eps
    assert c.sympd_tol == 100 * eps
    assert c.band_frac == 0.25
    assert c.precision == lib.PREC_MIXED
    assert c.ir_target_berr == 1e-13
    assert lib.lib().asolve_default_config(None) == lib.E_INVALID


def test_struct_sizes(lib):
    import ctypes as C
    assert C.sizeof(lib.Info) == 64
    assert C.sizeof(lib.ScanResult) == 56


def test_null_handles_rejected(lib):
    L = lib.lib()
    assert L.asolve_destroy(None) == lib.E_INVALID
    assert L.asolve_set_profiling(None, 1) == lib.E_INVALID
    assert L.asolve_create(None, None) == lib.E_INVALID


def test_binding_refuses_undersized_tensors(lib):
    """The binding checks tensor extents before a call reaches the library,
    which reads n*n elements of A and n*nrhs of B and X."""
    import torch
    need = lib._need
    need(torch.zeros(12, dtype=torch.float64), 12, "A")
    with pytest.raises(ValueError):
        need(torch.zeros(11, dtype=torch.float64), 12, "A")
    with pytest.raises(ValueError):
        need(torch.zeros(12, dtype=torch.float32), 12, "A")
    with pytest.raises(ValueError):
        need(torch.zeros(4, 6, dtype=torch.float64).t(), 12, "A")
    need(12345, 10 ** 9, "A")  # raw addresses are the caller's responsibility
