"""The C-ABI library builds, loads without a GPU, exports every entry point
include/tlsph.h declares, and rejects bad arguments on the host before any
device work."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

from paper_1901_07374_gb300 import build as B
from paper_1901_07374_gb300 import tlsph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists(B.LIB):
        pytest.skip("no nvcc and no prebuilt library")
    B.build()
    return tlsph.load()


def declared():
    src = open(os.path.join(ROOT, "include", "tlsph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tlsph_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(tlsph.EXPORTS) <= set(names)


def test_workspace_bytes(lib):
    cfg = tlsph.make_config(0.75e-3, 1.5e-3, 2e-8, 10.0)
    a = tlsph.workspace_bytes(cfg, 1000, 80000)
    b = tlsph.workspace_bytes(cfg, 1000, 160000)
    assert a > 0 and b - a >= 80000 * 4
    bad = tlsph.make_config(-1.0, 1.5e-3, 2e-8, 10.0)
    assert tlsph.workspace_bytes(bad, 1000, 10) == 0
    cfg_rc = tlsph.make_config(0.75e-3, 2e-3, 2e-8, 10.0)   # rc beyond 2h
    assert tlsph.workspace_bytes(cfg_rc, 1000, 10) == 0


def _create(lib, cfg, N, X, vol, mat=None):
    ctx = ctypes.c_void_p()
    p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    return lib.tlsph_create(ctypes.byref(cfg), N, p(X), p(vol), p(mat), None, None, None, None, 0, 0, None,
                            ctypes.byref(ctx))


def test_create_rejects_bad_arguments_on_host(lib):
    """Missing arrays, N and the configuration are checked on the host before
    any device call (the array contents are validated on the device after
    their upload: test_gpu_api.py)."""
    cfg = tlsph.make_config(0.75e-3, 1.5e-3, 2e-8, 10.0)
    X = np.zeros((4, 3))
    vol = np.ones(4)
    assert _create(lib, cfg, 4, None, vol) == -1
    assert b"required" in lib.tlsph_last_error(None)
    assert _create(lib, cfg, 4, X, None) == -1
    assert _create(lib, cfg, 0, X, vol) == -1
    bad = tlsph.make_config(0.75e-3, 1.5e-3, 0.0, 10.0)
    assert _create(lib, bad, 4, X, vol) == -1
    bad = tlsph.make_config(0.75e-3, 1.5e-3, 2e-8, 10.0, "fp64")
    bad.precision = 7
    assert _create(lib, bad, 4, X, vol) == -1


def test_null_context_calls(lib):
    assert lib.tlsph_step(None, 1) == -1
    assert lib.tlsph_sync(None) == -1
    assert lib.tlsph_destroy(None) == -1
    assert lib.tlsph_set_material(None, 0, None) == -1


def test_diagnostics_argument_errors(lib):
    import ctypes
    out = (ctypes.c_double * 11)()
    lib.tlsph_diagnostics.restype = ctypes.c_int
    lib.tlsph_diagnostics.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    assert lib.tlsph_diagnostics(None, out, 11) == -1
