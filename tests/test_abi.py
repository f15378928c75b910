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


def _header_constants():
    """Integer constants of include/tlsph.h: #define NAME value and enumerators NAME = value."""
    src = open(os.path.join(ROOT, "include", "tlsph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, val in re.findall(r"#define\s+(TLSPH_\w+)\s+(-?\d+)u?\b", src):
        out[name] = int(val)
    for name, val in re.findall(r"\b(TLSPH_\w+)\s*=\s*(-?\d+)", src):
        out[name] = int(val)
    return out


def test_binding_constants_match_the_header():
    """The binding's flags, precisions, field ids, status codes, status bits
    and counts are the header's values."""
    h = _header_constants()
    for k in ("SPATIAL_ORDER", "WALL", "LINE_ORDER", "AUTO_ORDER"):
        assert getattr(tlsph, "FLAG_" + k) == h["TLSPH_FLAG_" + k], k
    for k, v in tlsph.PRECISION.items():
        assert v == h["TLSPH_PRECISION_" + k.upper()], k
    for k, v in tlsph.FIELD.items():
        assert v == h["TLSPH_FIELD_" + k], k
    assert len(tlsph.FIELD) == h["TLSPH_FIELD_COUNT"]
    for v, k in tlsph.STATUS.items():
        assert v == h["TLSPH_" + k], k
    for k in ("POLAR_CAP", "NEWTON_CAP", "BAD_J", "NONFINITE"):
        assert getattr(tlsph, "ST_" + k) == h["TLSPH_ST_" + k], k
    assert tlsph.DIAG_COUNT == h["TLSPH_DIAG_COUNT"]


def test_workspace_bytes(lib):
    cfg = tlsph.make_config(0.75e-3, 1.5e-3, 2e-8, 10.0)
    a = tlsph.workspace_bytes(cfg, 1000, 80000)
    b = tlsph.workspace_bytes(cfg, 1000, 160000)
    assert a > 0 and b - a >= 80000 * 4
    bad = tlsph.make_config(-1.0, 1.5e-3, 2e-8, 10.0)
    assert tlsph.workspace_bytes(bad, 1000, 10) == 0
    cfg_rc = tlsph.make_config(0.75e-3, 2e-3, 2e-8, 10.0)   # rc beyond 2h
    assert tlsph.workspace_bytes(cfg_rc, 1000, 10) == 0


def test_order_flags_are_validated(lib):
    """At most one internal-order flag; unknown flag bits are rejected (a
    configuration the library rejects has no workspace size)."""
    ok = [0, tlsph.FLAG_SPATIAL_ORDER, tlsph.FLAG_LINE_ORDER, tlsph.FLAG_AUTO_ORDER,
          tlsph.FLAG_AUTO_ORDER | tlsph.FLAG_WALL]
    bad = [tlsph.FLAG_SPATIAL_ORDER | tlsph.FLAG_LINE_ORDER, tlsph.FLAG_AUTO_ORDER | tlsph.FLAG_LINE_ORDER,
           tlsph.FLAG_AUTO_ORDER | tlsph.FLAG_SPATIAL_ORDER, 16]
    for precision in ("fp64", "mixed"):
        for f in ok:
            assert tlsph.workspace_bytes(tlsph.make_config(0.75e-3, 1.5e-3, 2e-8, 10.0, precision, f), 1000, 10) > 0
        for f in bad:
            assert tlsph.workspace_bytes(tlsph.make_config(0.75e-3, 1.5e-3, 2e-8, 10.0, precision, f), 1000, 10) == 0


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
    lib.tlsph_diagnostics_async.restype = ctypes.c_int
    lib.tlsph_diagnostics_async.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    assert lib.tlsph_diagnostics_async(None, out, 11) == -1


def test_tensor_bindings_reject_bad_tensors_before_any_launch():
    """The bindings that pass torch data pointers straight to the kernels
    (tlsph_neighbors_noalloc, tlsph_material_point_batch) check dtype, shape,
    layout and device first: each bad argument raises ValueError on the host
    (CPU tensors of the right form fail the device check last)."""
    torch = pytest.importorskip("torch")
    N = 8
    X = torch.zeros((N, 3), dtype=torch.float64)
    rp = torch.zeros(N + 1, dtype=torch.int64)
    col = torch.zeros(100, dtype=torch.int32)
    bad = [
        (X.float(), rp, col, "float64"),                                  # X in FP32
        (torch.zeros((N, 4), dtype=torch.float64), rp, col, "shape"),     # X not (N, 3)
        (torch.zeros((N, 6), dtype=torch.float64)[:, ::2], rp, col, "contiguous"),
        (X, rp.int(), col, "int64"),                                      # row_ptr in int32
        (X, torch.zeros(N, dtype=torch.int64), col, "at least"),          # row_ptr too short
        (X, rp, col.long(), "int32"),                                     # col in int64
        (X, rp, torch.zeros((10, 10), dtype=torch.int32), "1-dimensional"),
        (X, rp, col, "CUDA"),                                             # host tensors
        ([[0.0, 0.0, 0.0]], rp, col, "torch tensor"),
    ]
    for x, r, c, msg in bad:
        with pytest.raises(ValueError, match=msg):
            tlsph.neighbors_noalloc(x, 1e-3, r, c)
    n = 4
    deps, J, st = torch.zeros((n, 9), dtype=torch.float64), torch.ones(n, dtype=torch.float64), \
        torch.zeros((n, 16), dtype=torch.float64)
    from paper_1901_07374_gb300 import specimen as S
    m = S.aluminium_cl()
    for args, msg in [((deps.float(), J, st), "float64"), ((deps, J, st[:, :15]), "shape"),
                      ((deps.t().contiguous().t(), J, st), "contiguous"), ((deps, J, st), "CUDA")]:
        with pytest.raises(ValueError, match=msg):
            tlsph.material_point_batch(m, 1e-7, *args)
