"""ctypes binding of libtlsph.so (the C ABI in include/tlsph.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels behind the ABI.  PyTorch provides device memory (the optional arena)
and the CUDA stream.  There is no CPU fallback: if the library is missing or
the GPU is absent, constructing a Simulation raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

PRECISION = {"fp64": 0, "mixed": 1}
# precision bench.py reports by default
DEFAULT_PRECISION = "mixed"
# precisions the smoke check runs, with the field tolerance against the oracle
SMOKE_PRECISIONS = (("fp64", 1e-10), ("mixed", 1e-4))

FIELD = dict(X=0, U=1, V=2, F=3, SIGMA=4, STRESS_DEV=5, EPSP=6, EPSP_RATE=7, DINIT=8, DAMAGE=9,
             POROSITY=10, FAIL_STEP=11, FORCE=12, A=13, LINV=14, NBR_ROWPTR=15, NBR_COL=16, STEP=17, ENERGY=18)
# (numpy dtype, components per particle); None = special count
_FIELD_SHAPE = dict(X=(np.float64, 3), U=(np.float64, 3), V=(np.float64, 3), F=(np.float64, 9),
                    SIGMA=(np.float64, 9), STRESS_DEV=(np.float64, 9), EPSP=(np.float64, 1),
                    EPSP_RATE=(np.float64, 1), DINIT=(np.float64, 1), DAMAGE=(np.float64, 1),
                    POROSITY=(np.float64, 1), FAIL_STEP=(np.int32, 1), FORCE=(np.float64, 3),
                    A=(np.float64, 9), LINV=(np.float64, 9), NBR_ROWPTR=(np.int64, None),
                    NBR_COL=(np.int32, None), STEP=(np.int64, None), ENERGY=(np.float64, 1))

# fields that together are the resumable state of a context
CHECKPOINT_FIELDS = ("U", "V", "F", "STRESS_DEV", "SIGMA", "EPSP", "EPSP_RATE", "DINIT", "DAMAGE", "POROSITY",
                     "ENERGY", "FAIL_STEP", "FORCE", "STEP")

# doubles returned by tlsph_diagnostics (TLSPH_DIAG_COUNT)
DIAG_COUNT = 11


def diagnostics_dict(out) -> dict:
    """The named values of a tlsph_diagnostics result (a sequence or tensor of
    DIAG_COUNT doubles)."""
    v = [float(x) for x in out[:DIAG_COUNT]]
    return {"momentum": tuple(v[0:3]), "force_sum": tuple(v[3:6]), "kinetic_energy": v[6], "failed": int(v[7]),
            "max_damage": v[8], "max_epsp": v[9], "internal_energy": v[10]}

STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_SINGULAR_L", -3: "ERR_NUMERICS", -4: "ERR_NOMEM",
          -5: "ERR_CUDA", -6: "ERR_STATE"}
ST_POLAR_CAP, ST_NEWTON_CAP, ST_BAD_J, ST_NONFINITE = 1, 2, 4, 8


class TlsphError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("rc", ctypes.c_double), ("dt", ctypes.c_double),
                ("hg_alpha", ctypes.c_double), ("precision", ctypes.c_int32), ("flags", ctypes.c_int32)]


class Material(ctypes.Structure):
    _fields_ = [("rho0", ctypes.c_double), ("E", ctypes.c_double), ("nu", ctypes.c_double),
                ("eos", ctypes.c_int32),
                ("c0", ctypes.c_double), ("S_alpha", ctypes.c_double), ("Gamma0", ctypes.c_double),
                ("A", ctypes.c_double), ("B", ctypes.c_double), ("n", ctypes.c_double),
                ("C", ctypes.c_double), ("epsdot0", ctypes.c_double),
                ("damage", ctypes.c_int32),
                ("Wcr", ctypes.c_double),
                ("D1", ctypes.c_double), ("D2", ctypes.c_double), ("D3", ctypes.c_double),
                ("D4", ctypes.c_double), ("D5", ctypes.c_double),
                ("q1", ctypes.c_double), ("q2", ctypes.c_double), ("q3", ctypes.c_double),
                ("fN", ctypes.c_double), ("eN", ctypes.c_double), ("sN", ctypes.c_double),
                ("fc", ctypes.c_double), ("fF", ctypes.c_double), ("komega", ctypes.c_double)]


def make_material(d: dict) -> Material:
    m = Material()
    for name, _ in Material._fields_:
        setattr(m, name, d[name])
    return m


EXPORTS = ("tlsph_workspace_bytes", "tlsph_create", "tlsph_set_material", "tlsph_step", "tlsph_sync",
           "tlsph_status_bits", "tlsph_info", "tlsph_get_state", "tlsph_set_state", "tlsph_last_error",
           "tlsph_destroy", "tlsph_material_point_batch", "tlsph_profile_enable", "tlsph_profile_read",
           "tlsph_set_plan", "tlsph_get_plan", "tlsph_batch_create", "tlsph_batch_set", "tlsph_batch_step",
           "tlsph_batch_sync", "tlsph_batch_last_error", "tlsph_batch_destroy", "tlsph_batch_set_shape",
           "tlsph_batch_get_shape", "tlsph_neighbor_layout",
           "tlsph_fma_peak", "tlsph_set_guard", "tlsph_diagnostics", "tlsph_diagnostics_async",
           "tlsph_set_grip_ramp")

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libtlsph.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: build it first (paper_1901_07374_gb300.build.build())")
            _build.build()
        L = ctypes.CDLL(path)
        vp, i64, i32, dbl, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        L.tlsph_workspace_bytes.restype = sz
        L.tlsph_workspace_bytes.argtypes = [ctypes.POINTER(Config), i64, i64]
        L.tlsph_create.restype = i32
        L.tlsph_create.argtypes = [ctypes.POINTER(Config), i64, vp, vp, vp, vp, vp, vp, vp, sz, i64, vp,
                                   ctypes.POINTER(vp)]
        L.tlsph_set_material.restype = i32
        L.tlsph_set_material.argtypes = [vp, i32, ctypes.POINTER(Material)]
        L.tlsph_step.restype = i32
        L.tlsph_step.argtypes = [vp, i32]
        L.tlsph_sync.restype = i32
        L.tlsph_sync.argtypes = [vp]
        L.tlsph_status_bits.restype = i32
        L.tlsph_status_bits.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
        L.tlsph_info.restype = i32
        L.tlsph_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.tlsph_get_state.restype = i32
        L.tlsph_get_state.argtypes = [vp, i32, vp, sz, i32]
        L.tlsph_set_state.restype = i32
        L.tlsph_set_state.argtypes = [vp, i32, vp, sz, i32]
        L.tlsph_last_error.restype = ctypes.c_char_p
        L.tlsph_last_error.argtypes = [vp]
        L.tlsph_destroy.restype = i32
        L.tlsph_destroy.argtypes = [vp]
        L.tlsph_profile_enable.restype = i32
        L.tlsph_profile_enable.argtypes = [vp, i32]
        L.tlsph_profile_read.restype = i32
        L.tlsph_profile_read.argtypes = [vp, ctypes.POINTER(dbl), i32, ctypes.POINTER(i64)]
        L.tlsph_set_plan.restype = i32
        L.tlsph_set_plan.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), i32]
        L.tlsph_get_plan.restype = i32
        L.tlsph_get_plan.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), i32]
        L.tlsph_diagnostics.restype = i32
        L.tlsph_diagnostics.argtypes = [vp, ctypes.POINTER(dbl), i32]
        L.tlsph_diagnostics_async.restype = i32
        L.tlsph_diagnostics_async.argtypes = [vp, ctypes.POINTER(dbl), i32]
        L.tlsph_set_guard.restype = i32
        L.tlsph_set_guard.argtypes = [vp, dbl]
        L.tlsph_set_grip_ramp.restype = i32
        L.tlsph_set_grip_ramp.argtypes = [vp, dbl]
        L.tlsph_fma_peak.restype = i32
        L.tlsph_fma_peak.argtypes = [i32, i32, ctypes.POINTER(dbl)]
        L.tlsph_neighbor_layout.restype = i32
        L.tlsph_neighbor_layout.argtypes = [vp] + [ctypes.POINTER(i64)] * 4
        L.tlsph_batch_create.restype = i32
        L.tlsph_batch_create.argtypes = [i32, vp, ctypes.POINTER(vp)]
        L.tlsph_batch_set.restype = i32
        L.tlsph_batch_set.argtypes = [vp, ctypes.POINTER(vp), i32]
        L.tlsph_batch_step.restype = i32
        L.tlsph_batch_step.argtypes = [vp, i32, i32]
        L.tlsph_batch_sync.restype = i32
        L.tlsph_batch_sync.argtypes = [vp]
        L.tlsph_batch_last_error.restype = ctypes.c_char_p
        L.tlsph_batch_last_error.argtypes = [vp]
        L.tlsph_batch_destroy.restype = i32
        L.tlsph_batch_destroy.argtypes = [vp]
        L.tlsph_batch_set_shape.restype = i32
        L.tlsph_batch_set_shape.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), i32]
        L.tlsph_batch_get_shape.restype = i32
        L.tlsph_batch_get_shape.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), i32]
        L.tlsph_material_point_batch.restype = i32
        L.tlsph_material_point_batch.argtypes = [ctypes.POINTER(Material), dbl, i64, vp, vp, vp, vp]
        _lib = L
        return L


def _check(code: int, ctx=None):
    if code != 0:
        msg = load().tlsph_last_error(ctx).decode(errors="replace")
        raise TlsphError(code, msg)


def mixed_algorithmic_bytes(N: int, list_words: int):
    """HBM bytes per step of (pass 1, pass 2) in the mixed path that the method
    must move with the library's state layout: the neighbour lists once per
    pass (`list_words` 4-byte words: 4 per pair for the CSR or explicit
    slices, a few bits per pair for aligned slices) plus each particle's own
    records and state read and written once (an elastic particle; gathered
    neighbour records count as on-chip reuse).
    pass 1: position 16, v record 16, L^-1 36, F (compensated) rw 144,
            deviator (compensated) rw 96, eps_p / rate / D_init r 24, D r+w 16,
            fail 4, material 4, V 8, u 24, E 8, sigma r+w 48,
            internal energy r+w 16, pass-2 record w 96                  = 556
    pass 2: position 16, own pass-2 record 96, S0 16, V 8, D 8, E 8,
            1/m 8, v_half rw 48, v w 24, force w 24, u r+w 48, fail 4, bc 1,
            v record w 16                                               = 325"""
    return 4 * list_words + 556 * N, 4 * list_words + 325 * N


# FP32 operations per pair-interaction of the mixed path's pair terms (an FMA,
# a compare-and-select, a reciprocal or a reciprocal square root counts as
# one), from the formulas as written in the pair functions of the library:
#  pass 1 (velocity gradient): X_ij from fixed-point positions 6, r^2 3, 1/r 1,
#         q 2, W'(q) 8, weight 2, v_ij 6, 9 sums                          = 37
#  pass 2 (forces): X_ij 6, r^2 3, 1/r 1, q 2, W'(q) 8, weights 3, 3 sums of
#         the S0 term, (A_j - A_i) X_ij 18, 3 sums                        = 47
#         hourglass: u_ij 3, x_ij 3, 1/|x_ij|^2 4, error vector 21,
#         projection 3, W(q) from the W' terms 5, pair modulus 2,
#         coefficient 5, 3 sums                                           = 49
# (an integer-to-float conversion of a position difference counts as one)
MIXED_FP32_OPS_PER_PAIR = {"pass1": 37, "pass2": 47, "pass2_hourglass": 49}


def mixed_fp32_ops(nnz: int, hourglass: bool = True):
    """Algorithmic FP32 operations per step of (pass 1, pass 2)."""
    o = MIXED_FP32_OPS_PER_PAIR
    return o["pass1"] * nnz, (o["pass2"] + (o["pass2_hourglass"] if hourglass else 0)) * nnz


# FP32 issue peak of one GB300: 152 SMs x 128 FP32 lanes x clock (Hz)
FP32_LANES = 152 * 128


def fma_peak(fp64: bool = False, iters: int = 4096) -> float:
    """Measured FMA rate (FMAs per second) of the current device."""
    v = ctypes.c_double()
    _check(load().tlsph_fma_peak(1 if fp64 else 0, int(iters), ctypes.byref(v)))
    return v.value


FLAG_SPATIAL_ORDER = 1
FLAG_WALL = 2
FLAG_LINE_ORDER = 4
FLAG_AUTO_ORDER = 8


def make_config(h, rc, dt, hg_alpha, precision="fp64", flags=0) -> Config:
    return Config(float(h), float(rc), float(dt), float(hg_alpha), PRECISION[precision], int(flags))


def workspace_bytes(cfg: Config, N: int, nnz_cap: int) -> int:
    return int(load().tlsph_workspace_bytes(ctypes.byref(cfg), int(N), int(nnz_cap)))


def _host(a, dtype, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Simulation:
    """One specimen resident on the GPU, advanced by the library's step.

    X, vol, mat_id, bc_mask, bc_vel, f0: host arrays (see tlsph_create).
    materials: list of material dicts (index = material id).
    arena: optional torch.uint8 CUDA tensor the library carves (with
    nnz_cap); otherwise the library owns its memory.
    stream: torch.cuda.Stream or raw handle; default the current stream.
    spatial_order / line_order: internal particle order (TLSPH_FLAG_SPATIAL_ORDER
    / TLSPH_FLAG_LINE_ORDER); line_order=False keeps the caller's order, and
    the default (None) lets a mixed-precision context choose between the two
    (TLSPH_FLAG_AUTO_ORDER).
    wall: the rigid wall on z = 0 (TLSPH_FLAG_WALL)."""

    def __init__(self, X, vol, mat_id, bc_mask, bc_vel, f0, materials, h, rc, dt, hg_alpha,
                 precision="fp64", arena=None, nnz_cap=0, stream=None, spatial_order=False, wall=False,
                 line_order=None):
        L = load()
        X = _host(X, np.float64)
        self.N = N = X.shape[0]
        X = X.reshape(N, 3)
        vol = _host(vol, np.float64)
        mat_id = _host(mat_id, np.int32)
        bc_mask = _host(bc_mask, np.uint8)
        bc_vel = _host(bc_vel, np.float64, (N, 3))
        f0 = _host(f0, np.float64)
        if line_order is None:
            order = FLAG_AUTO_ORDER if precision == "mixed" and not spatial_order else 0
        else:
            order = FLAG_LINE_ORDER if line_order else 0
        self.cfg = make_config(h, rc, dt, hg_alpha, precision,
                               (FLAG_SPATIAL_ORDER if spatial_order else 0) | (FLAG_WALL if wall else 0) | order)
        self.precision = precision
        self.arena = arena
        self.stream = _stream_handle(stream)
        ctx = ctypes.c_void_p()
        if arena is not None:
            aptr, abytes = ctypes.c_void_p(arena.data_ptr()), arena.numel() * arena.element_size()
        else:
            aptr, abytes = None, 0
        code = L.tlsph_create(ctypes.byref(self.cfg), N, _ptr(X), _ptr(vol), _ptr(mat_id), _ptr(bc_mask),
                              _ptr(bc_vel), _ptr(f0), aptr, abytes, int(nnz_cap), ctypes.c_void_p(self.stream),
                              ctypes.byref(ctx))
        _check(code, None)
        self.ctx = ctx
        self._mats = []
        for k, m in enumerate(materials):
            mm = make_material(m)
            self._mats.append(mm)
            _check(L.tlsph_set_material(self.ctx, k, ctypes.byref(mm)), self.ctx)

    @classmethod
    def from_workload(cls, w, precision="fp64", **kw):
        sp = w.specimen
        kw.setdefault("wall", getattr(w, "wall", False))
        sim = cls(sp.X, sp.vol, sp.mat_id, sp.bc_mask, sp.bc_vel, sp.f0, w.materials, w.h, w.rc, w.dt,
                  w.hg_alpha, precision=precision, **kw)
        if getattr(w, "grip_ramp", 0.0):
            sim.set_grip_ramp(w.grip_ramp)
        return sim

    # ---------------------------------------------------------------- stepping
    def step(self, n: int = 1) -> None:
        _check(load().tlsph_step(self.ctx, int(n)), self.ctx)

    def sync(self) -> None:
        _check(load().tlsph_sync(self.ctx), self.ctx)

    def status_bits(self) -> int:
        b = ctypes.c_uint32(0)
        _check(load().tlsph_status_bits(self.ctx, ctypes.byref(b)), self.ctx)
        return int(b.value)

    def profile(self, enable: bool = True) -> None:
        _check(load().tlsph_profile_enable(self.ctx, 1 if enable else 0), self.ctx)

    def profile_read(self):
        """(ms of pass 1, ms of pass 2, profiled steps)."""
        ms = (ctypes.c_double * 2)()
        n = ctypes.c_int64()
        _check(load().tlsph_profile_read(self.ctx, ms, 2, ctypes.byref(n)), self.ctx)
        return ms[0], ms[1], n.value

    def set_plan(self, plan) -> None:
        """Mixed-path launch plan (pass-1 form, block, pass-2 form, block)."""
        a = (ctypes.c_int32 * 4)(*[int(x) for x in plan])
        _check(load().tlsph_set_plan(self.ctx, a, 4), self.ctx)

    def get_plan(self):
        a = (ctypes.c_int32 * 4)()
        _check(load().tlsph_get_plan(self.ctx, a, 4), self.ctx)
        return tuple(a)

    def info(self):
        N, nnz, steps = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().tlsph_info(self.ctx, ctypes.byref(N), ctypes.byref(nnz), ctypes.byref(steps)), self.ctx)
        return N.value, nnz.value, steps.value

    def diagnostics(self) -> dict:
        """Momentum, force sum, kinetic energy, failed count, largest D and
        plastic strain, and internal energy of the current state
        (tlsph_diagnostics)."""
        out = (ctypes.c_double * DIAG_COUNT)()
        _check(load().tlsph_diagnostics(self.ctx, out, DIAG_COUNT), self.ctx)
        return diagnostics_dict(out)

    def diagnostics_async(self, out) -> None:
        """Queue the diagnostics of the state after the steps queued so far
        into `out`, a page-locked float64 CPU tensor of DIAG_COUNT elements,
        without waiting (tlsph_diagnostics_async); read it with
        diagnostics_dict(out) once the stream has passed the call."""
        import torch
        _check_tensor("out", out, torch.float64, min_numel=DIAG_COUNT, ndim=1)
        if out.is_cuda or not out.is_pinned():
            raise ValueError("out must be a page-locked (pinned) CPU tensor")
        _check(load().tlsph_diagnostics_async(self.ctx, ctypes.cast(out.data_ptr(), ctypes.POINTER(ctypes.c_double)),
                                              DIAG_COUNT), self.ctx)

    def set_guard(self, band: float) -> None:
        """Guard band of the mixed path's FP32 elastic screen (tlsph_set_guard)."""
        _check(load().tlsph_set_guard(self.ctx, float(band)), self.ctx)

    def set_grip_ramp(self, tau: float) -> None:
        """Prescribed velocities ramp up as bc_vel (1 - exp(-t / tau)) (Sec. 6
        grip loading; tlsph_set_grip_ramp); 0 keeps them constant."""
        _check(load().tlsph_set_grip_ramp(self.ctx, float(tau)), self.ctx)

    def neighbor_layout(self) -> dict:
        """Form of the sliced neighbour lists of a mixed-precision context:
        slices, aligned slices, slots and 4-byte words."""
        v = [ctypes.c_int64() for _ in range(4)]
        _check(load().tlsph_neighbor_layout(self.ctx, *[ctypes.byref(x) for x in v]), self.ctx)
        return dict(zip(("slices", "aligned_slices", "slots", "words"), (x.value for x in v)))

    @property
    def nnz(self) -> int:
        return self.info()[1]

    @property
    def steps(self) -> int:
        return self.info()[2]

    # ---------------------------------------------------------------- state
    def _shape(self, name):
        dt, w = _FIELD_SHAPE[name]
        if name == "NBR_ROWPTR":
            return dt, (self.N + 1,)
        if name == "NBR_COL":
            return dt, (self.nnz,)
        if name == "STEP":
            return dt, (1,)
        return dt, ((self.N,) if w == 1 else (self.N, w))

    def get(self, name: str) -> np.ndarray:
        """Copy a field to a new host array."""
        dt, shape = self._shape(name)
        out = np.empty(shape, dt)
        _check(load().tlsph_get_state(self.ctx, FIELD[name], _ptr(out), out.nbytes, 0), self.ctx)
        return out

    def get_device(self, name: str, out=None):
        """Copy a field into a torch CUDA tensor (device to device)."""
        import torch
        dt, shape = self._shape(name)
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dt]
        if out is None:
            out = torch.empty(shape, dtype=tdt, device="cuda")
        _check(load().tlsph_get_state(self.ctx, FIELD[name], ctypes.c_void_p(out.data_ptr()),
                                      out.numel() * out.element_size(), 1), self.ctx)
        return out

    def set(self, name: str, value) -> None:
        dt, shape = self._shape(name)
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(value, dt), shape))
        _check(load().tlsph_set_state(self.ctx, FIELD[name], _ptr(a), a.nbytes, 0), self.ctx)

    def checkpoint(self, device: bool = True) -> dict:
        """Every resumable field (torch CUDA tensors if device, else numpy)."""
        if device:
            return {k: (self.get_device(k) if k != "STEP" else self.get("STEP")) for k in CHECKPOINT_FIELDS}
        return {k: self.get(k) for k in CHECKPOINT_FIELDS}

    def restore(self, ck: dict) -> None:
        """Load a checkpoint taken by checkpoint() (same particle count)."""
        L = load()
        for k, v in ck.items():
            if hasattr(v, "data_ptr"):
                _check(L.tlsph_set_state(self.ctx, FIELD[k], ctypes.c_void_p(v.data_ptr()),
                                         v.numel() * v.element_size(), 1), self.ctx)
            else:
                self.set(k, v)

    def state(self) -> dict:
        names = ("U", "V", "F", "SIGMA", "STRESS_DEV", "EPSP", "EPSP_RATE", "DINIT", "DAMAGE", "POROSITY",
                 "ENERGY", "FAIL_STEP", "FORCE", "A")
        return {k: self.get(k) for k in names}

    def close(self) -> None:
        if getattr(self, "ctx", None):
            load().tlsph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _check_tensor(name, t, dtype, shape=None, min_numel=None, ndim=None):
    """Validate the form of a torch tensor whose data pointer crosses the ABI:
    dtype, shape, contiguity.  Raises ValueError."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must be {ndim}-dimensional, got {t.dim()} dimensions")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name} needs at least {min_numel} elements, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _check_device(**tensors):
    """Every tensor is a CUDA tensor, all on one device.  Raises ValueError."""
    dev = None
    for name, t in tensors.items():
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if dev is not None and t.device != dev:
            raise ValueError(f"{name} is on {t.device}, the other arguments on {dev}")
        dev = t.device


def material_point_batch(mat: dict, dt: float, deps, J, state, stream=None) -> None:
    """Constitutive update of n material points on the GPU (torch CUDA float64
    tensors: deps (n, 9), J (n,), state (n, 16) updated in place)."""
    import torch
    n = int(J.numel())
    _check_tensor("J", J, torch.float64, shape=(n,))
    _check_tensor("deps", deps, torch.float64, shape=(n, 9))
    _check_tensor("state", state, torch.float64, shape=(n, 16))
    _check_device(J=J, deps=deps, state=state)
    L = load()
    m = make_material(mat)
    code = L.tlsph_material_point_batch(ctypes.byref(m), float(dt), n, ctypes.c_void_p(deps.data_ptr()),
                                        ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(state.data_ptr()),
                                        ctypes.c_void_p(_stream_handle(stream)))
    _check(code, None)


def neighbors_noalloc(X, rc: float, row_ptr, col, stream=None) -> int:
    """tlsph_neighbors_noalloc on torch CUDA tensors: X (N, 3) float64,
    row_ptr (N + 1,) int64, col (capacity,) int32.  Returns the pair count;
    raises TlsphError (code -4) when col is too small, ValueError before any
    launch when a tensor has the wrong dtype, shape, layout or device."""
    import torch
    if not isinstance(X, torch.Tensor) or X.dim() != 2:
        raise ValueError("X must be a torch tensor of shape (N, 3)")
    N = int(X.shape[0])
    _check_tensor("X", X, torch.float64, shape=(N, 3))
    _check_tensor("row_ptr", row_ptr, torch.int64, min_numel=N + 1, ndim=1)
    if col is not None:
        _check_tensor("col", col, torch.int32, ndim=1)
    _check_device(X=X, row_ptr=row_ptr, col=col)
    L = load()
    fn = L.tlsph_neighbors_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    nnz = ctypes.c_int64(0)
    cap = int(col.numel()) if col is not None else 0
    code = fn(ctypes.c_void_p(X.data_ptr()), int(X.shape[0]), float(rc), ctypes.c_void_p(row_ptr.data_ptr()),
              ctypes.c_void_p(col.data_ptr()) if col is not None else None, cap, ctypes.byref(nnz),
              ctypes.c_void_p(_stream_handle(stream)))
    if code != 0:
        err = TlsphError(code, L.tlsph_last_error(None).decode(errors="replace"))
        err.nnz = nnz.value
        raise err
    return nnz.value


class Batch:
    """Many mixed-precision Simulations advanced together (tlsph_batch_*):
    one persistent launch per kernel kind and step over all members, replayed
    from a CUDA graph when graph=True.  Members can change between steps."""

    def __init__(self, capacity: int, stream=None):
        L = load()
        self.stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        code = L.tlsph_batch_create(int(capacity), ctypes.c_void_p(self.stream), ctypes.byref(h))
        if code != 0:
            raise TlsphError(code, "tlsph_batch_create failed")
        self.h = h
        self.members = []

    def _check(self, code):
        if code != 0:
            raise TlsphError(code, load().tlsph_batch_last_error(self.h).decode(errors="replace"))

    def set(self, sims) -> None:
        sims = list(sims)
        arr = (ctypes.c_void_p * max(1, len(sims)))(*[s.ctx.value for s in sims])
        self._check(load().tlsph_batch_set(self.h, arr, len(sims)))
        self.members = sims

    def step(self, n: int = 1, graph: bool = True) -> None:
        self._check(load().tlsph_batch_step(self.h, int(n), 1 if graph else 0))

    def set_shape(self, shape) -> None:
        """Launch-shape variant of each batch kernel kind (tlsph_batch_set_shape)."""
        arr = (ctypes.c_int32 * 3)(*[int(x) for x in shape])
        self._check(load().tlsph_batch_set_shape(self.h, arr, 3))

    def get_shape(self):
        """(current variant per kernel kind, number of variants per kind)."""
        cur, nv = (ctypes.c_int32 * 3)(), (ctypes.c_int32 * 3)()
        self._check(load().tlsph_batch_get_shape(self.h, cur, nv, 3))
        return tuple(cur), tuple(nv)

    def sync(self) -> None:
        self._check(load().tlsph_batch_sync(self.h))

    def close(self) -> None:
        if getattr(self, "h", None):
            load().tlsph_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
