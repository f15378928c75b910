"""FP64 CPU oracle of the damage-weighted TLSPH step (arXiv 1901.07374).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference the CUDA
library is checked against.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library (``paper_1901_07374_gb300``) and never imports it; the only
common input is the seeded specimen generator, which holds no method
arithmetic.

The arithmetic lives in ``tlsph_oracle.c`` (plain C, FP64, compiled with
``-O2 -ffp-contract=off``); this module builds it with gcc and wraps it with
ctypes.  Every C function cites the paper passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tlsph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

ST_POLAR_CAP, ST_NEWTON_CAP, ST_BAD_J, ST_NONFINITE = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                        "-Wall", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


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


class Config(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("rc", ctypes.c_double), ("dt", ctypes.c_double),
                ("hg_alpha", ctypes.c_double), ("wall", ctypes.c_int32), ("grip_ramp", ctypes.c_double)]


_P = ctypes.POINTER
_d = _P(ctypes.c_double)


class System(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64),
                ("X", _d), ("vol", _d), ("mat_id", _P(ctypes.c_int32)),
                ("bc_mask", _P(ctypes.c_uint8)), ("bc_vel", _d),
                ("row_ptr", _P(ctypes.c_int64)), ("col", _P(ctypes.c_int32)), ("Linv", _d),
                ("mats", _P(Material)),
                ("u", _d), ("v", _d), ("F", _d), ("sd", _d), ("sigma", _d), ("A", _d),
                ("ep", _d), ("epdot", _d), ("dinit", _d), ("D", _d), ("f", _d), ("e", _d),
                ("force", _d), ("fail_step", _P(ctypes.c_int32)),
                ("step", ctypes.c_int64), ("status", ctypes.c_uint32),
                ("vh", _d), ("Fdot", _d)]


def lib():
    """The loaded oracle library (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            L.orc_kernel_w.restype = ctypes.c_double
            L.orc_kernel_w.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_kernel_dw.restype = ctypes.c_double
            L.orc_kernel_dw.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_neighbors.restype = ctypes.c_int64
            L.orc_neighbors.argtypes = [ctypes.c_int64, vp, ctypes.c_double, vp, vp, ctypes.c_int64]
            L.orc_shape_matrix.restype = ctypes.c_int64
            L.orc_shape_matrix.argtypes = [ctypes.c_int64, vp, vp, vp, vp, ctypes.c_double, vp, vp]
            L.orc_velocity_gradient.restype = None
            L.orc_velocity_gradient.argtypes = [ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp,
                                                ctypes.c_double, vp]
            L.orc_polar.restype = ctypes.c_int
            L.orc_polar.argtypes = [vp, vp, vp]
            L.orc_eig_sym.restype = None
            L.orc_eig_sym.argtypes = [vp, vp]
            L.orc_eos_mean_stress.restype = ctypes.c_double
            L.orc_eos_mean_stress.argtypes = [_P(Material), ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.orc_flow_stress.restype = ctypes.c_double
            L.orc_flow_stress.argtypes = [_P(Material), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double]
            L.orc_gtn_fstar.restype = ctypes.c_double
            L.orc_gtn_fstar.argtypes = [_P(Material), ctypes.c_double]
            L.orc_gtn_omega.restype = ctypes.c_double
            L.orc_gtn_omega.argtypes = [vp, ctypes.c_double, ctypes.c_double]
            L.orc_gtn_solve_x.restype = ctypes.c_double
            L.orc_gtn_solve_x.argtypes = [_P(Material), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _P(ctypes.c_int32)]
            L.orc_gtn_phi.restype = ctypes.c_double
            L.orc_gtn_phi.argtypes = [_P(Material), ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double]
            L.orc_material_point.restype = ctypes.c_uint
            L.orc_material_point.argtypes = [_P(Material), ctypes.c_double, ctypes.c_int64, vp, vp,
                                             vp, vp]
            L.orc_forces.restype = None
            L.orc_forces.argtypes = [_P(System), _P(Config)]
            L.orc_step.restype = None
            L.orc_step.argtypes = [_P(System), _P(Config), ctypes.c_int64]
            for name in ("orc_step_predict", "orc_step_pass1", "orc_step_pass2"):
                getattr(L, name).restype = None
                getattr(L, name).argtypes = [_P(System), _P(Config)]
            L.orc_init_state.restype = None
            L.orc_init_state.argtypes = [_P(System)]
            L.orc_apply_grip_ramp.restype = None
            L.orc_apply_grip_ramp.argtypes = [_P(System), _P(Config)]
            L.orc_mat_det.restype = ctypes.c_double
            L.orc_mat_det.argtypes = [vp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_material(d: dict) -> Material:
    """ctypes material from a specimen-module material dict."""
    m = Material()
    for name, _ in Material._fields_:
        setattr(m, name, d[name])
    return m


# ---------------------------------------------------------------- primitives

def kernel_w(r: float, h: float) -> float:
    return lib().orc_kernel_w(float(r), float(h))


def kernel_dw(r: float, h: float) -> float:
    return lib().orc_kernel_dw(float(r), float(h))


def neighbors(X: np.ndarray, rc: float) -> tuple[np.ndarray, np.ndarray]:
    """Brute-force neighbour CSR (row_ptr int64, col int32, rows ascending)."""
    X = np.ascontiguousarray(X, np.float64)
    N = X.shape[0]
    row_ptr = np.zeros(N + 1, np.int64)
    cap = max(1, 128 * N)
    col = np.zeros(cap, np.int32)
    nnz = lib().orc_neighbors(N, _ptr(X), float(rc), _ptr(row_ptr), _ptr(col), cap)
    if nnz > cap:
        col = np.zeros(nnz, np.int32)
        lib().orc_neighbors(N, _ptr(X), float(rc), _ptr(row_ptr), _ptr(col), nnz)
    return row_ptr, col[:nnz].copy()


def shape_matrix(X, vol, row_ptr, col, h):
    """Correction matrices L_i and their inverses; returns (L, Linv, n_singular)."""
    X = np.ascontiguousarray(X, np.float64)
    vol = np.ascontiguousarray(vol, np.float64)
    N = X.shape[0]
    L = np.zeros((N, 9))
    Linv = np.zeros((N, 9))
    bad = lib().orc_shape_matrix(N, _ptr(X), _ptr(vol), _ptr(row_ptr), _ptr(col), float(h),
                                 _ptr(L), _ptr(Linv))
    return L, Linv, int(bad)


def velocity_gradient(X, vol, v, D, Linv, row_ptr, col, h):
    """Damage-weighted Fdot of every particle (N, 9)."""
    N = X.shape[0]
    out = np.zeros((N, 9))
    args = [np.ascontiguousarray(a, np.float64) for a in (X, vol, v, D, Linv)]
    lib().orc_velocity_gradient(N, *[_ptr(a) for a in args], _ptr(row_ptr), _ptr(col), float(h),
                                _ptr(out))
    return out


def polar(F: np.ndarray):
    """Polar decomposition F = R U; returns (R, U, converged)."""
    F = np.ascontiguousarray(F, np.float64).reshape(9)
    R = np.zeros(9)
    U = np.zeros(9)
    rc = lib().orc_polar(_ptr(F), _ptr(R), _ptr(U))
    return R.reshape(3, 3), U.reshape(3, 3), rc == 0


def eig_sym(S: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, np.float64).reshape(9)
    ev = np.zeros(3)
    lib().orc_eig_sym(_ptr(S), _ptr(ev))
    return ev


def eos_mean_stress(mat: dict, J: float, D: float = 0.0, e: float = 0.0) -> float:
    """Tension-positive mean stress of Eq. pH at J = det F, damage D and
    specific internal energy e."""
    m = make_material(mat)
    return lib().orc_eos_mean_stress(ctypes.byref(m), float(J), float(D), float(e))


def flow_stress(mat: dict, ep: float, epdot: float = 0.0, D: float = 0.0) -> float:
    m = make_material(mat)
    return lib().orc_flow_stress(ctypes.byref(m), float(ep), float(epdot), float(D))


def gtn_fstar(mat: dict, f: float) -> float:
    m = make_material(mat)
    return lib().orc_gtn_fstar(ctypes.byref(m), float(f))


def gtn_omega(s: np.ndarray, seq: float, K: float) -> float:
    s = np.ascontiguousarray(s, np.float64).reshape(9)
    return lib().orc_gtn_omega(_ptr(s), float(seq), float(K))


def gtn_solve_x(mat: dict, fstar: float, tri: float, x0: float = 1.0):
    m = make_material(mat)
    its = ctypes.c_int32(0)
    x = lib().orc_gtn_solve_x(ctypes.byref(m), float(fstar), float(tri), float(x0), ctypes.byref(its))
    return x, its.value


def gtn_phi(mat: dict, fstar: float, tri: float, x: float) -> float:
    m = make_material(mat)
    return lib().orc_gtn_phi(ctypes.byref(m), float(fstar), float(tri), float(x))


MP_FIELDS = ("sd", "sm", "ep", "epdot", "dinit", "D", "f", "failed")


def material_point(mat: dict, dt: float, deps: np.ndarray, J: np.ndarray, init: dict | None = None):
    """Drive one material point through n strain increments (n, 3, 3) with the
    given J per increment.  Returns (out (n, 16), status): columns 0-8 the
    unrotated deviator, then sm, ep, epdot, dinit, D, f, failed."""
    deps = np.ascontiguousarray(deps, np.float64).reshape(-1, 9)
    n = deps.shape[0]
    J = np.ascontiguousarray(np.broadcast_to(np.asarray(J, np.float64), (n,)))
    st = np.zeros(16)
    init = init or {}
    if "sd" in init:
        st[:9] = np.asarray(init["sd"], np.float64).reshape(9)
    for k, name in enumerate(MP_FIELDS[1:], start=9):
        if name in init:
            st[k] = float(init[name])
    out = np.zeros((n, 16))
    m = make_material(mat)
    status = lib().orc_material_point(ctypes.byref(m), float(dt), n, _ptr(deps), _ptr(J), _ptr(st),
                                      _ptr(out))
    return out, int(status)


def mat_det(a: np.ndarray) -> float:
    return lib().orc_mat_det(_ptr(np.ascontiguousarray(a, np.float64).reshape(9)))


# ---------------------------------------------------------------- full system

STATE_FIELDS = {"u": 3, "v": 3, "F": 9, "sd": 9, "sigma": 9, "A": 9, "ep": 1, "epdot": 1,
                "dinit": 1, "D": 1, "f": 1, "e": 1, "force": 3}


class Simulation:
    """A whole specimen advanced by the oracle's velocity-Verlet step.

    Inputs are copied; neighbours are found by brute force and the correction
    matrices computed on construction (Sec. 2.2: both fixed for the run)."""

    def __init__(self, X, vol, mat_id, bc_mask, bc_vel, f0, materials, h, rc, dt, hg_alpha,
                 neighbors_csr=None, wall=False, grip_ramp=0.0):
        self.N = N = int(np.asarray(X).shape[0])
        self.X = np.ascontiguousarray(X, np.float64).reshape(N, 3).copy()
        self.vol = np.ascontiguousarray(vol, np.float64).copy()
        self.mat_id = np.ascontiguousarray(mat_id, np.int32).copy()
        self.bc_mask = np.ascontiguousarray(bc_mask, np.uint8).copy()
        self.bc_vel = np.ascontiguousarray(bc_vel, np.float64).reshape(N, 3).copy()
        if not (grip_ramp >= 0.0 and np.isfinite(grip_ramp)):
            raise ValueError("grip_ramp must be finite and >= 0")
        self.cfg = Config(float(h), float(rc), float(dt), float(hg_alpha), 1 if wall else 0, float(grip_ramp))
        mats = [make_material(m) for m in materials]
        self._mats = (Material * len(mats))(*mats)
        if neighbors_csr is None:
            self.row_ptr, self.col = neighbors(self.X, rc)
        else:
            self.row_ptr = np.ascontiguousarray(neighbors_csr[0], np.int64).copy()
            self.col = np.ascontiguousarray(neighbors_csr[1], np.int32).copy()
        self.L, self.Linv, self.n_singular = shape_matrix(self.X, self.vol, self.row_ptr, self.col, h)
        self.arr = {k: np.zeros((N, w)) if w > 1 else np.zeros(N) for k, w in STATE_FIELDS.items()}
        self.arr["f"][:] = np.asarray(f0, np.float64)
        self.fail_step = np.full(N, -1, np.int32)
        self._vh = np.zeros((N, 3))
        self._Fdot = np.zeros((N, 9))
        s = System()
        s.N = N
        for name in ("X", "vol", "bc_vel", "Linv"):
            setattr(s, name, getattr(self, name).ctypes.data_as(_d))
        s.mat_id = self.mat_id.ctypes.data_as(_P(ctypes.c_int32))
        s.bc_mask = self.bc_mask.ctypes.data_as(_P(ctypes.c_uint8))
        s.row_ptr = self.row_ptr.ctypes.data_as(_P(ctypes.c_int64))
        s.col = self.col.ctypes.data_as(_P(ctypes.c_int32))
        s.mats = ctypes.cast(self._mats, _P(Material))
        for k in STATE_FIELDS:
            setattr(s, k, self.arr[k].ctypes.data_as(_d))
        s.fail_step = self.fail_step.ctypes.data_as(_P(ctypes.c_int32))
        s.vh = self._vh.ctypes.data_as(_d)
        s.Fdot = self._Fdot.ctypes.data_as(_d)
        self.sys = s
        lib().orc_init_state(ctypes.byref(self.sys))
        if grip_ramp > 0.0:
            lib().orc_apply_grip_ramp(ctypes.byref(self.sys), ctypes.byref(self.cfg))

    @classmethod
    def from_workload(cls, w, **kw):
        sp = w.specimen
        kw.setdefault("wall", getattr(w, "wall", False))
        kw.setdefault("grip_ramp", getattr(w, "grip_ramp", 0.0))
        return cls(sp.X, sp.vol, sp.mat_id, sp.bc_mask, sp.bc_vel, sp.f0, w.materials,
                   w.h, w.rc, w.dt, w.hg_alpha, **kw)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def step_count(self) -> int:
        return int(self.sys.step)

    @property
    def status(self) -> int:
        return int(self.sys.status)

    def step(self, n: int = 1) -> None:
        lib().orc_step(ctypes.byref(self.sys), ctypes.byref(self.cfg), int(n))

    def step_phase(self, phase: str) -> None:
        """One phase of a step: "predict" (half kick, drift, constraints),
        "pass1" (velocity gradients and the per-particle update) or "pass2"
        (forces and the second half kick); the three in order are one step."""
        fn = {"predict": lib().orc_step_predict, "pass1": lib().orc_step_pass1, "pass2": lib().orc_step_pass2}[phase]
        fn(ctypes.byref(self.sys), ctypes.byref(self.cfg))

    @property
    def vh(self) -> np.ndarray:
        """The half-step velocity v^{n+1/2} (N x 3, live view)."""
        return self._vh

    def forces(self) -> np.ndarray:
        """Recompute the nodal forces from the current A, D, F, u (no step)."""
        lib().orc_forces(ctypes.byref(self.sys), ctypes.byref(self.cfg))
        return self.arr["force"].copy()

    def __getitem__(self, name):
        if name == "fail_step":
            return self.fail_step
        return self.arr[name]

    def state(self) -> dict:
        out = {k: v.copy() for k, v in self.arr.items()}
        out["fail_step"] = self.fail_step.copy()
        return out
