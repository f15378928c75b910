"""Seeded synthetic specimens and the workload configurations.

This module only makes INPUTS: reference positions, particle volumes,
material ids, velocity-constraint masks, initial porosity and the material and
time-step parameters of each workload.  It holds none of the TLSPH method's
arithmetic, so both the CUDA library and the CPU oracle can be fed from it.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state_k = seed + k * golden,
then the published three-step mixer.  A uniform double is the top 53 bits.

Geometry follows the paper's specimens (Sec. 6: simple cubic particle arrays,
top and bottom rows pulled at +-v along the specimen axis) with the sizes of
the tensile-bar, notched-bar, batched and served workloads.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n consecutive splitmix64 outputs of the sequence seeded by (seed, stream)."""
    base = np.uint64((int(seed) * 0x100000001B3 + int(stream) * 0xC2B2AE3D27D4EB4F) & ((1 << 64) - 1))
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = base + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from the top 53 bits of splitmix64."""
    z = splitmix64(seed, n, stream)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class Specimen:
    """Inputs of one simulation (all float64 / int32 / uint8, row-major)."""

    name: str
    X: np.ndarray          # (N, 3) reference positions [m]
    vol: np.ndarray        # (N,) reference volumes [m^3]
    mat_id: np.ndarray     # (N,) int32 material index
    bc_mask: np.ndarray    # (N,) uint8, 1 = prescribed velocity
    bc_vel: np.ndarray     # (N, 3) prescribed velocity [m/s]
    f0: np.ndarray         # (N,) initial void fraction (GTN), zeros otherwise
    spacing: float         # lattice spacing [m]
    dims: tuple = ()       # lattice dimensions when the specimen is a full box

    @property
    def N(self) -> int:
        return int(self.X.shape[0])


def lattice_box(nx: int, ny: int, nz: int, spacing: float) -> tuple[np.ndarray, np.ndarray]:
    """Simple cubic lattice, x fastest; returns positions and (ix, iy, iz)."""
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
    return idx.astype(np.float64) * spacing, idx


def tensile_bar(nx: int, ny: int, nz: int, spacing: float, jitter: float = 0.01, seed: int = 0,
                grip_layers: int = 2, v_grip: float = 1.0, name: str = "tensile_bar") -> Specimen:
    """Bar along z on a jittered simple cubic lattice (uniform +-jitter*spacing
    per coordinate from the seed); the bottom and top `grip_layers` layers are
    pulled apart at -v_grip / +v_grip along z."""
    X, idx = lattice_box(nx, ny, nz, spacing)
    N = X.shape[0]
    if jitter:
        X = X + (2.0 * uniform(seed, 3 * N, stream=1).reshape(N, 3) - 1.0) * (jitter * spacing)
    bc_mask = np.zeros(N, np.uint8)
    bc_vel = np.zeros((N, 3))
    bot = idx[:, 2] < grip_layers
    top = idx[:, 2] >= nz - grip_layers
    bc_mask[bot | top] = 1
    bc_vel[bot, 2] = -v_grip
    bc_vel[top, 2] = v_grip
    return Specimen(name, np.ascontiguousarray(X), np.full(N, spacing ** 3), np.zeros(N, np.int32),
                    bc_mask, bc_vel, np.zeros(N), spacing, (nx, ny, nz))


def notched_round_bar(radius: float, height: float, spacing: float, notch_radius: float,
                      seed: int = 0, f0_range=(0.0008, 0.0012), grip_layers: int = 2,
                      v_grip: float = 1.0, name: str = "notched_round_bar") -> Specimen:
    """Round bar along z cut from an exact cubic lattice, with a circumferential
    notch: a torus of radius `notch_radius` centred on the bar surface at
    mid-height is removed.  Initial porosity is uniform in f0_range per
    particle from the seed."""
    n_r = int(math.floor(radius / spacing))
    nz = int(round(height / spacing)) + 1
    n = 2 * n_r + 1
    X, idx = lattice_box(n, n, nz, spacing)
    X[:, 0] -= n_r * spacing
    X[:, 1] -= n_r * spacing
    r = np.hypot(X[:, 0], X[:, 1])
    keep = r <= radius + 1e-9 * spacing
    zc = 0.5 * (nz - 1) * spacing
    dnotch = np.hypot(r - radius, X[:, 2] - zc)
    keep &= dnotch >= notch_radius
    X, idx = X[keep], idx[keep]
    N = X.shape[0]
    bc_mask = np.zeros(N, np.uint8)
    bc_vel = np.zeros((N, 3))
    bot = idx[:, 2] < grip_layers
    top = idx[:, 2] >= nz - grip_layers
    bc_mask[bot | top] = 1
    bc_vel[bot, 2] = -v_grip
    bc_vel[top, 2] = v_grip
    lo, hi = f0_range
    f0 = lo + (hi - lo) * uniform(seed, N, stream=2)
    return Specimen(name, np.ascontiguousarray(X), np.full(N, spacing ** 3), np.zeros(N, np.int32),
                    bc_mask, bc_vel, f0, spacing, ())


def taylor_cylinder(n_particles_target: int, spacing: float, v_impact: float, aspect: float = 3.2,
                    seed: int = 0, name: str = "taylor_cylinder") -> Specimen:
    """Cylinder of length/diameter `aspect` standing on z = 0 and moving at
    -v_impact along z (every particle starts with that velocity; nothing is
    prescribed).  The diameter is chosen so the particle count is close to the
    target."""
    d_over_s = (4.0 * n_particles_target / (math.pi * aspect)) ** (1.0 / 3.0)
    radius = 0.5 * d_over_s * spacing
    length = aspect * 2.0 * radius
    n_r = int(math.floor(radius / spacing))
    nz = max(2, int(round(length / spacing)))
    n = 2 * n_r + 1
    X, idx = lattice_box(n, n, nz, spacing)
    X[:, 0] -= n_r * spacing
    X[:, 1] -= n_r * spacing
    X[:, 2] += 0.5 * spacing
    keep = np.hypot(X[:, 0], X[:, 1]) <= radius
    X = np.ascontiguousarray(X[keep])
    N = X.shape[0]
    bc_vel = np.zeros((N, 3))
    bc_vel[:, 2] = -v_impact
    return Specimen(name, X, np.full(N, spacing ** 3), np.zeros(N, np.int32),
                    np.zeros(N, np.uint8), bc_vel, np.zeros(N), spacing, ())


# --------------------------------------------------------------------------
# Materials (SI units).  Keys follow the paper's symbols.
# --------------------------------------------------------------------------

DAMAGE_NONE, DAMAGE_CL, DAMAGE_JC, DAMAGE_GTN = 0, 1, 2, 3


def material(**kw) -> dict:
    """A material dict with every field present (zeros where unused)."""
    m = dict(rho0=2700.0, E=70e9, nu=0.3, eos=0, c0=0.0, S_alpha=0.0, Gamma0=0.0,
             A=324e6, B=114e6, n=0.42, C=0.0, epsdot0=1.0, damage=DAMAGE_NONE, Wcr=0.0,
             D1=0.0, D2=0.0, D3=0.0, D4=0.0, D5=0.0,
             q1=1.5, q2=1.0, q3=2.25, fN=0.0, eN=0.3, sN=0.1, fc=0.15, fF=0.25, komega=0.0)
    unknown = set(kw) - set(m)
    if unknown:
        raise KeyError(f"unknown material fields {sorted(unknown)}")
    m.update(kw)
    return m


def aluminium_cl(wcr: float = 50e6) -> dict:
    """Tensile-bar material: E 70 GPa, nu 0.3, rho 2700, JC A 324 MPa,
    B 114 MPa, n 0.42, C 0, Cockcroft-Latham critical work `wcr`."""
    return material(damage=DAMAGE_CL, Wcr=wcr)


def aluminium_jc(scale: float = 1.0, C: float = 0.002) -> dict:
    """Johnson-Cook damage D1 = D2 = 0.13, D3 = -1.5, D4 = D5 = 0, rate
    C = 0.002 at reference rate 1/s; `scale` multiplies D1 and D2."""
    return material(damage=DAMAGE_JC, C=C, epsdot0=1.0, D1=0.13 * scale, D2=0.13 * scale,
                    D3=-1.5, D4=0.0, D5=0.0)


def aluminium_gtn() -> dict:
    """GTN porous plasticity: q1 1.5, q2 1, q3 2.25, fN 0.04, eN 0.3, sN 0.1,
    fc 0.15, fF 0.25, k_omega 0; Johnson-Cook hardening with C = 0."""
    return material(damage=DAMAGE_GTN, q1=1.5, q2=1.0, q3=2.25, fN=0.04, eN=0.3, sN=0.1,
                    fc=0.15, fF=0.25, komega=0.0)


def weldox(alloy: str) -> dict:
    """Weldox steels from the paper's Tables 1-3 (Sec. 6): rho0 7750, E 211 GPa,
    nu 0.33, c0 5166 m/s, S_alpha 1.5, Gamma0 0, JC flow and damage constants,
    Cockcroft-Latham W_cr and GTN f_c, f_F, k_omega."""
    tab = {
        "460E": dict(A=499e6, B=382e6, n=0.458, Wcr=1219e6, D1=0.636, D2=1.936, D3=-2.969,
                     D4=-0.0140, D5=1.014, f0=0.0001, fc=0.01, fF=0.2, komega=5.5),
        "700E": dict(A=859e6, B=329e6, n=0.579, Wcr=1424e6, D1=0.361, D2=4.768, D3=-5.107,
                     D4=-0.0013, D5=1.333, f0=0.005, fc=0.25, fF=0.3, komega=3.5),
        "900E": dict(A=992e6, B=364e6, n=0.568, Wcr=1510e6, D1=0.294, D2=5.149, D3=-5.583,
                     D4=0.0023, D5=0.951, f0=0.005, fc=0.18, fF=0.2, komega=3.5),
    }[alloy]
    f0 = tab.pop("f0")
    m = material(rho0=7750.0, E=211e9, nu=0.33, eos=1, c0=5166.0, S_alpha=1.5, Gamma0=0.0,
                 C=0.0, **tab)
    m["_f0"] = f0
    return m


def moduli(m: dict) -> tuple[float, float]:
    """Bulk and shear modulus of an isotropic material from E and nu."""
    K = m["E"] / (3.0 * (1.0 - 2.0 * m["nu"]))
    G = m["E"] / (2.0 * (1.0 + m["nu"]))
    return K, G


def cfl_dt(m: dict, spacing: float, factor: float = 0.3) -> float:
    """Time step: factor * spacing / c_L with the longitudinal wave speed
    c_L = sqrt((K + 4G/3) / rho0)."""
    K, G = moduli(m)
    return factor * spacing / math.sqrt((K + 4.0 * G / 3.0) / m["rho0"])


@dataclasses.dataclass
class Workload:
    """A specimen plus its materials and step parameters."""

    name: str
    specimen: Specimen
    materials: list
    h: float
    rc: float
    dt: float
    hg_alpha: float
    steps: int
    wall: bool = False     # rigid frictionless wall on the plane z = 0
    grip_ramp: float = 0.0  # tau (s): prescribed velocities ramp up as 1 - exp(-t / tau) (Sec. 6); 0: constant

    def sim_params(self) -> dict:
        return dict(h=self.h, rc=self.rc, dt=self.dt, hg_alpha=self.hg_alpha)


HG_ALPHA = 10.0


def _workload(name, sp, mats, steps, hg_alpha=HG_ALPHA):
    h = 1.5 * sp.spacing
    return Workload(name, sp, mats, h, 2.0 * h, cfl_dt(mats[0], sp.spacing), hg_alpha, steps)


def tensile_bar_cl(nx=8, ny=8, nz=32, spacing=0.5e-3, seed=0, v_grip=1.0, wcr=50e6, steps=500,
                   hg_alpha=HG_ALPHA) -> Workload:
    """Cockcroft-Latham tensile bar: 8x8x32 lattice (2048 particles) at 0.5 mm,
    +-1% jitter, h = 1.5 spacing, neighbours within 2h, grips +-1 m/s,
    dt = 0.3 CFL, 500 steps."""
    sp = tensile_bar(nx, ny, nz, spacing, 0.01, seed, 2, v_grip, name="tensile_bar_cl")
    return _workload(f"tensile_bar_cl_{nx}x{ny}x{nz}", sp, [aluminium_cl(wcr)], steps, hg_alpha)


def tensile_bar_jc(nx=40, ny=40, nz=640, spacing=0.5e-3, seed=0, v_grip=1.0, scale=1.0, steps=2000,
                   hg_alpha=HG_ALPHA) -> Workload:
    """Johnson-Cook tensile bar: 40x40x640 lattice (1,024,000 particles) at
    0.5 mm with JC damage D1 = D2 = 0.13, D3 = -1.5, C = 0.002; 2000 steps."""
    sp = tensile_bar(nx, ny, nz, spacing, 0.01, seed, 2, v_grip, name="tensile_bar_jc")
    return _workload(f"tensile_bar_jc_{nx}x{ny}x{nz}", sp, [aluminium_jc(scale)], steps, hg_alpha)


def notched_bar_gtn(radius=5e-3, height=20e-3, spacing=0.15e-3, notch_radius=1e-3, seed=0,
                    v_grip=1.0, steps=3000, hg_alpha=HG_ALPHA) -> Workload:
    """GTN circumferentially notched round bar: radius 5 mm, notch radius 1 mm,
    height 20 mm, exact lattice at 0.15 mm (about 4.5e5 particles), f0 uniform
    in [0.0008, 0.0012]; 3000 steps."""
    sp = notched_round_bar(radius, height, spacing, notch_radius, seed, v_grip=v_grip)
    return _workload("notched_bar_gtn", sp, [aluminium_gtn()], steps, hg_alpha)


def paper_loading(w: Workload, v_max: float = 10.0, tau: float = 1e-3) -> Workload:
    """The grip loading of the paper's tensile simulations (Sec. 6): the end
    layers move apart at +-v_max (1 - exp(-t / tau)) along the bar axis, with
    v_max = 10 mm/ms and t in ms, i.e. tau = 1 ms."""
    sp = dataclasses.replace(w.specimen)
    sp.bc_vel = np.where(sp.bc_vel > 0, v_max, np.where(sp.bc_vel < 0, -v_max, 0.0))
    return dataclasses.replace(w, specimen=sp, grip_ramp=tau, name=w.name + "_ramp")


def failure_variant(w: Workload, v_grip: float = 20.0, scale: float = 0.02) -> Workload:
    """The failure-exercising variant of a tensile workload: grips at
    +-v_grip and the damage thresholds (W_cr, D1, D2) scaled by `scale`."""
    sp = dataclasses.replace(w.specimen)
    sp.bc_vel = np.sign(sp.bc_vel) * v_grip
    mats = []
    for m in w.materials:
        m = dict(m)
        m["Wcr"] *= scale
        m["D1"] *= scale
        m["D2"] *= scale
        mats.append(m)
    return dataclasses.replace(w, name=w.name + "_failure", specimen=sp, materials=mats)


def plastic_flow_state(w: Workload, strain: float = 0.01) -> dict:
    """A starting state in which every particle of a bar pulled along z by
    its grips (tensile or notched round bar) flows plastically: an affine isochoric stretch F = diag(1 - e/2, 1 - e/2, 1 + e)
    about the bar's centroid, the matching affine velocity field of the grip
    rate (strain rate 2 v_grip / length), and an uniaxial unrotated stress
    deviator diag(-1, -1, 2) A / 3 whose von Mises value is the yield stress A
    of the first material.  Returned as caller-order fields (U, V, F,
    STRESS_DEV; tensors as 9 row-major components per particle) to load
    with set_state before stepping."""
    sp = w.specimen
    X = sp.X
    c = X.mean(axis=0)
    length = float(X[:, 2].max() - X[:, 2].min())
    vz = float(np.abs(sp.bc_vel[:, 2]).max())
    rate = 2.0 * vz / length if length > 0 else 0.0
    shape = np.array([-0.5, -0.5, 1.0])
    N = sp.N
    F = np.zeros((N, 3, 3))
    F[:, [0, 1, 2], [0, 1, 2]] = 1.0 + strain * shape
    U = (X - c) * (strain * shape)
    V = (X - c) * (rate * shape)
    bc = sp.bc_mask.astype(bool)
    V[bc] = sp.bc_vel[bc]
    A = float(w.materials[0]["A"])
    S = np.zeros((N, 3, 3))
    S[:, [0, 1, 2], [0, 1, 2]] = np.array([-1.0, -1.0, 2.0]) * (A / 3.0)
    return {"U": U, "V": V, "F": F.reshape(N, 9), "STRESS_DEV": S.reshape(N, 9)}


def taylor_impact(n_particles: int = 12000, spacing: float = 0.5e-3, v_impact: float = 200.0, seed: int = 0,
                  steps: int = 1000, scale: float = 1.0, hg_alpha: float = HG_ALPHA) -> Workload:
    """Taylor impact: a cylinder (length/diameter 3.2, about n_particles
    particles on a cubic lattice) moving at v_impact onto a rigid wall at
    z = 0, Johnson-Cook material of the 1M-particle bar (damage constants x
    scale)."""
    sp = taylor_cylinder(n_particles, spacing, v_impact, seed=seed)
    mat = aluminium_jc(scale)
    w = _workload(f"taylor_{sp.N}", sp, [mat], steps, hg_alpha)
    w.wall = True
    return w


def batched_specimens(count: int = 256, seed: int = 0, n_min: int = 2000, n_max: int = 200000,
                      spacing: float = 0.5e-3, jitter: float = 0.01) -> list:
    """Independent tensile bars with particle counts log-uniform in
    [n_min, n_max] (lattice nx = ny, nz = 4 nx drawn from the seed) and
    Johnson-Cook damage constants D1, D2, D3 and C each drawn uniformly within
    +-20% of the 1M-particle bar's."""
    u = uniform(seed, 5 * count, stream=11).reshape(count, 5)
    out = []
    for k in range(count):
        n = math.exp(math.log(n_min) + u[k, 0] * (math.log(n_max) - math.log(n_min)))
        nx = max(3, int(round((n / 4.0) ** (1.0 / 3.0))))
        nz = 4 * nx
        mat = aluminium_jc()
        for c, key in enumerate(("D1", "D2", "D3", "C"), start=1):
            mat[key] *= 0.8 + 0.4 * u[k, c]
        sp = tensile_bar(nx, nx, nz, spacing, jitter, seed=seed * 100003 + k, name=f"bar_{k}")
        out.append(_workload(f"batched_bar_{k}_{nx}x{nx}x{nz}", sp, [mat], 0))
    return out


def serving_requests(count: int = 64, rate: float = 20.0, seed: int = 0, steps_range=(1000, 5000),
                     taylor_fraction: float = 0.5, n_range=(12000, 500000), bar_range=(2000, 200000)) -> list:
    """A Poisson request stream: (arrival time [s], workload, steps).  Half the
    requests (in expectation) are Taylor-impact cylinders (12k-500k particles
    log-uniform, v_impact uniform in [150, 300] m/s), the others tensile bars
    as in the batched workload; each asks for a uniform number of steps in
    steps_range."""
    u = uniform(seed, 6 * count, stream=13).reshape(count, 6)
    t = 0.0
    out = []
    for k in range(count):
        t += -math.log(1.0 - u[k, 0]) / rate
        steps = int(steps_range[0] + u[k, 1] * (steps_range[1] - steps_range[0]))
        if u[k, 2] < taylor_fraction:
            n = math.exp(math.log(n_range[0]) + u[k, 3] * (math.log(n_range[1]) - math.log(n_range[0])))
            w = taylor_impact(int(n), v_impact=150.0 + 150.0 * u[k, 4], seed=seed * 7919 + k, steps=steps)
        else:
            n = math.exp(math.log(bar_range[0]) + u[k, 3] * (math.log(bar_range[1]) - math.log(bar_range[0])))
            nx = max(3, int(round((n / 4.0) ** (1.0 / 3.0))))
            sp = tensile_bar(nx, nx, 4 * nx, 0.5e-3, 0.01, seed=seed * 7919 + k, name=f"req_bar_{k}")
            w = _workload(f"req_bar_{k}", sp, [aluminium_jc()], steps)
        out.append((t, w, steps))
    return out
