"""Helpers shared by the GPU parity tests: error norms with field floors,
mapping between the oracle's state and the library's fields, and the
extraction of a ball of particles around sampled particles so the oracle can
reproduce single particles of a full-size run."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1901_07374_gb300 import specimen as S

# library field name -> oracle state key
ORACLE_KEY = {"U": "u", "V": "v", "F": "F", "SIGMA": "sigma", "STRESS_DEV": "sd", "EPSP": "ep",
              "EPSP_RATE": "epdot", "DINIT": "dinit", "DAMAGE": "D", "POROSITY": "f", "FORCE": "force",
              "A": "A", "FAIL_STEP": "fail_step", "ENERGY": "e"}

# FP64 tolerance: normwise relative, per field (the FP64 GPU path reorders
# the sums over j, nothing else)
TOL_FP64 = 1e-10


def floors(w) -> dict:
    """Scale of each field, the floor of its normwise relative error: the
    lattice spacing for lengths, the grip speed for velocities, the yield
    stress for stresses (and A = P L^{-T}), yield stress x spacing^2 for
    forces, 1e-3 for the dimensionless strains, damage and porosity."""
    sp = w.specimen
    m = w.materials[0]
    L = sp.spacing
    vref = float(np.abs(sp.bc_vel).max()) or 1.0
    s = max(m["A"], 1e6)
    return dict(U=L, V=vref, F=1.0, SIGMA=s, STRESS_DEV=s, A=s, EPSP=1e-3, EPSP_RATE=1e-3 / w.dt,
                DINIT=1e-3, DAMAGE=1e-3, POROSITY=1e-3, FORCE=s * L * L, ENERGY=1e-3 * s / m["rho0"])


def relerr(a, b, floor):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), floor))


def compare_state(gpu, orc, w, tol=TOL_FP64, fields=None, idx=None):
    """Per-field normwise errors; returns {field: err} and asserts <= tol."""
    fl = floors(w)
    out = {}
    for f in fields or ("U", "V", "F", "SIGMA", "STRESS_DEV", "EPSP", "EPSP_RATE", "DINIT", "DAMAGE",
                        "POROSITY", "FORCE", "A", "ENERGY"):
        g = gpu[f]
        o = orc[ORACLE_KEY[f]]
        if idx is not None:
            g, o = g[idx], o[idx]
        out[f] = relerr(g.reshape(len(g), -1), o.reshape(len(o), -1), fl[f])
    bad = {k: v for k, v in out.items() if not v <= tol}
    assert not bad, f"fields above {tol}: {bad}"
    return out


def oracle_from_state(w, state: dict, step: int = 0) -> oracle.Simulation:
    """A fresh oracle simulation of workload w whose state is overwritten by
    `state` (oracle keys)."""
    sim = oracle.Simulation.from_workload(w)
    for k, v in state.items():
        if k == "fail_step":
            sim.fail_step[:] = v
        else:
            sim[k][:] = v
    sim.sys.step = step
    return sim


def ball(X, centres, radius):
    """Indices of all particles within `radius` of any centre (sorted)."""
    keep = np.zeros(X.shape[0], bool)
    for c in centres:
        keep |= np.sum((X - X[c]) ** 2, axis=1) < radius * radius
    return np.nonzero(keep)[0]


def sub_workload(w, idx):
    """The workload restricted to the particles idx (same materials, dt)."""
    import dataclasses
    sp = w.specimen
    sub = dataclasses.replace(sp, X=np.ascontiguousarray(sp.X[idx]), vol=sp.vol[idx], mat_id=sp.mat_id[idx],
                              bc_mask=sp.bc_mask[idx], bc_vel=np.ascontiguousarray(sp.bc_vel[idx]), f0=sp.f0[idx],
                              dims=())
    return dataclasses.replace(w, specimen=sub)


def taylor_energy_terms(mass, dt, v_n, f_n, v_n1, f_n1):
    """Per-step terms of the velocity-Verlet energy balance with the rigid
    wall, from the full-step velocities and forces alone (any path).

    The half-step velocity the drift used is v_post = v^{n+1} - dt/2 f^{n+1}/m,
    the one before the wall's projection is v_pre = v^n + dt/2 f^n/m; the wall
    removes  W = 1/2 m (v_pre - v_post) . (2 v^n - v_pre + v_post)  in the
    step (zero for a free particle and for one at rest against the wall), and
    the conserved quantity of the scheme is the kinetic energy less
    dt^2/8 sum |f|^2/m (the scheme's shadow term) plus the internal energy."""
    m = mass[:, None]
    v_pre = v_n + 0.5 * dt * f_n / m
    v_post = v_n1 - 0.5 * dt * f_n1 / m
    wall = 0.5 * np.sum(m * (v_pre - v_post) * (2.0 * v_n - v_pre + v_post))
    return wall


def shadow_energy(mass, dt, v, f, e):
    return 0.5 * np.sum(mass[:, None] * v * v) - dt * dt / 8.0 * np.sum(f * f / mass[:, None]) + np.sum(mass * e)


def taylor_energy_workload():
    """Taylor impact at 250 m/s onto the wall, no damage and no hourglass term
    (its work is not part of the internal energy), through 200 steps of plastic
    impact."""
    import dataclasses
    w = S.taylor_impact(3000, v_impact=250.0, steps=200)
    m = dict(w.materials[0])
    m["damage"] = S.DAMAGE_NONE
    return dataclasses.replace(w, materials=[m], hg_alpha=0.0)
