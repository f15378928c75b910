"""Hourglass control across a material interface (reading H, pair modulus
(E_i + E_j) / 2) on the GPU against the FP64 oracle, in both precisions.

The benchmark specimens are single-material, so only a body with two
materials exercises the pair modulus: the upper half of a tensile bar is a
stiffer material, pulled hard enough to yield and fail near the interface."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1901_07374_gb300 import specimen as S
from paper_1901_07374_gb300 import tlsph
from parity import TOL_FP64, compare_state

pytestmark = pytest.mark.gpu

MIXED_TOL = 2e-4
TRAJ_TOL = 1e-7


def _bimaterial(v_grip=10.0):
    w = S.failure_variant(S.tensile_bar_cl(nx=6, ny=6, nz=16), v_grip=v_grip, scale=0.05)
    sp = w.specimen
    mid = np.where(sp.X[:, 2] > np.median(sp.X[:, 2]), 1, 0).astype(np.int32)
    stiff = S.material(rho0=7800.0, E=200e9, nu=0.29, A=500e6, B=300e6, n=0.3, damage=S.DAMAGE_CL, Wcr=4e6)
    dt = min(S.cfl_dt(w.materials[0], sp.spacing), S.cfl_dt(stiff, sp.spacing))
    sp2 = dataclasses.replace(sp, mat_id=mid)
    return dataclasses.replace(w, specimen=sp2, materials=[w.materials[0], stiff], dt=dt)


def test_bimaterial_fp64_vs_oracle():
    w = _bimaterial()
    assert w.hg_alpha > 0
    g = tlsph.Simulation.from_workload(w, precision="fp64")
    o = oracle.Simulation.from_workload(w)
    for n in (1, 4):
        g.step(n)
        o.step(n)
        compare_state(g.state(), o.state(), w, tol=TOL_FP64)
    g.step(295)
    o.step(295)
    compare_state(g.state(), o.state(), w, tol=TRAJ_TOL)
    assert np.array_equal(g.get("FAIL_STEP"), o.fail_step)


def test_bimaterial_mixed_vs_oracle():
    w = _bimaterial()
    g = tlsph.Simulation.from_workload(w, precision="mixed")
    o = oracle.Simulation.from_workload(w)
    for n in (1, 9, 30):
        g.step(n)
        o.step(n)
        compare_state(g.state(), o.state(), w, tol=MIXED_TOL,
                      fields=("U", "V", "F", "SIGMA", "STRESS_DEV", "FORCE", "A"))
