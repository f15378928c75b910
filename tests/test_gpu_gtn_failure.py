"""GTN failure on the GPU against the FP64 oracle (Sec. 5.4: D = q1 f*,
f* = 1/q1 once f reaches f_F, so D = 1 and the particle fails, Sec. 3.1).

Two levels: material points driven to f = f_F through the constitutive
update alone, and a small circumferentially notched GTN bar pulled through
fracture at the notch."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1901_07374_gb300 import specimen as S
from paper_1901_07374_gb300 import tlsph
from parity import compare_state, relerr

pytestmark = pytest.mark.gpu

TRAJ_TOL = 1e-7


def test_gtn_material_points_fail_at_the_final_porosity():
    """Hydrostatic tension plus shear grows the voids of every point to f_F:
    the failed flag and its step are bit-exact, D is exactly 1 and the stress
    exactly 0 from the failing increment on, f is clamped to f_F."""
    import torch
    m = S.material(damage=S.DAMAGE_GTN, fN=0.0, komega=0.0)
    rng = np.random.default_rng(7)
    n, steps, dt = 48, 200, 1e-7
    f0 = rng.uniform(0.005, 0.02, n)
    base = np.diag([1e-3, 1e-3, 1e-3])
    deps = np.empty((steps, n, 3, 3))
    J = np.empty((steps, n))
    for p in range(n):
        e = base * rng.uniform(0.5, 1.5)
        e[0, 1] = e[1, 0] = 0.5 * rng.uniform(1e-3, 3e-3)
        deps[:, p] = e
        J[:, p] = np.cumprod(np.full(steps, np.linalg.det(np.eye(3) + e)))
    state = np.zeros((n, 16))
    state[:, 14] = f0
    state[:, 13] = [m["q1"] * oracle.gtn_fstar(m, f) for f in f0]
    ref = np.zeros((steps, n, 16))
    for p in range(n):
        ref[:, p], _ = oracle.material_point(m, dt, deps[:, p], J[:, p], init={"f": f0[p], "D": state[p, 13]})
    st = torch.tensor(state, device="cuda")
    fail_gpu = np.full(n, -1)
    for k in range(steps):
        tlsph.material_point_batch(m, dt, torch.tensor(deps[k].reshape(n, 9), device="cuda"),
                                   torch.tensor(J[k], device="cuda"), st)
        got = st.cpu().numpy()
        assert np.array_equal(got[:, 15], ref[k, :, 15]), k
        fail_gpu[(got[:, 15] == 1) & (fail_gpu < 0)] = k
        assert relerr(got[:, :10], ref[k, :, :10], 1e-3 * m["A"]) <= 1e-10
        for c in (10, 12, 13, 14):
            assert relerr(got[:, c], ref[k, :, c], 1e-9) <= 1e-10, (k, c)
        failed = got[:, 15] == 1
        assert np.all(got[failed, 13] == 1.0) and np.all(got[failed, 14] == m["fF"])
        assert np.all(got[failed, :10] == 0.0)
    fail_ref = np.array([int(np.argmax(ref[:, p, 15] == 1)) if ref[-1, p, 15] == 1 else -1 for p in range(n)])
    assert np.array_equal(fail_gpu, fail_ref)
    assert (fail_gpu >= 0).sum() == n and len(np.unique(fail_gpu)) > 5


def gtn_fracture_bar():
    """Small notched GTN round bar (R 1.2 mm, notch 0.4 mm, 630 particles at
    0.3 mm) whose voids nucleate early (eps_N 0.05, s_N 0.02) and reach a low
    final porosity (f_c 0.02, f_F 0.04), pulled at +-20 m/s: the notch
    layers fail within about 200 steps."""
    w = S.notched_bar_gtn(radius=1.2e-3, height=4e-3, spacing=0.3e-3, notch_radius=0.4e-3, v_grip=20.0,
                          steps=250)
    m = dict(w.materials[0])
    m.update(fc=0.02, fF=0.04, eN=0.05, sN=0.02, fN=0.04)
    return dataclasses.replace(w, materials=[m], name="gtn_fracture")


def test_gtn_notched_bar_fracture_fp64():
    w = gtn_fracture_bar()
    g = tlsph.Simulation.from_workload(w, precision="fp64")
    o = oracle.Simulation.from_workload(w)
    g.step(w.steps)
    o.step(w.steps)
    fs = g.get("FAIL_STEP")
    assert (o.fail_step >= 0).sum() > 20
    assert np.array_equal(fs, o.fail_step)
    failed = fs >= 0
    assert np.all(g.get("DAMAGE")[failed] == 1.0) and np.all(g.get("SIGMA")[failed] == 0.0)
    assert np.all(g.get("POROSITY")[failed] == w.materials[0]["fF"])
    compare_state(g.state(), o.state(), w, tol=TRAJ_TOL)


def test_gtn_notched_bar_fracture_mixed():
    """The mixed path through the same fracture: its failure set against the
    oracle's is stated (printed) and bounded; particles failing in both fail
    within a few steps of each other."""
    w = gtn_fracture_bar()
    g = tlsph.Simulation.from_workload(w, precision="mixed")
    o = oracle.Simulation.from_workload(w)
    g.step(w.steps)
    o.step(w.steps)
    fa, fb = o.fail_step >= 0, g.get("FAIL_STEP") >= 0
    both = fa & fb
    dstep = np.abs(o.fail_step[both] - g.get("FAIL_STEP")[both])
    print(f"GTN fracture, mixed vs oracle: failed {fa.sum()} / {fb.sum()}, symmetric difference {(fa ^ fb).sum()}, "
          f"failure steps differing {int((dstep > 0).sum())}, largest {int(dstep.max()) if both.any() else 0}")
    assert fa.sum() > 20
    assert (fa ^ fb).sum() <= 0.05 * fa.sum()
    assert dstep.max() <= 3
