"""Batched stepping (one persistent launch per kernel kind over all members,
optionally replayed from a CUDA graph).

A specimen's rows are computed by the same kernels whatever else is in the
batch, so its result in a batch of one and in any mix is identical bit for
bit, with or without the graph.  Against the same context advanced by its own
launches (other kernels, sums fused differently by the compiler) the results
agree to FP32 rounding."""
import numpy as np
import pytest

from paper_1901_07374_gb300 import specimen as S
from paper_1901_07374_gb300 import tlsph
from parity import ORACLE_KEY, compare_state

pytestmark = pytest.mark.gpu


def _specimens():
    return [S.tensile_bar_jc(nx=9, ny=7, nz=30, seed=1),
            S.failure_variant(S.tensile_bar_cl(nx=8, ny=8, nz=24)),
            S.tensile_bar_jc(nx=13, ny=11, nz=40, seed=2, scale=0.8),
            S.notched_bar_gtn(radius=1.5e-3, height=5e-3, spacing=0.3e-3, notch_radius=0.5e-3, v_grip=20.0),
            S.failure_variant(S.tensile_bar_jc(nx=6, ny=6, nz=20, seed=4)),
            S.paper_loading(S.tensile_bar_cl(nx=7, ny=6, nz=22, seed=5), v_max=20.0, tau=5e-7)]


def _make(ws):
    return [tlsph.Simulation.from_workload(w, precision="mixed") for w in ws]


def _alone_in_batch(w, schedule, graph=True):
    """w advanced by a batch of one, `schedule` = step counts per call."""
    g = tlsph.Simulation.from_workload(w, precision="mixed")
    b = tlsph.Batch(capacity=1)
    b.set([g])
    for n in schedule:
        b.step(n, graph=graph)
    return g


@pytest.mark.parametrize("graph", [False, True])
def test_alone_and_in_the_mix_are_identical(graph):
    ws = _specimens()
    mix = _make(ws)
    b = tlsph.Batch(capacity=8)
    b.set(mix)
    b.step(25, graph=graph)
    b.step(15, graph=graph)
    for w, g in zip(ws, mix):
        assert g.steps == 40
        a = _alone_in_batch(w, (40,), graph=not graph)
        for k, v in a.state().items():
            assert np.array_equal(v, g.get(k)), k


def test_membership_changes_between_steps():
    ws = _specimens()
    mix = _make(ws)
    b = tlsph.Batch(capacity=8)
    b.set(mix[:3])
    b.step(10)
    b.set(mix[1:])                 # one leaves, two join
    b.step(10)
    b.set([mix[0], mix[4]])
    b.step(5)
    for w, g, n in zip(ws, mix, (15, 20, 20, 10, 15)):
        assert g.steps == n
        a = _alone_in_batch(w, (n,))
        for k, v in a.state().items():
            assert np.array_equal(v, g.get(k)), k


def test_batch_matches_own_launches_to_fp32_rounding():
    ws = _specimens()
    mix = _make(ws)
    own = _make(ws)
    b = tlsph.Batch(capacity=8)
    b.set(mix)
    b.step(30)
    for w, g, o in zip(ws, mix, own):
        o.step(30)
        ref = {ORACLE_KEY[k]: v for k, v in o.state().items()}
        compare_state(g.state(), ref, w, tol=2e-5, fields=("U", "V", "F", "SIGMA", "STRESS_DEV", "FORCE"))
        assert np.array_equal(g.get("FAIL_STEP") >= 0, o.get("FAIL_STEP") >= 0)


def test_batch_rejects_fp64_and_stale_members():
    w = S.tensile_bar_cl(nx=5, ny=5, nz=10)
    b = tlsph.Batch(capacity=2)
    with pytest.raises(tlsph.TlsphError) as e:
        b.set([tlsph.Simulation.from_workload(w, precision="fp64")])
    assert e.value.code == -1
    g = tlsph.Simulation.from_workload(w, precision="mixed")
    b.set([g])
    b.step(2)
    g.step(1)                          # stepped outside the batch
    with pytest.raises(tlsph.TlsphError) as e:
        b.step(1)
    assert e.value.code == -6
    b.set([g])
    b.step(1)
    assert g.steps == 4
