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


def test_every_launch_shape_computes_the_same_rows():
    """Each variant of each batch kernel kind (register cap, pairs in flight)
    changes only the launch: the members' states after the same steps agree
    to FP32 rounding (under another register cap the compiler may fuse
    multiply-adds differently), and with any one shape a member alone equals
    the member in the mix bit for bit."""
    ws = _specimens()[:4]
    ref = None
    b = tlsph.Batch(capacity=4)
    _, nv = b.get_shape()
    shapes = [(0, 0, 0)] + [tuple(v if k == kind else 0 for k in range(3)) for kind in range(3)
                            for v in range(1, nv[kind])]
    for shape in shapes:
        mix = _make(ws)
        b.set(mix)
        b.set_shape(shape)
        assert b.get_shape()[0] == shape
        b.step(12)
        st = [g.state() for g in mix]
        if ref is None:
            ref = st
            continue
        for a, r in zip(st, ref):
            for k in ("U", "V", "F", "SIGMA", "STRESS_DEV"):
                x, y = a[k], r[k]
                assert np.max(np.abs(x - y)) <= 1e-5 * max(np.max(np.abs(y)), 1e-30), (shape, k)
            assert np.array_equal(a["FAIL_STEP"] >= 0, r["FAIL_STEP"] >= 0)
    last = shapes[-1]
    alone = tlsph.Simulation.from_workload(ws[0], precision="mixed")
    b1 = tlsph.Batch(capacity=1)
    b1.set([alone])
    b1.set_shape(last)
    b1.step(12)
    for k, v in alone.state().items():
        assert np.array_equal(v, st[0][k]), (last, k)
    with pytest.raises(tlsph.TlsphError) as e:
        b.set_shape((nv[0], 0, 0))
    assert e.value.code == -1


def test_weight_table_variant_equals_the_default_bitwise():
    """Pass-1 variant 4 reads the members' per-slot weight tables (built when
    the shape is set) and otherwise runs the default gather: the two batches
    step bit for bit alike.  Releasing a member's table (its own plan leaves
    form 5) stops the batch until it is set again."""
    ws = _specimens()[:4]
    base = _make(ws)
    b0 = tlsph.Batch(capacity=4)
    b0.set(base)
    b0.step(15)
    tab = _make(ws)
    b1 = tlsph.Batch(capacity=4)
    b1.set(tab)
    b1.set_shape((4, 0, 0))
    b1.step(15)
    for a, r in zip(tab, base):
        for k, v in r.state().items():
            assert np.array_equal(a.get(k), v), k
    tab[0].set_plan((4, 128, 7, 128))       # leaves form 5 (never set): its table is released
    with pytest.raises(tlsph.TlsphError):
        b1.step(1)
    b1.set(tab)                             # rebuilds the table
    b1.step(1)
    b0.step(1)
    for a, r in zip(tab, base):
        assert np.array_equal(a.get("V"), r.get("V"))


def test_tuned_batch_restores_the_state_and_equals_the_shape_set_by_hand(tmp_path, monkeypatch):
    """The batch autotuner times the launch shapes on the members' live state
    and then restores every member bit for bit: its tuned batch steps exactly
    like a batch that ran the same steps and was given the chosen shape by
    hand."""
    from paper_1901_07374_gb300 import autotune
    monkeypatch.setenv("TLSPH_PLAN_CACHE", str(tmp_path / "plans.json"))
    ws = _specimens()
    tuned = _make(ws)
    b = tlsph.Batch(capacity=8)
    b.set(tuned)
    b.step(7)
    before = [g.checkpoint(device=False) for g in tuned]
    rec = []
    shape = autotune.tune_batch(b, tuned, steps=2, warmup=1, record=rec)
    _, nv = b.get_shape()
    assert len(rec) == sum(nv) and b.get_shape()[0] == shape
    for g, ck in zip(tuned, before):
        assert g.steps == 7
        for k, v in ck.items():         # every resumable field, bit for bit
            assert np.array_equal(v, g.get(k)), k
    b.step(11)
    # by hand: the same 7 steps with the default shape, then the tuned shape
    byhand = _make(ws)
    b2 = tlsph.Batch(capacity=8)
    b2.set(byhand)
    b2.step(7)
    b2.set_shape(shape)
    b2.step(11)
    for g, h in zip(tuned, byhand):
        assert g.steps == h.steps == 18
        for k, v in h.state().items():
            assert np.array_equal(v, g.get(k)), k
    # the cached shape is reused without timing
    rec2 = []
    assert autotune.tune_batch(b2, byhand, record=rec2) == shape and rec2 == []
