"""The mixed-precision path (FP32 pair gathers and sums, FP64 state and
constitutive update) against the FP64 oracle and the FP64 GPU path.

Its error is a stated property, not parity: these tests bound it loosely
(MIXED_TOL per field after a few steps of an elastic run; first-order
completeness and momentum to FP32 rounding) and the benchmark reports the
measured per-field errors."""
import numpy as np
import pytest

import oracle
from paper_1901_07374_gb300 import specimen as S
from paper_1901_07374_gb300 import tlsph
from parity import compare_state

pytestmark = pytest.mark.gpu

MIXED_TOL = 2e-4


def test_mixed_first_steps_vs_oracle():
    w = S.tensile_bar_cl()
    g = tlsph.Simulation.from_workload(w, precision="mixed")
    o = oracle.Simulation.from_workload(w)
    for steps in (1, 9, 40):
        g.step(steps)
        o.step(steps)
        errs = compare_state(g.state(), o.state(), w, tol=MIXED_TOL,
                             fields=("U", "V", "F", "SIGMA", "STRESS_DEV", "FORCE", "A"))
        print("mixed vs oracle", g.steps, errs)


def test_mixed_patch_test_and_momentum():
    w = S.tensile_bar_cl(nx=10, ny=9, nz=20)
    w.specimen.bc_mask[:] = 0
    w.specimen.bc_vel[:] = 0
    g = tlsph.Simulation.from_workload(w, precision="mixed")
    B = np.random.default_rng(0).normal(size=(3, 3)) * 5.0
    g.set("V", w.specimen.X @ B.T)
    g.step(1)
    F = g.get("F")
    assert np.max(np.abs(F - (np.eye(3).ravel() + w.dt * B.ravel()))) <= 1e-6 * w.dt * np.abs(B).max()
    g.step(5)
    f = g.get("FORCE")
    assert np.all(np.abs(f.sum(0)) <= 1e-5 * np.abs(f).sum(0))


def test_mixed_failure_variant_runs_and_fails_close_to_fp64():
    """Plastic flow, damage and failure in mixed precision: status clean, the
    failure set close to the FP64 path's (the decisions are FP64, their inputs
    carry the FP32 pair sums)."""
    w = S.failure_variant(S.tensile_bar_cl())
    a = tlsph.Simulation.from_workload(w, precision="fp64")
    b = tlsph.Simulation.from_workload(w, precision="mixed")
    a.step(500)
    b.step(500)
    b.sync()
    fa, fb = a.get("FAIL_STEP") >= 0, b.get("FAIL_STEP") >= 0
    assert fa.sum() > 50
    assert (fa ^ fb).sum() <= 0.05 * fa.sum()


def test_mixed_resume_is_bitwise():
    w = S.failure_variant(S.tensile_bar_cl(nx=6, ny=6, nz=16))
    names = tlsph.CHECKPOINT_FIELDS
    a = tlsph.Simulation.from_workload(w, precision="mixed")
    a.step(120)
    ck = {k: a.get(k) for k in names}
    a.step(80)
    ref = a.state()
    b = tlsph.Simulation.from_workload(w, precision="mixed")
    for k, v in ck.items():
        b.set(k, v)
    b.step(80)
    for k, v in b.state().items():
        assert np.array_equal(v, ref[k]), k


def test_mixed_resume_is_bitwise_with_partial_damage():
    """A GTN bar, whose every particle carries 0 < D = q1 f* < 1: the pass-1
    record's weight V (1 - D) rebuilt after a reload equals the one the
    uninterrupted run carries, so the resumed run is identical bit for bit."""
    w = S.notched_bar_gtn(radius=1.5e-3, height=5e-3, spacing=0.3e-3, notch_radius=0.5e-3, v_grip=20.0, steps=60)
    names = tlsph.CHECKPOINT_FIELDS
    a = tlsph.Simulation.from_workload(w, precision="mixed")
    a.step(30)
    ck = {k: a.get(k) for k in names}
    D = ck["DAMAGE"]
    assert np.all((D > 0) & (D < 1))
    a.step(30)
    ref = a.state()
    b = tlsph.Simulation.from_workload(w, precision="mixed")
    for k, v in ck.items():
        b.set(k, v)
    b.step(30)
    for k, v in b.state().items():
        assert np.array_equal(v, ref[k]), k


PLANS = [(0, 128, 0, 128), (1, 64, 1, 64), (2, 256, 1, 256), (3, 128, 0, 128), (1, 128, 1, 256), (4, 64, 3, 128),
         (2, 128, 4, 128), (4, 128, 2, 64), (4, 128, 5, 128), (4, 64, 6, 128), (4, 128, 7, 128),
         (4, 128, 8, 128), (5, 128, 8, 128)]


def test_every_launch_plan_computes_the_same_step():
    """The launch plans only regroup the FP32 sums: each stays within the mixed
    tolerance of the oracle and within FP32 rounding of the others."""
    w = S.failure_variant(S.tensile_bar_cl(), v_grip=10.0, scale=0.05)
    o = oracle.Simulation.from_workload(w)
    o.step(30)
    ref = o.state()
    states = []
    for plan in PLANS:
        g = tlsph.Simulation.from_workload(w, precision="mixed")
        g.set_plan(plan)
        assert g.get_plan() == plan
        g.step(30)
        st = g.state()
        compare_state(st, ref, w, tol=MIXED_TOL, fields=("U", "V", "F", "SIGMA", "FORCE"))
        states.append(st)
    for st in states[1:]:
        for k in ("U", "V", "F", "SIGMA"):
            a, b = st[k], states[0][k]
            assert np.max(np.abs(a - b)) <= 1e-5 * max(np.max(np.abs(b)), 1e-30), k


def _reordered(w, perm):
    import dataclasses
    sp = w.specimen
    sp2 = dataclasses.replace(sp, X=sp.X[perm].copy(), vol=sp.vol[perm].copy(), mat_id=sp.mat_id[perm].copy(),
                              bc_mask=sp.bc_mask[perm].copy(), bc_vel=sp.bc_vel[perm].copy(), f0=sp.f0[perm].copy())
    return dataclasses.replace(w, specimen=sp2)


@pytest.mark.parametrize("shuffle", ["all", "second_half"])
def test_aligned_and_explicit_slices_compute_the_same_step(shuffle):
    """Caller order kept (no internal reordering): lattice order gives aligned
    slices (one shared offset table per 32 rows); a shuffled caller order
    leaves the index offsets irregular, so its slices keep the explicit form
    (shuffling half the particles mixes both forms in one context).  The thread-per-row plans then compute the same
    step in both layouts to FP32 rounding, within MIXED_TOL of the oracle."""
    w = S.failure_variant(S.tensile_bar_cl(nx=8, ny=8, nz=24), v_grip=10.0, scale=0.05)
    N = w.specimen.N
    perm = np.arange(N)
    rng = np.random.default_rng(3)
    if shuffle == "all":
        perm = rng.permutation(N)
    else:
        perm[N // 2:] = N // 2 + rng.permutation(N - N // 2)
    a = tlsph.Simulation.from_workload(w, precision="mixed", line_order=False)
    b = tlsph.Simulation.from_workload(_reordered(w, perm), precision="mixed", line_order=False)
    la, lb = a.neighbor_layout(), b.neighbor_layout()
    assert la["slices"] == lb["slices"] == (N + 31) // 32
    # lattice order: all slices aligned but those within 3 layers of either end
    # of the index range (there i + o_k would leave the particle range)
    assert la["aligned_slices"] >= 0.6 * la["slices"]
    if shuffle == "all":
        assert lb["aligned_slices"] <= 0.1 * lb["slices"]
    else:
        assert 0.15 * lb["slices"] <= lb["aligned_slices"] <= 0.7 * lb["slices"]
    assert la["words"] < lb["words"]
    for plan in [(4, 128, 1, 128), (1, 64, 2, 256)]:
        a = tlsph.Simulation.from_workload(w, precision="mixed", line_order=False)
        b = tlsph.Simulation.from_workload(_reordered(w, perm), precision="mixed", line_order=False)
        a.set_plan(plan)
        b.set_plan(plan)
        a.step(30)
        b.step(30)
        for k in ("U", "V", "F", "SIGMA"):
            x, y = a.get(k)[perm], b.get(k)
            assert np.max(np.abs(x - y)) <= 1e-5 * max(np.max(np.abs(x)), 1e-30), (plan, k)
    o = oracle.Simulation.from_workload(w)
    o.step(30)
    compare_state(a.state(), o.state(), w, tol=MIXED_TOL, fields=("U", "V", "F", "SIGMA", "FORCE"))


def test_weight_table_form_equals_the_computed_weights():
    """Pass-1 form 5 reads W'(q)/r of every slot from a table built when the
    form is set; the weights are formed by the same explicitly rounded
    expression as form 4 forms them in place, so the two step bit for bit
    alike, also after switching back and forth (the table is freed and
    rebuilt).  A context in a caller arena has no table: the form is refused."""
    import torch
    w = S.failure_variant(S.tensile_bar_cl(nx=8, ny=8, nz=40), v_grip=10.0, scale=0.05)
    a = tlsph.Simulation.from_workload(w, precision="mixed", line_order=False)
    b = tlsph.Simulation.from_workload(w, precision="mixed", line_order=False)
    a.set_plan((4, 128, 7, 128))
    b.set_plan((5, 128, 7, 128))
    a.step(300)
    b.step(150)
    b.set_plan((4, 128, 7, 128))
    b.step(30)
    b.set_plan((5, 64, 7, 128))
    b.step(120)
    for k, v in a.state().items():
        assert np.array_equal(b.get(k), v), k
    nnz = a.nnz
    cfg = tlsph.make_config(w.h, w.rc, w.dt, w.hg_alpha, "mixed")
    arena = torch.empty(tlsph.workspace_bytes(cfg, w.specimen.N, nnz), dtype=torch.uint8, device="cuda")
    c = tlsph.Simulation.from_workload(w, precision="mixed", arena=arena, nnz_cap=nnz, line_order=False)
    with pytest.raises(tlsph.TlsphError) as e:
        c.set_plan((5, 128, 7, 128))
    assert e.value.code == -1
    assert c.get_plan() != (5, 128, 7, 128)
    c.step(2)


def test_plans_out_of_range_are_rejected():
    g = tlsph.Simulation.from_workload(S.tensile_bar_cl(nx=5, ny=5, nz=8), precision="mixed")
    for plan in [(6, 128, 1, 128), (1, 128, 9, 128), (1, 100, 1, 128), (1, 128, 6, 256), (1, 128, 4, 256),
                 (1, 128, 5, 256), (1, 128, 7, 256), (1, 128, 8, 256), (1, 512, 1, 128),
                 (5, 256, 1, 128)]:
        with pytest.raises(tlsph.TlsphError) as e:
            g.set_plan(plan)
        assert e.value.code == -1, plan


def test_autotune_restores_the_state_bitwise(tmp_path, monkeypatch):
    from paper_1901_07374_gb300 import autotune
    monkeypatch.setenv("TLSPH_PLAN_CACHE", str(tmp_path / "plans.json"))
    w = S.failure_variant(S.tensile_bar_cl(nx=8, ny=8, nz=24))
    a = tlsph.Simulation.from_workload(w, precision="mixed")
    a.step(40)
    before = a.checkpoint(device=False)
    rec = []
    plan = autotune.tune(a, steps=2, warmup=1, record=rec)
    assert len(rec) == len(autotune.PASS1) + len(autotune.PASS2)
    after = a.checkpoint(device=False)
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    assert a.get_plan() == tuple(plan)
    # the tuned run continues exactly like an untuned one with the same plan
    b = tlsph.Simulation.from_workload(w, precision="mixed")
    b.step(40)
    b.set_plan(plan)
    a.step(20)
    b.step(20)
    for k, v in a.state().items():
        assert np.array_equal(v, b.get(k)), k
    # a second call is served from the cache without stepping
    steps = a.steps
    assert autotune.tune(a) == tuple(plan) and a.steps == steps


def _order_layouts(w):
    a = tlsph.Simulation.from_workload(w, precision="mixed")                     # TLSPH_FLAG_AUTO_ORDER
    c = tlsph.Simulation.from_workload(w, precision="mixed", line_order=False)
    l = tlsph.Simulation.from_workload(w, precision="mixed", line_order=True)
    return a, c, l


@pytest.mark.parametrize("name", ["box_bar", "notched_bar_gtn"])
def test_auto_order_takes_the_better_aligned_order(name):
    """The binding's default for mixed contexts (TLSPH_FLAG_AUTO_ORDER) keeps
    the caller's order when nine in ten neighbour slices are aligned and takes
    lattice-line order when that aligns more; the chosen context equals the
    explicitly ordered one bit for bit.  On the 455,958-particle GTN notched
    bar, whose x-lines change length across the round cross-section, the
    caller's order leaves 28 % of the slices explicit and line order is taken."""
    if name == "box_bar":
        w = S.tensile_bar_jc(nx=12, ny=12, nz=96, steps=20)
    else:
        w = S.notched_bar_gtn()
    a, c, l = _order_layouts(w)
    la, lc, ll = a.neighbor_layout(), c.neighbor_layout(), l.neighbor_layout()
    if 10 * lc["aligned_slices"] >= 9 * lc["slices"]:
        expect, ref = lc, c
    else:
        expect, ref = (ll, l) if ll["aligned_slices"] > lc["aligned_slices"] else (lc, c)
    assert la == expect
    if name == "notched_bar_gtn":
        assert expect is ll and lc["aligned_slices"] < 0.8 * lc["slices"]
    a.step(3)
    ref.step(3)
    for k in ("U", "V", "F", "SIGMA", "FORCE", "DAMAGE"):
        assert np.array_equal(a.get(k), ref.get(k)), k


def test_auto_order_in_a_caller_arena():
    """The automatic order builds a shuffled bar (its caller order leaves the
    slices explicit) a second time, in line order, in the same caller-owned
    arena; the context equals an explicitly line-ordered one in its own arena
    bit for bit."""
    import torch
    w0 = S.failure_variant(S.tensile_bar_cl(nx=8, ny=8, nz=24), v_grip=10.0, scale=0.05)
    w = _reordered(w0, np.random.default_rng(5).permutation(w0.specimen.N))
    nnz = tlsph.Simulation.from_workload(w, precision="fp64").nnz
    cfg = tlsph.make_config(w.h, w.rc, w.dt, w.hg_alpha, "mixed")
    nbytes = tlsph.workspace_bytes(cfg, w.specimen.N, nnz)
    arenas = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    a = tlsph.Simulation.from_workload(w, precision="mixed", arena=arenas[0], nnz_cap=nnz)
    b = tlsph.Simulation.from_workload(w, precision="mixed", arena=arenas[1], nnz_cap=nnz, line_order=True)
    c = tlsph.Simulation.from_workload(w, precision="mixed", line_order=False)
    assert a.neighbor_layout() == b.neighbor_layout()
    assert c.neighbor_layout()["aligned_slices"] < a.neighbor_layout()["aligned_slices"]
    a.step(20)
    b.step(20)
    for k, v in b.state().items():
        assert np.array_equal(a.get(k), v), k


def test_line_order_removes_padding_slots():
    """Lattice lines along the longest axis as the internal order: every row of
    a slice shares its neighbourhood shape, so the aligned slices carry far
    less padding than in the caller's x-fastest order (where a slice mixes
    surface and interior rows), and the step agrees with the caller-order
    context to FP32 rounding."""
    w = S.failure_variant(S.tensile_bar_cl(nx=6, ny=6, nz=64), v_grip=10.0, scale=0.05)
    a = tlsph.Simulation.from_workload(w, precision="mixed", line_order=False)
    b = tlsph.Simulation.from_workload(w, precision="mixed", line_order=True)
    la, lb = a.neighbor_layout(), b.neighbor_layout()
    nnz = a.nnz
    assert b.nnz == nnz
    # jittered lattice: the pairs at exactly 3 spacings are in or out per row, so
    # even line order pads about 13 % (x-fastest order on this bar: about 70 %)
    assert lb["slots"] <= 1.2 * nnz and la["slots"] >= 1.4 * nnz
    assert lb["aligned_slices"] >= 0.8 * lb["slices"]
    a.step(30)
    b.step(30)
    for k in ("U", "V", "F", "SIGMA"):
        x, y = a.get(k), b.get(k)
        assert np.max(np.abs(x - y)) <= 1e-5 * max(np.max(np.abs(x)), 1e-30), k


def test_guard_band_changes_only_which_kernel_updates():
    """The FP32 elastic screen's guard band only moves particles between the
    FP32 elastic branch and the FP64 update: band 1 (every particle in FP64)
    agrees with the default band to FP32 rounding through plastic flow with
    elastic unloading near the free surfaces, and bands below the
    conservative 1e-5 are refused."""
    w = S.tensile_bar_jc(nx=9, ny=9, nz=20, steps=20)
    st = S.plastic_flow_state(w)
    a = tlsph.Simulation.from_workload(w, precision="mixed")
    b = tlsph.Simulation.from_workload(w, precision="mixed")
    for g in (a, b):
        for k, v in st.items():
            g.set(k, v)
    b.set_guard(1.0)
    for bad in (0.0, 1e-6, float("nan"), float("inf")):
        with pytest.raises(tlsph.TlsphError) as e:
            a.set_guard(bad)
        assert e.value.code == -1
    a.step(20)
    b.step(20)
    assert a.status_bits() == 0 and b.status_bits() == 0
    assert np.mean(a.get("EPSP") > 0) > 0.5
    for k in ("U", "V", "F", "SIGMA", "STRESS_DEV"):
        x, y = a.get(k), b.get(k)
        assert np.max(np.abs(x - y)) <= 1e-5 * max(np.max(np.abs(x)), 1e-30), k
    o = oracle.Simulation.from_workload(w)
    o["u"][:] = st["U"]
    o["v"][:] = st["V"]
    o["F"][:] = st["F"]
    o["sd"][:] = st["STRESS_DEV"]
    o.step(20)
    errs = compare_state(b.state(), o.state(), w, tol=MIXED_TOL, fields=PLASTIC_FIELDS)
    print("plastic-flow window, band 1, vs oracle", errs)
    errs = compare_state(a.state(), o.state(), w, tol=MIXED_TOL, fields=PLASTIC_FIELDS)
    print("plastic-flow window, default band, vs oracle", errs)


def test_gtn_mixed_screen_against_fp64_update_and_oracle():
    """GTN porous plasticity in the mixed path: particles clearly inside the
    GTN yield surface take the FP32 elastic branch, the others the FP64
    return.  Through 300 steps of a small notched bar (plastic flow near the
    notch, elastic elsewhere) it agrees with every particle in the FP64 update
    (guard band 1) to FP32 rounding and with the oracle within MIXED_TOL."""
    w = S.notched_bar_gtn(radius=2.0e-3, height=6e-3, spacing=0.3e-3, notch_radius=0.6e-3, v_grip=20.0, steps=300)
    a = tlsph.Simulation.from_workload(w, precision="mixed")
    b = tlsph.Simulation.from_workload(w, precision="mixed")
    b.set_guard(1.0)
    a.step(300)
    b.step(300)
    assert a.status_bits() == 0 and b.status_bits() == 0
    ep = a.get("EPSP")
    assert (ep > 0).any() and (ep == 0).any()
    for k in ("U", "V", "F", "SIGMA", "POROSITY"):
        x, y = a.get(k), b.get(k)
        assert np.max(np.abs(x - y)) <= 1e-4 * max(np.max(np.abs(x)), 1e-30), k
    o = oracle.Simulation.from_workload(w)
    o.step(300)
    compare_state(a.state(), o.state(), w, tol=MIXED_TOL, fields=("U", "V", "F", "SIGMA", "FORCE"))


def test_gtn_plastic_flow_seeded_return():
    """Every particle of a GTN notched bar in plastic flow, so every update
    goes through the mixed path's FP64 return, whose two Newton solves
    (Algorithm 2) start from single-precision seeds.  After 10 steps no solve
    has hit its iteration cap, and the state agrees with the FP64 GPU path
    (unseeded solves) to the FP32 rounding of the kinematics and with the
    oracle within MIXED_TOL."""
    w = S.notched_bar_gtn(radius=2.0e-3, height=6e-3, spacing=0.3e-3, notch_radius=0.6e-3, steps=10)
    st = S.plastic_flow_state(w)
    a = tlsph.Simulation.from_workload(w, precision="mixed")
    b = tlsph.Simulation.from_workload(w, precision="fp64")
    for g in (a, b):
        for k, v in st.items():
            g.set(k, v)
    a.step(10)
    b.step(10)
    assert a.status_bits() == 0 and b.status_bits() == 0
    assert np.all(a.get("EPSP") > 0)
    for k in ("U", "F", "SIGMA", "EPSP", "POROSITY"):
        x, y = a.get(k), b.get(k)
        assert np.max(np.abs(x - y)) <= 1e-4 * max(np.max(np.abs(y)), 1e-30), k
    o = oracle.Simulation.from_workload(w)
    o["u"][:] = st["U"]
    o["v"][:] = st["V"]
    o["F"][:] = st["F"]
    o["sd"][:] = st["STRESS_DEV"]
    o.step(10)
    compare_state(a.state(), o.state(), w, tol=MIXED_TOL, fields=("U", "V", "F", "SIGMA", "FORCE"))


PLASTIC_FIELDS = ("U", "V", "F", "SIGMA", "STRESS_DEV", "EPSP", "DINIT", "DAMAGE", "FORCE")


def _plastic_window(w, steps, mixed=False):
    """The mixed path (or the oracle) from the plastic-flow state of w after
    `steps` steps."""
    st = S.plastic_flow_state(w)
    if not mixed:
        o = oracle.Simulation.from_workload(w)
        o["u"][:] = st["U"]
        o["v"][:] = st["V"]
        o["F"][:] = st["F"]
        o["sd"][:] = st["STRESS_DEV"]
        o.step(steps)
        return o.state()
    g = tlsph.Simulation.from_workload(w, precision="mixed")
    for k, v in st.items():
        g.set(k, v)
    g.step(steps)
    assert g.status_bits() == 0
    return g.state()


def test_plastic_flow_window_long_bar_against_the_oracle():
    """A long Johnson-Cook bar (rate term C = 0.002) with every particle in
    plastic flow: plastic strain, damage initiation and damage are gated with
    the other fields within the mixed tolerance of the oracle."""
    w = S.tensile_bar_jc(nx=6, ny=6, nz=200, steps=12)
    errs = compare_state(_plastic_window(w, 12, mixed=True), _plastic_window(w, 12), w, tol=MIXED_TOL,
                         fields=PLASTIC_FIELDS)
    print("plastic-flow window, long bar, vs oracle", errs)
