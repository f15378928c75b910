"""C-ABI behaviour on the GPU: caller-owned arenas, checkpoint/resume,
error reporting and status bits (raised from the host or from inputs the
kernels handle, never by faulting the device)."""
import numpy as np
import pytest

from paper_1901_07374_gb300 import specimen as S
from paper_1901_07374_gb300 import tlsph

pytestmark = pytest.mark.gpu

WRITABLE = tlsph.CHECKPOINT_FIELDS


def test_resume_is_bitwise():
    """Checkpoint at step k into a new context, continue: identical bits to
    the uninterrupted run."""
    w = S.failure_variant(S.tensile_bar_cl())
    a = tlsph.Simulation.from_workload(w)
    a.step(150)
    ck = {k: a.get(k) for k in WRITABLE}
    a.step(100)
    ref = a.state()
    b = tlsph.Simulation.from_workload(w)
    for k, v in ck.items():
        b.set(k, v)
    b.step(100)
    got = b.state()
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


def test_arena_matches_owned_memory():
    import torch
    w = S.tensile_bar_cl(nx=6, ny=6, nz=16)
    a = tlsph.Simulation.from_workload(w)
    nnz = a.nnz
    cfg = tlsph.make_config(w.h, w.rc, w.dt, w.hg_alpha)
    nbytes = tlsph.workspace_bytes(cfg, w.specimen.N, nnz)
    arena = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    b = tlsph.Simulation.from_workload(w, arena=arena, nnz_cap=nnz)
    a.step(20)
    b.step(20)
    for k, v in a.state().items():
        assert np.array_equal(b.get(k), v), k


def test_arena_too_small_and_capacity_errors():
    import torch
    w = S.tensile_bar_cl(nx=5, ny=5, nz=8)
    cfg = tlsph.make_config(w.h, w.rc, w.dt, w.hg_alpha)
    need = tlsph.workspace_bytes(cfg, w.specimen.N, 10)
    arena = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(tlsph.TlsphError) as e:
        tlsph.Simulation.from_workload(w, arena=arena, nnz_cap=10)
    assert e.value.code == -4 and "nnz_cap" in str(e.value)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(tlsph.TlsphError) as e:
        tlsph.Simulation.from_workload(w, arena=small, nnz_cap=10)
    assert e.value.code == -4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_create_validates_inputs_on_device(precision):
    """The array contents are validated on the device after their upload, in
    the pass that also forms the bounding box, the materials in use and the
    bulk velocity: a non-positive or non-finite volume, a non-finite position
    and a material index out of range are argument errors with their
    messages, with library memory or a caller arena, and a valid create
    afterwards works."""
    import torch
    w = S.tensile_bar_cl(nx=4, ny=4, nz=6)
    sp = w.specimen
    N = sp.N
    mats = [S.aluminium_cl()]

    def make(X=sp.X, vol=sp.vol, mat=sp.mat_id, **kw):
        return tlsph.Simulation(X, vol, mat, sp.bc_mask, sp.bc_vel, sp.f0, mats, w.h, w.rc, w.dt, w.hg_alpha,
                                precision=precision, **kw)

    Xn = sp.X.copy()
    Xn[N - 1, 2] = np.nan
    vinf = sp.vol.copy()
    vinf[5] = np.inf
    mbad = sp.mat_id.copy()
    mbad[N // 2] = 99
    cases = [(dict(vol=-sp.vol), "vol"), (dict(vol=vinf), "vol"), (dict(X=Xn), "X must be finite"),
             (dict(mat=mbad), "mat_id")]
    cfg = tlsph.make_config(w.h, w.rc, w.dt, w.hg_alpha, precision)
    arena = torch.empty(tlsph.workspace_bytes(cfg, N, 200 * N), dtype=torch.uint8, device="cuda")
    for extra in ({}, dict(arena=arena, nnz_cap=200 * N)):
        for kw, msg in cases:
            with pytest.raises(tlsph.TlsphError) as e:
                make(**kw, **extra)
            assert e.value.code == -1 and msg in str(e.value), (kw.keys(), str(e.value))
        g = make(**extra)
        g.step(2)
        assert g.status_bits() == 0 and np.all(np.isfinite(g.get("V")))
        g.close()


def test_isolated_particle_is_singular():
    sp = S.tensile_bar(4, 4, 6, 1e-3, jitter=0.0)
    X = np.vstack([sp.X, [[1.0, 1.0, 1.0]]])
    N = X.shape[0]
    with pytest.raises(tlsph.TlsphError) as e:
        tlsph.Simulation(X, np.full(N, 1e-9), None, None, None, None, [S.aluminium_cl()], 1.5e-3, 3e-3, 1e-8, 0.0)
    assert e.value.code == -2


def test_unset_material_is_reported():
    w = S.tensile_bar_cl(nx=4, ny=4, nz=6)
    sp = w.specimen
    sp.mat_id[:] = 1
    g = tlsph.Simulation(sp.X, sp.vol, sp.mat_id, sp.bc_mask, sp.bc_vel, sp.f0, [S.aluminium_cl()], w.h, w.rc, w.dt,
                         w.hg_alpha)
    with pytest.raises(tlsph.TlsphError) as e:
        g.step(1)
    assert e.value.code == -6


def test_nonfinite_input_sets_status_bits():
    """A NaN velocity (set from the host) propagates to a non-finite state:
    tlsph_sync reports ERR_NUMERICS with the status bits, the context stays
    usable for reading."""
    w = S.tensile_bar_cl(nx=5, ny=5, nz=8)
    g = tlsph.Simulation.from_workload(w)
    v = g.get("V")
    interior = int(np.nonzero(w.specimen.bc_mask == 0)[0][len(v) // 4])
    v[interior] = np.nan
    g.set("V", v)
    g.step(2)
    with pytest.raises(tlsph.TlsphError) as e:
        g.sync()
    assert e.value.code == -3
    assert g.status_bits() != 0
    assert g.get("U").shape == (w.specimen.N, 3)


def test_step_counter_is_part_of_the_checkpoint():
    w = S.tensile_bar_cl(nx=5, ny=5, nz=8)
    g = tlsph.Simulation.from_workload(w)
    g.step(7)
    assert g.get("STEP")[0] == 7 == g.steps
    g.set("STEP", np.array([41], np.int64))
    assert g.steps == 41
    g.step(2)
    assert g.get("STEP")[0] == 43


@pytest.mark.parametrize("order", ["spatial_order", "line_order"])
def test_internal_order_is_invisible(order):
    """A reordered context (brick order, or lattice lines along the longest
    axis) and one keeping the caller's order return the same neighbour CSR bit
    for bit and the same fields to FP64 rounding (only the order of the sums
    over j differs)."""
    from parity import ORACLE_KEY, compare_state
    w = S.failure_variant(S.tensile_bar_jc(nx=9, ny=7, nz=30, seed=2, steps=60))
    a = tlsph.Simulation.from_workload(w, **{order: True})
    b = tlsph.Simulation.from_workload(w)
    assert np.array_equal(a.get("NBR_ROWPTR"), b.get("NBR_ROWPTR"))
    assert np.array_equal(a.get("NBR_COL"), b.get("NBR_COL"))
    assert np.array_equal(a.get("X"), w.specimen.X)
    a.step(60)
    b.step(60)
    ref = {ORACLE_KEY[k]: v for k, v in b.state().items()}
    compare_state(a.state(), ref, w, tol=1e-9)
    assert np.array_equal(a.get("FAIL_STEP"), b.get("FAIL_STEP"))
    if order == "line_order":
        with pytest.raises(tlsph.TlsphError) as e:
            tlsph.Simulation.from_workload(w, spatial_order=True, line_order=True)
        assert e.value.code == -1
    for precision in ("mixed",):
        c = tlsph.Simulation.from_workload(w, precision=precision, **{order: True})
        c.step(60)
        compare_state(c.state(), ref, w, tol=2e-4, fields=("U", "V", "F", "SIGMA", "FORCE"))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_diagnostics_async_equals_the_synchronous_call(precision):
    """tlsph_diagnostics_async queues the same reductions behind the queued
    steps: two calls in flight (after steps 3 and 4) hold, once the stream has
    passed them, the bits the synchronous call gives at those states.  The
    binding takes only a page-locked float64 CPU tensor."""
    import torch
    w = S.failure_variant(S.tensile_bar_cl(nx=6, ny=6, nz=20))
    a = tlsph.Simulation.from_workload(w, precision=precision)
    b = tlsph.Simulation.from_workload(w, precision=precision)
    bufs = [torch.zeros(tlsph.DIAG_COUNT, dtype=torch.float64).pin_memory() for _ in range(2)]
    a.step(3)
    a.diagnostics_async(bufs[0])
    a.step(1)
    a.diagnostics_async(bufs[1])
    a.sync()
    b.step(3)
    assert tlsph.diagnostics_dict(bufs[0]) == b.diagnostics()
    b.step(1)
    assert tlsph.diagnostics_dict(bufs[1]) == b.diagnostics()
    with pytest.raises(ValueError):
        a.diagnostics_async(torch.zeros(tlsph.DIAG_COUNT, dtype=torch.float64))           # pageable
    with pytest.raises(ValueError):
        a.diagnostics_async(torch.zeros(tlsph.DIAG_COUNT, dtype=torch.float32).pin_memory())


def test_fma_peak_microbenchmark():
    """The FMA-rate probe: FP32 well above FP64 on this part, both positive
    and below the nominal unit counts x 2.2 GHz."""
    f32 = tlsph.fma_peak(False, 512)
    f64 = tlsph.fma_peak(True, 16)
    assert 1e12 < f32 < 152 * 128 * 2.2e9
    assert 0 < f64 < f32 / 8
    with pytest.raises(tlsph.TlsphError) as e:
        tlsph.fma_peak(False, 0)
    assert e.value.code == -1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_diagnostics_match_the_fields(precision):
    """Momentum, force sum, kinetic energy, failed count and the largest D and
    plastic strain equal the same reductions of the fields read back, and the
    device reduction returns the same bits every time."""
    w = S.failure_variant(S.tensile_bar_cl(nx=6, ny=6, nz=20))
    g = tlsph.Simulation.from_workload(w, precision=precision)
    g.step(300)
    d = g.diagnostics()
    assert d == g.diagnostics()
    m = w.materials[0]["rho0"] * w.specimen.vol
    v, f = g.get("V"), g.get("FORCE")
    mom = (m[:, None] * v).sum(0)
    assert np.allclose(d["momentum"], mom, rtol=1e-12, atol=1e-12 * np.abs(m[:, None] * v).sum())
    assert np.allclose(d["force_sum"], f.sum(0), rtol=1e-12, atol=1e-12 * np.abs(f).sum())
    assert d["kinetic_energy"] == pytest.approx(0.5 * (m * (v * v).sum(1)).sum(), rel=1e-12)
    assert d["failed"] == int((g.get("FAIL_STEP") >= 0).sum())
    assert d["max_damage"] == g.get("DAMAGE").max()
    assert d["max_epsp"] == g.get("EPSP").max()
    assert d["internal_energy"] == pytest.approx((m * g.get("ENERGY")).sum(), rel=1e-12)
    assert d["internal_energy"] > 0
    assert d["max_epsp"] > 0
