"""Edge cases of the step through the C ABI, in both precisions, against the
FP64 oracle: the smallest bodies (one partial warp of rows), particle counts
on either side of a 32-row slice boundary, very wide neighbour rows, and the
degenerate inputs the method has (no particles, a particle without
neighbours: a singular correction matrix, Sec. 2.2)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1901_07374_gb300 import specimen as S
from paper_1901_07374_gb300 import tlsph
from parity import TOL_FP64, compare_state

pytestmark = pytest.mark.gpu

MIXED_TOL = 2e-4
MIXED_FIELDS = ("U", "V", "F", "SIGMA", "STRESS_DEV", "FORCE")


def _body(X, base, seed=0, h_factor=None):
    """Workload of the free body with positions X (no constraints), the
    material and step of `base`, a random initial velocity field of a few m/s
    and, optionally, a wider kernel (h = h_factor x spacing, rc = 2h)."""
    N = X.shape[0]
    rng = np.random.default_rng(seed)
    d = base.specimen.spacing
    v0 = rng.normal(size=(N, 3)) * 2.0
    sp = S.Specimen("edge", X, np.full(N, d ** 3), np.zeros(N, np.int32), np.zeros(N, np.uint8), v0,
                    np.zeros(N), d)
    w = dataclasses.replace(base, specimen=sp, name="edge")
    if h_factor is not None:
        h = h_factor * d
        w = dataclasses.replace(w, h=h, rc=2.0 * h)
    return w


def _lattice(nx, ny, nz, base, seed=0, n=None):
    d = base.specimen.spacing
    X, _ = S.lattice_box(nx, ny, nz, d)
    X = X + np.random.default_rng(seed + 11).uniform(-0.01, 0.01, X.shape) * d
    return X[:n] if n is not None else X


def _both(w, steps, precision, plan=None):
    g = tlsph.Simulation.from_workload(w, precision=precision)
    if plan is not None:
        g.set_plan(plan)
    o = oracle.Simulation.from_workload(w)
    g.step(steps)
    o.step(steps)
    g.sync()
    return g.state(), o.state()


# the launch plans the benchmark tunes to: the per-slot weight table in pass 1
# (padded, zero-filled slice tails) with packed or scalar pass-2 terms
BENCH_PLANS = [(5, 128, 8, 128), (5, 64, 7, 128)]


def _check(w, steps):
    gs, os_ = _both(w, steps, "fp64")
    compare_state(gs, os_, w, tol=TOL_FP64)
    for plan in [None] + BENCH_PLANS:
        gm, om = _both(w, steps, "mixed", plan)
        compare_state(gm, om, w, tol=MIXED_TOL, fields=MIXED_FIELDS)


def test_smallest_body_one_partial_warp():
    """27 particles: a single slice of rows, 5 of its lanes empty."""
    base = S.tensile_bar_cl()
    _check(_body(_lattice(3, 3, 3, base), base), 6)


@pytest.mark.parametrize("n", [31, 33, 63, 65])
def test_ragged_counts_around_a_slice(n):
    """Particle counts one below and one above a multiple of the 32-row slice."""
    base = S.tensile_bar_cl()
    w = _body(_lattice(4, 4, 5, base, seed=n, n=n), base, seed=n)
    _check(w, 5)


def test_wide_rows():
    """h = 3 spacings, rc = 6 spacings: about 500 neighbours per row on a 9^3
    lattice (rows longer than the warp sort's register form, sliced lists
    with long offset unions)."""
    base = S.tensile_bar_cl()
    w = _body(_lattice(9, 9, 9, base, seed=3), base, seed=3, h_factor=3.0)
    g = tlsph.Simulation.from_workload(w, precision="fp64")
    rp = g.get("NBR_ROWPTR")
    assert np.diff(rp).max() > 400
    o = oracle.Simulation.from_workload(w)
    assert np.array_equal(rp, o.row_ptr) and np.array_equal(g.get("NBR_COL"), o.col)
    _check(w, 3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_degenerate_inputs(precision):
    base = S.tensile_bar_cl()
    # no particles: rejected on the host
    w0 = _body(np.zeros((0, 3)), base)
    with pytest.raises((tlsph.TlsphError, ValueError)):
        tlsph.Simulation.from_workload(w0, precision=precision)
    # a lone particle, and a body with one particle far from the rest: no
    # neighbours, singular correction matrix
    w1 = _body(np.zeros((1, 3)), base)
    with pytest.raises(tlsph.TlsphError) as e:
        tlsph.Simulation.from_workload(w1, precision=precision)
    assert e.value.code == -2
    X = _lattice(4, 4, 4, base)
    X = np.vstack([X, X[:1] + 1.0])
    with pytest.raises(tlsph.TlsphError) as e:
        tlsph.Simulation.from_workload(_body(X, base), precision=precision)
    assert e.value.code == -2
    # the library stays usable after the failures
    _check(_body(_lattice(3, 3, 4, base, seed=5), base, seed=5), 2)
