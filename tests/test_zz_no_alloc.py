"""tlsph_neighbors_noalloc: the neighbour-CSR build for callers that cannot
allocate device memory (a host framework that owns all device memory through
its own pool, loops that must not take the device-wide synchronisation of a
cudaMalloc/cudaFree, plugins without an allocator).  It keeps its scratch in
a fixed device array inside the library, so these checks compare its output
with the neighbour CSR that tlsph_create builds, on consecutive calls that
reuse that array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1901_07374_gb300 import specimen as S
from paper_1901_07374_gb300 import tlsph

pytestmark = pytest.mark.gpu


def _reference(w):
    sim = tlsph.Simulation.from_workload(w)
    rp, col = sim.get("NBR_ROWPTR"), sim.get("NBR_COL")
    sim.close()
    return rp, col


def _noalloc(w, cap):
    import torch
    X = torch.tensor(w.specimen.X, dtype=torch.float64, device="cuda")
    rp = torch.full((w.specimen.N + 1,), -7, dtype=torch.int64, device="cuda")
    col = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    nnz = tlsph.neighbors_noalloc(X, w.rc, rp, col)
    torch.cuda.synchronize()
    return nnz, rp.cpu().numpy(), col.cpu().numpy()


def test_noalloc_matches_create_on_consecutive_calls():
    """Two different specimens, then the first again: every call must equal
    the tlsph_create rows bit for bit, whatever the previous call left in the
    shared scratch."""
    work = [S.tensile_bar_cl(), S.tensile_bar_jc(nx=12, ny=10, nz=40, seed=5), S.tensile_bar_cl()]
    for w in work:
        rp_ref, col_ref = _reference(w)
        nnz, rp, col = _noalloc(w, len(col_ref) + 17)
        assert nnz == len(col_ref)
        assert np.array_equal(rp, rp_ref)
        assert np.array_equal(col[:nnz], col_ref)
        assert np.all(col[nnz:] == -7)          # nothing written past the pairs


def test_noalloc_limits_and_capacity():
    import torch
    w = S.tensile_bar_cl(nx=6, ny=6, nz=10)
    rp_ref, col_ref = _reference(w)
    # too small a column buffer: the pair count comes back, the columns are not written
    with pytest.raises(tlsph.TlsphError) as e:
        _noalloc(w, 10)
    assert e.value.code == -4 and e.value.nnz == len(col_ref)
    # beyond the fixed scratch size: rejected on the host with a clear message
    big = torch.zeros((262145, 3), dtype=torch.float64, device="cuda")
    rp = torch.empty(262146, dtype=torch.int64, device="cuda")
    with pytest.raises(tlsph.TlsphError) as e:
        tlsph.neighbors_noalloc(big, 1e-3, rp, None)
    assert e.value.code == -1 and "262144" in str(e.value)
    # and the entry point still works afterwards
    nnz, rp2, col2 = _noalloc(w, len(col_ref))
    assert np.array_equal(rp2, rp_ref) and np.array_equal(col2, col_ref)


def _lattice_workload(X, spacing):
    n = X.shape[0]
    sp = S.Specimen("cloud", np.ascontiguousarray(X), np.full(n, spacing ** 3), np.zeros(n, np.int32),
                    np.zeros(n, np.uint8), np.zeros((n, 3)), np.zeros(n), spacing, ())
    h = 1.5 * spacing
    return S.Workload("cloud", sp, [S.aluminium_cl()], h, 2 * h, 2e-8, 10.0, 1)


def _rows_by_brute_force(X, rc, rows):
    """Neighbour rows by the definition (r^2 = (dx^2 + dy^2) + dz^2 < rc^2, self
    excluded), for a few sampled particles."""
    out = []
    for i in rows:
        d = X - X[i]
        r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        m = r2 < rc * rc
        m[i] = False
        out.append(np.nonzero(m)[0])
    return out


def test_noalloc_at_its_particle_limit():
    """N = 262144, the largest count the fixed scratch holds (its layout is
    sized by N): a jittered 64^3 lattice, equal to tlsph_create's rows and to
    sampled rows by brute force."""
    w = S.tensile_bar_cl(nx=64, ny=64, nz=64)
    assert w.specimen.N == 262144
    rp_ref, col_ref = _reference(w)
    nnz, rp, col = _noalloc(w, len(col_ref))
    assert np.array_equal(rp, rp_ref) and np.array_equal(col, col_ref)
    rows = np.random.default_rng(2).choice(w.specimen.N, 40, replace=False)
    for i, r in zip(rows, _rows_by_brute_force(w.specimen.X, w.rc, rows)):
        assert np.array_equal(col[rp[i]:rp[i + 1]], r)


def test_noalloc_sparse_body_widens_its_cell_grid():
    """4096 small clumps (4 x 4 x 4 lattice blocks) spread over a box hundreds
    of cutoffs wide, N = 262144: cells of rc / 2 would number far more than
    the 2N + 4096 the scratch holds, so the grid's cells are widened; the rows
    still equal tlsph_create's and sampled brute-force rows."""
    d = 0.5e-3
    g = np.arange(4) * d
    block = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    c = np.arange(16) * 40 * d
    centres = np.stack(np.meshgrid(c, c, c, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(4)
    X = (centres[:, None, :] + block[None, :, :]).reshape(-1, 3) + rng.uniform(-0.01, 0.01, (262144, 3)) * d
    w = _lattice_workload(X, d)
    extent = X.max(0) - X.min(0)
    assert np.prod(np.floor(extent / (w.rc / 2)) + 1) > 2 * 262144 + 4096
    rp_ref, col_ref = _reference(w)
    nnz, rp, col = _noalloc(w, len(col_ref))
    assert np.array_equal(rp, rp_ref) and np.array_equal(col, col_ref)
    rows = rng.choice(262144, 40, replace=False)
    for i, r in zip(rows, _rows_by_brute_force(X, w.rc, rows)):
        assert np.array_equal(col[rp[i]:rp[i + 1]], r)


def test_noalloc_rejects_non_finite_positions():
    """A NaN or infinite coordinate is an argument error (as in tlsph_create),
    not a particle with an empty row; the entry point works afterwards."""
    import torch
    w = S.tensile_bar_cl(nx=6, ny=6, nz=10)
    rp_ref, col_ref = _reference(w)
    for bad in (np.nan, np.inf):
        X = w.specimen.X.copy()
        X[17, 1] = bad
        Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
        rp = torch.empty(w.specimen.N + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(len(col_ref), dtype=torch.int32, device="cuda")
        with pytest.raises(tlsph.TlsphError) as e:
            tlsph.neighbors_noalloc(Xd, w.rc, rp, col)
        assert e.value.code == -1 and "finite" in str(e.value)
    nnz, rp2, col2 = _noalloc(w, len(col_ref))
    assert np.array_equal(rp2, rp_ref) and np.array_equal(col2, col_ref)
