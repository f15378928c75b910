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
