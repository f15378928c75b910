"""Pins of the oracle's kernel, neighbour sets, correction matrix, velocity
gradient, polar decomposition and eigenvalues against facts the paper and the
mathematics fix (normalisation, library routines, first-order completeness,
closed-form lattice counts)."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg
import scipy.spatial

import oracle
from paper_1901_07374_gb300 import specimen as S

H = 1.5  # smoothing length in lattice units


# ------------------------------------------------------------------ kernel

def test_kernel_normalised_in_3d():
    """The kernel integrates to one over its support (Sec. 2.2, Eq. condition_1)."""
    for h in (1.0, 0.75e-3):
        val, _ = scipy.integrate.quad(lambda r: 4 * math.pi * r * r * oracle.kernel_w(r, h), 0, 2 * h,
                                      points=[h], epsabs=0, epsrel=1e-13)
        assert abs(val - 1.0) < 1e-12


def test_kernel_derivative_is_dw_dr():
    h = 0.75e-3
    for q in (0.1, 0.5, 0.9, 1.2, 1.7, 1.95):
        r = q * h
        e = 1e-7 * h
        fd = (oracle.kernel_w(r + e, h) - oracle.kernel_w(r - e, h)) / (2 * e)
        assert abs(fd - oracle.kernel_dw(r, h)) <= 1e-6 * abs(oracle.kernel_dw(r, h))


def test_kernel_compact_and_continuous():
    h = 1.0
    assert oracle.kernel_w(2 * h, h) == 0.0 and oracle.kernel_dw(2 * h, h) == 0.0
    assert oracle.kernel_dw(0.0, h) == 0.0
    for q in (1.0, 2.0):
        a, b = oracle.kernel_w(q * h * (1 - 1e-12), h), oracle.kernel_w(q * h * (1 + 1e-12), h)
        assert abs(a - b) < 1e-9
        a, b = oracle.kernel_dw(q * h * (1 - 1e-12), h), oracle.kernel_dw(q * h * (1 + 1e-12), h)
        assert abs(a - b) < 1e-9


# ------------------------------------------------------------------ neighbours

def _rows(row_ptr, col):
    return [col[row_ptr[i]:row_ptr[i + 1]] for i in range(len(row_ptr) - 1)]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_neighbors_match_kdtree(seed):
    """Brute-force neighbour rows equal scipy's kd-tree ball query (strict <),
    on a jittered lattice with no distance within 1e-9 of the cutoff."""
    sp = S.tensile_bar(6, 5, 9, 1.0, jitter=0.01, seed=seed)
    rc = 2 * H
    row_ptr, col = oracle.neighbors(sp.X, rc)
    d = scipy.spatial.distance.cdist(sp.X, sp.X)
    assert np.min(np.abs(d - rc)) > 1e-9
    tree = scipy.spatial.cKDTree(sp.X)
    ref = tree.query_ball_point(sp.X, r=rc * (1 - 1e-12))
    for i, row in enumerate(_rows(row_ptr, col)):
        expect = sorted(j for j in ref[i] if j != i)
        assert list(row) == expect


def test_neighbors_interior_count_exact_lattice():
    """On an exact cubic lattice with rc = 3 spacings the interior rows hold the
    92 lattice vectors with 0 < |k|^2 < 9 (count 6+12+8+6+24+24+12)."""
    sp = S.tensile_bar(9, 9, 9, 1.0, jitter=0.0)
    row_ptr, col = oracle.neighbors(sp.X, 3.0)
    counts = np.diff(row_ptr)
    centre = 4 + 9 * 4 + 81 * 4
    assert counts[centre] == 92
    assert counts.max() == 92
    # corners keep only the octant: lattice vectors with all k >= 0, 0 < |k|^2 < 9
    octant = sum(1 for a in range(3) for b in range(3) for c in range(3) if 0 < a * a + b * b + c * c < 9)
    assert counts[0] == octant


def test_neighbors_symmetric_sorted_no_self_and_bounded():
    sp = S.tensile_bar(8, 8, 12, 0.5e-3, jitter=0.01, seed=3)
    row_ptr, col = oracle.neighbors(sp.X, 3 * 0.5e-3)
    rows = _rows(row_ptr, col)
    pairs = set()
    for i, r in enumerate(rows):
        assert np.all(np.diff(r) > 0)
        assert i not in set(r.tolist())
        pairs.update((i, int(j)) for j in r)
    assert all((j, i) in pairs for i, j in pairs)
    # +-1% jitter cannot bring |k|^2 = 10 inside 3 spacings, so rows hold at
    # most the 92 + 30 vectors with |k|^2 <= 9
    assert np.diff(row_ptr).max() <= 122


# ------------------------------------------------------------------ correction matrix and gradient

def _bar(seed=0, dims=(6, 5, 8), jitter=0.01):
    sp = S.tensile_bar(*dims, 1.0, jitter=jitter, seed=seed)
    row_ptr, col = oracle.neighbors(sp.X, 2 * H)
    L, Linv, bad = oracle.shape_matrix(sp.X, sp.vol, row_ptr, col, H)
    assert bad == 0
    return sp, row_ptr, col, L, Linv


def test_correction_matrix_inverse_matches_numpy():
    sp, row_ptr, col, L, Linv = _bar()
    ref = np.linalg.inv(L.reshape(-1, 3, 3)).reshape(-1, 9)
    assert np.max(np.abs(ref - Linv)) <= 1e-12 * np.max(np.abs(ref))


def test_correction_matrix_is_kernel_moment():
    """L_i assembled independently with numpy from Eq. (correction_matrix)."""
    sp, row_ptr, col, L, _ = _bar(seed=4)
    i = 37
    js = col[row_ptr[i]:row_ptr[i + 1]]
    d = sp.X[js] - sp.X[i]
    r = np.linalg.norm(d, axis=1)
    dw = np.array([oracle.kernel_dw(x, H) for x in r])
    grad = dw[:, None] * d / r[:, None]
    Lref = np.einsum("j,jk,jl->kl", sp.vol[js], d, grad)
    assert np.allclose(Lref.ravel(), L[i], rtol=1e-13, atol=0)


@pytest.mark.parametrize("seed", [0, 5])
def test_patch_test_affine_velocity(seed):
    """First-order completeness (Sec. 2.2, corrected gradient): an affine
    velocity v = B X + c gives Fdot_i = B at every particle, surface included."""
    sp, row_ptr, col, L, Linv = _bar(seed=seed)
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(3, 3))
    v = sp.X @ B.T + rng.normal(size=3)
    Fd = oracle.velocity_gradient(sp.X, sp.vol, v, np.zeros(sp.N), Linv, row_ptr, col, H)
    err = np.max(np.abs(Fd - B.ravel()[None, :]))
    assert err <= 1e-12 * np.max(np.abs(B))


def test_damage_weight_removes_contribution():
    """Eq. (Crack_approx_Fdot): a particle with D_j = 1 no longer enters any
    neighbour's Fdot, and D_j = 1/2 halves its contribution."""
    sp, row_ptr, col, L, Linv = _bar(seed=2)
    rng = np.random.default_rng(7)
    v = rng.normal(size=(sp.N, 3))
    D = np.zeros(sp.N)
    j = 123
    D[j] = 1.0
    Fd1 = oracle.velocity_gradient(sp.X, sp.vol, v, D, Linv, row_ptr, col, H)
    v2 = v.copy()
    v2[j] += rng.normal(size=3) * 10
    Fd2 = oracle.velocity_gradient(sp.X, sp.vol, v2, D, Linv, row_ptr, col, H)
    nb = [i for i in range(sp.N) if i != j]
    assert np.array_equal(Fd1[nb], Fd2[nb])
    # half weight: the difference between D_j = 0 and D_j = 1/2 is half the
    # difference between D_j = 0 and D_j = 1
    F0 = oracle.velocity_gradient(sp.X, sp.vol, v, np.zeros(sp.N), Linv, row_ptr, col, H)
    Dh = np.zeros(sp.N)
    Dh[j] = 0.5
    Fh = oracle.velocity_gradient(sp.X, sp.vol, v, Dh, Linv, row_ptr, col, H)
    assert np.allclose(F0 - Fh, 0.5 * (F0 - Fd1), rtol=1e-10, atol=1e-12 * np.abs(F0).max())


# ------------------------------------------------------------------ polar / eigen

def test_polar_matches_scipy():
    rng = np.random.default_rng(11)
    for _ in range(200):
        F = np.eye(3) + 0.6 * rng.normal(size=(3, 3))
        if np.linalg.det(F) <= 0.05:
            continue
        R, U, ok = oracle.polar(F)
        assert ok
        Rs, Us = scipy.linalg.polar(F, side="right")
        assert np.allclose(R, Rs, atol=1e-13)
        assert np.allclose(U, Us, atol=1e-12 * np.abs(F).max())
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert np.all(np.linalg.eigvalsh(U) > 0)


def test_polar_of_rotation_is_itself():
    th = 0.7
    R0 = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    R, U, ok = oracle.polar(R0)
    assert ok and np.allclose(R, R0, atol=1e-15) and np.allclose(U, np.eye(3), atol=1e-15)


def test_eig_sym_matches_numpy():
    rng = np.random.default_rng(3)
    for _ in range(200):
        A = rng.normal(size=(3, 3))
        A = A + A.T
        ev = np.sort(oracle.eig_sym(A))
        assert np.allclose(ev, np.linalg.eigvalsh(A), atol=1e-13 * np.abs(A).max())
    # repeated eigenvalues
    ev = np.sort(oracle.eig_sym(np.diag([2.0, 2.0, -1.0])))
    assert np.allclose(ev, [-1, 2, 2])
