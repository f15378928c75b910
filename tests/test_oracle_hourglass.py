"""Pins of the oracle's hourglass control term (reading H).

Sec. 2 names Ganzenmueller's hourglass control without giving a formula; the
reading is a penalty on the mismatch between where a particle's own
deformation gradient puts a neighbour and where the neighbour is:

    eps_i = F_i X_ij - x_ij,  eps_j = F_j X_ij - x_ij,  delta = (eps_i + eps_j) . xhat_ij,
    f_i^HG = -1/2 alpha sum_j (1 - D_i)(1 - D_j) V_i V_j W(X_ij) E_ij / X_ij^2 delta xhat_ij,
    E_ij = (E_i + E_j) / 2.

Each pin below checks a property that a plausible slip in that formula
breaks: the term must vanish for every affine motion (not only rigid
rotation), rotate with the body, be linear in alpha, act as a restoring
spring along the current bond whose stiffness falls off as W(X)/X^2, lose
each partner's damage fraction, and use the mean of the two moduli.  The
stress term is switched off (A = 0) so that the forces are the hourglass
term alone."""
import numpy as np
import pytest

import oracle
from paper_1901_07374_gb300 import specimen as S

SPACING = 0.5e-3
E0, E1 = 70e9, 210e9


def _body(alpha=10.0, mats=None, mat_id=None, dims=(6, 6, 8), seed=1):
    """A jittered free body (no constraints) with zero stress."""
    sp = S.tensile_bar(*dims, SPACING, jitter=0.01, seed=seed)
    sp.bc_mask[:] = 0
    sp.bc_vel[:] = 0
    mats = mats or [S.material(E=E0, A=1e12), S.material(E=E1, A=1e12)]
    mid = np.zeros(sp.N, np.int32) if mat_id is None else np.asarray(mat_id, np.int32)
    h = 1.5 * SPACING
    sim = oracle.Simulation(sp.X, sp.vol, mid, sp.bc_mask, sp.bc_vel, sp.f0, mats, h, 2 * h,
                            S.cfl_dt(mats[0], SPACING), alpha)
    sim["A"][:] = 0.0
    return sim, sp


def _interior(sp):
    """Index of the particle closest to the body's centre."""
    c = sp.X.mean(0)
    return int(np.argmin(np.sum((sp.X - c) ** 2, 1)))


def _nbrs(sim, p):
    return sim.col[sim.row_ptr[p]:sim.row_ptr[p + 1]].astype(np.int64)


def _displaced(alpha=10.0, d=None, D=None, mat_id=None):
    """Undeformed body (F = I, u = 0) except one interior particle p moved by
    d: only the bonds of p are out of balance.  Returns the forces, p, its
    neighbours, the current bond vectors x_jp and the body."""
    sim, sp = _body(alpha, mat_id=mat_id)
    p = _interior(sp)
    d = np.array([0.7e-6, -0.4e-6, 1.1e-6]) if d is None else np.asarray(d, float)
    sim["u"][p] = d
    if D is not None:
        sim["D"][:] = D
    f = sim.forces()
    nb = _nbrs(sim, p)
    x = (sp.X[p] + d)[None, :] - sp.X[nb]
    return f, p, nb, x, sim, sp


def test_vanishes_for_any_affine_motion():
    """u = (F - I) X with a consistent, non-orthogonal F at every particle:
    each particle's F predicts its neighbours exactly, so the term is zero to
    rounding whatever the damage field (a transposed F, a flipped u_ij or a
    reference-frame direction would leave a force)."""
    rng = np.random.default_rng(3)
    sim, sp = _body()
    G = 0.2 * rng.normal(size=(3, 3))
    F = np.eye(3) + G
    assert abs(np.linalg.det(F @ F.T - np.eye(3))) > 1e-3      # not a rotation
    sim["F"][:] = F.ravel()
    sim["u"][:] = sp.X @ G.T
    sim["D"][:] = rng.uniform(0.0, 0.6, sim.N)
    f_affine = sim.forces()
    # the same body with a non-affine perturbation of 1e-3 spacing gives the force scale
    sim["u"][:] += 1e-3 * SPACING * rng.normal(size=(sim.N, 3))
    f_scale = np.abs(sim.forces()).max()
    assert f_scale > 0.0
    assert np.abs(f_affine).max() <= 1e-9 * f_scale


def test_objective_under_rotation_of_the_deformed_body():
    """Rotating a non-affinely deformed body (x -> Q x, F -> Q F) rotates
    every hourglass force (f -> Q f)."""
    rng = np.random.default_rng(4)
    sim, sp = _body()
    F = np.eye(3)[None] + 0.05 * rng.normal(size=(sim.N, 3, 3))
    u = 2e-6 * rng.normal(size=(sim.N, 3))
    D = rng.uniform(0.0, 0.5, sim.N)
    sim["F"][:] = F.reshape(-1, 9)
    sim["u"][:] = u
    sim["D"][:] = D
    f = sim.forces()
    a = rng.normal(size=3)
    a /= np.linalg.norm(a)
    th = 1.1
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    Q = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    sim["F"][:] = np.einsum("kl,nlm->nkm", Q, F).reshape(-1, 9)
    sim["u"][:] = (sp.X + u) @ Q.T - sp.X
    f_rot = sim.forces()
    assert np.abs(f_rot - f @ Q.T).max() <= 1e-11 * np.abs(f).max()


def test_linear_in_alpha():
    """The term is alpha times a fixed vector field; alpha = 0 switches it off."""
    fs = {}
    for alpha in (0.0, 1.0, 10.0, 37.5):
        rng = np.random.default_rng(5)           # the same state for every alpha
        sim, sp = _body(alpha)
        sim["F"][:] = (np.eye(3)[None] + 0.03 * rng.normal(size=(sim.N, 3, 3))).reshape(-1, 9)
        sim["u"][:] = 1e-6 * rng.normal(size=(sim.N, 3))
        sim["D"][:] = rng.uniform(0, 0.4, sim.N)
        sim["A"][:] = 1e8 * rng.normal(size=(sim.N, 9))
        fs[alpha] = sim.forces()
    unit = fs[1.0] - fs[0.0]
    assert np.abs(unit).max() > 0.0
    for alpha in (10.0, 37.5):
        assert np.abs((fs[alpha] - fs[0.0]) - alpha * unit).max() <= 1e-12 * alpha * np.abs(unit).max()


def test_restoring_spring_along_the_current_bond():
    """One displaced particle in an undeformed body: each of its neighbours
    feels a force along the current bond direction, attractive when the bond
    is stretched and repulsive when compressed, and nothing else moves."""
    f, p, nb, x, sim, sp = _displaced()
    xhat = x / np.linalg.norm(x, axis=1)[:, None]
    d = sim["u"][p]
    fj = f[nb]
    along = np.sum(fj * xhat, 1)
    perp = fj - along[:, None] * xhat
    assert np.abs(perp).max() <= 1e-10 * np.abs(fj).max()
    stretch = xhat @ d                      # d . xhat > 0: the bond j-p got longer
    big = np.abs(stretch) > 1e-3 * np.abs(d).max()
    assert np.all(np.sign(along[big]) == np.sign(stretch[big]))
    others = np.setdiff1d(np.arange(sim.N), np.append(nb, p))
    assert np.abs(f[others]).max() == 0.0
    assert np.allclose(f[p], -fj.sum(0), rtol=1e-13, atol=1e-13 * np.abs(fj).max())


def test_bond_stiffness_falls_off_as_w_over_distance_squared():
    """The bond stiffness k_j = (f_j . xhat) / (alpha d . xhat) of the
    displaced particle's bonds, compared between bonds of different reference
    lengths, scales as V_j W(X_jp) / X_jp^2 (the kernel pinned separately);
    its absolute value is E V_j V_p W / X^2, the reading's spring on the mean
    of the two particles' errors (both equal to -d here, so the 1/2 and the
    sum of the two errors cancel)."""
    alpha = 10.0
    f, p, nb, x, sim, sp = _displaced(alpha)
    xhat = x / np.linalg.norm(x, axis=1)[:, None]
    d = sim["u"][p]
    den = alpha * (xhat @ d)
    ok = np.abs(xhat @ d) > 0.2 * np.linalg.norm(d)
    k = np.sum(f[nb] * xhat, 1)[ok] / den[ok]
    X = np.linalg.norm(sp.X[p][None] - sp.X[nb], axis=1)[ok]
    V = sp.vol[nb][ok] * sp.vol[p]
    Wr = np.array([oracle.kernel_w(r, sim.cfg.h) for r in X])
    # three bonds of clearly different lengths: ratios only
    order = np.argsort(X)
    picks = [order[0], order[len(order) // 2], order[-1]]
    assert X[picks[-1]] > 2.0 * X[picks[0]]
    ratio = k / (V * Wr / X ** 2)
    for a in picks[1:]:
        assert ratio[a] / ratio[picks[0]] == pytest.approx(1.0, rel=1e-9)
    # every bond: the same constant, the mean Young modulus of the pair
    assert np.allclose(ratio, E0, rtol=1e-9)


def test_each_partner_damage_scales_the_bond():
    """Bond forces of the displaced particle lose the damaged fraction of
    both partners, (1 - D_p)(1 - D_j); a fully damaged partner transmits
    nothing (Sec. 3.1)."""
    rng = np.random.default_rng(12)
    f0, p, nb, x, sim, sp = _displaced()
    D = rng.uniform(0.0, 0.8, sim.N)
    D[p] = 0.35
    fD, *_ = _displaced(D=D)
    scale = (1 - D[p]) * (1 - D[nb])
    assert np.allclose(fD[nb], f0[nb] * scale[:, None], rtol=1e-12, atol=1e-12 * np.abs(f0).max())
    D[p] = 1.0
    f1, *_ = _displaced(D=D)
    assert np.abs(f1).max() == 0.0
    D[p] = 0.0
    j = nb[3]
    D[j] = 1.0
    fj, *_ = _displaced(D=D)
    assert np.abs(fj[j]).max() == 0.0 and np.abs(fj[p]).max() > 0.0


def test_two_materials_use_the_mean_modulus():
    """Bonds across a material interface: the force is the mean of the two
    single-material bodies' forces (a pair modulus linear in each partner's
    modulus, i.e. their arithmetic mean), and swapping which side carries
    which material leaves every bond force unchanged."""
    sim, sp = _body()
    p = _interior(sp)
    N = sp.N
    mid_p1 = np.zeros(N, np.int32)
    mid_p1[p] = 1
    f_mix, _, nb, *_ = _displaced(mat_id=mid_p1)
    f_all0, *_ = _displaced(mat_id=np.zeros(N, np.int32))
    f_all1, *_ = _displaced(mat_id=np.ones(N, np.int32))
    assert np.allclose(f_mix[nb], 0.5 * (f_all0[nb] + f_all1[nb]), rtol=1e-12,
                       atol=1e-12 * np.abs(f_all1).max())
    swapped = 1 - mid_p1
    f_swap, *_ = _displaced(mat_id=swapped)
    assert np.allclose(f_swap[nb], f_mix[nb], rtol=1e-12, atol=1e-12 * np.abs(f_mix).max())
    # single-material bodies scale with E
    assert np.allclose(f_all1[nb], (E1 / E0) * f_all0[nb], rtol=1e-12, atol=1e-12 * np.abs(f_all1).max())


def test_bond_force_acts_on_the_mean_of_the_two_errors():
    """All positions at the reference, but one particle p carries a wrong
    deformation gradient F_p = I + G: only p's own prediction of its
    neighbours is off (eps_p = G X, eps_j = 0), so every bond of p -- whichever
    particle has the lower index -- carries the bond stiffness measured on the
    displaced particle times the mean of the two projected errors."""
    alpha = 10.0
    # bond stiffness of each of p's bonds from the displaced-particle body
    f, p, nb, x, sim, sp = _displaced(alpha)
    xhat = x / np.linalg.norm(x, axis=1)[:, None]
    d = sim["u"][p]
    ok = np.abs(xhat @ d) > 0.2 * np.linalg.norm(d)
    k = np.sum(f[nb] * xhat, 1) / (alpha * (xhat @ d))
    # the same body, u = 0, F_p = I + G
    rng = np.random.default_rng(21)
    G = 1e-3 * rng.normal(size=(3, 3))
    sim2, _ = _body(alpha)
    sim2["F"][p] = (np.eye(3) + G).ravel()
    f2 = sim2.forces()
    X = sp.X[p][None, :] - sp.X[nb]                 # bond j -> p
    Xh = X / np.linalg.norm(X, axis=1)[:, None]
    err_p = X @ G.T                                 # F_p X - x with x = X
    mean_err = 0.5 * np.sum(err_p * Xh, 1)          # (eps_j + eps_p) / 2 projected, eps_j = 0
    expect = -(alpha * k * mean_err)[:, None] * Xh
    assert (nb > p).any() and (nb < p).any()
    assert np.allclose(f2[nb][ok], expect[ok], rtol=1e-6, atol=1e-9 * np.abs(expect).max())
    others = np.setdiff1d(np.arange(sim2.N), np.append(nb, p))
    assert np.abs(f2[others]).max() == 0.0
