"""Pins of the oracle's constitutive and damage updates (Secs. 4-5,
Algorithms 1 and 2) against closed forms, special cases and invariants."""
import math
import os

import numpy as np
import pytest
import scipy.optimize
import scipy.stats

import oracle
from paper_1901_07374_gb300 import specimen as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _moduli(m):
    return S.moduli(m)


def shear_increment(dg):
    """Symmetric strain increment of an engineering shear dg in the xy plane."""
    e = np.zeros((3, 3))
    e[0, 1] = e[1, 0] = 0.5 * dg
    return e


# ------------------------------------------------------------------ moduli and EOS

def test_table1_sound_speed_pins_bulk_modulus():
    """Table 1 prints c0 = 5166 m/s for rho0 7750, E 211 GPa, nu 0.33; that is
    sqrt(K/rho0) with K = E/(3(1-2nu)), the bulk modulus the linear EOS uses."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "weldox_table1.txt")) if not l.startswith("#")]
    rho0, E, nu, c0 = (float(x) for x in rows[0][:4])
    m = S.material(rho0=rho0, E=E, nu=nu)
    # the linear EOS slope dsigma_m/dJ at J = 1 is K
    K = (oracle.eos_mean_stress(m, 1.0 + 1e-7) - oracle.eos_mean_stress(m, 1.0 - 1e-7)) / 2e-7
    assert abs(math.sqrt(K / rho0) - c0) < 1.0


def test_weldox_presets_match_tables():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "weldox_tables23.txt")) if not l.startswith("#")]
    for r in rows:
        m = S.weldox(r[0])
        A, B, n, Wcr, D1, D2, D3, D4, D5, f0, fc, fF, kw = (float(x) for x in r[1:])
        assert (m["A"], m["B"], m["n"], m["Wcr"]) == (A * 1e6, B * 1e6, n, Wcr * 1e6)
        assert (m["D1"], m["D2"], m["D3"], m["D4"], m["D5"]) == (D1, D2, D3, D4, D5)
        assert (m["_f0"], m["fc"], m["fF"], m["komega"]) == (f0, fc, fF, kw)


def test_eos_linear_and_damaged_tension():
    m = S.aluminium_cl()
    K, _ = _moduli(m)
    for J in (0.97, 1.0, 1.002):
        assert oracle.eos_mean_stress(m, J) == pytest.approx(K * (J - 1), rel=1e-15, abs=0)
    # (1 - D) scales the tensile branch only (Eq. pH)
    assert oracle.eos_mean_stress(m, 1.01, 0.4) == pytest.approx(0.6 * K * 0.01, rel=1e-14)
    assert oracle.eos_mean_stress(m, 0.99, 0.4) == pytest.approx(-K * 0.01, rel=1e-14)


def test_mie_grueneisen_reduces_to_linear_and_is_compressive_positive_pressure():
    m_lin = S.aluminium_cl()
    K, _ = _moduli(m_lin)
    m_mg = dict(m_lin, eos=1, c0=math.sqrt(K / m_lin["rho0"]), S_alpha=0.0, Gamma0=0.0)
    for J in (0.95, 0.999, 1.0, 1.003):
        # with S_alpha = Gamma0 = 0 the pressure is rho0 c0^2 (eta - 1) / eta
        # = K (1 - J): the tension-positive mean stress is exactly K (J - 1)
        eta = 1 / J
        p = m_mg["rho0"] * m_mg["c0"] ** 2 * (eta - 1) / eta
        assert oracle.eos_mean_stress(m_mg, J) == pytest.approx(-p, rel=1e-12, abs=1e-3)
        assert oracle.eos_mean_stress(m_mg, J) == pytest.approx(oracle.eos_mean_stress(m_lin, J),
                                                                rel=1e-12, abs=1e-3)
    w = S.weldox("700E")
    assert oracle.eos_mean_stress(w, 0.99) < 0 < oracle.eos_mean_stress(w, 1.01)


# ------------------------------------------------------------------ elastic response

def test_small_strain_elastic_response_is_hooke():
    """Below yield one increment gives sigma_d = 2G e_d and sigma_m = K (J - 1)."""
    m = S.aluminium_cl()
    K, G = _moduli(m)
    rng = np.random.default_rng(0)
    e = rng.normal(size=(3, 3)) * 1e-5
    e = 0.5 * (e + e.T)
    J = np.linalg.det(np.eye(3) + e)
    out, st = oracle.material_point(m, 1e-8, e[None], [J])
    ed = e - np.trace(e) / 3 * np.eye(3)
    assert np.allclose(out[0, :9], (2 * G * ed).ravel(), rtol=1e-13, atol=1e-6)
    assert out[0, 9] == pytest.approx(K * (J - 1), rel=1e-14)
    assert out[0, 10] == 0.0 and st == 0


# ------------------------------------------------------------------ Algorithm 1

@pytest.mark.parametrize("nsteps", [7, 40, 300])
def test_perfect_plasticity_pure_shear_closed_form(nsteps):
    """With B = 0 radial return is exact for proportional loading: the shear
    stress is min(G gamma, A/sqrt(3)) at every step, whatever the step size,
    and eps_p = (gamma - tau/G)/sqrt(3)."""
    m = S.material(B=0.0, damage=0)
    K, G = _moduli(m)
    gmax = 0.05
    dg = gmax / nsteps
    deps = np.repeat(shear_increment(dg)[None], nsteps, 0)
    out, _ = oracle.material_point(m, 1e-7, deps, np.ones(nsteps))
    gam = dg * np.arange(1, nsteps + 1)
    tau = np.minimum(G * gam, m["A"] / math.sqrt(3))
    assert np.allclose(out[:, 1], tau, rtol=1e-12)
    assert np.allclose(out[:, 10], (gam - tau / G) / math.sqrt(3), rtol=1e-9, atol=1e-15)


def _exact_jc_shear(m, gam):
    """Continuous JC pure-shear response: tau = sigma_f(eps_p)/sqrt(3) with
    eps_p = (gamma - tau/G)/sqrt(3), solved by Brent's method."""
    K, G = _moduli(m)
    ty = m["A"] / math.sqrt(3)
    if G * gam <= ty:
        return G * gam

    def res(tau):
        ep = (gam - tau / G) / math.sqrt(3)
        return tau - (m["A"] + m["B"] * ep ** m["n"]) / math.sqrt(3)
    return scipy.optimize.brentq(res, ty, G * gam, xtol=1e-6, rtol=1e-15)


def test_jc_radial_return_converges_to_continuous_response():
    """Algorithm 1 evaluates sigma_f at eps_p^n (explicit), so it converges at
    first order to the continuous Johnson-Cook pure-shear curve."""
    m = S.material(damage=0)
    gmax = 0.08
    errs = []
    for nsteps in (400, 800, 1600, 3200):
        dg = gmax / nsteps
        deps = np.repeat(shear_increment(dg)[None], nsteps, 0)
        out, _ = oracle.material_point(m, 1e-7, deps, np.ones(nsteps))
        errs.append(abs(out[-1, 1] - _exact_jc_shear(m, gmax)) / _exact_jc_shear(m, gmax))
    rates = [errs[k] / errs[k + 1] for k in range(3)]
    assert all(1.7 < r < 2.3 for r in rates), (errs, rates)
    assert errs[-1] < 2e-4


def test_plastic_return_lands_on_yield_surface_and_is_radial():
    m = S.material(damage=0)
    K, G = _moduli(m)
    rng = np.random.default_rng(5)
    e = rng.normal(size=(3, 3)) * 3e-3
    e = 0.5 * (e + e.T)
    sd0 = rng.normal(size=(3, 3)) * 50e6
    sd0 = 0.5 * (sd0 + sd0.T)
    sd0 -= np.trace(sd0) / 3 * np.eye(3)
    out, _ = oracle.material_point(m, 1e-7, e[None], [1.0], init={"sd": sd0, "ep": 0.01})
    sd = out[0, :9].reshape(3, 3)
    seq = math.sqrt(1.5 * np.sum(sd * sd))
    sf = m["A"] + m["B"] * 0.01 ** m["n"]
    assert seq == pytest.approx(sf, rel=1e-13)
    trial = sd0 + 2 * G * (e - np.trace(e) / 3 * np.eye(3))
    assert np.allclose(sd / np.linalg.norm(sd), trial / np.linalg.norm(trial), atol=1e-14)
    tseq = math.sqrt(1.5 * np.sum(trial * trial))
    assert out[0, 10] - 0.01 == pytest.approx((tseq - sf) / (3 * G), rel=1e-12)


def test_rate_term_is_non_negative_log():
    m = S.material(C=0.002, epsdot0=1.0)
    base = oracle.flow_stress(m, 0.02, 0.0)
    assert oracle.flow_stress(m, 0.02, 0.5) == base          # below the reference rate
    assert oracle.flow_stress(m, 0.02, 1e3) == pytest.approx(base * (1 + 0.002 * math.log(1e3)), rel=1e-14)
    assert oracle.flow_stress(m, 0.02, 0.0, D=0.3) == pytest.approx(0.7 * base, rel=1e-15)


# ------------------------------------------------------------------ damage (Sec. 5.1-5.3)

def test_cockcroft_latham_pure_shear_closed_form():
    """Perfectly plastic pure shear keeps sigma_1 = tau = A/sqrt(3) on every
    plastic step, so D_init = (A/sqrt(3)) eps_p / W_cr exactly."""
    m = S.material(B=0.0, damage=S.DAMAGE_CL, Wcr=5e6)
    nsteps = 200
    deps = np.repeat(shear_increment(0.03 / nsteps)[None], nsteps, 0)
    out, _ = oracle.material_point(m, 1e-7, deps, np.ones(nsteps))
    ep, dinit = out[:, 10], out[:, 12]
    assert np.allclose(dinit, (m["A"] / math.sqrt(3)) * ep / m["Wcr"], rtol=1e-12, atol=1e-15)


def test_johnson_cook_damage_closed_form_fixed_triaxiality():
    """At fixed J (constant mean stress) and perfect plasticity the triaxiality
    is K(J-1)/A after yield, so D_init = eps_p / (D1 + D2 exp(D3 sigma*))."""
    m = S.material(B=0.0, damage=S.DAMAGE_JC, D1=0.05, D2=0.4, D3=-1.5)
    K, _ = _moduli(m)
    J = 1.0 + 0.5 * m["A"] / K        # sigma* = 0.5
    nsteps = 300
    deps = np.repeat(shear_increment(0.05 / nsteps)[None], nsteps, 0)
    out, _ = oracle.material_point(m, 1e-7, deps, np.full(nsteps, J))
    ef = 0.05 + 0.4 * math.exp(-1.5 * 0.5)
    pl = out[:, 10] > 0
    assert np.allclose(out[pl, 12], out[pl, 10] / ef, rtol=1e-9)


def test_damage_evolution_and_failure():
    """D = 10 (D_init - 1) once D_init >= 1 (Sec. 5.3); at D = 1 the particle
    fails and carries no stress."""
    m = S.material(B=0.0, damage=S.DAMAGE_JC, D1=0.01, D2=0.0, D3=0.0)
    nsteps = 400
    deps = np.repeat(shear_increment(0.04 / nsteps)[None], nsteps, 0)
    out, _ = oracle.material_point(m, 1e-7, deps, np.ones(nsteps))
    dinit, D, failed = out[:, 12], out[:, 13], out[:, 15]
    alive = failed == 0
    expect = np.where(dinit >= 1, np.minimum(1.0, 10 * (dinit - 1)), 0.0)
    assert np.allclose(D[alive], expect[alive], rtol=0, atol=1e-14)
    k = int(np.argmax(failed))
    assert failed[k] == 1 and dinit[k] >= 1.1 and dinit[k - 1] < 1.1
    assert np.all(out[k:, :10] == 0.0) and np.all(D[k:] == 1.0)


def test_damage_is_monotone_under_cyclic_loading():
    rng = np.random.default_rng(9)
    for dmg, extra in ((S.DAMAGE_CL, dict(Wcr=2e6)), (S.DAMAGE_JC, dict(D1=0.02, D2=0.05, D3=-1.5))):
        m = S.material(damage=dmg, **extra)
        n = 600
        deps = np.zeros((n, 3, 3))
        amp = 2e-3 * np.sin(np.arange(n) / 15.0)
        for k in range(n):
            e = rng.normal(size=(3, 3)) * 2e-4 + np.diag([amp[k], -0.5 * amp[k], -0.5 * amp[k]])
            deps[k] = 0.5 * (e + e.T)
        J = 1 + 0.01 * np.sin(np.arange(n) / 10.0)
        out, _ = oracle.material_point(m, 1e-7, deps, J)
        for c in (10, 12, 13, 15):
            assert np.all(np.diff(out[:, c]) >= 0)


# ------------------------------------------------------------------ GTN (Sec. 5.4, Algorithm 2)

def gtn(**kw):
    base = dict(damage=S.DAMAGE_GTN, fN=0.0, komega=0.0)
    base.update(kw)
    return S.material(**base)


def test_gtn_without_voids_is_consistent_linear_hardening_return():
    """f = 0 makes x = 1 and Algorithm 2 the consistent J2 return; with n = 1
    the plastic increment is (s_eq_trial - sigma_f(eps_n)) / (3G + B)."""
    m = gtn(n=1.0, B=500e6)
    K, G = _moduli(m)
    ep0 = 0.02
    e = shear_increment(0.01)
    out, st = oracle.material_point(m, 1e-7, e[None], [1.0], init={"ep": ep0, "f": 0.0})
    tseq = math.sqrt(3) * G * 0.01
    expect = (tseq - (m["A"] + m["B"] * ep0)) / (3 * G + m["B"])
    assert out[0, 10] - ep0 == pytest.approx(expect, rel=1e-12)
    assert st == 0


def test_gtn_pure_shear_yield_ratio_is_one_minus_damage():
    """With zero triaxiality cosh = 1 and the yield function gives
    x = 1 - q1 f* (Eq. yield_GTN_2 with D = q1 f*)."""
    m = gtn()
    for fs in (0.0, 0.001, 0.05, 0.3):
        x, _ = oracle.gtn_solve_x(m, fs, 0.0, 1.0)
        assert x == pytest.approx(1 - m["q1"] * fs, rel=1e-14)


def test_gtn_x_root_matches_bracketed_root_of_damage_form():
    """Newton's x is the unique positive root of Eq. (yield_GTN_2),
    x^2 + 2 D cosh(1.5 q2 sigma* x) - (1 + D^2) with D = q1 f*."""
    m = gtn()
    rng = np.random.default_rng(1)
    for _ in range(100):
        fs = rng.uniform(0, 0.6)
        tri = rng.uniform(-3, 3)
        D = m["q1"] * fs

        def phi(x):
            return x * x + 2 * D * math.cosh(1.5 * m["q2"] * tri * x) - (1 + D * D)
        ref = scipy.optimize.brentq(phi, 0.0, 1.0, xtol=1e-16, rtol=1e-15)
        x, its = oracle.gtn_solve_x(m, fs, tri, 1.0)
        assert abs(x - ref) <= 1e-13 and its < 50


def _gtn_state_after(m, e, J, f, ep=0.0, sd=None):
    init = {"f": f, "ep": ep, "D": m["q1"] * oracle.gtn_fstar(m, f)}
    if sd is not None:
        init["sd"] = sd
    out, st = oracle.material_point(m, 1e-7, e[None], [J], init=init)
    return out[0], st


def test_gtn_return_keeps_triaxiality_and_plastic_work_balance():
    """After the return the triaxiality equals the trial one (the assumption
    of the derivation), and the matrix and macroscopic plastic work agree:
    (1-f) sigma_M d eps_M = sigma_y (d eps_p^eq + sigma* tr d eps_p)."""
    m = gtn(fN=0.04)
    K, G = _moduli(m)
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(50):
        e = rng.normal(size=(3, 3)) * 4e-3
        e = 0.5 * (e + e.T)
        J = 1 + rng.uniform(-2e-3, 4e-3)
        f = rng.uniform(0.001, 0.1)
        ep = rng.uniform(0, 0.2)
        D = m["q1"] * oracle.gtn_fstar(m, f)
        out, st = _gtn_state_after(m, e, J, f, ep)
        dem = out[10] - ep
        if dem <= 0:
            continue
        ed = e - np.trace(e) / 3 * np.eye(3)
        trial = 2 * G * (1 - D) * ed
        tseq = math.sqrt(1.5 * np.sum(trial * trial))
        sm_tr = oracle.eos_mean_stress(m, J, D)
        tri = sm_tr / tseq
        sd = out[:9].reshape(3, 3)
        seq = math.sqrt(1.5 * np.sum(sd * sd))
        assert out[9] / seq == pytest.approx(tri, rel=1e-11, abs=1e-12)
        sM = m["A"] + m["B"] * out[10] ** m["n"]
        x = seq / sM
        depeq = (tseq - seq) / (3 * G * (1 - D))
        alpha = 1.5 / x * m["q1"] * m["q2"] * f * math.sinh(1.5 * m["q2"] * tri * x)
        lhs = (1 - f) * sM * dem
        rhs = seq * (depeq + tri * alpha * depeq)
        assert lhs == pytest.approx(rhs, rel=1e-10)
        checked += 1
    assert checked > 20


def test_gtn_nucleation_integrates_to_normal_cdf():
    """In pure shear with k_omega = 0 only nucleation changes f; summed over
    small steps it approaches f_N [Phi((eps - eps_N)/s_N) - Phi(-eps_N/s_N)]."""
    m = gtn(fN=0.04, eN=0.05, sN=0.02, B=0.0)
    nsteps = 3000
    deps = np.repeat(shear_increment(0.3 / nsteps)[None], nsteps, 0)
    out, st = oracle.material_point(m, 1e-7, deps, np.ones(nsteps), init={"f": 0.0})
    ep = out[-1, 10]
    expect = 0.04 * (scipy.stats.norm.cdf((ep - 0.05) / 0.02) - scipy.stats.norm.cdf(-0.05 / 0.02))
    assert out[-1, 14] == pytest.approx(expect, rel=5e-3)
    assert np.all(np.diff(out[:, 14]) >= 0)


def test_gtn_omega_special_cases():
    """omega = 0 for an axisymmetric deviator and 1 for pure shear (Eq. omega)."""
    K = 1.0
    ax = np.diag([2.0, -1.0, -1.0])
    assert oracle.gtn_omega(ax, math.sqrt(1.5 * np.sum(ax * ax)), K) == pytest.approx(0.0, abs=1e-14)
    sh = np.diag([1.0, -1.0, 0.0])
    assert oracle.gtn_omega(sh, math.sqrt(1.5 * np.sum(sh * sh)), K) == pytest.approx(1.0, abs=1e-14)


def test_gtn_void_fraction_function():
    m = gtn()
    assert oracle.gtn_fstar(m, 0.1) == 0.1
    assert oracle.gtn_fstar(m, m["fc"]) == pytest.approx(m["fc"])
    assert oracle.gtn_fstar(m, m["fF"]) == pytest.approx(1 / m["q1"])
    mid = 0.5 * (m["fc"] + m["fF"])
    assert oracle.gtn_fstar(m, mid) == pytest.approx(0.5 * (m["fc"] + 1 / m["q1"]))


def test_gtn_growth_sign_and_failure():
    """Hydrostatic tension grows voids; the porosity saturates at f_F, where
    D = 1 and the point fails."""
    m = gtn(fN=0.0)
    K, G = _moduli(m)
    n = 400
    e = np.diag([3e-3, 3e-3, 3e-3]) + shear_increment(2e-3)
    deps = np.repeat(e[None], n, 0)
    J = np.cumprod(np.full(n, np.linalg.det(np.eye(3) + e)))
    out, st = oracle.material_point(m, 1e-7, deps, J, init={"f": 0.01, "D": 1.5 * 0.01})
    f = out[:, 14]
    alive = out[:, 15] == 0
    assert np.all(np.diff(f[alive]) >= 0) and f[alive][-1] > 0.01
    assert out[-1, 15] == 1 and out[-1, 13] == 1.0 and f[-1] == m["fF"]
