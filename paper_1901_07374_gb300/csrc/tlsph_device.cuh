// Device-side building blocks of the TLSPH step: the cubic-spline kernel,
// 3x3 algebra on registers, the polar decomposition, the largest principal
// stress and the constitutive + damage update of one particle.
//
// Paper passages: kernel gradient (Sec. 2.2, Eq. SPH_gradient_kernel),
// equation of state (Sec. 4, Eq. pH), Johnson-Cook flow stress and radial
// return (Sec. 4, Eq. JC_viscoplastic_model, Algorithm 1), Cockcroft-Latham
// (Sec. 5.1), Johnson-Cook damage (Sec. 5.2), damage evolution (Sec. 5.3),
// GTN yield, void fraction function, nucleation, growth and return
// (Sec. 5.4, Eqs. yield_GTN, void_fraction_function, GTN_damage_nucleation,
// GTN_damage_growth, omega, Algorithm 2).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tlsph_internal.cuh"

namespace tlsph {

// ---------------------------------------------------------------- kernel
// M4 cubic spline in q = r / h, support q < 2.  Returned without the
// normalisation 1/(pi h^3) (value) or 1/(pi h^4) (derivative): callers fold
// those constants into their per-row factors.
__device__ __forceinline__ double spline_w(double q)
{
    if (q < 1.0) return 1.0 - q * q * (1.5 - 0.75 * q);
    if (q < 2.0) { double t = 2.0 - q; return 0.25 * t * t * t; }
    return 0.0;
}
__device__ __forceinline__ double spline_dw(double q)
{
    if (q < 1.0) return q * (2.25 * q - 3.0);
    if (q < 2.0) { double t = 2.0 - q; return -0.75 * t * t; }
    return 0.0;
}
__device__ __forceinline__ float spline_w(float q)
{
    if (q < 1.0f) return 1.0f - q * q * (1.5f - 0.75f * q);
    if (q < 2.0f) { float t = 2.0f - q; return 0.25f * t * t * t; }
    return 0.0f;
}
__device__ __forceinline__ float spline_dw(float q)
{
    if (q < 1.0f) return q * (2.25f * q - 3.0f);
    if (q < 2.0f) { float t = 2.0f - q; return -0.75f * t * t; }
    return 0.0f;
}

// grip ramp of Sec. 6: a prescribed velocity v_bc holds as v_bc (1 - exp(-t / tau))
// at time t; tau = 0 keeps it constant
__device__ __forceinline__ double grip_factor(double tau, double t) { return tau > 0.0 ? -expm1(-t / tau) : 1.0; }

// Velocity-Verlet half kick v + h (f / m) (f / m as f times the stored 1/m) and
// drift u + dt v, each rounding written out, so that every kernel that forms
// them -- the predictor, the FP64 and mixed pass-2 epilogues in any launch
// form -- produces the same bits whatever multiply-adds the compiler would
// otherwise fuse (a state reloaded from a checkpoint then continues exactly
// like the uninterrupted run)
__device__ __forceinline__ double kick(double v, double h, double f, double inv_m)
{
    return __fma_rn(h, __dmul_rn(f, inv_m), v);
}
__device__ __forceinline__ double drift(double u, double dt, double v) { return __fma_rn(dt, v, u); }

// ---------------------------------------------------------------- 3x3 algebra
struct M3 { double a[9]; };

__device__ __forceinline__ double det3(const double *m)
{
    return m[0] * (m[4] * m[8] - m[5] * m[7]) + m[1] * (m[5] * m[6] - m[3] * m[8])
         + m[2] * (m[3] * m[7] - m[4] * m[6]);
}

// cofactor matrix: cof(M) = det(M) M^{-T}
__device__ __forceinline__ void cof3(const double *m, double *c)
{
    c[0] = m[4] * m[8] - m[5] * m[7];
    c[1] = m[5] * m[6] - m[3] * m[8];
    c[2] = m[3] * m[7] - m[4] * m[6];
    c[3] = m[2] * m[7] - m[1] * m[8];
    c[4] = m[0] * m[8] - m[2] * m[6];
    c[5] = m[1] * m[6] - m[0] * m[7];
    c[6] = m[1] * m[5] - m[2] * m[4];
    c[7] = m[2] * m[3] - m[0] * m[5];
    c[8] = m[0] * m[4] - m[1] * m[3];
}

__device__ __forceinline__ void mul3(const double *a, const double *b, double *c)
{
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            c[3 * k + l] = a[3 * k] * b[l] + a[3 * k + 1] * b[3 + l] + a[3 * k + 2] * b[6 + l];
}

// c = a b^T
__device__ __forceinline__ void mul3_bt(const double *a, const double *b, double *c)
{
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            c[3 * k + l] = a[3 * k] * b[3 * l] + a[3 * k + 1] * b[3 * l + 1] + a[3 * k + 2] * b[3 * l + 2];
}

// symmetric 6-vector (xx, yy, zz, xy, yz, zx) <-> full
__device__ __forceinline__ void sym_to_full(const double *s, double *m)
{
    m[0] = s[0]; m[4] = s[1]; m[8] = s[2];
    m[1] = m[3] = s[3];
    m[5] = m[7] = s[4];
    m[2] = m[6] = s[5];
}

__device__ __forceinline__ double sym_ddot(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + 2.0 * (a[3] * b[3] + a[4] * b[4] + a[5] * b[5]);
}

__device__ __forceinline__ double sym_det(const double *s)
{
    return s[0] * (s[1] * s[2] - s[4] * s[4]) - s[3] * (s[3] * s[2] - s[4] * s[5])
         + s[5] * (s[3] * s[4] - s[1] * s[5]);
}

// Q^T S Q for symmetric S (6) and a general Q: result symmetric (6)
__device__ __forceinline__ void sym_rotate_t(const double *Q, const double *s, double *out)
{
    double S[9], T[9];
    sym_to_full(s, S);
    // T = S Q
    mul3(S, Q, T);
    // out = Q^T T
#define QTT(k, l) (Q[k] * T[l] + Q[3 + k] * T[3 + l] + Q[6 + k] * T[6 + l])
    out[0] = QTT(0, 0); out[1] = QTT(1, 1); out[2] = QTT(2, 2);
    out[3] = QTT(0, 1); out[4] = QTT(1, 2); out[5] = QTT(2, 0);
#undef QTT
}

// Q S Q^T for symmetric S (6)
__device__ __forceinline__ void sym_rotate(const double *Q, const double *s, double *out)
{
    double S[9], T[9];
    sym_to_full(s, S);
    mul3_bt(S, Q, T);       // T = S Q^T
#define QT(k, l) (Q[3 * k] * T[l] + Q[3 * k + 1] * T[3 + l] + Q[3 * k + 2] * T[6 + l])
    out[0] = QT(0, 0); out[1] = QT(1, 1); out[2] = QT(2, 2);
    out[3] = QT(0, 1); out[4] = QT(1, 2); out[5] = QT(2, 0);
#undef QT
}

// Rotation factor of the polar decomposition F = R U by Newton's iteration
// X <- (g X + X^{-T} / g) / 2 with the determinant scaling g = |det X|^{-1/3}
// (N. J. Higham, "Computing the polar decomposition -- with applications",
// SIAM J. Sci. Stat. Comput. 7, 1986).  Converges quadratically; the loop
// stops once a step moves X by less than 1e-10 (the next iterate is then
// exact to rounding) and is capped at 30 steps (status bit on the cap).
__device__ __forceinline__ bool polar_rotation(const double *F, double *R)
{
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = F[k];
    bool last = false;
    for (int it = 0; it < 30; ++it) {
        double c[9];
        cof3(R, c);
        double d = R[0] * c[0] + R[1] * c[1] + R[2] * c[2];
        double g = rcbrt(fabs(d));
        double ginv_d = 1.0 / (g * d);
        double diff = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double xn = 0.5 * (g * R[k] + c[k] * ginv_d);
            double e = xn - R[k];
            diff += e * e;
            R[k] = xn;
        }
        if (last) return true;
        if (diff < 1e-20) last = true;
    }
    return false;
}

// Largest eigenvalue of a symmetric 3x3 (6) by the trigonometric solution of
// the characteristic cubic (O. K. Smith, "Eigenvalues of a symmetric 3x3
// matrix", Commun. ACM 4, 1961).
__device__ __forceinline__ double sym_max_eig(const double *s)
{
    double q = (s[0] + s[1] + s[2]) * (1.0 / 3.0);
    double p1 = s[3] * s[3] + s[4] * s[4] + s[5] * s[5];
    double a = s[0] - q, b = s[1] - q, c = s[2] - q;
    double p2 = a * a + b * b + c * c + 2.0 * p1;
    if (p2 <= 0.0) return q;
    double p = sqrt(p2 * (1.0 / 6.0));
    double ip = 1.0 / p;
    double B[6] = { a * ip, b * ip, c * ip, s[3] * ip, s[4] * ip, s[5] * ip };
    double r = 0.5 * sym_det(B);
    r = fmin(1.0, fmax(-1.0, r));
    double phi = acos(r) * (1.0 / 3.0);
    return q + 2.0 * p * cos(phi);
}

// ---------------------------------------------------------------- material point
struct MPState {
    double sd[6];   // unrotated stress deviator
    double sm;      // mean stress
    double ep, epdot, dinit, D, f;
    double e;       // specific internal energy at the start of the update (enters the EOS)
    int failed;
};

__device__ __forceinline__ double vm_eq(const double *s) { return sqrt(1.5 * sym_ddot(s, s)); }

// tension-positive mean stress from the equation of state (Eq. pH): the
// Mie-Grueneisen pressure with eta = 1/J, negated; the tensile branch is
// scaled by (1 - D).  eos 0 is its S_alpha = Gamma0 = 0 case K (J - 1).
__device__ __forceinline__ double eos_sm(const DevMat &m, double J, double D, double e)
{
    double sm;
    if (m.eos == 0) {
        sm = m.K * (J - 1.0);
    } else {
        double eta = 1.0 / J, mu = eta - 1.0;
        double den = eta - m.S_alpha * mu;
        // the energy term of Eq. pH read as Gamma0 rho0 e with e per unit mass
        sm = -(m.rho0c02 * mu * (eta - 0.5 * m.Gamma0 * mu) / (den * den) + m.g0rho0 * e);
    }
    return sm > 0.0 ? sm * (1.0 - D) : sm;
}

// Johnson-Cook strain-rate factor with the normalised rate clamped at 1
__device__ __forceinline__ double jc_rate(const DevMat &m, double epdot)
{
    if (m.C == 0.0 || m.inv_epsdot0 <= 0.0) return 1.0;
    const double r = epdot * m.inv_epsdot0;
    return r > 1.0 ? 1.0 + m.C * log(r) : 1.0;   // log(1) = 0 exactly below the reference rate
}
__device__ __forceinline__ double jc_hard(const DevMat &m, double ep)
{
    return ep > 0.0 ? m.A + m.B * pow(ep, m.n) : m.A;
}
__device__ __forceinline__ double jc_hard_slope(const DevMat &m, double ep)
{
    return ep > 0.0 ? m.B * m.n * pow(ep, m.n - 1.0) : INFINITY;
}

__device__ __forceinline__ double gtn_fstar(const DevMat &m, double f)
{
    if (f <= m.fc) return f;
    if (f >= m.fF) return 1.0 / m.q1;
    return m.fc + m.fstar_slope * (f - m.fc);
}

// Single-precision starting points for the two Newton solves of Algorithm 2
// (the mixed path).  Each returns a value <= 0 when its iteration does not
// settle; the FP64 iteration then starts where it does without a seed.  The
// FP64 iteration that follows keeps its own convergence test, so a seed only
// shortens it: from a start within FP32 rounding of the root, Newton's
// quadratic convergence reaches the FP64 tolerance in one or two steps.
//
// First solve: x with x^2 + 2 q1 f* cosh(a1 x) - c0 = 0 (Eq. yield_GTN_2 at
// fixed triaxiality), convex and increasing on x > 0.
__device__ __forceinline__ float gtn_x_seed32(float a1, float q1f2, float c0, float x)
{
    for (int it = 0; it < 20; ++it) {
        const float e = expf(a1 * x), ie = 1.0f / e;
        const float phi = x * x + q1f2 * (0.5f * (e + ie)) - c0;
        const float dphi = 2.0f * x + q1f2 * a1 * (0.5f * (e - ie));
        const float dx = -phi / dphi;
        x += dx;
        if (!(x > 0.0f) || !isfinite(x)) return -1.0f;
        if (fabsf(dx) <= 1e-5f * x) return x;
    }
    return -1.0f;
}
// Second solve: de with de - kf (seq - x rate sigma_hard(ep0 + de)) = 0,
// written as g(de) = de - r0kf + xrk dH(de) with r0kf = (seq - x rate
// sigma_hard(ep0)) kf, xrk = x rate kf and the hardening increment
// dH(de) = sigma_hard(ep0 + de) - sigma_hard(ep0): H0 ((1 + de/ep0)^n - 1)
// with H0 = B ep0^n, or B de^n at ep0 = 0.  In this form no FP32 sum
// ep0 + de and no difference of two flow stresses is rounded, so the seed is
// accurate to FP32 rounding of de itself.  g is increasing with its root in
// [0, r0kf]; Newton steps that leave the bracket are replaced by bisection.
__device__ __forceinline__ float gtn_de_seed32(float ep0, float H0, float B, float n, float r0kf, float xrk)
{
    float lo = 0.0f, hi = r0kf, de = r0kf;
    for (int it = 0; it < 40; ++it) {
        const float dH = ep0 > 0.0f ? H0 * expm1f(n * log1pf(de / ep0)) : (de > 0.0f ? B * powf(de, n) : 0.0f);
        const float g = de - r0kf + xrk * dH;
        if (g > 0.0f) hi = de; else lo = de;
        const float ep = ep0 + de;
        const float gp = 1.0f + xrk * n * (H0 + dH) / ep;
        float dn = de - g / gp;
        if (!(dn > lo && dn < hi)) dn = 0.5f * (lo + hi);
        const float stp = dn - de;
        de = dn;
        if (!isfinite(de)) return -1.0f;
        if (fabsf(stp) <= 1e-5f * de || hi - lo <= 1e-6f * r0kf) return de;
    }
    return -1.0f;
}

// Algorithm 2.  Returns the matrix plastic strain increment.  SEED32 starts
// both Newton solves from their single-precision seeds (above), takes cosh
// and sinh of the first solve from one exponential, and the hardening slope
// of the second from the identity B n e^(n-1) = n (sigma_hard(e) - A) / e
// (one pow per step); the FP64 convergence tests are unchanged.
template <bool SEED32 = false>
__device__ __forceinline__ double gtn_update(const DevMat &m, double dt, const double *ed, double J,
                                            MPState &s, uint32_t &status)
{
    const double D = s.D, omD = 1.0 - D, f = s.f;
    const double fs = gtn_fstar(m, f);
    const double sm_tr = eos_sm(m, J, D, s.e);
    double tr[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) tr[k] = s.sd[k] + 2.0 * m.G * omD * ed[k];
    const double seq = vm_eq(tr);
    bool elastic = seq < 1e-12 * m.K;
    double tri = 0.0, rate = 1.0, sM = 0.0;
    double h0 = 0.0;
    if (!elastic) {
        tri = sm_tr / seq;
        rate = jc_rate(m, s.epdot);
        h0 = jc_hard(m, s.ep);
        sM = h0 * rate;
        double xt = seq / sM;
        double phi = xt * xt + 2.0 * m.q1 * fs * cosh(1.5 * m.q2 * tri * xt) - (1.0 + m.q3 * fs * fs);
        elastic = phi <= 0.0;
    }
    if (elastic) {
#pragma unroll
        for (int k = 0; k < 6; ++k) s.sd[k] = tr[k];
        s.sm = sm_tr;
        s.epdot = 0.0;
        return 0.0;
    }
    // x = sigma_y / sigma_M at fixed triaxiality (first Newton solve)
    const double a1 = 1.5 * m.q2 * tri;
    const double c0 = 1.0 + m.q3 * fs * fs;
    double x = fmin(1.0, seq / sM);
    if (SEED32) {
        const float xs = gtn_x_seed32((float)a1, (float)(2.0 * m.q1 * fs), (float)c0, (float)x);
        if (xs > 0.0f) x = (double)xs;
    }
    bool conv = false;
    for (int it = 0; it < 50; ++it) {
        double ch, sh;
        if (SEED32) {
            const double e = exp(a1 * x), ie = 1.0 / e;
            ch = 0.5 * (e + ie);
            sh = 0.5 * (e - ie);   // enters the derivative only
        } else {
            sh = sinh(a1 * x);
            ch = cosh(a1 * x);
        }
        double phi = x * x + 2.0 * m.q1 * fs * ch - c0;
        double dphi = 2.0 * x + 2.0 * m.q1 * fs * a1 * sh;
        double dx = -phi / dphi;
        x += dx;
        if (fabs(dx) <= 1e-14) { conv = true; break; }
    }
    if (!conv) status |= TLSPH_ST_NEWTON_CAP;
    const double shx = sinh(a1 * x);
    const double kf = (x + 1.5 * m.q1 * m.q2 * f * tri * shx) / (3.0 * m.G * omD * (1.0 - f));
    // matrix strain increment: root of g(de) = de - (seq - x sigma_f(ep + de)) kf,
    // Newton steps kept inside the bracket [lo, hi] (bisection otherwise)
    const double ep0 = s.ep;
    double de = (seq - x * sM) * kf;
    double lo = 0.0, hi = fmax(de, 0.0);
    const double tol = 1e-14 * (seq * kf + fabs(de));
    if (SEED32 && de > 0.0) {
        const float ds = gtn_de_seed32((float)ep0, (float)(h0 - m.A), (float)m.B, (float)m.n, (float)de,
                                       (float)(x * rate * kf));
        if (ds > 0.0f && (double)ds < hi) de = (double)ds;
    }
    conv = false;
    for (int it = 0; it < 50; ++it) {
        const double ep = ep0 + de;
        const double h = jc_hard(m, ep);
        double g = de - (seq - x * h * rate) * kf;
        if (g > 0.0) hi = de; else lo = de;
        const double slope = SEED32 ? (ep > 0.0 ? m.n * (h - m.A) / ep : INFINITY) : jc_hard_slope(m, ep);
        double gp = 1.0 + x * slope * rate * kf;
        double dn = de - g / gp;
        if (!(dn > lo && dn < hi)) dn = 0.5 * (lo + hi);
        double stp = dn - de;
        de = dn;
        if (fabs(stp) <= tol || hi - lo <= tol) { conv = true; break; }
    }
    if (!conv) status |= TLSPH_ST_NEWTON_CAP;
    s.ep = ep0 + de;
    const double sMn = jc_hard(m, s.ep) * rate;
    const double sy = x * sMn;
    const double scale = sy / seq;
#pragma unroll
    for (int k = 0; k < 6; ++k) s.sd[k] = scale * tr[k];
    const double depeq = (seq - sy) / (3.0 * m.G * omD);
    s.sm = sm_tr - 3.0 * m.G * omD * tri * depeq;
    const double alpha = 1.5 * (sMn / sy) * m.q1 * m.q2 * f * shx;
    double om = 0.0;
    if (m.komega != 0.0) {
        double r = 27.0 * sym_det(tr) / (2.0 * seq * seq * seq);
        om = fmin(1.0, fmax(0.0, 1.0 - r * r));
    }
    const double z = (s.ep - m.eN) / m.sN;
    const double nucl = m.nucl_coef * exp(-0.5 * z * z) * de;
    const double grow = (1.0 - f) / (alpha * tri + 1.0) * (sMn / sy) * (alpha * (1.0 - f) + f * m.komega * om) * de;
    s.f = fmin(m.fF, fmax(0.0, f + nucl + grow));
    s.epdot = de / dt;
    return de;
}

// Constitutive and damage update of one particle from the symmetric strain
// increment de (unrotated frame) and J = det F^{n+1}.  D^n enters, D^{n+1}
// leaves.  Returns status bits.
template <bool SEED32 = false>
__device__ __forceinline__ uint32_t material_update(const DevMat &m, double dt, const double *de, double J,
                                                    MPState &s)
{
    uint32_t status = 0;
    if (s.failed) return 0;
    const double trc = (de[0] + de[1] + de[2]) * (1.0 / 3.0);
    const double ed[6] = { de[0] - trc, de[1] - trc, de[2] - trc, de[3], de[4], de[5] };
    double dep;
    if (m.damage == TLSPH_DAMAGE_GTN) {
        dep = gtn_update<SEED32>(m, dt, ed, J, s, status);
    } else {
        // Algorithm 1: elastic trial, von Mises check, radial scale-back
        const double omD = 1.0 - s.D;
        double tr[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) tr[k] = s.sd[k] + 2.0 * m.G * omD * ed[k];
        const double s2 = 1.5 * sym_ddot(tr, tr);
        const double sf = jc_hard(m, s.ep) * jc_rate(m, s.epdot) * omD;
        dep = 0.0;
        if (s2 <= sf * sf) {            // sigma_eq <= sigma_f, decided without the square root
#pragma unroll
            for (int k = 0; k < 6; ++k) s.sd[k] = tr[k];
        } else {
            const double seq = sqrt(s2);
            dep = (seq - sf) / (3.0 * m.G * omD);
            const double sc = sf / seq;
#pragma unroll
            for (int k = 0; k < 6; ++k) s.sd[k] = sc * tr[k];
        }
        s.ep += dep;
        s.epdot = dep > 0.0 ? dep / dt : 0.0;
        s.sm = eos_sm(m, J, s.D, s.e);
    }
    // damage initiation and evolution (no plastic increment: D_init unchanged)
    if (dep == 0.0) {
    } else if (m.damage == TLSPH_DAMAGE_CL) {
        double full[6] = { s.sd[0] + s.sm, s.sd[1] + s.sm, s.sd[2] + s.sm, s.sd[3], s.sd[4], s.sd[5] };
        double s1 = sym_max_eig(full);
        s.dinit += fmax(s1, 0.0) * dep * m.inv_Wcr;
    } else if (m.damage == TLSPH_DAMAGE_JC) {
        const double seq = vm_eq(s.sd);
        const double tri = seq < 1e-12 * m.K ? 0.0 : s.sm / seq;
        const double rstar = m.inv_epsdot0 > 0.0 ? (dep / dt) * m.inv_epsdot0 : 0.0;
        double ef = (m.D1 + m.D2 * exp(m.D3 * tri));
        if (m.D4 != 0.0) ef *= pow(1.0 + rstar, m.D4);
        ef = fmax(ef, 1e-12);
        s.dinit += dep / ef;
    }
    if (m.damage == TLSPH_DAMAGE_CL || m.damage == TLSPH_DAMAGE_JC) {
        double D = 0.0;
        if (s.dinit >= 1.0) D = fmin(1.0, 10.0 * (s.dinit - 1.0));
        s.D = D;
        if (D >= 1.0) s.failed = 1;
    } else if (m.damage == TLSPH_DAMAGE_GTN) {
        if (s.f >= m.fF) { s.D = 1.0; s.failed = 1; }
        else s.D = m.q1 * gtn_fstar(m, s.f);
    }
    if (s.failed) {
#pragma unroll
        for (int k = 0; k < 6; ++k) s.sd[k] = 0.0;
        s.sm = 0.0;
    }
    return status;
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ double warp_allsum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ float warp_allsum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

}  // namespace tlsph
