/*
 * tlsph_oracle.c -- plain, slow FP64 CPU oracle of the damage-weighted
 * Total-Lagrangian SPH step of de Vaucorbeil & Hutchinson (arXiv 1901.07374).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may build, load or call it.  It shares no code, header,
 * table or helper with the CUDA library; the two are written independently
 * from the paper.
 *
 * Style: every quantity is computed from its definition, sums over a
 * neighbour row run sequentially in ascending neighbour index, and the file is
 * compiled with -O2 -ffp-contract=off (no fused multiply-add).  Nothing is
 * blocked, fused or reordered beyond what the cited equation states.
 *
 * Conventions
 *   3x3 tensors are row-major double[9]:  T[3*k + l] = T_kl.
 *   a (x) b is the dyadic product:          (a (x) b)_kl = a_k b_l.
 *   Stress is tension-positive; sigma_m is the mean stress.
 *
 * Paper passages (section / equation / algorithm):
 *   kinematics u = x - X, F = I + du/dX          Sec. 2.1, Eq. (deformation_gradient)
 *   rho J = rho_0                                  Sec. 2.1, Eq. (conservation1)
 *   kernel gradient grad W_i(X_ij)                 Sec. 2.2, Eq. (SPH_gradient_kernel)
 *   correction matrix L_i                          Sec. 2.2, Eq. (correction_matrix)
 *   damage-weighted F-dot and F                    Sec. 3.1, Eqs. (Crack_approx_Fdot), (Crack_approx_F)
 *   damage-weighted nodal forces                   Sec. 3.1, unnumbered equation after (Crack_approx_F)
 *   fully damaged particle: no stress, v = 0       Sec. 3.1, text before (Crack_approx_Fdot)
 *   stress split, equation of state                Sec. 4, Eq. (pH)
 *   Johnson-Cook flow stress                       Sec. 4, Eq. (JC_viscoplastic_model)
 *   radial return                                  Sec. 4, Algorithm 1
 *   Cockcroft-Latham                               Sec. 5.1, Eq. (cockcroft-latham)
 *   Johnson-Cook damage initiation                 Sec. 5.2
 *   damage evolution D = 10 (D_init - 1)           Sec. 5.3
 *   GTN yield, f*, D = q1 f*                       Sec. 5.4, Eqs. (yield_GTN), (void_fraction_function), (yield_GTN_2)
 *   GTN nucleation, growth, omega                  Sec. 5.4, Eqs. (GTN_damage_nucleation), (GTN_damage_growth), (omega)
 *   GTN return with two Newton solves              Sec. 5.4, Algorithm 2 and the derivation after it
 *   grip velocity ramp v_max (1 - e^{-t})          Sec. 6 (specimens and loading)
 *   internal energy de/dt = Fdot : P / rho0        Sec. 2.1, Eq. (conservation3); enters Eq. (pH)
 *
 * Where the paper is silent or garbled the oracle takes the readings listed
 * in the design notes (kernel form, integrator, frame, EOS sign, lagged rate,
 * Alg. 1 denominator, GTN nucleation exponent and pressure scale-back,
 * hourglass form).  Each reading is marked "Reading:" below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Public structs (mirrored by ctypes in oracle/__init__.py)                */
/* ------------------------------------------------------------------------ */

typedef struct {
    double rho0, E, nu;
    int32_t eos;              /* 0 = linear (Mie-Grueneisen with S=Gamma0=0), 1 = Mie-Grueneisen */
    double c0, S_alpha, Gamma0;
    double A, B, n, C, epsdot0;
    int32_t damage;           /* 0 none, 1 Cockcroft-Latham, 2 Johnson-Cook, 3 GTN */
    double Wcr;
    double D1, D2, D3, D4, D5;
    double q1, q2, q3, fN, eN, sN, fc, fF, komega;
} orc_material;

typedef struct {
    double h, rc, dt, hg_alpha;
    int32_t wall;             /* 1: rigid frictionless wall on the plane z = 0 */
    double grip_ramp;         /* tau > 0: prescribed velocities ramp up as 1 - exp(-t / tau); 0: constant */
} orc_config;

/* status bits */
#define ORC_ST_POLAR_CAP   1u
#define ORC_ST_NEWTON_CAP  2u
#define ORC_ST_BAD_J       4u
#define ORC_ST_NONFINITE   8u

/* ------------------------------------------------------------------------ */
/* Small dense helpers                                                       */
/* ------------------------------------------------------------------------ */

static void mat_mul(const double *a, const double *b, double *c)
{
    double t[9];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            double s = 0.0;
            for (int m = 0; m < 3; ++m) s += a[3 * k + m] * b[3 * m + l];
            t[3 * k + l] = s;
        }
    memcpy(c, t, sizeof t);
}

static void mat_transpose(const double *a, double *t)
{
    double r[9];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) r[3 * k + l] = a[3 * l + k];
    memcpy(t, r, sizeof r);
}

static double mat_det(const double *a)
{
    return a[0] * (a[4] * a[8] - a[5] * a[7])
         - a[1] * (a[3] * a[8] - a[5] * a[6])
         + a[2] * (a[3] * a[7] - a[4] * a[6]);
}

/* inverse by the adjugate divided by the determinant */
static int mat_inv(const double *a, double *inv)
{
    double det = mat_det(a);
    if (det == 0.0 || !isfinite(det)) return -1;
    double c[9];
    c[0] = a[4] * a[8] - a[5] * a[7];
    c[1] = a[2] * a[7] - a[1] * a[8];
    c[2] = a[1] * a[5] - a[2] * a[4];
    c[3] = a[5] * a[6] - a[3] * a[8];
    c[4] = a[0] * a[8] - a[2] * a[6];
    c[5] = a[2] * a[3] - a[0] * a[5];
    c[6] = a[3] * a[7] - a[4] * a[6];
    c[7] = a[1] * a[6] - a[0] * a[7];
    c[8] = a[0] * a[4] - a[1] * a[3];
    for (int k = 0; k < 9; ++k) inv[k] = c[k] / det;
    return 0;
}

static double frob(const double *a)
{
    double s = 0.0;
    for (int k = 0; k < 9; ++k) s += a[k] * a[k];
    return sqrt(s);
}

static double ddot9(const double *a, const double *b)
{
    double s = 0.0;
    for (int k = 0; k < 9; ++k) s += a[k] * b[k];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Kernel.  Reading: the paper gives no kernel form; the M4 cubic spline with */
/* smoothing length h and support 2h is used (3D normalisation 1/(pi h^3)).  */
/* ------------------------------------------------------------------------ */

double orc_kernel_w(double r, double h)
{
    double q = r / h;
    double s = 1.0 / (M_PI * h * h * h);
    if (q < 1.0) return s * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q < 2.0) { double t = 2.0 - q; return s * 0.25 * t * t * t; }
    return 0.0;
}

/* dW/dr */
double orc_kernel_dw(double r, double h)
{
    double q = r / h;
    double s = 1.0 / (M_PI * h * h * h * h);
    if (q < 1.0) return s * (-3.0 * q + 2.25 * q * q);
    if (q < 2.0) { double t = 2.0 - q; return s * (-0.75 * t * t); }
    return 0.0;
}

/* grad W_i(X_ij) = dW/dX_ij (X_j - X_i)/X_ij   (Eq. SPH_gradient_kernel) */
static void kernel_grad(const double *Xi, const double *Xj, double h, double *g)
{
    double d[3] = { Xj[0] - Xi[0], Xj[1] - Xi[1], Xj[2] - Xi[2] };
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double w = orc_kernel_dw(r, h);
    for (int k = 0; k < 3; ++k) g[k] = w * d[k] / r;
}

/* ------------------------------------------------------------------------ */
/* a0: neighbour sets S_i, fixed in the reference configuration (Sec. 1,     */
/* Sec. 2.2).  Definition: S_i = { j != i : |X_j - X_i| < rc }, rc = 2h.     */
/* The predicate is evaluated as ((dx*dx + dy*dy) + dz*dz) < rc*rc in FP64.  */
/* Brute force over all pairs; rows come out in ascending j.                 */
/* Returns nnz; if nnz > cap the columns are not all written (call again).   */
/* ------------------------------------------------------------------------ */

static int in_support(const double *Xi, const double *Xj, double rc2)
{
    double dx = Xj[0] - Xi[0];
    double dy = Xj[1] - Xi[1];
    double dz = Xj[2] - Xi[2];
    double r2 = (dx * dx + dy * dy) + dz * dz;
    return r2 < rc2;
}

int64_t orc_neighbors(int64_t N, const double *X, double rc,
                      int64_t *row_ptr, int32_t *col, int64_t cap)
{
    double rc2 = rc * rc;
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            if (in_support(X + 3 * i, X + 3 * j, rc2)) {
                if (nnz < cap) col[nnz] = (int32_t)j;
                ++nnz;
            }
        }
        row_ptr[i + 1] = nnz;
    }
    return nnz;
}

/* ------------------------------------------------------------------------ */
/* a1: correction matrix L_i = sum_j V_j (X_j - X_i) (x) grad W_i(X_ij)      */
/* (Eq. correction_matrix) and its inverse.  Returns the number of rows     */
/* whose L is singular (their Linv is left at zero).                        */
/* ------------------------------------------------------------------------ */

int64_t orc_shape_matrix(int64_t N, const double *X, const double *vol,
                         const int64_t *row_ptr, const int32_t *col, double h,
                         double *L_out, double *Linv_out)
{
    int64_t bad = 0;
    for (int64_t i = 0; i < N; ++i) {
        double L[9] = { 0 };
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int64_t j = col[p];
            double g[3];
            kernel_grad(X + 3 * i, X + 3 * j, h, g);
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l)
                    L[3 * k + l] += vol[j] * (X[3 * j + k] - X[3 * i + k]) * g[l];
        }
        if (L_out) memcpy(L_out + 9 * i, L, sizeof L);
        double Li[9];
        if (mat_inv(L, Li) != 0) { memset(Li, 0, sizeof Li); ++bad; }
        memcpy(Linv_out + 9 * i, Li, sizeof Li);
    }
    return bad;
}

/* corrected gradient g_ij = L_i^{-T} grad W_i(X_ij)  (row vector grad W L^{-1}) */
static void corrected_grad(const double *Linv, const double *Xi, const double *Xj,
                           double h, double *g)
{
    double w[3];
    kernel_grad(Xi, Xj, h, w);
    for (int l = 0; l < 3; ++l)
        g[l] = w[0] * Linv[0 * 3 + l] + w[1] * Linv[1 * 3 + l] + w[2] * Linv[2 * 3 + l];
}

/* ------------------------------------------------------------------------ */
/* a3: damage-weighted velocity gradient (Eq. Crack_approx_Fdot)             */
/* Fdot_i = sum_j V_j (1 - D_j) (v_j - v_i) (x) g_ij                          */
/* ------------------------------------------------------------------------ */

static void fdot_row(int64_t i, const double *X, const double *vol, const double *v,
                     const double *D, const double *Linv,
                     const int64_t *row_ptr, const int32_t *col, double h, double *Fd)
{
    memset(Fd, 0, 9 * sizeof(double));
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        int64_t j = col[p];
        double g[3];
        corrected_grad(Linv + 9 * i, X + 3 * i, X + 3 * j, h, g);
        double w = vol[j] * (1.0 - D[j]);
        for (int k = 0; k < 3; ++k) {
            double dv = v[3 * j + k] - v[3 * i + k];
            for (int l = 0; l < 3; ++l) Fd[3 * k + l] += w * dv * g[l];
        }
    }
}

void orc_velocity_gradient(int64_t N, const double *X, const double *vol, const double *v,
                           const double *D, const double *Linv,
                           const int64_t *row_ptr, const int32_t *col, double h, double *Fdot)
{
    for (int64_t i = 0; i < N; ++i)
        fdot_row(i, X, vol, v, D, Linv, row_ptr, col, h, Fdot + 9 * i);
}

/* ------------------------------------------------------------------------ */
/* a4: polar decomposition F = R U, Higham's scaled Newton iteration        */
/*   X_{k+1} = (gamma X_k + X_k^{-T} / gamma) / 2,                          */
/*   gamma = sqrt(|X_k^{-1}|_F / |X_k|_F)   (N. J. Higham, SIAM J. Sci.      */
/*   Stat. Comput. 7, 1986).  Capped at 100 iterations (status bit).        */
/* ------------------------------------------------------------------------ */

int orc_polar(const double *F, double *R, double *U)
{
    double Xk[9];
    memcpy(Xk, F, sizeof Xk);
    int ok = 0;
    for (int it = 0; it < 100; ++it) {
        double Xi[9], XiT[9], Xn[9];
        if (mat_inv(Xk, Xi) != 0) return -1;
        mat_transpose(Xi, XiT);
        double gam = sqrt(frob(Xi) / frob(Xk));
        /* once close to convergence the unscaled iteration is used */
        if (it > 0 && fabs(gam - 1.0) < 1e-3) gam = 1.0;
        for (int k = 0; k < 9; ++k) Xn[k] = 0.5 * (gam * Xk[k] + XiT[k] / gam);
        double diff[9];
        for (int k = 0; k < 9; ++k) diff[k] = Xn[k] - Xk[k];
        double dn = frob(diff), xn = frob(Xn);
        memcpy(Xk, Xn, sizeof Xk);
        if (dn <= 1e-15 * xn) { ok = 1; break; }
    }
    memcpy(R, Xk, sizeof Xk);
    if (U) {
        double RT[9], Um[9];
        mat_transpose(R, RT);
        mat_mul(RT, F, Um);
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) U[3 * k + l] = 0.5 * (Um[3 * k + l] + Um[3 * l + k]);
    }
    return ok ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Symmetric 3x3 eigenvalues by the cyclic Jacobi method (textbook).        */
/* ------------------------------------------------------------------------ */

void orc_eig_sym(const double *S, double *ev)
{
    double a[9];
    memcpy(a, S, sizeof a);
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = a[1] * a[1] + a[2] * a[2] + a[5] * a[5];
        double diag = a[0] * a[0] + a[4] * a[4] + a[8] * a[8];
        if (off <= 1e-36 * diag || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double apq = a[3 * p + q];
                if (apq == 0.0) continue;
                double app = a[3 * p + p], aqq = a[3 * q + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* a <- J^T a J with the rotation in the (p, q) plane */
                for (int k = 0; k < 3; ++k) {
                    double akp = a[3 * k + p], akq = a[3 * k + q];
                    a[3 * k + p] = c * akp - s * akq;
                    a[3 * k + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = a[3 * p + k], aqk = a[3 * q + k];
                    a[3 * p + k] = c * apk - s * aqk;
                    a[3 * q + k] = s * apk + c * aqk;
                }
            }
    }
    ev[0] = a[0]; ev[1] = a[4]; ev[2] = a[8];
}

static double max_eig(const double *S)
{
    double ev[3];
    orc_eig_sym(S, ev);
    double m = ev[0];
    if (ev[1] > m) m = ev[1];
    if (ev[2] > m) m = ev[2];
    return m;
}

/* ------------------------------------------------------------------------ */
/* Material: moduli, equation of state, flow stress                          */
/* ------------------------------------------------------------------------ */

static double bulk_modulus(const orc_material *m) { return m->E / (3.0 * (1.0 - 2.0 * m->nu)); }
static double shear_modulus(const orc_material *m) { return m->E / (2.0 * (1.0 + m->nu)); }

/* Eq. (pH).  Reading: the printed Mie-Grueneisen expression is a pressure
 * (positive in compression); the tension-positive mean stress is its
 * negative with eta = rho/rho0 = 1/J, multiplied by (1 - D) when tensile.
 * With S_alpha = Gamma0 = 0 and rho0 c0^2 = K this is sigma_m = K (J - 1)
 * exactly; the linear EOS (eos = 0) uses K = E / (3 (1 - 2 nu)).
 * e is the specific internal energy of Eq. (conservation3) at the start of
 * the step; it enters through the Gamma0 rho0 e term below. */
double orc_eos_mean_stress(const orc_material *m, double J, double D, double e)
{
    double sm;
    if (m->eos == 0) {
        sm = bulk_modulus(m) * (J - 1.0);
    } else {
        double eta = 1.0 / J;
        double mu = eta - 1.0;
        double den = eta - m->S_alpha * mu;
        /* Hugoniot part plus the energy term: Eq. pH writes Gamma0 e, which has
         * the units of a pressure only with e per unit reference volume;
         * reading: e per unit mass (Eq. conservation3), term Gamma0 rho0 e */
        double p = m->rho0 * m->c0 * m->c0 * mu * (eta - 0.5 * m->Gamma0 * mu) / (den * den)
                 + m->Gamma0 * m->rho0 * e;
        sm = -p;
    }
    if (sm > 0.0) sm *= (1.0 - D);
    return sm;
}

/* Eq. (JC_viscoplastic_model) without the (1 - D) factor, T* = 0.
 * Reading: the normalised rate is max(epsdot/epsdot0, 1) (lagged one step),
 * so the logarithm is non-negative. */
static double jc_rate_factor(const orc_material *m, double epsdot)
{
    if (m->C == 0.0 || m->epsdot0 <= 0.0) return 1.0;
    double r = epsdot / m->epsdot0;
    if (r < 1.0) r = 1.0;
    return 1.0 + m->C * log(r);
}

static double jc_hardening(const orc_material *m, double ep)
{
    return m->A + m->B * (ep > 0.0 ? pow(ep, m->n) : 0.0);
}

static double jc_hardening_slope(const orc_material *m, double ep)
{
    if (ep <= 0.0) return INFINITY;
    return m->B * m->n * pow(ep, m->n - 1.0);
}

double orc_flow_stress(const orc_material *m, double ep, double epsdot, double D)
{
    return jc_hardening(m, ep) * jc_rate_factor(m, epsdot) * (1.0 - D);
}

/* GTN void fraction function f* (Eq. void_fraction_function); beyond f_F it
 * stays at 1/q1. */
double orc_gtn_fstar(const orc_material *m, double f)
{
    if (f <= m->fc) return f;
    if (f >= m->fF) return 1.0 / m->q1;
    return m->fc + (1.0 / m->q1 - m->fc) / (m->fF - m->fc) * (f - m->fc);
}

/* Eq. (omega) for a deviator s with von Mises stress seq. */
double orc_gtn_omega(const double *s, double seq, double K)
{
    if (seq < 1e-12 * K) return 0.0;
    double r = 27.0 * mat_det(s) / (2.0 * seq * seq * seq);
    double w = 1.0 - r * r;
    if (w < 0.0) w = 0.0;
    if (w > 1.0) w = 1.0;
    return w;
}

/* ------------------------------------------------------------------------ */
/* Material-point state and the constitutive update (a5-a8)                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    double sd[9];      /* unrotated stress deviator, symmetric */
    double sm;         /* mean stress of the last update */
    double ep;         /* equivalent plastic strain (matrix strain for GTN) */
    double epdot;      /* plastic strain rate of the last step */
    double dinit;      /* damage initiation variable */
    double D;          /* damage */
    double f;          /* void volume fraction (GTN) */
    double e;          /* specific internal energy at the start of the update (enters the EOS) */
    int32_t failed;
    int32_t newton_its;/* diagnostics: iterations of the last GTN solves */
} orc_mp_state;

static void deviator(const double *e, double *ed, double *tr)
{
    double t = e[0] + e[4] + e[8];
    memcpy(ed, e, 9 * sizeof(double));
    ed[0] -= t / 3.0; ed[4] -= t / 3.0; ed[8] -= t / 3.0;
    if (tr) *tr = t;
}

static double von_mises(const double *s) { return sqrt(1.5 * ddot9(s, s)); }

/* Algorithm 1 (Johnson-Cook radial return).  Returns the plastic strain
 * increment.  Reading: Delta eps_p = (s_eq - s_f) / (3 G (1 - D)) -- the
 * printed 3G is taken with the same damaged modulus as the trial step, which
 * is what Algorithm 2 uses; sigma_f is evaluated at eps_p^n (explicit). */
static double radial_return_jc(const orc_material *m, double dt, const double *ded,
                               double D, orc_mp_state *st)
{
    double G = shear_modulus(m);
    double tr_s[9];
    for (int k = 0; k < 9; ++k) tr_s[k] = st->sd[k] + 2.0 * G * (1.0 - D) * ded[k];
    double seq = von_mises(tr_s);
    double sf = orc_flow_stress(m, st->ep, st->epdot, D);
    double dep = 0.0;
    if (seq <= sf) {
        memcpy(st->sd, tr_s, sizeof tr_s);
    } else {
        dep = (seq - sf) / (3.0 * G * (1.0 - D));
        for (int k = 0; k < 9; ++k) st->sd[k] = sf / seq * tr_s[k];
    }
    st->ep += dep;
    st->epdot = dep / dt;
    return dep;
}

/* GTN yield function in x = sigma_eq / sigma_M at fixed triaxiality and its
 * derivative (Algorithm 2, first Newton loop). */
static double gtn_phi(const orc_material *m, double fs, double tri, double x)
{
    return x * x + 2.0 * m->q1 * fs * cosh(1.5 * m->q2 * tri * x) - (1.0 + m->q3 * fs * fs);
}
static double gtn_dphi(const orc_material *m, double fs, double tri, double x)
{
    return 2.0 * x + 3.0 * m->q1 * m->q2 * fs * tri * sinh(1.5 * m->q2 * tri * x);
}

/* Algorithm 2 (GTN return).  Readings: q1^2 in the yield function is q3;
 * sigma_M is the undamaged matrix flow stress (no (1 - D) factor); the
 * nucleation term is the Chu-Needleman normal density in eps_M with its
 * square restored, times the matrix plastic strain increment; the pressure is
 * scaled back with Delta eps_p^eq = (s_eq_trial - s_y) / (3 G (1 - D)) as in
 * the derivation after the algorithm; both Newton solves are safeguarded by a
 * bracket (bisection when a Newton step leaves it) and capped at 50 steps.
 * Returns the matrix plastic strain increment. */
static double gtn_return(const orc_material *m, double dt, const double *ded, double J,
                         double D, orc_mp_state *st, unsigned *status)
{
    double G = shear_modulus(m), K = bulk_modulus(m);
    double f = st->f;
    double fs = orc_gtn_fstar(m, f);
    double sm_tr = orc_eos_mean_stress(m, J, D, st->e);
    double tr_s[9];
    for (int k = 0; k < 9; ++k) tr_s[k] = st->sd[k] + 2.0 * G * (1.0 - D) * ded[k];
    double seq = von_mises(tr_s);
    st->newton_its = 0;
    if (seq < 1e-12 * K) {           /* purely hydrostatic: elastic step */
        memcpy(st->sd, tr_s, sizeof tr_s);
        st->sm = sm_tr;
        st->epdot = 0.0;
        return 0.0;
    }
    double tri = sm_tr / seq;
    double rate = jc_rate_factor(m, st->epdot);
    double sM = jc_hardening(m, st->ep) * rate;
    double phi_tr = gtn_phi(m, fs, tri, seq / sM);
    if (phi_tr <= 0.0) {
        memcpy(st->sd, tr_s, sizeof tr_s);
        st->sm = sm_tr;
        st->epdot = 0.0;
        return 0.0;
    }
    /* first Newton loop: x = sigma_y / sigma_M on the yield surface; x lies
     * in (0, 1] and the yield function is O(1), so the stop is absolute */
    double x = seq / sM;
    if (x > 1.0) x = 1.0;
    int its = 0, conv = 0;
    for (its = 0; its < 50; ++its) {
        double dx = -gtn_phi(m, fs, tri, x) / gtn_dphi(m, fs, tri, x);
        x += dx;
        if (fabs(dx) <= 1e-14) { conv = 1; break; }
    }
    if (!conv) *status |= ORC_ST_NEWTON_CAP;
    double sh = sinh(1.5 * m->q2 * tri * x);
    double kfac = (x + 1.5 * m->q1 * m->q2 * f * tri * sh) / (3.0 * G * (1.0 - D) * (1.0 - f));
    /* second Newton loop on g(de) = de - (s_eq_tr - x sigma_f(ep + de)) kfac */
    double ep0 = st->ep;
    double lo = 0.0;
    double de = (seq - x * sM) * kfac;
    double hi = de;
    if (hi < 0.0) hi = 0.0;
    /* converged once the increment moves the stress by less than 1e-14 of
     * the trial stress (the data do not resolve it further) */
    double tol = 1e-14 * (seq * kfac + fabs(de));
    conv = 0;
    int its2;
    for (its2 = 0; its2 < 50; ++its2) {
        double sf = jc_hardening(m, ep0 + de) * rate;
        double g = de - (seq - x * sf) * kfac;
        if (g > 0.0) hi = de; else lo = de;
        double gp = 1.0 + x * jc_hardening_slope(m, ep0 + de) * rate * kfac;
        double dn = de - g / gp;
        if (!(dn > lo && dn < hi)) dn = 0.5 * (lo + hi);
        double step = dn - de;
        de = dn;
        if (fabs(step) <= tol || hi - lo <= tol) { conv = 1; break; }
    }
    if (!conv) *status |= ORC_ST_NEWTON_CAP;
    st->newton_its = its + its2;
    st->ep = ep0 + de;
    double sMn = jc_hardening(m, st->ep) * rate;
    double sy = x * sMn;
    for (int k = 0; k < 9; ++k) st->sd[k] = sy / seq * tr_s[k];
    double depeq = (seq - sy) / (3.0 * G * (1.0 - D));
    st->sm = sm_tr - 3.0 * G * (1.0 - D) * tri * depeq;
    double alpha = 1.5 * (sMn / sy) * m->q1 * m->q2 * f * sinh(1.5 * m->q2 * tri * x);
    double om = orc_gtn_omega(tr_s, seq, K);
    double z = (st->ep - m->eN) / m->sN;
    double nucl = m->fN / (m->sN * sqrt(2.0 * M_PI)) * exp(-0.5 * z * z) * de;
    double grow = (1.0 - f) / (alpha * tri + 1.0) * (sMn / sy)
                * (alpha * (1.0 - f) + f * m->komega * om) * de;
    double fn = f + nucl + grow;
    if (fn < 0.0) fn = 0.0;
    if (fn > m->fF) fn = m->fF;
    st->f = fn;
    st->epdot = de / dt;
    return de;
}

/* Damage after the return (Sec. 5.1-5.4).  sd/sm is the updated stress. */
static void damage_update(const orc_material *m, double dt, double dep, orc_mp_state *st)
{
    double K = bulk_modulus(m);
    if (m->damage == 1) {                 /* Cockcroft-Latham */
        double s[9];
        memcpy(s, st->sd, sizeof s);
        s[0] += st->sm; s[4] += st->sm; s[8] += st->sm;
        double s1 = max_eig(s);
        double pos = s1 > 0.0 ? s1 : 0.0;
        st->dinit += pos * dep / m->Wcr;
    } else if (m->damage == 2) {          /* Johnson-Cook */
        double seq = von_mises(st->sd);
        double tri = seq < 1e-12 * K ? 0.0 : st->sm / seq;
        double rstar = (m->epsdot0 > 0.0) ? (dep / dt) / m->epsdot0 : 0.0;
        double ef = (m->D1 + m->D2 * exp(m->D3 * tri)) * pow(1.0 + rstar, m->D4) * (1.0 + m->D5 * 0.0);
        if (ef < 1e-12) ef = 1e-12;
        st->dinit += dep / ef;
    }
    if (m->damage == 1 || m->damage == 2) {
        double D = 0.0;
        if (st->dinit >= 1.0) {
            D = 10.0 * (st->dinit - 1.0);
            if (D > 1.0) D = 1.0;
        }
        st->D = D;
        if (D >= 1.0) st->failed = 1;
    } else if (m->damage == 3) {          /* GTN: D = q1 f*, failure at f = f_F */
        if (st->f >= m->fF) { st->D = 1.0; st->failed = 1; }
        else st->D = m->q1 * orc_gtn_fstar(m, st->f);
    }
}

/* One constitutive update of a material point: strain increment deps (the
 * unrotated rate times dt, symmetric 3x3) and J = det F^{n+1}.  D^n enters
 * the return; D^{n+1} leaves it.  Used by the full step and by the
 * material-point tests. */
unsigned orc_constitutive(const orc_material *m, double dt, const double *deps, double J,
                          orc_mp_state *st)
{
    unsigned status = 0;
    if (st->failed) return 0;
    double ded[9], tr;
    deviator(deps, ded, &tr);
    double D = st->D;
    double dep;
    if (m->damage == 3) {
        dep = gtn_return(m, dt, ded, J, D, st, &status);
    } else {
        dep = radial_return_jc(m, dt, ded, D, st);
        st->sm = orc_eos_mean_stress(m, J, D, st->e);
    }
    damage_update(m, dt, dep, st);
    if (st->failed) {
        memset(st->sd, 0, sizeof st->sd);
        st->sm = 0.0;
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Whole system and the time step                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t N;
    /* fixed inputs */
    const double *X;          /* N*3 reference positions */
    const double *vol;        /* N   reference volumes */
    const int32_t *mat_id;    /* N   material index */
    const uint8_t *bc_mask;   /* N   1 = prescribed velocity */
    const double *bc_vel;     /* N*3 prescribed velocity */
    const int64_t *row_ptr;   /* N+1 */
    const int32_t *col;       /* nnz */
    const double *Linv;       /* N*9 */
    const orc_material *mats; /* material table */
    /* state at step n */
    double *u, *v, *F;        /* N*3, N*3, N*9 */
    double *sd;               /* N*9 unrotated deviatoric stress */
    double *sigma;            /* N*9 Cauchy stress (current frame) */
    double *A;                /* N*9 P L^{-T} */
    double *ep, *epdot, *dinit, *D, *f;  /* N each */
    double *e;                /* N   specific internal energy */
    double *force;            /* N*3 */
    int32_t *fail_step;       /* N, -1 while intact */
    int64_t step;
    uint32_t status;
    /* scratch, N*3 and N*9 */
    double *vh, *Fdot;
} orc_system;

/* Canonical pair force between a < b, acting on a (the force on b is its
 * negative): the damage-weighted PK1 term (Sec. 3.1) plus hourglass control.
 *
 * Reading (hourglass; the paper cites Ganzenmueller 2015 without a formula):
 *   eps_a = F_a X_ab - x_ab,  eps_b = F_b X_ab - x_ab,
 *   delta = (eps_a + eps_b) . xhat_ab,
 *   f_hg = -1/2 alpha (1-D_a)(1-D_b) V_a V_b W(X_ab) E / X_ab^2 delta xhat_ab,
 * with x_ab = X_ab + u_b - u_a and E the arithmetic mean (E_a + E_b) / 2
 * of the pair's Young moduli (symmetric in a, b; E itself for one material:
 * the bond's stiffness is the average of the two particles' stiffnesses, as
 * delta is the sum of the two particles' errors). */
static void pair_force(const orc_system *s, const orc_config *c, int64_t a, int64_t b, double *t)
{
    const double *Xa = s->X + 3 * a, *Xb = s->X + 3 * b;
    double gw[3];
    kernel_grad(Xa, Xb, c->h, gw);
    double Va = s->vol[a], Vb = s->vol[b];
    double Da = s->D[a], Db = s->D[b];
    const double *Aa = s->A + 9 * a, *Ab = s->A + 9 * b;
    for (int k = 0; k < 3; ++k) {
        double sa = 0.0, sb = 0.0;
        for (int l = 0; l < 3; ++l) { sa += Aa[3 * k + l] * gw[l]; sb += Ab[3 * k + l] * gw[l]; }
        t[k] = Va * Vb * ((1.0 - Db) * sa + (1.0 - Da) * sb);
    }
    if (c->hg_alpha != 0.0) {
        double X[3] = { Xb[0] - Xa[0], Xb[1] - Xa[1], Xb[2] - Xa[2] };
        double r = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
        double x[3];
        for (int k = 0; k < 3; ++k) x[k] = X[k] + s->u[3 * b + k] - s->u[3 * a + k];
        double xl = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (xl > 0.0) {
            double xh[3] = { x[0] / xl, x[1] / xl, x[2] / xl };
            const double *Fa = s->F + 9 * a, *Fb = s->F + 9 * b;
            double delta = 0.0;
            for (int k = 0; k < 3; ++k) {
                double ea = 0.0, eb = 0.0;
                for (int l = 0; l < 3; ++l) { ea += Fa[3 * k + l] * X[l]; eb += Fb[3 * k + l] * X[l]; }
                ea -= x[k]; eb -= x[k];
                delta += (ea + eb) * xh[k];
            }
            double E = 0.5 * (s->mats[s->mat_id[a]].E + s->mats[s->mat_id[b]].E);
            double coef = -0.5 * c->hg_alpha * (1.0 - Da) * (1.0 - Db) * Va * Vb
                        * orc_kernel_w(r, c->h) * E / (r * r) * delta;
            for (int k = 0; k < 3; ++k) t[k] += coef * xh[k];
        }
    }
}

/* nodal forces f_i = sum_j f_ij, sequential in ascending j */
void orc_forces(const orc_system *s, const orc_config *c)
{
    for (int64_t i = 0; i < s->N; ++i) {
        double fi[3] = { 0, 0, 0 };
        for (int64_t p = s->row_ptr[i]; p < s->row_ptr[i + 1]; ++p) {
            int64_t j = s->col[p];
            double t[3];
            if (i < j) {
                pair_force(s, c, i, j, t);
                for (int k = 0; k < 3; ++k) fi[k] += t[k];
            } else {
                pair_force(s, c, j, i, t);
                for (int k = 0; k < 3; ++k) fi[k] -= t[k];
            }
        }
        for (int k = 0; k < 3; ++k) s->force[3 * i + k] = fi[k];
    }
}

/* Per-particle kinematics + constitutive update + PK1 (a4-a9) given Fdot. */
static void particle_update(orc_system *s, const orc_config *c, int64_t i)
{
    const orc_material *m = &s->mats[s->mat_id[i]];
    double *F = s->F + 9 * i;
    if (s->fail_step[i] >= 0) {          /* fully damaged: no stress, F frozen */
        memset(s->sigma + 9 * i, 0, 9 * sizeof(double));
        memset(s->A + 9 * i, 0, 9 * sizeof(double));
        memset(s->sd + 9 * i, 0, 9 * sizeof(double));
        return;
    }
    const double *Fd = s->Fdot + 9 * i;
    for (int k = 0; k < 9; ++k) F[k] += c->dt * Fd[k];
    double J = mat_det(F);
    double Finv[9];
    if (!(J > 0.0) || !isfinite(J) || mat_inv(F, Finv) != 0) {
        s->status |= ORC_ST_BAD_J;
        return;
    }
    /* rate of deformation d = sym(Fdot F^{-1}), rotated to the unrotated frame */
    double Lv[9], d[9], R[9], RT[9], tmp[9], dh[9];
    mat_mul(Fd, Finv, Lv);
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) d[3 * k + l] = 0.5 * (Lv[3 * k + l] + Lv[3 * l + k]);
    if (orc_polar(F, R, NULL) != 0) s->status |= ORC_ST_POLAR_CAP;
    mat_transpose(R, RT);
    mat_mul(RT, d, tmp);
    mat_mul(tmp, R, dh);
    double deps[9];
    for (int k = 0; k < 9; ++k) deps[k] = c->dt * dh[k];
    orc_mp_state st;
    memcpy(st.sd, s->sd + 9 * i, sizeof st.sd);
    st.sm = 0.0;
    st.ep = s->ep[i]; st.epdot = s->epdot[i]; st.dinit = s->dinit[i];
    st.D = s->D[i]; st.f = s->f[i]; st.e = s->e[i]; st.failed = 0; st.newton_its = 0;
    s->status |= orc_constitutive(m, c->dt, deps, J, &st);
    memcpy(s->sd + 9 * i, st.sd, sizeof st.sd);
    s->ep[i] = st.ep; s->epdot[i] = st.epdot; s->dinit[i] = st.dinit;
    s->f[i] = st.f;
    s->D[i] = st.D;
    /* internal energy, Eq. (conservation3): de/dt = Fdot : P / rho0 = J sigma : d / rho0.
     * Reading: trapezoidal in the step (second order, like the velocity-Verlet
     * kinetic energy), in the current frame with the step's J and d:
     *   e^{n+1} = e^n + dt J / rho0 * (sigma^n + sigma^{n+1}) / 2 : d
     * with sigma^n the stress at the start of the step and sigma^{n+1} = 0
     * for a particle that fails in the step (the EOS of the step used e^n). */
    const double *sg_n = s->sigma + 9 * i;
    if (st.failed) {
        double w = 0.0;
        for (int k = 0; k < 9; ++k) w += 0.5 * sg_n[k] * d[k];
        s->e[i] += c->dt * J / m->rho0 * w;
        s->fail_step[i] = (int32_t)(s->step + 1);
        memset(s->sigma + 9 * i, 0, 9 * sizeof(double));
        memset(s->A + 9 * i, 0, 9 * sizeof(double));
        return;
    }
    /* Cauchy stress sigma = R (sigma_m I + s_hat) R^T, P = J sigma F^{-T},
     * A = P L^{-T} (the per-particle factor of the nodal force) */
    double sh[9], sg[9], FiT[9], P[9], LiT[9];
    memcpy(sh, st.sd, sizeof sh);
    sh[0] += st.sm; sh[4] += st.sm; sh[8] += st.sm;
    mat_mul(R, sh, tmp);
    mat_mul(tmp, RT, sg);
    {
        double w = 0.0;
        for (int k = 0; k < 9; ++k) w += 0.5 * (sg_n[k] + sg[k]) * d[k];
        s->e[i] += c->dt * J / m->rho0 * w;
    }
    memcpy(s->sigma + 9 * i, sg, sizeof sg);
    mat_transpose(Finv, FiT);
    mat_mul(sg, FiT, P);
    for (int k = 0; k < 9; ++k) P[k] *= J;
    mat_transpose(s->Linv + 9 * i, LiT);
    mat_mul(P, LiT, s->A + 9 * i);
    for (int k = 0; k < 9; ++k)
        if (!isfinite(s->A[9 * i + k]) || !isfinite(F[k])) s->status |= ORC_ST_NONFINITE;
}

static double particle_mass(const orc_system *s, int64_t i)
{
    return s->mats[s->mat_id[i]].rho0 * s->vol[i];
}

/* Sec. 6 drives the grips with v_max (1 - e^{-t}) (v_max in mm/ms, so t in
 * ms).  Reading: the prescribed velocity v_bc is scaled by
 * 1 - exp(-t / tau) = -expm1(-t / tau), t the time at which the velocity
 * holds (t_n + dt/2 for the half-step velocity, t_{n+1} for the full step);
 * tau = 0 keeps v_bc constant. */
static double grip_factor(const orc_config *c, double t)
{
    return c->grip_ramp > 0.0 ? -expm1(-t / c->grip_ramp) : 1.0;
}

/* velocity boundary conditions at time t: prescribed particles move with
 * their (ramped) prescribed velocity; fully damaged particles are held at
 * rest (Sec. 3.1) */
static void apply_bc(const orc_system *s, const orc_config *c, int64_t i, double t, double *vi)
{
    if (s->fail_step[i] >= 0) { vi[0] = vi[1] = vi[2] = 0.0; return; }
    if (s->bc_mask[i]) {
        const double r = grip_factor(c, t);
        for (int k = 0; k < 3; ++k) vi[k] = s->bc_vel[3 * i + k] * r;
    }
}

/* the velocities of the prescribed particles at the current time (step * dt),
 * e.g. zero at t = 0 under a ramp; called when the ramp is switched on */
void orc_apply_grip_ramp(orc_system *s, const orc_config *c)
{
    const double t = (double)s->step * c->dt;
    for (int64_t i = 0; i < s->N; ++i) apply_bc(s, c, i, t, s->v + 3 * i);
}

/* One velocity-Verlet step (Reading: the paper does not state its
 * integrator; kick-drift-kick with a fixed dt).
 *   v^{n+1/2} = v^n + dt/2 f^n/m          (BCs applied)
 *   u^{n+1}   = u^n + dt v^{n+1/2}
 *   Fdot from v^{n+1/2} and D^n; F^{n+1} = F^n + dt Fdot (Reading of Eq.
 *   Crack_approx_F: the time integral inside the sum equals per-particle
 *   integration because g_ij and the neighbour set are constant)
 *   constitutive update, damage -> D^{n+1}, P^{n+1}
 *   f^{n+1} from P^{n+1}, D^{n+1}, F^{n+1}, u^{n+1}
 *   v^{n+1}   = v^{n+1/2} + dt/2 f^{n+1}/m (BCs applied)                */
/* One time step in three phases (the whole step is the three in order):
 *  predict: half-step kick v^{n+1/2} = v^n + dt/2 f^n/m (constraints applied)
 *           and drift u^{n+1} = u^n + dt v^{n+1/2} (rigid wall applied);
 *  pass 1:  velocity gradients of every row from v^{n+1/2} and D^n, then the
 *           per-particle update (F, kinematics, constitutive, damage, A);
 *  pass 2:  forces from A, D^{n+1}, F, u^{n+1}, then the second half kick. */
void orc_step_predict(orc_system *s, const orc_config *c)
{
    int64_t N = s->N;
    const double t_half = ((double)s->step + 0.5) * c->dt;
    for (int64_t i = 0; i < N; ++i) {
        double m = particle_mass(s, i);
        for (int k = 0; k < 3; ++k)
            s->vh[3 * i + k] = s->v[3 * i + k] + 0.5 * c->dt * s->force[3 * i + k] / m;
        apply_bc(s, c, i, t_half, s->vh + 3 * i);
    }
    for (int64_t i = 0; i < 3 * N; ++i) s->u[i] += c->dt * s->vh[i];
    /* Reading (rigid wall; the paper has no contact): a kinematic plane
     * z = 0 -- a particle that drifted below it is put back on it and its
     * velocity may not point into it */
    if (c->wall)
        for (int64_t i = 0; i < N; ++i)
            if (s->X[3 * i + 2] + s->u[3 * i + 2] < 0.0) {
                s->u[3 * i + 2] = -s->X[3 * i + 2];
                if (s->vh[3 * i + 2] < 0.0) s->vh[3 * i + 2] = 0.0;
            }
}

void orc_step_pass1(orc_system *s, const orc_config *c)
{
    int64_t N = s->N;
    orc_velocity_gradient(N, s->X, s->vol, s->vh, s->D, s->Linv, s->row_ptr, s->col, c->h, s->Fdot);
    for (int64_t i = 0; i < N; ++i) particle_update(s, c, i);
}

void orc_step_pass2(orc_system *s, const orc_config *c)
{
    int64_t N = s->N;
    orc_forces(s, c);
    const double t_full = ((double)s->step + 1.0) * c->dt;
    for (int64_t i = 0; i < N; ++i) {
        double m = particle_mass(s, i);
        for (int k = 0; k < 3; ++k)
            s->v[3 * i + k] = s->vh[3 * i + k] + 0.5 * c->dt * s->force[3 * i + k] / m;
        apply_bc(s, c, i, t_full, s->v + 3 * i);
    }
    s->step += 1;
}

void orc_step(orc_system *s, const orc_config *c, int64_t nsteps)
{
    for (int64_t it = 0; it < nsteps; ++it) {
        orc_step_predict(s, c);
        orc_step_pass1(s, c);
        orc_step_pass2(s, c);
    }
}

/* Initial state: u = 0, F = I, no stress, v = bc_vel (the prescribed
 * velocity on constrained particles, the initial velocity elsewhere); GTN
 * starts from D = q1 f*(f0). */
void orc_init_state(orc_system *s)
{
    for (int64_t i = 0; i < s->N; ++i) {
        const orc_material *m = &s->mats[s->mat_id[i]];
        for (int k = 0; k < 3; ++k) {
            s->u[3 * i + k] = 0.0;
            s->v[3 * i + k] = s->bc_vel[3 * i + k];
            s->force[3 * i + k] = 0.0;
        }
        for (int k = 0; k < 9; ++k) {
            s->F[9 * i + k] = (k % 4 == 0) ? 1.0 : 0.0;
            s->sd[9 * i + k] = 0.0; s->sigma[9 * i + k] = 0.0; s->A[9 * i + k] = 0.0;
        }
        s->ep[i] = 0.0; s->epdot[i] = 0.0; s->dinit[i] = 0.0; s->e[i] = 0.0;
        s->D[i] = (m->damage == 3) ? m->q1 * orc_gtn_fstar(m, s->f[i]) : 0.0;
        s->fail_step[i] = -1;
    }
    s->step = 0;
    s->status = 0;
}

/* Material-point driver for the tests: applies n strain increments deps_k
 * (n x 9) with the given J_k (n) to one state, recording the state after
 * each increment into out (n x 16: sd[9], sm, ep, epdot, dinit, D, f, failed). */
unsigned orc_material_point(const orc_material *m, double dt, int64_t n, const double *deps,
                            const double *J, const double *init /* 16 */, double *out)
{
    orc_mp_state st;
    memcpy(st.sd, init, 9 * sizeof(double));
    st.sm = init[9]; st.ep = init[10]; st.epdot = init[11]; st.dinit = init[12];
    st.D = init[13]; st.f = init[14]; st.failed = (int32_t)init[15]; st.newton_its = 0;
    st.e = 0.0;        /* the material-point driver holds the internal energy at zero */
    unsigned status = 0;
    for (int64_t k = 0; k < n; ++k) {
        status |= orc_constitutive(m, dt, deps + 9 * k, J[k], &st);
        double *o = out + 16 * k;
        memcpy(o, st.sd, 9 * sizeof(double));
        o[9] = st.sm; o[10] = st.ep; o[11] = st.epdot; o[12] = st.dinit;
        o[13] = st.D; o[14] = st.f; o[15] = (double)st.failed;
    }
    return status;
}

/* GTN first Newton solve exposed for the tests: root x of the yield function
 * at fixed f* and triaxiality, from the starting guess x0. */
double orc_gtn_solve_x(const orc_material *m, double fs, double tri, double x0, int32_t *its)
{
    double x = x0;
    int k;
    for (k = 0; k < 50; ++k) {
        double dx = -gtn_phi(m, fs, tri, x) / gtn_dphi(m, fs, tri, x);
        x += dx;
        if (fabs(dx) <= 1e-14) break;
    }
    if (its) *its = k;
    return x;
}

double orc_gtn_phi(const orc_material *m, double fs, double tri, double x)
{
    return gtn_phi(m, fs, tri, x);
}

double orc_mat_det(const double *a) { return mat_det(a); }
int orc_mat_inv(const double *a, double *inv) { return mat_inv(a, inv); }
