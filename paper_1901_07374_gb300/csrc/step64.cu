// The FP64 time step: two gather passes over the fixed neighbour CSR.
//
// Pass 1 (per particle i):  damage-weighted velocity gradient
//   Fdot_i = sum_j V_j (1 - D_j^n) (v_j - v_i) (x) L_i^{-T} grad W_i(X_ij)
// (Sec. 3.1, Eq. Crack_approx_Fdot), F^{n+1} = F^n + dt Fdot (Eq.
// Crack_approx_F with g_ij and S_i constant in time), polar decomposition,
// strain increment in the unrotated frame, constitutive and damage update
// (Secs. 4-5), sigma = R s_hat R^T, P = J sigma F^{-T}, A_i = P_i L_i^{-T}.
//
// Pass 2 (per particle i):  damage-weighted nodal force (Sec. 3.1)
//   f_i = sum_j V_i V_j [(1 - D_j) A_i + (1 - D_i) A_j] grad W_i(X_ij)
// plus hourglass control, then the velocity-Verlet update with the
// velocity constraints and the fully damaged particles held at rest.
//
// Work decomposition: a warp owns 32 consecutive rows.  For each of them the
// 32 lanes stride over the row's neighbours and the partial sums meet in a
// butterfly reduction; lane r keeps row r's sums.  The per-particle epilogue
// then runs on all 32 lanes at once, one particle per lane, so the heavy
// FP64 constitutive work never leaves lanes idle.  Sums over j are therefore
// grouped by lane; the oracle sums sequentially, and the two agree to
// rounding.
#include <math.h>

#include <algorithm>

#include "tlsph_device.cuh"
#include "tlsph_internal.cuh"

namespace tlsph {

static constexpr int STEP_THREADS = 128;

struct StepConst {
    double dt, half_dt, inv_h, dw_norm, w_norm, hg_coef;
    int64_t step_index;
    int ucur, dcur, wall;
};

static StepConst make_const(const tlsph_config &cfg, int ucur, int dcur, int64_t step_index)
{
    StepConst c;
    c.dt = cfg.dt;
    c.half_dt = 0.5 * cfg.dt;
    c.inv_h = 1.0 / cfg.h;
    c.dw_norm = 1.0 / (M_PI * cfg.h * cfg.h * cfg.h * cfg.h);
    c.w_norm = 1.0 / (M_PI * cfg.h * cfg.h * cfg.h);
    c.hg_coef = -0.5 * cfg.hg_alpha;
    c.step_index = step_index;
    c.ucur = ucur;
    c.dcur = dcur;
    c.wall = (cfg.flags & TLSPH_FLAG_WALL) != 0;
    return c;
}

// velocity constraints at time t: a fully damaged particle is held at rest
// (Sec. 3.1); a prescribed particle moves with v_bc, ramped as
// v_bc (1 - exp(-t / tau)) when the context has a grip ramp (Sec. 6)
__device__ __forceinline__ void apply_bc(const DevState &s, int64_t i, int fail, double t, double *v)
{
    if (fail >= 0) {
        v[0] = v[1] = v[2] = 0.0;
    } else if (s.bcm[i]) {
        const double r = grip_factor(s.grip_ramp, t);
        v[0] = s.bcv[3 * i] * r; v[1] = s.bcv[3 * i + 1] * r; v[2] = s.bcv[3 * i + 2] * r;
    }
}

// ------------------------------------------------------------------ pass 1
__global__ void __launch_bounds__(STEP_THREADS) k_pass1_fp64(DevState s, StepConst c)
{
    const int lane = threadIdx.x & 31;
    const int64_t row0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5;
    if (row0 >= s.N) return;
    const int nrows = (int)min((int64_t)32, s.N - row0);
    const double *__restrict__ Dn = s.D[c.dcur];
    const double *__restrict__ X = s.X;
    const double *__restrict__ vh = s.vh;
    const double *__restrict__ vol = s.vol;
    double keep[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) keep[k] = 0.0;

    for (int r = 0; r < nrows; ++r) {
        const int64_t i = row0 + r;
        const double xi = X[3 * i], yi = X[3 * i + 1], zi = X[3 * i + 2];
        const double ui = vh[3 * i], vi = vh[3 * i + 1], wi = vh[3 * i + 2];
        const int64_t p0 = s.row_ptr[i], p1 = s.row_ptr[i + 1];
        double m[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) m[k] = 0.0;
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int64_t j = s.col[p];
            const double dx = X[3 * j] - xi, dy = X[3 * j + 1] - yi, dz = X[3 * j + 2] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double rinv = rsqrt(r2);
            const double q = r2 * rinv * c.inv_h;
            const double cw = vol[j] * (1.0 - Dn[j]) * spline_dw(q) * rinv;
            const double cx = cw * (vh[3 * j] - ui), cy = cw * (vh[3 * j + 1] - vi), cz = cw * (vh[3 * j + 2] - wi);
            m[0] += cx * dx; m[1] += cx * dy; m[2] += cx * dz;
            m[3] += cy * dx; m[4] += cy * dy; m[5] += cy * dz;
            m[6] += cz * dx; m[7] += cz * dy; m[8] += cz * dz;
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double t = warp_allsum(m[k]);
            keep[k] = (lane == r) ? t : keep[k];
        }
    }
    if (lane >= nrows) return;

    // ---- per-particle epilogue (one particle per lane)
    const int64_t i = row0 + lane;
    double *__restrict__ Dnext = s.D[c.dcur ^ 1];
    const int fail = s.fail[i];
    if (fail >= 0) {            // fully damaged: no stress, F frozen (Sec. 3.1)
        Dnext[i] = Dn[i];
        return;
    }
    double Li[9], Fd[9], Fn[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Li[k] = s.Linv[9 * i + k];
    // Fdot = M L^{-1} with M_km = sum_j w_j (v_j - v_i)_k (X_j - X_i)_m W'/r
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            Fd[3 * k + l] = c.dw_norm * (keep[3 * k] * Li[l] + keep[3 * k + 1] * Li[3 + l] + keep[3 * k + 2] * Li[6 + l]);
#pragma unroll
    for (int k = 0; k < 9; ++k) Fn[k] = s.F[9 * i + k] + c.dt * Fd[k];
    double cf[9];
    cof3(Fn, cf);
    const double J = Fn[0] * cf[0] + Fn[1] * cf[1] + Fn[2] * cf[2];
#pragma unroll
    for (int k = 0; k < 9; ++k) s.F[9 * i + k] = Fn[k];
    if (!(J > 0.0) || !isfinite(J)) {
        atomicOr(s.status, TLSPH_ST_BAD_J);
        Dnext[i] = Dn[i];
        return;
    }
    // F^{-1} = cof^T / J ;  L_v = Fdot F^{-1} ;  d = sym(L_v)
    const double iJ = 1.0 / J;
    double Fi[9];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) Fi[3 * k + l] = cf[3 * l + k] * iJ;
    double Lv[9];
    mul3(Fd, Fi, Lv);
    const double d[6] = { Lv[0], Lv[4], Lv[8], 0.5 * (Lv[1] + Lv[3]), 0.5 * (Lv[5] + Lv[7]), 0.5 * (Lv[2] + Lv[6]) };
    double R[9];
    uint32_t st = polar_rotation(Fn, R) ? 0u : TLSPH_ST_POLAR_CAP;
    double dh[6];
    sym_rotate_t(R, d, dh);
    double de[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) de[k] = c.dt * dh[k];

    MPState mp;
#pragma unroll
    for (int k = 0; k < 6; ++k) mp.sd[k] = s.sd[6 * i + k];
    mp.sm = 0.0;
    mp.ep = s.ep[i];
    mp.epdot = s.epdot[i];
    mp.dinit = s.dinit[i];
    mp.D = Dn[i];
    mp.f = s.por[i];
    mp.e = s.e[i];
    mp.failed = 0;
    const DevMat &mat = s.mats[s.mat[i]];
    st |= material_update(mat, c.dt, de, J, mp);
    // internal energy (Eq. conservation3, de/dt = J sigma : d / rho0), trapezoidal in the step with the
    // stress at its start and at its end (zero after a failure), current frame, d scaled by dt below
    double sgn[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) sgn[k] = s.sig[6 * i + k];
    double e_new = mp.e + c.dt * J * mat.inv_rho0 * (0.5 * sym_ddot(sgn, d));

#pragma unroll
    for (int k = 0; k < 6; ++k) s.sd[6 * i + k] = mp.sd[k];
    s.ep[i] = mp.ep;
    s.epdot[i] = mp.epdot;
    s.dinit[i] = mp.dinit;
    s.por[i] = mp.f;
    Dnext[i] = mp.D;
    if (mp.failed) {
        s.fail[i] = (int32_t)(c.step_index + 1);
        s.e[i] = e_new;
#pragma unroll
        for (int k = 0; k < 6; ++k) s.sig[6 * i + k] = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) s.A[9 * i + k] = 0.0;
    } else {
        // sigma = R (sigma_m I + s_hat) R^T
        double sh[6] = { mp.sd[0] + mp.sm, mp.sd[1] + mp.sm, mp.sd[2] + mp.sm, mp.sd[3], mp.sd[4], mp.sd[5] };
        double sg[6];
        sym_rotate(R, sh, sg);
        s.e[i] = e_new + c.dt * J * mat.inv_rho0 * (0.5 * sym_ddot(sg, d));
#pragma unroll
        for (int k = 0; k < 6; ++k) s.sig[6 * i + k] = sg[k];
        // P = J sigma F^{-T};  A = P L^{-T}
        double S[9], P[9], A[9];
        sym_to_full(sg, S);
        mul3_bt(S, Fi, P);
#pragma unroll
        for (int k = 0; k < 9; ++k) P[k] *= J;
        mul3_bt(P, Li, A);
        bool fin = true;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            s.A[9 * i + k] = A[k];
            fin &= isfinite(A[k]);
        }
        if (!fin) st |= TLSPH_ST_NONFINITE;
    }
    if (st) atomicOr(s.status, st);
}

// ------------------------------------------------------------------ pass 2
template <bool HG>
__global__ void __launch_bounds__(STEP_THREADS) k_pass2_fp64(DevState s, StepConst c)
{
    const int lane = threadIdx.x & 31;
    const int64_t row0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5;
    if (row0 >= s.N) return;
    const int nrows = (int)min((int64_t)32, s.N - row0);
    const double *__restrict__ D1 = s.D[c.dcur ^ 1];
    const double *__restrict__ X = s.X;
    const double *__restrict__ un = s.u[c.ucur ^ 1];   // u^{n+1}
    const double *__restrict__ vol = s.vol;
    const double *__restrict__ Aa = s.A;
    const double *__restrict__ Fa = s.F;
    double keep[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) keep[k] = 0.0;

    for (int r = 0; r < nrows; ++r) {
        const int64_t i = row0 + r;
        const double xi = X[3 * i], yi = X[3 * i + 1], zi = X[3 * i + 2];
        double uxi = 0, uyi = 0, uzi = 0, Ei = 0;
        double Fi[9];
        if (HG) {
            uxi = un[3 * i]; uyi = un[3 * i + 1]; uzi = un[3 * i + 2];
            Ei = s.youngs[i];
#pragma unroll
            for (int k = 0; k < 9; ++k) Fi[k] = Fa[9 * i + k];
        }
        const int64_t p0 = s.row_ptr[i], p1 = s.row_ptr[i + 1];
        double acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = 0.0;
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int64_t j = s.col[p];
            const double dx = X[3 * j] - xi, dy = X[3 * j + 1] - yi, dz = X[3 * j + 2] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double rinv = rsqrt(r2);
            const double q = r2 * rinv * c.inv_h;
            const double Vj = vol[j];
            const double omd = 1.0 - D1[j];
            const double g = spline_dw(q) * rinv;
            // s1 = sum V_j (1 - D_j) grad W ; s2 = sum V_j A_j grad W
            const double c1 = Vj * omd * g;
            acc[0] += c1 * dx; acc[1] += c1 * dy; acc[2] += c1 * dz;
            const double *Aj = Aa + 9 * j;
            const double c2 = Vj * g;
            acc[3] += c2 * (Aj[0] * dx + Aj[1] * dy + Aj[2] * dz);
            acc[4] += c2 * (Aj[3] * dx + Aj[4] * dy + Aj[5] * dz);
            acc[5] += c2 * (Aj[6] * dx + Aj[7] * dy + Aj[8] * dz);
            if (HG) {
                const double xx = dx + un[3 * j] - uxi, xy = dy + un[3 * j + 1] - uyi, xz = dz + un[3 * j + 2] - uzi;
                const double lx2 = xx * xx + xy * xy + xz * xz;
                if (lx2 > 0.0) {
                    const double lxi = rsqrt(lx2);
                    const double *Fj = Fa + 9 * j;
                    const double gx = (Fi[0] + Fj[0]) * dx + (Fi[1] + Fj[1]) * dy + (Fi[2] + Fj[2]) * dz;
                    const double gy = (Fi[3] + Fj[3]) * dx + (Fi[4] + Fj[4]) * dy + (Fi[5] + Fj[5]) * dz;
                    const double gz = (Fi[6] + Fj[6]) * dx + (Fi[7] + Fj[7]) * dy + (Fi[8] + Fj[8]) * dz;
                    // delta = (eps_i + eps_j) . xhat = ((F_i + F_j) X_ij) . xhat - 2 |x_ij|
                    const double delta = (gx * xx + gy * xy + gz * xz) * lxi - 2.0 * lx2 * lxi;
                    // pair modulus (E_i + E_j) / 2; the 1/2 is in the epilogue's coefficient
                    const double ch = (Ei + s.youngs[j]) * omd * Vj * spline_w(q) * rinv * rinv * delta * lxi;
                    acc[6] += ch * xx; acc[7] += ch * xy; acc[8] += ch * xz;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (!HG && k >= 6) continue;
            const double t = warp_allsum(acc[k]);
            keep[k] = (lane == r) ? t : keep[k];
        }
    }
    if (lane >= nrows) return;

    // ---- epilogue: nodal force and velocity-Verlet update of particle i
    const int64_t i = row0 + lane;
    const double Vi = vol[i];
    const double omdi = 1.0 - D1[i];
    double Ai[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Ai[k] = Aa[9 * i + k];
    double f[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        f[k] = Vi * c.dw_norm * (Ai[3 * k] * keep[0] + Ai[3 * k + 1] * keep[1] + Ai[3 * k + 2] * keep[2] + omdi * keep[3 + k]);
    if (HG) {
        const double hc = 0.5 * c.hg_coef * omdi * Vi * c.w_norm;
#pragma unroll
        for (int k = 0; k < 3; ++k) f[k] += hc * keep[6 + k];
    }
    const double im = s.inv_mass[i];
    const int fail = s.fail[i];
    double vn[3], v2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        s.force[3 * i + k] = f[k];
        vn[k] = kick(s.vh[3 * i + k], c.half_dt, f[k], im);
    }
    apply_bc(s, i, fail, ((double)c.step_index + 1.0) * c.dt, vn);
#pragma unroll
    for (int k = 0; k < 3; ++k) v2[k] = kick(vn[k], c.half_dt, f[k], im);
    apply_bc(s, i, fail, ((double)(c.step_index + 1) + 0.5) * c.dt, v2);
    double *__restrict__ unext = s.u[c.ucur];
    double un2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) un2[k] = drift(un[3 * i + k], c.dt, v2[k]);
    if (c.wall) wall_contact(s.X[3 * i + 2], un2[2], v2[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        s.v[3 * i + k] = vn[k];
        s.vh[3 * i + k] = v2[k];
        unext[3 * i + k] = un2[k];
    }
    if (!(isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]))) atomicOr(s.status, TLSPH_ST_NONFINITE);
}

// ------------------------------------------------------------------ set-up and helpers
__global__ void k_init_state(DevState s)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        s.u[0][3 * i + k] = 0.0;
        s.u[1][3 * i + k] = 0.0;
        s.v[3 * i + k] = s.bcv[3 * i + k];
        s.vh[3 * i + k] = s.bcv[3 * i + k];
        s.force[3 * i + k] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        s.F[9 * i + k] = (k == 0 || k == 4 || k == 8) ? 1.0 : 0.0;
        s.A[9 * i + k] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        s.sd[6 * i + k] = 0.0;
        s.sig[6 * i + k] = 0.0;
    }
    s.ep[i] = 0.0;
    s.epdot[i] = 0.0;
    s.dinit[i] = 0.0;
    s.e[i] = 0.0;
    s.D[0][i] = 0.0;
    s.D[1][i] = 0.0;
    s.fail[i] = -1;
}

// material-dependent per-particle constants; before the first step a GTN
// material also sets D = q1 f*(f0) (Sec. 5.4)
__global__ void k_material_fields(DevState s, int mat_id, int dcur, int set_gtn_damage)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N || s.mat[i] != mat_id) return;
    const DevMat &m = s.mats[mat_id];
    const_cast<double *>(s.mass)[i] = m.rho0 * s.vol[i];
    const_cast<double *>(s.inv_mass)[i] = 1.0 / (m.rho0 * s.vol[i]);
    const_cast<double *>(s.youngs)[i] = m.E;
    if (set_gtn_damage && m.damage == TLSPH_DAMAGE_GTN) s.D[dcur][i] = m.q1 * gtn_fstar(m, s.por[i]);
}

// v^{n+1/2} = v^n + dt/2 f^n / m and u^{n+1} = u^n + dt v^{n+1/2} (constraints applied)
__global__ void k_predict(DevState s, int ucur, double dt, int wall, double t_half)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    const double im = s.inv_mass[i];
    double v[3], u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = kick(s.v[3 * i + k], 0.5 * dt, s.force[3 * i + k], im);
    apply_bc(s, i, s.fail[i], t_half, v);
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = drift(s.u[ucur][3 * i + k], dt, v[k]);
    if (wall) wall_contact(s.X[3 * i + 2], u[2], v[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        s.vh[3 * i + k] = v[k];
        s.u[ucur ^ 1][3 * i + k] = u[k];
    }
}

// the velocities of the prescribed particles at time t (a ramp switched on)
__global__ void k_apply_grip(DevState s, double t)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    apply_bc(s, i, s.fail[i], t, s.v + 3 * i);
}

__global__ void k_material_point(const DevMat m, double dt, int64_t n, const double *deps, const double *J,
                                 double *state)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double *e = deps + 9 * t;
    double *x = state + 16 * t;
    const double de[6] = { e[0], e[4], e[8], 0.5 * (e[1] + e[3]), 0.5 * (e[5] + e[7]), 0.5 * (e[2] + e[6]) };
    MPState mp;
    mp.sd[0] = x[0]; mp.sd[1] = x[4]; mp.sd[2] = x[8];
    mp.sd[3] = 0.5 * (x[1] + x[3]); mp.sd[4] = 0.5 * (x[5] + x[7]); mp.sd[5] = 0.5 * (x[2] + x[6]);
    mp.sm = x[9]; mp.ep = x[10]; mp.epdot = x[11]; mp.dinit = x[12]; mp.D = x[13]; mp.f = x[14];
    mp.e = 0.0;        // the material-point driver holds the internal energy at zero
    mp.failed = x[15] != 0.0;
    material_update(m, dt, de, J[t], mp);
    sym_to_full(mp.sd, x);
    x[9] = mp.sm; x[10] = mp.ep; x[11] = mp.epdot; x[12] = mp.dinit; x[13] = mp.D; x[14] = mp.f;
    x[15] = mp.failed ? 1.0 : 0.0;
}

__global__ void k_export_sym(const double *src6, double *dst9, int64_t N)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) sym_to_full(src6 + 6 * i, dst9 + 9 * i);
}

__global__ void k_import_sym(const double *src9, double *dst6, int64_t N)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double *a = src9 + 9 * i;
    double *o = dst6 + 6 * i;
    o[0] = a[0]; o[1] = a[4]; o[2] = a[8];
    o[3] = 0.5 * (a[1] + a[3]); o[4] = 0.5 * (a[5] + a[7]); o[5] = 0.5 * (a[2] + a[6]);
}

__global__ void k_gather_inputs(const int32_t *perm, int64_t N, const double *X, const double *vol, const int32_t *mat,
                                const uint8_t *bcm, const double *bcv, const double *f0, DevState s)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int64_t i = perm[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const_cast<double *>(s.X)[3 * k + c] = X[3 * i + c];
        const_cast<double *>(s.bcv)[3 * k + c] = bcv[3 * i + c];
    }
    const_cast<double *>(s.vol)[k] = vol[i];
    const_cast<int32_t *>(s.mat)[k] = mat[i];
    const_cast<uint8_t *>(s.bcm)[k] = bcm[i];
    s.por[k] = f0[i];
}

template <class T>
__global__ void k_permute(const T *src, T *dst, const int32_t *perm, int64_t N, int comps, bool out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int64_t i = perm[k];
    if (out)
        for (int c = 0; c < comps; ++c) dst[comps * i + c] = src[comps * k + c];
    else
        for (int c = 0; c < comps; ++c) dst[comps * k + c] = src[comps * i + c];
}

__global__ void k_permute_sym(const double *src, double *dst, const int32_t *perm, int64_t N, bool out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int64_t i = perm[k];
    if (out) {
        sym_to_full(src + 6 * k, dst + 9 * i);
    } else {
        const double *a = src + 9 * i;
        double *o = dst + 6 * k;
        o[0] = a[0]; o[1] = a[4]; o[2] = a[8];
        o[3] = 0.5 * (a[1] + a[3]); o[4] = 0.5 * (a[5] + a[7]); o[5] = 0.5 * (a[2] + a[6]);
    }
}

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class T>
__global__ void k_to_caller(const T *__restrict__ src, T *__restrict__ dst, const int32_t *__restrict__ inv,
                            int64_t N, int comps, int scomps, bool sym)
{
    // row-major 3x3 index -> stored symmetric component (xx, yy, zz, xy, yz, zx)
    const int smap[9] = { 0, 3, 5, 3, 1, 4, 5, 4, 2 };
    const int64_t total = N * comps;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / comps;
        const int c = (int)(e - i * comps);
        const int64_t k = inv ? (int64_t)inv[i] : i;
        dst[e] = src[k * scomps + (sym ? smap[c] : c)];
    }
}

cudaError_t launch_to_caller(const void *src, void *dst, const int32_t *inv, int64_t N, int comps, int scomps,
                             int elem, bool sym, cudaStream_t st)
{
    const int64_t total = N * comps;
    const unsigned g = (unsigned)std::min<int64_t>(nblk(total, 256), 152 * 16);
    if (total <= 0) return cudaSuccess;
    if (elem == 8)
        k_to_caller<double><<<g, 256, 0, st>>>(static_cast<const double *>(src), static_cast<double *>(dst), inv, N,
                                               comps, scomps, sym);
    else if (elem == 4)
        k_to_caller<int32_t><<<g, 256, 0, st>>>(static_cast<const int32_t *>(src), static_cast<int32_t *>(dst), inv,
                                                N, comps, scomps, false);
    else
        k_to_caller<uint8_t><<<g, 256, 0, st>>>(static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst), inv,
                                                N, comps, scomps, false);
    return cudaGetLastError();
}

cudaError_t launch_gather_inputs(const int32_t *perm, int64_t N, const double *X, const double *vol,
                                 const int32_t *mat, const uint8_t *bcm, const double *bcv, const double *f0,
                                 const DevState &s, cudaStream_t st)
{
    k_gather_inputs<<<nblk(N, 256), 256, 0, st>>>(perm, N, X, vol, mat, bcm, bcv, f0, s);
    return cudaGetLastError();
}

cudaError_t launch_permute(const void *src, void *dst, const int32_t *perm, int64_t N, int comps, int elem,
                           bool out, bool sym, cudaStream_t st)
{
    const unsigned g = nblk(N, 256);
    if (sym)
        k_permute_sym<<<g, 256, 0, st>>>(static_cast<const double *>(src), static_cast<double *>(dst), perm, N, out);
    else if (elem == 8)
        k_permute<double><<<g, 256, 0, st>>>(static_cast<const double *>(src), static_cast<double *>(dst), perm, N,
                                             comps, out);
    else if (elem == 4)
        k_permute<int32_t><<<g, 256, 0, st>>>(static_cast<const int32_t *>(src), static_cast<int32_t *>(dst), perm,
                                              N, comps, out);
    else
        k_permute<uint8_t><<<g, 256, 0, st>>>(static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst), perm,
                                              N, comps, out);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const DevState &s, cudaStream_t st)
{
    k_init_state<<<nblk(s.N, 256), 256, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_material_fields(const DevState &s, int mat_id, int dcur, bool gtn_damage, cudaStream_t st)
{
    k_material_fields<<<nblk(s.N, 256), 256, 0, st>>>(s, mat_id, dcur, gtn_damage ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ diagnostics
// Block b reduces particles [b N / B, (b + 1) N / B) in a fixed order (thread
// stride, then a shared-memory tree); a second one-block kernel reduces the
// block partials in block order: the same N gives the same bits every time.
constexpr int DIAG_THREADS = 512;

// slots 8 and 9 are maxima (largest D, largest plastic strain), every other slot a sum
__device__ __forceinline__ bool diag_is_max(int k) { return k == 8 || k == 9; }

__device__ __forceinline__ void diag_combine(double *a, const double *b)
{
#pragma unroll
    for (int k = 0; k < TLSPH_DIAG_COUNT; ++k) a[k] = diag_is_max(k) ? fmax(a[k], b[k]) : a[k] + b[k];
}

// a[] of lane 0 becomes the combination over the warp (fixed butterfly order)
__device__ __forceinline__ void diag_warp(double *a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double b[TLSPH_DIAG_COUNT];
#pragma unroll
        for (int k = 0; k < TLSPH_DIAG_COUNT; ++k) b[k] = __shfl_down_sync(0xffffffffu, a[k], o);
        diag_combine(a, b);
    }
}

// combination over the block into sh[0][.]; every thread passes its a[]
__device__ __forceinline__ void diag_block(double *a, double (*sh)[TLSPH_DIAG_COUNT])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    diag_warp(a);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < TLSPH_DIAG_COUNT; ++k) sh[wid][k] = a[k];
    __syncthreads();
    if (wid == 0) {
        double b[TLSPH_DIAG_COUNT];
#pragma unroll
        for (int k = 0; k < TLSPH_DIAG_COUNT; ++k) b[k] = lane < nw ? sh[lane][k] : (diag_is_max(k) ? -INFINITY : 0.0);
        diag_warp(b);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < TLSPH_DIAG_COUNT; ++k) sh[0][k] = b[k];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(DIAG_THREADS) k_diag_blocks(DevState s, int dcur, double *partials)
{
    __shared__ double sh[32][TLSPH_DIAG_COUNT];
    const int64_t N = s.N;
    const int64_t lo = (int64_t)blockIdx.x * N / gridDim.x, hi = (int64_t)(blockIdx.x + 1) * N / gridDim.x;
    double a[TLSPH_DIAG_COUNT];
#pragma unroll
    for (int k = 0; k < TLSPH_DIAG_COUNT; ++k) a[k] = diag_is_max(k) ? -INFINITY : 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double m = s.mass[i];
        const double v0 = s.v[3 * i], v1 = s.v[3 * i + 1], v2 = s.v[3 * i + 2];
        double b[TLSPH_DIAG_COUNT] = { m * v0, m * v1, m * v2, s.force[3 * i], s.force[3 * i + 1], s.force[3 * i + 2],
                                       0.5 * m * (v0 * v0 + v1 * v1 + v2 * v2), s.fail[i] >= 0 ? 1.0 : 0.0,
                                       s.D[dcur][i], s.ep[i], m * s.e[i] };
        diag_combine(a, b);
    }
    diag_block(a, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < TLSPH_DIAG_COUNT; ++k) partials[(int64_t)blockIdx.x * TLSPH_DIAG_COUNT + k] = sh[0][k];
}

// one block over the per-block partials (nblocks <= blockDim.x)
__global__ void k_diag_final(double *partials, int nblocks)
{
    __shared__ double sh[32][TLSPH_DIAG_COUNT];
    double a[TLSPH_DIAG_COUNT];
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < TLSPH_DIAG_COUNT; ++k)
        a[k] = t < nblocks ? partials[(int64_t)t * TLSPH_DIAG_COUNT + k] : (diag_is_max(k) ? -INFINITY : 0.0);
    diag_block(a, sh);
    if (t == 0)
        for (int k = 0; k < TLSPH_DIAG_COUNT; ++k) partials[k] = sh[0][k];
}

cudaError_t launch_diagnostics(const DevState &s, int dcur, double *partials, cudaStream_t st)
{
    static_assert(DIAG_BLOCKS <= 256, "the final reduction takes one block of 256 threads");
    k_diag_blocks<<<DIAG_BLOCKS, DIAG_THREADS, 0, st>>>(s, dcur, partials);
    k_diag_final<<<1, 256, 0, st>>>(partials, DIAG_BLOCKS);
    return cudaGetLastError();
}

cudaError_t launch_apply_grip(const DevState &s, double t, cudaStream_t st)
{
    k_apply_grip<<<nblk(s.N, 256), 256, 0, st>>>(s, t);
    return cudaGetLastError();
}

cudaError_t launch_predict(const DevState &s, int ucur, double dt, bool wall, int64_t steps, cudaStream_t st)
{
    k_predict<<<nblk(s.N, 256), 256, 0, st>>>(s, ucur, dt, wall ? 1 : 0, ((double)steps + 0.5) * dt);
    return cudaGetLastError();
}

cudaError_t launch_step_fp64(const DevState &s, const tlsph_config &cfg, int ucur, int dcur,
                             int64_t step_index, cudaStream_t st, cudaEvent_t *ev)
{
    const StepConst c = make_const(cfg, ucur, dcur, step_index);
    const unsigned grid = nblk((s.N + 31) / 32 * 32, STEP_THREADS);
    if (ev) cudaEventRecord(ev[0], st);
    k_pass1_fp64<<<grid, STEP_THREADS, 0, st>>>(s, c);
    if (ev) cudaEventRecord(ev[1], st);
    if (cfg.hg_alpha != 0.0)
        k_pass2_fp64<true><<<grid, STEP_THREADS, 0, st>>>(s, c);
    else
        k_pass2_fp64<false><<<grid, STEP_THREADS, 0, st>>>(s, c);
    if (ev) cudaEventRecord(ev[2], st);
    return cudaGetLastError();
}

cudaError_t launch_material_point_value(const DevMat &m, double dt, int64_t n, const double *deps,
                                        const double *J, double *state, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_material_point<<<nblk(n, 128), 128, 0, st>>>(m, dt, n, deps, J, state);
    return cudaGetLastError();
}

cudaError_t launch_export_sym(const double *src6, double *dst9, int64_t N, cudaStream_t st)
{
    k_export_sym<<<nblk(N, 256), 256, 0, st>>>(src6, dst9, N);
    return cudaGetLastError();
}

cudaError_t launch_import_sym(const double *src9, double *dst6, int64_t N, cudaStream_t st)
{
    k_import_sym<<<nblk(N, 256), 256, 0, st>>>(src9, dst6, N);
    return cudaGetLastError();
}

}  // namespace tlsph
