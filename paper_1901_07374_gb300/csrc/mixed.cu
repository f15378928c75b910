// Mixed-precision time step: FP32 pair gathers and FP32 sums over j.
//
// What stays FP64: displacements and velocities (u, v, v^{n+1/2}), the
// correction matrix inverse (computed once in FP64, used rounded), the nodal
// force handed to the integrator and the velocity-Verlet update, and the
// constitutive + damage update of every particle that yields, is near yield,
// is a GTN particle or has reached damage initiation.
//
// Compensated FP32 (hi + lo float pairs): F and the unrotated stress deviator,
// so that small increments accumulate without loss over many steps.
//
// What is FP32: every per-pair term of both passes, the sums over j, J - 1
// (from the invariants of F - I), the polar decomposition, the rotations,
// P = J sigma F^{-T}, A = P L^{-T}, and the elastic branch of Algorithm 1 for
// particles whose trial stress is clearly inside the yield surface.
//
// The pair terms are arranged so the FP32 sums carry no large cancellation:
//  - a reference position is an int32 fixed-point triple about the specimen's
//    centre (unit a power of two, |coordinate| < 2^31), so X_ij is an exact
//    integer difference rounded once to FP32; every pair length is in those
//    units (the kernel argument q uses unit / h, the hourglass sums are
//    rescaled per particle);
//  - velocities are mirrored relative to a bulk reference velocity;
//  - the hourglass error vector uses F - I and u, e = (F_i - I) X_ij - u_ij;
//  - the stress term is written with differences (Sec. 3.1 force, rearranged):
//      f_i = V_i (1-D_i) sum_j V_j (A_j - A_i) grad W_ij
//          + V_i A_i [ (2 - D_i) S0_i - sum_j V_j D_j grad W_ij ],
//    with the static S0_i = sum_j V_j grad W_ij computed once in FP64.
//
// Data layout (16-byte records indexed by particle, "SoA of float4", so a warp
// gathering consecutive particles reads consecutive 16-byte words):
//   xo   int4 {fixed-point x, y, z, 0}
//   r1   {v^{n+1/2} - v_ref, V (1 - D)}                       pass-1 gather record
//   r2k  k = 0..5 (at r2 + k N):                               pass-2 gather record
//        {A00 A01 A02 A10} {A11 A12 A20 A21} {A22, V D, V, u_x}
//        {u_y, u_z, G00, G01} {G02 G10 G11 G12} {G20, G21, G22, E V (1-D)}
//        with G = F - I and u in fixed-point units.
// Thread-per-row kernels read their neighbours through the sliced neighbour
// lists (slices of 32 rows, aligned or explicit form, described below).
#include <math.h>

#include <algorithm>

#include "tlsph_device.cuh"
#include "tlsph_internal.cuh"

namespace tlsph {

static constexpr int MIX_THREADS = 128;

static MixConst make_mix_const(const tlsph_ctx &ctx, int64_t step_index)
{
    MixConst c;
    const tlsph_config &cfg = ctx.cfg;
    c.dt = cfg.dt;
    c.half_dt = 0.5 * cfg.dt;
    c.inv_h = (float)(ctx.s.pack.unit / cfg.h);
    c.dt_dw = (float)(cfg.dt / (M_PI * cfg.h * cfg.h * cfg.h * cfg.h));
    c.dw_norm = (float)(1.0 / (M_PI * cfg.h * cfg.h * cfg.h * cfg.h));
    c.w_norm = (float)(1.0 / (M_PI * cfg.h * cfg.h * cfg.h));
    c.hg_coef = (float)(-0.5 * cfg.hg_alpha);
    c.hg_w = (float)(-0.5 * cfg.hg_alpha / (M_PI * cfg.h * cfg.h * cfg.h) * ctx.s.pack.inv_unit);
    c.inv_unit = ctx.s.pack.inv_unit;
    c.yield_keep = ctx.guard >= 1.0 ? -1.0f : (float)(1.0 - ctx.guard);
    c.inv_unit_f = (float)ctx.s.pack.inv_unit;
    c.vref0 = ctx.s.vref[0];
    c.vref1 = ctx.s.vref[1];
    c.vref2 = ctx.s.vref[2];
    c.N = ctx.N;
    c.step_index = step_index;
    c.ucur = ctx.ucur;
    c.dcur = ctx.dcur;
    c.wall = (cfg.flags & TLSPH_FLAG_WALL) != 0;
    return c;
}

// ------------------------------------------------------------------ FP32 3x3 helpers
__device__ __forceinline__ void mul3f(const float *a, const float *b, float *c)
{
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            c[3 * k + l] = a[3 * k] * b[l] + a[3 * k + 1] * b[3 + l] + a[3 * k + 2] * b[6 + l];
}
__device__ __forceinline__ void mul3f_bt(const float *a, const float *b, float *c)
{
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            c[3 * k + l] = a[3 * k] * b[3 * l] + a[3 * k + 1] * b[3 * l + 1] + a[3 * k + 2] * b[3 * l + 2];
}
__device__ __forceinline__ void cof3f(const float *m, float *c)
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

// FP32 rotation of the polar decomposition, same iteration as the FP64
// path (determinant-scaled Newton), stop after a step below 1e-5, cap 30.
__device__ __forceinline__ bool polar_rotation_f(const float *F, float *R)
{
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = F[k];
    bool last = false;
    for (int it = 0; it < 30; ++it) {
        float c[9];
        cof3f(R, c);
        const float d = R[0] * c[0] + R[1] * c[1] + R[2] * c[2];
        const float g = rcbrtf(fabsf(d));
        const float gi = 1.0f / (g * d);
        float diff = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float xn = 0.5f * (g * R[k] + c[k] * gi);
            const float e = xn - R[k];
            diff += e * e;
            R[k] = xn;
        }
        if (last) return true;
        if (diff < 1e-10f) last = true;
    }
    return false;
}

// symmetric (6) sandwich products in FP32
__device__ __forceinline__ void sym_rotate_t_f(const float *Q, const float *s, float *out)
{
    float S[9] = { s[0], s[3], s[5], s[3], s[1], s[4], s[5], s[4], s[2] }, T[9];
    mul3f(S, Q, T);
#define QTT(k, l) (Q[k] * T[l] + Q[3 + k] * T[3 + l] + Q[6 + k] * T[6 + l])
    out[0] = QTT(0, 0); out[1] = QTT(1, 1); out[2] = QTT(2, 2);
    out[3] = QTT(0, 1); out[4] = QTT(1, 2); out[5] = QTT(2, 0);
#undef QTT
}
__device__ __forceinline__ void sym_rotate_f(const float *Q, const float *s, float *out)
{
    float S[9] = { s[0], s[3], s[5], s[3], s[1], s[4], s[5], s[4], s[2] }, T[9];
    mul3f_bt(S, Q, T);
#define QT(k, l) (Q[3 * k] * T[l] + Q[3 * k + 1] * T[3 + l] + Q[3 * k + 2] * T[6 + l])
    out[0] = QT(0, 0); out[1] = QT(1, 1); out[2] = QT(2, 2);
    out[3] = QT(0, 1); out[4] = QT(1, 2); out[5] = QT(2, 0);
#undef QT
}

// X_j - X_i in units of the fixed-point grid: an exact integer difference
// (modular, so a masked slot between distant particles stays finite), then
// rounded once to FP32
__device__ __forceinline__ float3 xdiff(const int4 oj, const int4 oi)
{
    return make_float3((float)(int)((unsigned)oj.x - (unsigned)oi.x), (float)(int)((unsigned)oj.y - (unsigned)oi.y),
                       (float)(int)((unsigned)oj.z - (unsigned)oi.z));
}

// M4 spline (normalisation in the step constants) in the branch-free form
//   W(q) = (2 - q)_+^3 / 4 - (1 - q)_+^3,   W'(q) = 3 (1 - q)_+^2 - 3/4 (2 - q)_+^2
__device__ __forceinline__ float spline_dw_ab(float q, float &a, float &b)
{
    a = fmaxf(2.0f - q, 0.0f);
    b = fmaxf(1.0f - q, 0.0f);
    return fmaf(3.0f * b, b, -0.75f * a * a);
}
__device__ __forceinline__ float spline_w_ab(float a, float b) { return fmaf(0.25f * a * a, a, -b * b * b); }

// kernel-argument offset of a padding slot: q >= 2 for any pair distance
constexpr float SLOT_PAD_Q = 4.0f;

// approximate reciprocal, one MUFU operation (relative error about 1 ulp)
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ------------------------------------------------------------------ sliced neighbour lists
// The thread-per-row kernels read neighbours slice by slice, a slice being the
// 32 consecutive rows of one warp.  A slice is stored in one of two forms:
//
//  explicit: ell_w[g] = W >= 0 slots; entry k of lane l at ell_off[g] + 32 k + l
//            holds the neighbour index j, or ~p for a padding slot (p a valid
//            particle index other than the row's, weight 0);
//  aligned:  ell_w[g] = ~(W | clamp << 24) < 0.  Slot k stands for the same
//            index offset o_k in every row of the slice (j = i + o_k); the
//            slice's union of offsets is stored once (o_k at ell_off[g] + k,
//            padded with the last offset to T = 32 ceil(W / 32) words)
//            followed by one mask word per row and 32 slots (bit k % 32 of
//            the word at ell_off[g] + T + 32 (k / 32) + l says whether row l
//            has j = i + o_k as a neighbour).  clamp = 0 when i + o_k is a
//            particle index for every row i < N of the slice and every
//            offset, so a masked slot reads a valid particle (j != i) as it
//            stands; slices near either end of the index range have clamp = 1
//            and their masked slots that would leave the range read i -+ 1.
//
// Rows are sorted by j, so slots run in ascending j in both forms: the sums
// over j are taken in CSR order either way.  Particles laid out with a regular
// index structure (lattice rows) have nearly the same neighbour offsets in
// all rows of a slice, so the aligned form replaces 4 bytes per pair with a
// few bits, and the 32 lanes' k-th neighbours are consecutive particles (one
// contiguous 512-byte record load per warp).  A slice whose offset union is
// much wider than its longest row keeps the explicit form.

// union of the slice's offsets (ascending), cut off once it exceeds `limit`;
// returns its width, the smallest and the largest offset
__device__ __forceinline__ int slice_union(const int64_t *row_ptr, const int32_t *col, int64_t i, int64_t N, int limit,
                                          int32_t *table, uint32_t *masks, int lane, int T, int &omin, int &omax)
{
    int64_t p = 0, e = 0;
    if (i < N) { p = row_ptr[i]; e = row_ptr[i + 1]; }
    int h = p < e ? (int)(col[p] - i) : INT_MAX;
    int cnt = 0;
    int myoff = 0;
    uint32_t mword = 0;
    omin = 0;
    omax = 0;
    while (true) {
        const int m = __reduce_min_sync(0xffffffffu, h);
        if (m == INT_MAX || cnt >= limit) break;
        if (cnt == 0) omin = m;
        omax = m;
        if (table) {
            if (lane == (cnt & 31)) myoff = m;
            if (h == m) mword |= 1u << (cnt & 31);
            if ((cnt & 31) == 31) {
                table[32 * (cnt >> 5) + lane] = myoff;
                masks[T + 32 * (cnt >> 5) + lane] = mword;
                myoff = 0;
                mword = 0;
            }
        }
        ++cnt;
        if (h == m) {
            ++p;
            h = p < e ? (int)(col[p] - i) : INT_MAX;
        }
    }
    if (table && (cnt & 31)) {
        if (lane >= (cnt & 31)) myoff = omax;      // table padding: a valid offset, its mask bits are 0
        table[32 * (cnt >> 5) + lane] = myoff;
        masks[T + 32 * (cnt >> 5) + lane] = mword;
    }
    return cnt;
}

// per slice: the form, its width and its word count (into ell_off, scanned later)
__global__ void k_ell_plan(const int64_t *row_ptr, const int32_t *col, int64_t N, int32_t *ell_w, int64_t *ell_off)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g = i >> 5;
    if (g >= (N + 31) / 32) return;       // whole warps: N rounded up to 32 rows
    const int lane = threadIdx.x & 31;
    const int len = i < N ? (int)(row_ptr[i + 1] - row_ptr[i]) : 0;
    const int wp = __reduce_max_sync(0xffffffffu, len);
    // aligned only when its slots stay within 5/4 of the explicit form's, its
    // words fit in the explicit form's and every row's i + o_k is a particle
    const int limit = (5 * wp) / 4 + 4;
    int omin, omax;
    const int wu = slice_union(row_ptr, col, i, N, limit + 1, nullptr, nullptr, lane, 0, omin, omax);
    const int64_t words_u = 64 * (int64_t)((wu + 31) / 32);
    const bool in_range = i >= N || (i + omin >= 0 && i + omax < N);
    const int clamp = __all_sync(0xffffffffu, in_range) ? 0 : 1;
    const bool aligned = wp > 0 && wu <= limit && words_u <= 32 * (int64_t)wp;
    if (lane == 0) {
        ell_w[g] = aligned ? ~(wu | (clamp << 24)) : wp;
        ell_off[g] = aligned ? words_u : 32 * (int64_t)wp;
    }
}

__global__ void k_ell_fill(const int64_t *row_ptr, const int32_t *col, int64_t N, const int32_t *ell_w,
                           const int64_t *ell_off, int32_t *colE)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g = i >> 5;
    if (g >= (N + 31) / 32) return;
    const int lane = threadIdx.x & 31;
    const int wv = ell_w[g];
    int32_t *o = colE + ell_off[g];
    if (wv < 0) {
        const int W = (~wv) & 0xffffff;
        const int T = 32 * ((W + 31) / 32);
        int omin, omax;
        slice_union(row_ptr, col, i, N, W, o, reinterpret_cast<uint32_t *>(o), lane, T, omin, omax);
        return;
    }
    const int64_t b = i < N ? row_ptr[i] : 0, n = i < N ? row_ptr[i + 1] - row_ptr[i] : 0;
    const int32_t pad = ~(int32_t)(i == 0 ? (N > 1 ? 1 : 0) : (i < N ? i - 1 : 0));
    for (int k = 0; k < wv; ++k) o[32 * k + lane] = k < n ? col[b + k] : pad;
}

// aligned slice: slots in groups of U; CLAMP replaces an index outside the
// particle range (only ever a masked slot) by alt
template <int U, bool CLAMP, class Body>
__device__ __forceinline__ void aligned_slots(const int32_t *__restrict__ base, int W, int lane, int ii, int alt,
                                              int N, Body &&body)
{
    const int T = 32 * ((W + 31) / 32);
    const uint32_t *__restrict__ mk = reinterpret_cast<const uint32_t *>(base) + T + lane;
    uint32_t bits = 0;
    for (int k = 0; k < W; k += U) {
        if ((k & 31) == 0) bits = mk[k];
        int o[U];
        // the table is 128-byte aligned and k a multiple of U: one 8- or 16-byte load for the group
        if (U == 2) {
            const int2 t = *reinterpret_cast<const int2 *>(base + k);
            o[0] = t.x;
            o[U - 1] = t.y;
        } else if (U == 4) {
            const int4 t = *reinterpret_cast<const int4 *>(base + k);
            o[0] = t.x;
            o[1 % U] = t.y;
            o[2 % U] = t.z;
            o[3 % U] = t.w;
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) o[u] = base[k + u];
        }
        int j[U];
        float w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned ju = (unsigned)ii + (unsigned)o[u];   // modular: a negative index wraps high
            j[u] = (CLAMP && ju >= (unsigned)N) ? alt : (int)ju;
            w[u] = (bits & (1u << u)) ? 0.0f : SLOT_PAD_Q;
        }
        bits >>= U;
        body(j, w, k);
    }
}

// Neighbour slots of row i in groups of U (U divides 32): body(j[U], qpad[U])
// for each group, qpad = 0 for a neighbour and SLOT_PAD_Q for a padding slot
// (whose j is a valid particle other than i, so its terms are finite).  The
// pair terms add qpad to the kernel argument q = r / h: a padding slot lands
// outside the kernel's support (q >= 2), where W and W' are exactly zero, so
// its terms vanish without a weight multiply.
template <int U, class Body>
__device__ __forceinline__ void for_slots(const DevState &s, int64_t i, Body &&body)
{
    const int64_t g = i >> 5;
    const int lane = (int)(i & 31);
    const int wv = s.ell_w[g];
    const int32_t *__restrict__ base = s.colE + s.ell_off[g];
    const int alt = i == 0 ? 1 : (int)i - 1;
    if (wv < 0) {
        const int W = (~wv) & 0xffffff;
        if ((~wv) >> 24) aligned_slots<U, true>(base, W, lane, (int)i, alt, (int)s.N, body);
        else aligned_slots<U, false>(base, W, lane, (int)i, alt, (int)s.N, body);
    } else {
        const int32_t *__restrict__ cp = base + lane;
        for (int k = 0; k < wv; k += U) {
            int j[U];
            float w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int kk = k + u;
                const int jj = kk < wv ? cp[32 * kk] : ~alt;
                j[u] = jj >= 0 ? jj : ~jj;
                w[u] = jj >= 0 ? 0.0f : SLOT_PAD_Q;
            }
            body(j, w, k);
        }
    }
}


// ------------------------------------------------------------------ compensated FP32
// A value carried as an unevaluated sum hi + lo of two floats keeps about 46
// significant bits, enough for quantities that accumulate small increments
// over many steps (F, the stress deviator).  The pair is kept canonical
// (hi = round(hi + lo)) and lo is rounded to 2^-45 of hi's binade, so
// hi + lo is exactly a double: export to FP64 and import back reproduce the
// pair bit for bit (checkpoints resume exactly).  The __fadd_rn forms keep
// the compiler from contracting or reordering the error-free transformations
// (Knuth's TwoSum, Dekker's FastTwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// canonical pair from h + l with |l| <= ulp(h): l on the grid 2^(E(h) - 45)
__device__ __forceinline__ void df_norm(float &h, float &l)
{
    const float p = __int_as_float(__float_as_int(h) & 0x7f800000);   // 2^E(h); 0 below the normal range
    const float C = p * 3.5762786865234375e-7f;                          // 1.5 * 2^(E - 22)
    const float lq = __fsub_rn(__fadd_rn(l, C), C);
    const float hn = __fadd_rn(h, lq);
    l = __fsub_rn(lq, __fsub_rn(hn, h));
    h = hn;
}
// (h, l) += x
__device__ __forceinline__ void df_add(float &h, float &l, float x)
{
    float s, e;
    two_sum(h, x, s, e);
    e = __fadd_rn(e, l);
    h = __fadd_rn(s, e);
    l = __fsub_rn(e, __fsub_rn(h, s));
    df_norm(h, l);
}
__device__ __forceinline__ void df_split(double x, float &h, float &l)
{
    h = (float)x;
    l = (float)(x - (double)h);
    df_norm(h, l);
}
__device__ __forceinline__ double df_value(float h, float l) { return (double)h + (double)l; }

// single-precision flow stress sigma_f of Algorithm 1 (Johnson-Cook hardening
// and lagged rate factor, as jc_hard * jc_rate)
__device__ __forceinline__ float jc_flow_f(const DevMat &m, float ep, float epdot)
{
    float r = 1.0f;
    if (m.Cf != 0.0f && m.inv_epsdot0f > 0.0f) {
        const float x = epdot * m.inv_epsdot0f;
        if (x > 1.0f) r = 1.0f + m.Cf * logf(x);
    }
    return (ep > 0.0f ? m.Af + m.Bf * powf(ep, m.nf) : m.Af) * r;
}
// single-precision mean stress (eos_sm) from J - 1
__device__ __forceinline__ float eos_sm_f(const DevMat &m, float Jm1, float J, float D, float e)
{
    float sm;
    if (m.eos == 0) {
        sm = m.Kf * Jm1;
    } else {
        const float eta = 1.0f / J, mu = -Jm1 * eta;
        const float den = eta - m.S_alphaf * mu;
        sm = -(m.rho0c02f * mu * (eta - 0.5f * m.Gamma0f * mu) / (den * den) + m.g0rho0f * e);
    }
    return sm > 0.0f ? sm * (1.0f - D) : sm;
}

// Single-precision elastic screen of the GTN return (Algorithm 2, Eq.
// yield_GTN): the trial state is inside the yield surface when
// Phi = x^2 + 2 q1 f* cosh(3/2 q2 T x) - (1 + q3 f*^2) <= 0 with x = sigma_eq / sigma_M
// and T = sigma_m / sigma_eq (elastic as well when sigma_eq < 1e-12 K).  In
// FP32 the terms of Phi are O(1) with rounding below 1e-6, so Phi <= -10 band
// (1 + q3 f*^2) implies the FP64 test passes; s2 = sigma_eq^2 of the trial.
__device__ __forceinline__ bool gtn_elastic_f(const DevMat &m, float s2, float sm, float ep, float epdot, float f,
                                              float keep)
{
    const float tiny = 1e-12f * m.Kf;
    if (s2 <= tiny * tiny * keep) return true;
    const float sM = jc_flow_f(m, ep, epdot);
    if (!(sM > 0.0f)) return false;
    const float fs = f <= m.fcf ? f : (f >= m.fFf ? 1.0f / m.q1f : m.fcf + m.fstar_slopef * (f - m.fcf));
    const float seq = sqrtf(s2);
    const float x = seq / sM, tri = sm / seq;
    const float c0 = 1.0f + m.q3f * fs * fs;
    const float phi = x * x + 2.0f * m.q1f * fs * coshf(1.5f * m.q2f * tri * x) - c0;
    return phi <= -10.0f * (1.0f - keep) * c0;
}

// The single-precision yield screen passes a particle when sigma_eq^2 <=
// sigma_f^2 (1 - band) in FP32.  The FP32 values of sigma_eq^2 and sigma_f^2
// are within 2e-6 of their FP64 counterparts, so any band >= 1e-5 (the
// default; tlsph_set_guard) implies the FP64 test passes; band >= 1 sends
// every particle to the FP64 update.

// ------------------------------------------------------------------ pass 1, per particle
// F^{n+1}, J, kinematics, constitutive and damage update, stress, A and the
// pass-2 record of particle i from its velocity-gradient sums keep[9].
//
// F and the stress deviator are compensated FP32 pairs.  J - 1 comes from the
// invariants of G = F - I (det(I + G) = 1 + tr G + m2(G) + det G), accurate
// to FP32 rounding of J - 1 itself.  A particle whose FP32 trial stress lies
// inside the yield surface by more than the guard band takes the elastic
// branch of Algorithm 1 in FP32 (no plastic increment, so no damage
// increment) in this kernel; every other particle (yielding, near yield,
// GTN, damage at or past initiation) is queued with its strain increment and
// finished by the FP64 material update in a separate kernel, so this kernel
// carries no FP64 return-mapping code (fewer registers, more resident warps).

// kinematics at F^{n+1}: G = F - I, J - 1, F^{-1} and the rotation R
struct Kin1 {
    float G[9], Fi[9], R[9];
    float Jm1, Jf;
};

__device__ __forceinline__ bool kin_from_F(const float *Fh, const float *Fl, Kin1 &k, uint32_t &st)
{
    // G = F - I (the diagonal's hi - 1 is exact for hi in [0.5, 2])
#pragma unroll
    for (int q = 0; q < 9; ++q) k.G[q] = ((q % 4 == 0) ? Fh[q] - 1.0f : Fh[q]) + Fl[q];
    const float *G = k.G;
    const float m2 = (G[0] * G[4] - G[1] * G[3]) + (G[4] * G[8] - G[5] * G[7]) + (G[0] * G[8] - G[2] * G[6]);
    const float m3 = G[0] * (G[4] * G[8] - G[5] * G[7]) + G[1] * (G[5] * G[6] - G[3] * G[8])
                   + G[2] * (G[3] * G[7] - G[4] * G[6]);
    k.Jm1 = (G[0] + G[4] + G[8]) + (m2 + m3);
    k.Jf = 1.0f + k.Jm1;
    if (!(k.Jf > 0.0f) || !isfinite(k.Jm1)) return false;
    float cf[9];
    cof3f(Fh, cf);
    const float iJ = 1.0f / k.Jf;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) k.Fi[3 * a + b] = cf[3 * b + a] * iJ;
    if (!polar_rotation_f(Fh, k.R)) st |= TLSPH_ST_POLAR_CAP;
    return true;
}

// Pass-2 record of a particle: six float4 components (tiled, r2_tile)
//   c0 {A00, A10, A01, A11}   c1 {A02, A12, A20, A21}   c2 {A22, V D, V, E V (1 - D)}
//   c3 {u0, u1, G00, G10}     c4 {G01, G11, G02, G12}   c5 {u2, G20, G21, G22}
// with A row-major (A[3r + c]), G = F - I and u in fixed-point units.  Rows 0
// and 1 of A and G and the first two components of u sit side by side in
// aligned float pairs, so that the pair terms take them two at a time with
// packed FP32x2 operations; a record without the hourglass term is c0..c2.
__device__ __forceinline__ void r2_store(float4 *__restrict__ r2, const float *A, float VD, float V, float EV,
                                         float u0, float u1, float u2, const float *G)
{
    r2[0] = make_float4(A[0], A[3], A[1], A[4]);
    r2[R2_STRIDE] = make_float4(A[2], A[5], A[6], A[7]);
    r2[2 * R2_STRIDE] = make_float4(A[8], VD, V, EV);
    r2[3 * R2_STRIDE] = make_float4(u0, u1, G[0], G[3]);
    r2[4 * R2_STRIDE] = make_float4(G[1], G[4], G[2], G[5]);
    r2[5 * R2_STRIDE] = make_float4(u2, G[6], G[7], G[8]);
}

// A (row-major) from the first three components of a pass-2 record
__device__ __forceinline__ void r2_A(const float4 c0, const float4 c1, const float4 c2, float *A)
{
    A[0] = c0.x; A[3] = c0.y; A[1] = c0.z; A[4] = c0.w;
    A[2] = c1.x; A[5] = c1.y; A[6] = c1.z; A[7] = c1.w;
    A[8] = c2.x;
}

// stress, A and the pass-2 record of a particle after its constitutive update
// internal-energy increment (Eq. conservation3, de/dt = J sigma : d / rho0), trapezoidal in the step:
// J / rho0 * (sigma^n + sigma^{n+1}) / 2 : dcur with dcur the step's strain increment in the current frame
__device__ __forceinline__ float sym_ddot_f(const float *a, const float *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + 2.0f * (a[3] * b[3] + a[4] * b[4] + a[5] * b[5]);
}

// The caller loads sigma^n and e^n before its first store (later loads could
// not be moved above stores through the other state pointers and would add
// two memory round trips per particle) and passes w0 = sigma^n : dcur.
__device__ __forceinline__ void epi1_finish(const DevState &s, const MixConst &c, int64_t i, const Kin1 &k,
                                            const float *Li, const float *sd, float sm, double Dnew, bool failed,
                                            const float *dcur, float w0, double e_n, float inv_rho0,
                                            float Vf, float u0, float u1, float u2, uint32_t st)
{
    const int64_t N = c.N;
    float4 *__restrict__ r2 = s.r2 + r2_tile(i);
    float A[9] = { 0, 0, 0, 0, 0, 0, 0, 0, 0 };
    float w = w0;
    const float ejr = 0.5f * k.Jf * inv_rho0;
    if (failed) {
        s.fail[i] = (int32_t)(c.step_index + 1);
#pragma unroll
        for (int q = 0; q < 6; ++q) s.sigf[q * N + i] = 0.0f;
    } else {
        // sigma = R (sigma_m I + s_hat) R^T ;  P = J sigma F^{-T} ;  A = P L^{-T}
        const float sh[6] = { sd[0] + sm, sd[1] + sm, sd[2] + sm, sd[3], sd[4], sd[5] };
        float sg[6];
        sym_rotate_f(k.R, sh, sg);
        w += sym_ddot_f(sg, dcur);
#pragma unroll
        for (int q = 0; q < 6; ++q) s.sigf[q * N + i] = sg[q];
        float S[9] = { sg[0], sg[3], sg[5], sg[3], sg[1], sg[4], sg[5], sg[4], sg[2] }, P[9];
        mul3f_bt(S, k.Fi, P);
#pragma unroll
        for (int q = 0; q < 9; ++q) P[q] *= k.Jf;
        mul3f_bt(P, Li, A);
        bool fin = true;
#pragma unroll
        for (int q = 0; q < 9; ++q) fin &= isfinite(A[q]);
        if (!fin) st |= TLSPH_ST_NONFINITE;
    }
    s.e[i] = e_n + (double)(ejr * w);
    const float omd = 1.0f - (float)Dnew;
    r2_store(r2, A, Vf * (float)Dnew, Vf, (float)s.youngs[i] * Vf * omd, u0, u1, u2, k.G);
    if (st) atomicOr(s.status, st);
}

__device__ __forceinline__ void load_u1(const DevState &s, const MixConst &c, int64_t i, float &u0, float &u1, float &u2)
{
    const double *un = s.u[c.ucur ^ 1];   // u^{n+1}, mirrored for pass 2's hourglass term (fixed-point units)
    u0 = (float)un[3 * i] * c.inv_unit_f;
    u1 = (float)un[3 * i + 1] * c.inv_unit_f;
    u2 = (float)un[3 * i + 2] * c.inv_unit_f;
}

__device__ __forceinline__ void epi1_mixed(const DevState &s, const MixConst &c, int64_t i, const float *keep)
{
    const double *__restrict__ Dn = s.D[c.dcur];
    double *__restrict__ Dnext = s.D[c.dcur ^ 1];
    const int64_t N = c.N;
    const int fail = s.fail[i];
    const float Vf = (float)s.vol[i];
    float Fh[9], Fl[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) { Fh[k] = s.Fh[k * N + i]; Fl[k] = s.Fl[k * N + i]; }
    float u0, u1, u2;
    load_u1(s, c, i, u0, u1, u2);
    // stress at the start of the step and internal energy, loaded before the first store (epi1_finish)
    float sgn[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) sgn[k] = s.sigf[k * N + i];
    const double e_n = s.e[i];
    if (fail >= 0) {            // fully damaged: no stress, F frozen, record with A = 0 and 1 - D = 0
        Dnext[i] = Dn[i];
        const float A0[9] = { 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f };
        float G[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) G[k] = ((k & 3) == 0 ? Fh[k] - 1.0f : Fh[k]) + Fl[k];
        r2_store(s.r2 + r2_tile(i), A0, Vf, Vf, 0.f, u0, u1, u2, G);    // V D with D = 1
        return;
    }
    float Li[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Li[k] = s.linv32[9 * i + k];
    // dF = dt Fdot (Fdot = M L^{-1}, Sec. 3.1); F^{n+1} = F^n + dF compensated
    float dF[9];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            dF[3 * k + l] = c.dt_dw * (keep[3 * k] * Li[l] + keep[3 * k + 1] * Li[3 + l] + keep[3 * k + 2] * Li[6 + l]);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        df_add(Fh[k], Fl[k], dF[k]);
        s.Fh[k * N + i] = Fh[k];
        s.Fl[k * N + i] = Fl[k];
    }
    Kin1 kin;
    uint32_t st = 0;
    if (!kin_from_F(Fh, Fl, kin, st)) {
        atomicOr(s.status, TLSPH_ST_BAD_J);
        Dnext[i] = Dn[i];
        return;
    }
    // unrotated strain increment dh = R^T sym(dt L_v) R with dt L_v = dF F^{-1}
    float Lv[9];
    mul3f(dF, kin.Fi, Lv);
    const float d[6] = { Lv[0], Lv[4], Lv[8], 0.5f * (Lv[1] + Lv[3]), 0.5f * (Lv[5] + Lv[7]), 0.5f * (Lv[2] + Lv[6]) };
    float dh[6];
    sym_rotate_t_f(kin.R, d, dh);

    const DevMat &mat = s.mats[s.mat[i]];
    const double Dd = Dn[i];
    const double dinit = s.dinit[i];
    const double epdot = s.epdot[i];
    float sdh[6], sdl[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) { sdh[k] = s.sdh[k * N + i]; sdl[k] = s.sdl[k * N + i]; }
    // FP32 screen (elastic branch of Algorithm 1)
    const float omDf = 1.0f - (float)Dd;
    const float trc = (dh[0] + dh[1] + dh[2]) * (1.0f / 3.0f);
    const float g2 = 2.0f * mat.Gf * omDf;
    float inc[6] = { g2 * (dh[0] - trc), g2 * (dh[1] - trc), g2 * (dh[2] - trc), g2 * dh[3], g2 * dh[4], g2 * dh[5] };
    float tr[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) tr[k] = sdh[k] + inc[k];
    const float s2 = 1.5f * ((tr[0] * tr[0] + tr[1] * tr[1] + tr[2] * tr[2]) +
                             2.0f * (tr[3] * tr[3] + tr[4] * tr[4] + tr[5] * tr[5]));
    const float sm = eos_sm_f(mat, kin.Jm1, kin.Jf, (float)Dd, (float)e_n);
    double por = 0.0;
    bool fast;
    if (mat.damage == TLSPH_DAMAGE_GTN) {
        por = s.por[i];
        fast = por < mat.fF && gtn_elastic_f(mat, s2, sm, (float)s.ep[i], (float)epdot, (float)por, c.yield_keep);
    } else {
        const float sf = jc_flow_f(mat, (float)s.ep[i], (float)epdot) * omDf;
        fast = dinit < 1.0 && sf > 0.0f && s2 <= sf * sf * c.yield_keep;
    }
    if (!fast) {
        // the FP64 update finishes this particle (k_epi1_slow): hand it the strain increment
#pragma unroll
        for (int k = 0; k < 6; ++k) s.fsum[k * N + i] = dh[k];
        const uint32_t q = atomicAdd(&s.slowq_n[c.step_index & 1], 1u);
        s.slowq[q] = (int32_t)i;
        if (st) atomicOr(s.status, st);
        return;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        df_add(sdh[k], sdl[k], inc[k]);
        s.sdh[k * N + i] = sdh[k];
        s.sdl[k * N + i] = sdl[k];
    }
    if (epdot != 0.0) s.epdot[i] = 0.0;
    // D of the unchanged damage variables: Sec. 5.3 with D_init < 1 (CL, JC), q1 f*(f) (GTN), unchanged (none)
    const double Dnew = mat.damage == TLSPH_DAMAGE_NONE ? Dd
                      : (mat.damage == TLSPH_DAMAGE_GTN ? mat.q1 * gtn_fstar(mat, por) : 0.0);
    Dnext[i] = Dnew;
    epi1_finish(s, c, i, kin, Li, sdh, sm, Dnew, false, d, sym_ddot_f(sgn, d), e_n, mat.inv_rho0f, Vf, u0, u1,
                u2, st);
}

// FP64 constitutive and damage update of a queued particle (F^{n+1} already
// stored, its unrotated strain increment in fsum[0..5])
__device__ __forceinline__ void epi1_slow(const DevState &s, const MixConst &c, int64_t i)
{
    const double *__restrict__ Dn = s.D[c.dcur];
    double *__restrict__ Dnext = s.D[c.dcur ^ 1];
    const int64_t N = c.N;
    const float Vf = (float)s.vol[i];
    float Fh[9], Fl[9], Li[9], sgn[6];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Fh[k] = s.Fh[k * N + i];
        Fl[k] = s.Fl[k * N + i];
        Li[k] = s.linv32[9 * i + k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) sgn[k] = s.sigf[k * N + i];
    float u0, u1, u2;
    load_u1(s, c, i, u0, u1, u2);
    Kin1 kin;
    uint32_t st = 0;
    kin_from_F(Fh, Fl, kin, st);     // same inputs and code as the first kernel: J was valid there
    const DevMat &mat = s.mats[s.mat[i]];
    MPState mp;
#pragma unroll
    for (int k = 0; k < 6; ++k) mp.sd[k] = df_value(s.sdh[k * N + i], s.sdl[k * N + i]);
    mp.sm = 0.0;
    mp.ep = s.ep[i];
    mp.epdot = s.epdot[i];
    mp.dinit = s.dinit[i];
    mp.D = Dn[i];
    mp.f = s.por[i];
    const double e_n = s.e[i];
    mp.e = e_n;
    mp.failed = 0;
    double de[6];
    float dh[6], dcur[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        dh[k] = s.fsum[k * N + i];
        de[k] = (double)dh[k];
    }
    sym_rotate_f(kin.R, dh, dcur);      // the strain increment back in the current frame
    st |= material_update<true>(mat, c.dt, de, 1.0 + (double)kin.Jm1, mp);
    float sdh[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float l;
        df_split(mp.sd[k], sdh[k], l);
        s.sdh[k * N + i] = sdh[k];
        s.sdl[k * N + i] = l;
    }
    s.ep[i] = mp.ep;
    s.epdot[i] = mp.epdot;
    s.dinit[i] = mp.dinit;
    s.por[i] = mp.f;
    Dnext[i] = mp.D;
    epi1_finish(s, c, i, kin, Li, sdh, (float)mp.sm, mp.D, mp.failed != 0, dcur, sym_ddot_f(sgn, dcur), e_n,
                mat.inv_rho0f, Vf, u0, u1, u2, st);
}

// persistent grid over the step's queue of FP64 updates; clears the queue
// counter of the next step (the two counters alternate with the step parity)
__global__ void __launch_bounds__(128) k_epi1_slow(DevState s, MixConst c)
{
    const uint32_t n = s.slowq_n[c.step_index & 1];
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        epi1_slow(s, c, s.slowq[q]);
    if (blockIdx.x == 0 && threadIdx.x == 0) s.slowq_n[(c.step_index + 1) & 1] = 0u;
}

// weight V (1 - D) of the pass-1 record, formed the same way (FP32, each
// rounding written out) by the pass-2 epilogue that refreshes the record every
// step and by the kernel that rebuilds it after a state change, so that a
// resumed run gathers exactly the records of the uninterrupted one
__device__ __forceinline__ float r1_weight(float V, float D) { return __fmul_rn(V, __fsub_rn(1.0f, D)); }

// ------------------------------------------------------------------ pass 1 pair terms
// W'(q)/r of a pair in fixed-point units (qpad as for the slots), every
// rounding spelled out, so that the per-slot weight table and the kernels that
// form the weight in place give the same bits
__device__ __forceinline__ float w1_weight(const float3 d, float inv_h, float qpad)
{
    const float r2 = __fmaf_rn(d.z, d.z, __fmaf_rn(d.y, d.y, __fmul_rn(d.x, d.x)));
    const float rinv = rsqrtf(r2);
    const float q = __fmaf_rn(__fmul_rn(r2, rinv), inv_h, qpad);
    const float a = fmaxf(__fsub_rn(2.0f, q), 0.0f), b = fmaxf(__fsub_rn(1.0f, q), 0.0f);
    return __fmul_rn(__fmaf_rn(__fmul_rn(3.0f, b), b, __fmul_rn(__fmul_rn(-0.75f, a), a)), rinv);
}

// the pair's terms of the nine sums M = sum_j V_j (1 - D_j) W'/r (v_j - v_i) (X_j - X_i)^T
__device__ __forceinline__ void pair1w(const float3 d, const float4 vi, const float4 vj, float w, float *m)
{
    const float cw = __fmul_rn(vj.w, w);       // V_j (1 - D_j) W'/r
    const float cx = cw * (vj.x - vi.x), cy = cw * (vj.y - vi.y), cz = cw * (vj.z - vi.z);
    m[0] += cx * d.x; m[1] += cx * d.y; m[2] += cx * d.z;
    m[3] += cy * d.x; m[4] += cy * d.y; m[5] += cy * d.z;
    m[6] += cz * d.x; m[7] += cz * d.y; m[8] += cz * d.z;
}

__device__ __forceinline__ void pair1(const MixConst &c, const int4 oi, const float4 vi, const int4 oj,
                                      const float4 vj, float qpad, float *m)
{
    const float3 d = xdiff(oj, oi);
    pair1w(d, vi, vj, w1_weight(d, c.inv_h, qpad), m);
}

// thread per row over the sliced neighbour lists, U pairs in flight; with TAB
// (four pairs in flight) the weights come from the per-slot table, one float4
// per group of four slots, laid out [group][lane] within the slice
template <int U, bool TAB = false>
__device__ __forceinline__ void gather1_row(const DevState &s, const MixConst &c, int64_t i, float *m)
{
    const int4 oi = s.xo[i];
    const float4 vi = s.r1[i];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = 0.0f;
    if constexpr (TAB) {
        static_assert(U == 4, "the weight table holds groups of four slots");
        const float4 *__restrict__ tb = s.w1t + s.w1t_off[i >> 5] + (i & 31);
        for_slots<U>(s, i, [&](const int *j, const float *, int k) {
            int4 o[U];
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) { o[u] = s.xo[j[u]]; v[u] = s.r1[j[u]]; }
            const float4 t = tb[8 * k];      // group k / 4: float4 index 32 (k / 4) + lane
            const float tw[4] = { t.x, t.y, t.z, t.w };
#pragma unroll
            for (int u = 0; u < U; ++u) pair1w(xdiff(o[u], oi), vi, v[u], tw[u % 4], m);
        });
        return;
    }
    for_slots<U>(s, i, [&](const int *j, const float *w, int) {
        int4 o[U];
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) { o[u] = s.xo[j[u]]; v[u] = s.r1[j[u]]; }
#pragma unroll
        for (int u = 0; u < U; ++u) pair1(c, oi, vi, o[u], v[u], w[u], m);
    });
}

// warp per 32 consecutive rows over the CSR (lanes stride a row)
__device__ __forceinline__ void gather1_w32(const DevState &s, const MixConst &c, int64_t row0, int nrows, int lane,
                                            float *keep)
{
#pragma unroll
    for (int k = 0; k < 9; ++k) keep[k] = 0.0f;
    for (int r = 0; r < nrows; ++r) {
        const int64_t i = row0 + r;
        const int4 oi = s.xo[i];
        const float4 vi = s.r1[i];
        const int64_t p0 = s.row_ptr[i], p1 = s.row_ptr[i + 1];
        float m[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) m[k] = 0.0f;
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int j = s.col[p];
            pair1(c, oi, vi, s.xo[j], s.r1[j], 0.0f, m);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float t = warp_allsum(m[k]);
            keep[k] = (lane == r) ? t : keep[k];
        }
    }
}

__global__ void __launch_bounds__(MIX_THREADS) k_pass1_mixed(DevState s, MixConst c)
{
    const int lane = threadIdx.x & 31;
    const int64_t row0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5;
    if (row0 >= s.N) return;
    const int nrows = (int)min((int64_t)32, s.N - row0);
    float keep[9];
    gather1_w32(s, c, row0, nrows, lane, keep);
    if (lane >= nrows) return;
    epi1_mixed(s, c, row0 + lane, keep);
}

__global__ void __launch_bounds__(256) k_pass1_mixed_t(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float m[9];
    gather1_row<2>(s, c, i, m);
    epi1_mixed(s, c, i, m);
}

// split form of pass 1: the gather kernel stores the 9 sums, a second kernel
// runs the per-particle update (lighter registers in the gather)
__global__ void __launch_bounds__(256) k_gather1_mixed_t(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float m[9];
    gather1_row<2>(s, c, i, m);
#pragma unroll
    for (int k = 0; k < 9; ++k) s.fsum[k * s.N + i] = m[k];
}

__global__ void __launch_bounds__(256) k_gather1_mixed_w32(DevState s, MixConst c)
{
    const int lane = threadIdx.x & 31;
    const int64_t row0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5;
    if (row0 >= s.N) return;
    const int nrows = (int)min((int64_t)32, s.N - row0);
    float keep[9];
    gather1_w32(s, c, row0, nrows, lane, keep);
    if (lane >= nrows) return;
#pragma unroll
    for (int k = 0; k < 9; ++k) s.fsum[k * s.N + row0 + lane] = keep[k];
}

#ifndef EPI1_MINB
#define EPI1_MINB 5
#endif
__global__ void __launch_bounds__(128, EPI1_MINB) k_epi1_mixed(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = s.fsum[k * s.N + i];
    epi1_mixed(s, c, i, m);
}

// ------------------------------------------------------------------ pass 2
// per-particle part: force (rearranged Sec. 3.1 form) and the velocity-Verlet
// update in FP64 from the pair sums keep[9]
template <bool HG>
__device__ __forceinline__ void epi2_mixed(const DevState &s, const MixConst &c, int64_t i, const float *keep)
{
    const float4 *ri = s.r2 + r2_tile(i);
    const float4 a0 = ri[0], a1 = ri[R2_STRIDE], a2 = ri[2 * R2_STRIDE];
    float Ai[9];
    r2_A(a0, a1, a2, Ai);
    const float Vf = a2.z;                           // V_i
    const float Df = (float)s.D[c.dcur ^ 1][i];      // D_i^{n+1}
    const float omdf = 1.0f - Df;
    const float4 s0 = s.s0[i];
    const float w2 = 2.0f - Df;
    const float bx = w2 * s0.x - keep[0], by = w2 * s0.y - keep[1], bz = w2 * s0.z - keep[2];
    const float vdw = Vf * c.dw_norm;
    float f[3];
    f[0] = vdw * ((Ai[0] * bx + Ai[1] * by + Ai[2] * bz) + omdf * keep[3]);
    f[1] = vdw * ((Ai[3] * bx + Ai[4] * by + Ai[5] * bz) + omdf * keep[4]);
    f[2] = vdw * ((Ai[6] * bx + Ai[7] * by + Ai[8] * bz) + omdf * keep[5]);
    if (HG) {
        // the pair sums are in fixed-point units (X_ij, u_ij and x_ij scaled by 1/unit): hg_w folds 1/unit in;
        // the sums carry (E_i + E_j) V_j (1 - D_j), the 1/2 of the pair modulus is taken here
        const float hc = c.hg_w * 0.5f * Vf * omdf;
        f[0] += hc * keep[6];
        f[1] += hc * keep[7];
        f[2] += hc * keep[8];
    }
    // the integrator in FP64 from the FP32 force; the half kick is the
    // predictor's (kick, explicitly rounded), so a state reloaded from a
    // checkpoint predicts exactly the v^{n+1/2} of the uninterrupted run
    const double im = s.inv_mass[i];
    const int fail = s.fail[i];
    double vn[3], v2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        s.force[3 * i + k] = (double)f[k];
        vn[k] = kick(s.vh[3 * i + k], c.half_dt, (double)f[k], im);
    }
    // velocity constraints (Sec. 3.1; grip ramp of Sec. 6 at t_{n+1} and at t_{n+3/2})
    if (fail >= 0) {
        vn[0] = vn[1] = vn[2] = 0.0;
    } else if (s.bcm[i]) {
        const double r = grip_factor(s.grip_ramp, ((double)c.step_index + 1.0) * c.dt);
        vn[0] = s.bcv[3 * i] * r; vn[1] = s.bcv[3 * i + 1] * r; vn[2] = s.bcv[3 * i + 2] * r;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) v2[k] = kick(vn[k], c.half_dt, (double)f[k], im);
    if (fail >= 0) {
        v2[0] = v2[1] = v2[2] = 0.0;
    } else if (s.bcm[i]) {
        const double r = grip_factor(s.grip_ramp, ((double)(c.step_index + 1) + 0.5) * c.dt);
        v2[0] = s.bcv[3 * i] * r; v2[1] = s.bcv[3 * i + 1] * r; v2[2] = s.bcv[3 * i + 2] * r;
    }
    const double *un = s.u[c.ucur ^ 1];
    double *unext = s.u[c.ucur];
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
    s.r1[i] = make_float4((float)(v2[0] - c.vref0), (float)(v2[1] - c.vref1), (float)(v2[2] - c.vref2),
                          r1_weight(Vf, Df));
    if (!(isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]))) atomicOr(s.status, TLSPH_ST_NONFINITE);
}

struct Row2 {   // row i's own pass-2 record, negated where the pair terms subtract it
    int4 o;
    float2 nA0, nA1, nA2;     // -(A_0c, A_1c), c = 0, 1, 2
    float nA20, nA21, nA22;   // -A_2c
    float2 nu01;              // -(u_0, u_1)
    float nu2;                // -u_2
    float2 G0, G1, G2;        // (G_0c, G_1c)
    float G20, G21, G22;
    float E;                  // Young modulus of row i's material (hourglass term)
};

__device__ __forceinline__ float2 neg2(const float a, const float b) { return make_float2(-a, -b); }

template <bool HG>
__device__ __forceinline__ Row2 load_row2(const DevState &s, const MixConst &c, int64_t i)
{
    const float4 *ri = s.r2 + r2_tile(i);
    Row2 w;
    w.o = s.xo[i];
    const float4 a0 = ri[0], a1 = ri[R2_STRIDE], a2 = ri[2 * R2_STRIDE];
    w.nA0 = neg2(a0.x, a0.y);
    w.nA1 = neg2(a0.z, a0.w);
    w.nA2 = neg2(a1.x, a1.y);
    w.nA20 = -a1.z;
    w.nA21 = -a1.w;
    w.nA22 = -a2.x;
    w.nu01 = make_float2(0.f, 0.f);
    w.G0 = w.G1 = w.G2 = make_float2(0.f, 0.f);
    w.nu2 = w.G20 = w.G21 = w.G22 = w.E = 0.0f;
    if (HG) {
        const float4 a3 = ri[3 * R2_STRIDE], a4 = ri[4 * R2_STRIDE], a5 = ri[5 * R2_STRIDE];
        w.E = (float)s.youngs[i];
        w.nu01 = neg2(a3.x, a3.y);
        w.nu2 = -a5.x;
        w.G0 = make_float2(a3.z, a3.w);
        w.G1 = make_float2(a4.x, a4.y);
        w.G2 = make_float2(a4.z, a4.w);
        w.G20 = a5.y;
        w.G21 = a5.z;
        w.G22 = a5.w;
    }
    return w;
}

// Pair terms of row i with neighbour j (qpad: 0, or SLOT_PAD_Q for a padding
// slot).  The row's own A and u are held negated, so the differences are sums.
// With PK, rows 0 and 1 of (A_j - A_i) X_ij are formed together by packed
// FP32x2 operations on the record's column pairs (same roundings as the
// scalar form); the scalar form is the faster one on most lists, the packed
// one on fully aligned lattice lists.
template <bool HG, bool PK = false>
__device__ __forceinline__ void pair2(const DevState &s, const MixConst &c, const Row2 &w, int j, float qpad,
                                      float *acc)
{
    const int4 oj = s.xo[j];
    const float4 *rj = s.r2 + r2_tile(j);
    const float4 b0 = rj[0], b1 = rj[R2_STRIDE], b2 = rj[2 * R2_STRIDE];
    const float3 d = xdiff(oj, w.o);
    const float r2v = d.x * d.x + d.y * d.y + d.z * d.z;
    const float rinv = rsqrtf(r2v);
    const float q = fmaf(r2v * rinv, c.inv_h, qpad);
    float a, b;
    const float g0 = spline_dw_ab(q, a, b) * rinv;
    const float g = b2.z * g0;                     // V_j W'/r
    const float gd = b2.y * g0;                    // V_j D_j W'/r
    acc[0] += gd * d.x; acc[1] += gd * d.y; acc[2] += gd * d.z;
    // (A_j - A_i) X_ij
    float t0, t1;
    if (PK) {
        const float2 dx2 = make_float2(d.x, d.x), dy2 = make_float2(d.y, d.y), dz2 = make_float2(d.z, d.z);
        const float2 t01 = __ffma2_rn(__fadd2_rn(make_float2(b1.x, b1.y), w.nA2), dz2,
                                      __ffma2_rn(__fadd2_rn(make_float2(b0.z, b0.w), w.nA1), dy2,
                                                 __fmul2_rn(__fadd2_rn(make_float2(b0.x, b0.y), w.nA0), dx2)));
        t0 = t01.x;
        t1 = t01.y;
    } else {
        t0 = (b0.x + w.nA0.x) * d.x + (b0.z + w.nA1.x) * d.y + (b1.x + w.nA2.x) * d.z;
        t1 = (b0.y + w.nA0.y) * d.x + (b0.w + w.nA1.y) * d.y + (b1.y + w.nA2.y) * d.z;
    }
    const float t2 = fmaf(b2.x + w.nA22, d.z, fmaf(b1.w + w.nA21, d.y, (b1.z + w.nA20) * d.x));
    acc[3] += g * t0; acc[4] += g * t1; acc[5] += g * t2;
    if (HG) {
        const float4 b3 = rj[3 * R2_STRIDE], b4 = rj[4 * R2_STRIDE], b5 = rj[5 * R2_STRIDE];
        // u_ij, x_ij = X_ij + u_ij, e = ((F_i - I) + (F_j - I)) X_ij - 2 u_ij
        const float ux = b3.x + w.nu01.x, uy = b3.y + w.nu01.y, uz = b5.x + w.nu2;
        const float xx = d.x + ux, xy = d.y + uy, xz = d.z + uz;
        const float lxi2 = rcp_approx(fmaf(xz, xz, fmaf(xy, xy, xx * xx)));   // 1 / |x_ij|^2
        const float ex = (b3.z + w.G0.x) * d.x + (b4.x + w.G1.x) * d.y + (b4.z + w.G2.x) * d.z - 2.0f * ux;
        const float ey = (b3.w + w.G0.y) * d.x + (b4.y + w.G1.y) * d.y + (b4.w + w.G2.y) * d.z - 2.0f * uy;
        const float ez = fmaf(b5.w + w.G22, d.z, fmaf(b5.z + w.G21, d.y, fmaf(b5.y + w.G20, d.x, -2.0f * uz)));
        // (E_i + E_j) V_j (1 - D_j) W / X_ij^2 * delta / |x_ij| with delta = (e . x_ij) / |x_ij|;
        // V_j (1 - D_j) = V_j - V_j D_j, and the record carries E_j V_j (1 - D_j)
        const float ev = fmaf(w.E, b2.z - b2.y, b2.w);
        const float ch = ev * spline_w_ab(a, b) * rinv * rinv * fmaf(ez, xz, fmaf(ey, xy, ex * xx)) * lxi2;
        acc[6] += ch * xx; acc[7] += ch * xy; acc[8] += ch * xz;
    }
}

template <bool HG>
__global__ void __launch_bounds__(MIX_THREADS) k_pass2_mixed(DevState s, MixConst c)
{
    const int lane = threadIdx.x & 31;
    const int64_t row0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5;
    if (row0 >= s.N) return;
    const int nrows = (int)min((int64_t)32, s.N - row0);
    float keep[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) keep[k] = 0.0f;
    for (int r = 0; r < nrows; ++r) {
        const int64_t i = row0 + r;
        const Row2 w = load_row2<HG>(s, c, i);
        const int64_t p0 = s.row_ptr[i], p1 = s.row_ptr[i + 1];
        float acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
        for (int64_t p = p0 + lane; p < p1; p += 32) pair2<HG>(s, c, w, s.col[p], 0.0f, acc);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (!HG && k >= 6) continue;
            const float t = warp_allsum(acc[k]);
            keep[k] = (lane == r) ? t : keep[k];
        }
    }
    if (lane >= nrows) return;
    epi2_mixed<HG>(s, c, row0 + lane, keep);
}

// pass-2 pair sums of row i over its slots, U pairs in flight
template <bool HG, int U, bool PK = false>
__device__ __forceinline__ void gather2_row(const DevState &s, const MixConst &c, int64_t i, float *acc)
{
    const Row2 w = load_row2<HG>(s, c, i);
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
    for_slots<U>(s, i, [&](const int *j, const float *wm, int) {
#pragma unroll
        for (int u = 0; u < U; ++u) pair2<HG, PK>(s, c, w, j[u], wm[u], acc);
    });
}

template <bool HG>
__global__ void __launch_bounds__(256) k_pass2_mixed_t(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float acc[9];
    gather2_row<HG, 2>(s, c, i, acc);
    epi2_mixed<HG>(s, c, i, acc);
}

// one pair in flight per thread (fewer registers, more resident warps)
template <bool HG>
__global__ void __launch_bounds__(256) k_pass2_mixed_t1(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float acc[9];
    gather2_row<HG, 1>(s, c, i, acc);
    epi2_mixed<HG>(s, c, i, acc);
}

// one pair in flight, registers capped so that eight blocks of 128 fit an SM
template <bool HG>
__global__ void __launch_bounds__(128, 8) k_pass2_mixed_t1c(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float acc[9];
    gather2_row<HG, 1>(s, c, i, acc);
    epi2_mixed<HG>(s, c, i, acc);
}

// two pairs in flight, registers capped so that seven blocks of 128 fit an SM
template <bool HG>
__global__ void __launch_bounds__(128, 7) k_pass2_mixed_tc7(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float acc[9];
    gather2_row<HG, 2>(s, c, i, acc);
    epi2_mixed<HG>(s, c, i, acc);
}

// two pairs in flight, registers capped so that five blocks of 128 fit an SM
template <bool HG>
__global__ void __launch_bounds__(128, 5) k_pass2_mixed_tc5(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float acc[9];
    gather2_row<HG, 2>(s, c, i, acc);
    epi2_mixed<HG>(s, c, i, acc);
}

// as k_pass2_mixed_tc5 with the packed FP32x2 stress rows
template <bool HG>
__global__ void __launch_bounds__(128, 5) k_pass2_mixed_tc5p(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float acc[9];
    gather2_row<HG, 2, true>(s, c, i, acc);
    epi2_mixed<HG>(s, c, i, acc);
}

// two pairs in flight, registers capped so that six blocks of 128 fit an SM
template <bool HG>
__global__ void __launch_bounds__(128, 6) k_pass2_mixed_tc(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float acc[9];
    gather2_row<HG, 2>(s, c, i, acc);
    epi2_mixed<HG>(s, c, i, acc);
}

__global__ void __launch_bounds__(256) k_gather1_mixed_t4(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float m[9];
    gather1_row<4>(s, c, i, m);
#pragma unroll
    for (int k = 0; k < 9; ++k) s.fsum[k * s.N + i] = m[k];
}

// as k_gather1_mixed_t4 with the weights from the per-slot table; registers
// capped for nine resident blocks of 128, as the gather now waits on the
// table's DRAM stream and more warps keep more of it in flight
__global__ void __launch_bounds__(128, 9) k_gather1_mixed_t4w(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float m[9];
    gather1_row<4, true>(s, c, i, m);
#pragma unroll
    for (int k = 0; k < 9; ++k) s.fsum[k * s.N + i] = m[k];
}

// split form of pass 2: a gather kernel with no FP64 epilogue stores the 9
// pair sums; a second kernel computes the force and integrates
template <bool HG>
__global__ void __launch_bounds__(256) k_gather2_mixed_t(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float acc[9];
    gather2_row<HG, 2>(s, c, i, acc);
#pragma unroll
    for (int k = 0; k < 9; ++k) s.fsum[k * s.N + i] = acc[k];
}

template <bool HG>
__global__ void __launch_bounds__(128) k_epi2_mixed(DevState s, MixConst c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    float m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = s.fsum[k * s.N + i];
    epi2_mixed<HG>(s, c, i, m);
}

// ------------------------------------------------------------------ mirrors
// static records from the FP64 inputs: fixed-point positions, S0, L^{-1}
__global__ void k_mixed_positions(DevState s, FixPack pk)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    int x[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = (int)llrint((s.X[3 * i + k] - pk.center[k]) * pk.inv_unit);
    s.xo[i] = make_int4(x[0], x[1], x[2], 0);
}

__global__ void k_mixed_static(DevState s, const double *S0)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    s.s0[i] = make_float4((float)S0[3 * i], (float)S0[3 * i + 1], (float)S0[3 * i + 2], 0.0f);
#pragma unroll
    for (int k = 0; k < 9; ++k) s.linv32[9 * i + k] = (float)s.Linv[9 * i + k];
}

// pass-1 record from the FP64 half-step velocity and D^n
__global__ void k_mixed_r1(DevState s, int dcur)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    s.r1[i] = make_float4((float)(s.vh[3 * i] - s.vref[0]), (float)(s.vh[3 * i + 1] - s.vref[1]),
                          (float)(s.vh[3 * i + 2] - s.vref[2]), r1_weight((float)s.vol[i], (float)s.D[dcur][i]));
}

// FP64 copy of A from the pass-2 records (for reading the state)
__global__ void k_mixed_export_A(DevState s)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    const float4 *ri = s.r2 + r2_tile(i);
    float A[9];
    r2_A(ri[0], ri[R2_STRIDE], ri[2 * R2_STRIDE], A);
#pragma unroll
    for (int k = 0; k < 9; ++k) s.A[9 * i + k] = (double)A[k];
}

// compensated F, stress deviator and FP32 stress -> FP64 arrays (which = bit
// set of 1 F, 2 stress deviator, 4 Cauchy stress)
__global__ void k_mixed_export(DevState s, int which)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = s.N;
    if (i >= N) return;
    if (which & 1)
#pragma unroll
        for (int k = 0; k < 9; ++k) s.F[9 * i + k] = df_value(s.Fh[k * N + i], s.Fl[k * N + i]);
    if (which & 2)
#pragma unroll
        for (int k = 0; k < 6; ++k) s.sd[6 * i + k] = df_value(s.sdh[k * N + i], s.sdl[k * N + i]);
    if (which & 4)
#pragma unroll
        for (int k = 0; k < 6; ++k) s.sig[6 * i + k] = (double)s.sigf[k * N + i];
}

// FP64 arrays -> compensated state (same bit set)
__global__ void k_mixed_import(DevState s, int which)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = s.N;
    if (i >= N) return;
    if (which & 1)
#pragma unroll
        for (int k = 0; k < 9; ++k) df_split(s.F[9 * i + k], s.Fh[k * N + i], s.Fl[k * N + i]);
    if (which & 2)
#pragma unroll
        for (int k = 0; k < 6; ++k) df_split(s.sd[6 * i + k], s.sdh[k * N + i], s.sdl[k * N + i]);
    if (which & 4)
#pragma unroll
        for (int k = 0; k < 6; ++k) s.sigf[k * N + i] = (float)s.sig[6 * i + k];
}

static int mixed_field_bits(int field)
{
    switch (field) {
    case -1: return 7;
    case TLSPH_FIELD_F: return 1;
    case TLSPH_FIELD_STRESS_DEV: return 2;
    case TLSPH_FIELD_SIGMA: return 4;
    default: return 0;
    }
}

static unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t mixed_import(const tlsph_ctx &ctx, int field, cudaStream_t st)
{
    const int bits = mixed_field_bits(field);
    if (bits == 0 || ctx.N == 0) return cudaSuccess;
    k_mixed_import<<<nb(ctx.N, 256), 256, 0, st>>>(ctx.s, bits);
    return cudaGetLastError();
}

cudaError_t mixed_init_positions(const DevState &s, const FixPack &pk, cudaStream_t st)
{
    k_mixed_positions<<<nb(s.N, 256), 256, 0, st>>>(s, pk);
    return cudaGetLastError();
}

cudaError_t mixed_init_static(const DevState &s, const double *S0, cudaStream_t st)
{
    k_mixed_static<<<nb(s.N, 256), 256, 0, st>>>(s, S0);
    return cudaGetLastError();
}

// Correction matrix (Sec. 2.2, Eq. correction_matrix) and S0 of a mixed
// context: thread per row over the sliced lists, with the X_ij the steps use
// (exact fixed-point differences rounded once to FP32) and FP32 pair terms;
// each row sum is Kahan-compensated in FP32 and finished in FP64, and the 3x3
// inversion is FP64 (same singularity test as the FP64 path).  In units u of
// the fixed-point grid, X_ij (x) X_ij / r = u d (x) d / |d| and X_ij / r = d / |d|.
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x)
{
    const float y = __fsub_rn(x, comp);
    const float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

__global__ void __launch_bounds__(256) k_shape_mixed(DevState s, float inv_h, double l_scale, double *Linv,
                                                     double *S0, uint32_t *n_singular)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.N) return;
    const int4 oi = s.xo[i];
    float sm[9], cp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) sm[k] = cp[k] = 0.0f;
    for_slots<2>(s, i, [&](const int *j, const float *w, int) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float3 d = xdiff(s.xo[j[u]], oi);
            const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
            const float rinv = rsqrtf(r2);
            float a, b;
            const float c0 = (float)s.vol[j[u]] * spline_dw_ab(fmaf(r2 * rinv, inv_h, w[u]), a, b) * rinv;
            kahan_add(sm[0], cp[0], c0 * d.x);
            kahan_add(sm[1], cp[1], c0 * d.y);
            kahan_add(sm[2], cp[2], c0 * d.z);
            kahan_add(sm[3], cp[3], c0 * d.x * d.x);
            kahan_add(sm[4], cp[4], c0 * d.y * d.y);
            kahan_add(sm[5], cp[5], c0 * d.z * d.z);
            kahan_add(sm[6], cp[6], c0 * d.x * d.y);
            kahan_add(sm[7], cp[7], c0 * d.y * d.z);
            kahan_add(sm[8], cp[8], c0 * d.z * d.x);
        }
    });
    double v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = (double)sm[k] - (double)cp[k];
    S0[3 * i] = v[0]; S0[3 * i + 1] = v[1]; S0[3 * i + 2] = v[2];
    const double l[6] = { l_scale * v[3], l_scale * v[4], l_scale * v[5], l_scale * v[6], l_scale * v[7],
                          l_scale * v[8] };
    double L[9], c[9];
    sym_to_full(l, L);
    cof3(L, c);
    const double det = L[0] * c[0] + L[1] * c[1] + L[2] * c[2];
    double fn2 = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) fn2 += L[k] * L[k];
    const double fn = sqrt(fn2);
    const bool ok = isfinite(det) && fabs(det) > 1e-12 * fn * fn * fn;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) Linv[9 * i + 3 * k + m] = ok ? c[3 * m + k] / det : 0.0;
    if (!ok) atomicAdd(n_singular, 1u);
}

cudaError_t mixed_shape_matrix(const DevState &s, double h, double *Linv, double *S0, uint32_t *n_singular,
                               cudaStream_t st)
{
    const double dw_norm = 1.0 / (M_PI * h * h * h * h);
    k_shape_mixed<<<nb(s.N, 256), 256, 0, st>>>(s, (float)(s.pack.unit / h), dw_norm * s.pack.unit, Linv, S0,
                                                  n_singular);
    return cudaGetLastError();
}

cudaError_t mixed_ell_widths(const DevState &s, int64_t *ell_off, cudaStream_t st)
{
    const int64_t rows = (s.N + 31) / 32 * 32;
    k_ell_plan<<<nb(rows, 256), 256, 0, st>>>(s.row_ptr, s.col, s.N, const_cast<int32_t *>(s.ell_w), ell_off);
    return cudaGetLastError();
}

cudaError_t mixed_ell_fill(const DevState &s, const int64_t *ell_off, int32_t *colE, cudaStream_t st)
{
    const int64_t rows = (s.N + 31) / 32 * 32;
    k_ell_fill<<<nb(rows, 256), 256, 0, st>>>(s.row_ptr, s.col, s.N, s.ell_w, ell_off, colE);
    return cudaGetLastError();
}

// the weight W'(q)/r of every slot of the sliced lists (zero for a padding
// slot), for pass-1 plan form 5: static, as it depends on the reference
// configuration only; thread per row, rows past N of the last slice zeroed
__global__ void __launch_bounds__(256) k_w1t_fill(DevState s, float inv_h)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g = i >> 5;
    if (g >= (s.N + 31) / 32) return;
    float4 *tb = const_cast<float4 *>(s.w1t) + s.w1t_off[g] + (i & 31);
    if (i >= s.N) {
        const int wv = s.ell_w[g];
        const int W = wv < 0 ? ((~wv) & 0xffffff) : wv;
        for (int k = 0; k < W; k += 4) tb[8 * k] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const int4 oi = s.xo[i];
    for_slots<4>(s, i, [&](const int *j, const float *w, int k) {
        float t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u] = w1_weight(xdiff(s.xo[j[u]], oi), inv_h, w[u]);
        tb[8 * k] = make_float4(t[0], t[1], t[2], t[3]);
    });
}

cudaError_t mixed_w1t_fill(const DevState &s, float inv_h, cudaStream_t st)
{
    const int64_t rows = (s.N + 31) / 32 * 32;
    k_w1t_fill<<<nb(rows, 256), 256, 0, st>>>(s, inv_h);
    return cudaGetLastError();
}

cudaError_t mixed_after_predict(const DevState &s, int dcur, cudaStream_t st)
{
    k_mixed_r1<<<nb(s.N, 256), 256, 0, st>>>(s, dcur);
    // the state may have been replaced (set_state, restore): start both step-parity queues empty
    return cudaMemsetAsync(s.slowq_n, 0, 2 * sizeof(uint32_t), st);
}

// persistent grid of the FP64-update kernel on the current device: SMs x
// resident blocks of 128 (each context computes it once, at creation)
int mixed_slow_grid()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_epi1_slow, 128, 0);
    return std::max(1, sms) * std::max(1, per);
}

// Launch plans (chosen per context, e.g. by the autotuner):
//   pass 1: 0 = warp per 32 rows, fused;  1 = thread per row, fused;
//           2 = thread-per-row gather + per-particle kernel;  3 = warp-per-32-rows gather + per-particle kernel;
//           4 = as 2 with four pairs in flight per thread;  5 = as 4 with the weights W'/r from the per-slot table
//   pass 2: 0 = warp per 32 rows;  1 = thread per row;  2 = thread-per-row gather + per-particle kernel;
//           3 = thread per row, one pair in flight;  4 = thread per row, registers capped for 6 blocks of 128;
//           5 = as 3 with registers capped for 8 blocks of 128;  6 = as 1 with registers capped for 7 blocks of 128;
//           7 = as 1 with registers capped for 5 blocks of 128;  8 = as 7 with packed FP32x2 stress rows
// block sizes are multiples of 32 up to 256 (128 for the fused warp forms and pass-2 forms 4 to 8).
cudaError_t launch_step_mixed(tlsph_ctx &ctx, int64_t step_index, cudaStream_t st, cudaEvent_t *ev)
{
    const MixConst c = make_mix_const(ctx, step_index);
    const DevState &s = ctx.s;
    const int v1 = ctx.plan[0], b1 = ctx.plan[1], v2 = ctx.plan[2], b2 = ctx.plan[3];
    const bool hg = ctx.cfg.hg_alpha != 0.0;
    const int64_t rows32 = (s.N + 31) / 32 * 32;
    if (ev) cudaEventRecord(ev[0], st);
    switch (v1) {
    case 1: k_pass1_mixed_t<<<nb(s.N, b1), b1, 0, st>>>(s, c); break;
    case 2:
        k_gather1_mixed_t<<<nb(s.N, b1), b1, 0, st>>>(s, c);
        k_epi1_mixed<<<nb(s.N, 128), 128, 0, st>>>(s, c);
        break;
    case 3:
        k_gather1_mixed_w32<<<nb(rows32, b1), b1, 0, st>>>(s, c);
        k_epi1_mixed<<<nb(s.N, 128), 128, 0, st>>>(s, c);
        break;
    case 4:
        k_gather1_mixed_t4<<<nb(s.N, b1), b1, 0, st>>>(s, c);
        k_epi1_mixed<<<nb(s.N, 128), 128, 0, st>>>(s, c);
        break;
    case 5:
        k_gather1_mixed_t4w<<<nb(s.N, b1), b1, 0, st>>>(s, c);
        k_epi1_mixed<<<nb(s.N, 128), 128, 0, st>>>(s, c);
        break;
    default: k_pass1_mixed<<<nb(rows32, MIX_THREADS), MIX_THREADS, 0, st>>>(s, c); break;
    }
    k_epi1_slow<<<ctx.slow_grid, 128, 0, st>>>(s, c);
    if (ev) cudaEventRecord(ev[1], st);
    if (v2 == 1) {
        if (hg) k_pass2_mixed_t<true><<<nb(s.N, b2), b2, 0, st>>>(s, c);
        else k_pass2_mixed_t<false><<<nb(s.N, b2), b2, 0, st>>>(s, c);
    } else if (v2 == 3) {
        if (hg) k_pass2_mixed_t1<true><<<nb(s.N, b2), b2, 0, st>>>(s, c);
        else k_pass2_mixed_t1<false><<<nb(s.N, b2), b2, 0, st>>>(s, c);
    } else if (v2 == 4) {
        if (hg) k_pass2_mixed_tc<true><<<nb(s.N, b2), b2, 0, st>>>(s, c);
        else k_pass2_mixed_tc<false><<<nb(s.N, b2), b2, 0, st>>>(s, c);
    } else if (v2 == 6) {
        if (hg) k_pass2_mixed_tc7<true><<<nb(s.N, b2), b2, 0, st>>>(s, c);
        else k_pass2_mixed_tc7<false><<<nb(s.N, b2), b2, 0, st>>>(s, c);
    } else if (v2 == 7) {
        if (hg) k_pass2_mixed_tc5<true><<<nb(s.N, b2), b2, 0, st>>>(s, c);
        else k_pass2_mixed_tc5<false><<<nb(s.N, b2), b2, 0, st>>>(s, c);
    } else if (v2 == 8) {
        if (hg) k_pass2_mixed_tc5p<true><<<nb(s.N, b2), b2, 0, st>>>(s, c);
        else k_pass2_mixed_tc5p<false><<<nb(s.N, b2), b2, 0, st>>>(s, c);
    } else if (v2 == 5) {
        if (hg) k_pass2_mixed_t1c<true><<<nb(s.N, b2), b2, 0, st>>>(s, c);
        else k_pass2_mixed_t1c<false><<<nb(s.N, b2), b2, 0, st>>>(s, c);
    } else if (v2 == 2) {
        if (hg) {
            k_gather2_mixed_t<true><<<nb(s.N, b2), b2, 0, st>>>(s, c);
            k_epi2_mixed<true><<<nb(s.N, 128), 128, 0, st>>>(s, c);
        } else {
            k_gather2_mixed_t<false><<<nb(s.N, b2), b2, 0, st>>>(s, c);
            k_epi2_mixed<false><<<nb(s.N, 128), 128, 0, st>>>(s, c);
        }
    } else {
        if (hg) k_pass2_mixed<true><<<nb(rows32, MIX_THREADS), MIX_THREADS, 0, st>>>(s, c);
        else k_pass2_mixed<false><<<nb(rows32, MIX_THREADS), MIX_THREADS, 0, st>>>(s, c);
    }
    if (ev) cudaEventRecord(ev[2], st);
    return cudaGetLastError();
}

int mixed_kernels_per_step(const tlsph_ctx &ctx) { return (ctx.plan[0] >= 2 ? 2 : 1) + 1 + (ctx.plan[2] == 2 ? 2 : 1); }

cudaError_t mixed_sync_to_fp64(tlsph_ctx &ctx, int field, cudaStream_t st)
{
    if (ctx.N == 0) return cudaSuccess;
    if ((field == TLSPH_FIELD_A || field == -1) && ctx.steps > 0)
        k_mixed_export_A<<<nb(ctx.N, 256), 256, 0, st>>>(ctx.s);
    const int bits = mixed_field_bits(field);
    if (bits) k_mixed_export<<<nb(ctx.N, 256), 256, 0, st>>>(ctx.s, bits);
    return cudaGetLastError();
}

void mixed_release(tlsph_ctx &) {}

}  // namespace tlsph

// ====================================================================== batched step
// Many contexts advance together: a device table holds one slot per context
// (its device arrays and step constants).  Every kernel runs a persistent
// grid that strides over the flattened work list of (context, block of rows);
// a block finds its context by binary search on the slots' first work block.
// The ping-pong indices and the step counter live in the slots and are
// advanced on the device at the end of each step, so one captured step can be
// replayed as a CUDA graph, and the membership can change by rewriting the
// table without touching the graph.  A context's rows are computed by these
// kernels alone, independently of the other members, so its result does not
// depend on the company it keeps.
namespace tlsph {

// member of work block w: binary search over the members' first blocks (a
// contiguous array next to the table)
__device__ __forceinline__ int batch_find(const int64_t *blk0, int n, int64_t w)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk0[mid] <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// A block keeps its current member's slot in shared memory (copied when the
// block's work moves to another member), so the kernels read the member's
// arrays and constants from registers and shared memory rather than through
// global loads that stores into the state could alias.  Blocks take their work
// in chunks of BATCH_CHUNK consecutive work blocks: its first chunk by its own
// index, every later one from a counter (dynamic balance across members of
// different cost; blocks of a grid larger than the work leave at once, so a
// batch of a few small members pays no contention on the counter).  Measured on 256 bars of 2k-200k
// particles: one work block per grab 9.54 ms per step, 4 per grab 9.78 ms, 16
// per grab 10.8 ms, and a static strided assignment 11.3 ms.  The member of a
// chunk is found by a search over the first-block table (a few hundred bytes,
// cached) and then stepped forward.  Every row is computed independently, so
// the order in which chunks are taken changes no result.
#ifndef BATCH_CHUNK
#define BATCH_CHUNK 1
#endif

// Launch-shape variants of the batch kernels, chosen per batch
// (tlsph_batch_set_shape, by the autotuner): resident blocks of 128 per SM the
// kernel's registers are capped for, and pairs in flight per thread in the
// gathers.  Variant 0 of each kind is the default.  The variants agree with
// each other to FP32 rounding (a register cap can change which multiply-adds
// the compiler fuses).
//   pass-1 gather:        (8, 4)  (6, 4)  (10, 4)  (8, 2)  (8, 4) with the members' per-slot weight tables
//   per-particle update:  5  4  3
//   pass 2:               (5, 2)  (6, 2)  (4, 2)  (8, 1)  (5, 2) with packed FP32x2 stress rows
const int BATCH_VARIANTS[BATCH_KINDS] = { 5, 3, 5 };

// ALT selects the alternative pair-term form of a kind: the per-slot weight
// table in the pass-1 gather (members must hold one), the packed stress rows
// in pass 2
template <int KIND, bool HG, int MINB, int U, bool ALT = false>
__global__ void __launch_bounds__(128, MINB) k_batch(BatchHdr *hdr, const BatchSlot *slots)
{
    __shared__ uint64_t slot_words[(sizeof(BatchSlot) + 7) / 8];
    __shared__ int64_t grab;
    const BatchSlot &sl = *reinterpret_cast<const BatchSlot *>(slot_words);
    const int nspec = hdr->nspec;
    const int64_t total = hdr->total_blk;
    const int64_t *blk0 = hdr->blk0;
    int cur = -1;
    // the first chunk is the block's own (blocks without one leave at once, touching no counter);
    // later chunks come from the counter, after the grid's first chunks
    int64_t wb = (int64_t)blockIdx.x * BATCH_CHUNK;
    for (;;) {
        if (wb >= total) break;         // uniform over the block
        const int64_t we = min(total, wb + (int64_t)BATCH_CHUNK);
        int m = batch_find(blk0, nspec, wb);
        for (int64_t w = wb; w < we; ++w) {
            while (m + 1 < nspec && blk0[m + 1] <= w) ++m;
            if (m != cur) {             // uniform over the block
                __syncthreads();        // every thread is done with the previous slot
                const uint64_t *src = reinterpret_cast<const uint64_t *>(slots + m);
                for (int k = threadIdx.x; k < (int)((sizeof(BatchSlot) + 7) / 8); k += blockDim.x)
                    slot_words[k] = src[k];
                cur = m;
                __syncthreads();
            }
            const DevState &st = sl.s;
            const MixConst &c = sl.c;
            const int64_t i = (w - sl.blk0) * blockDim.x + threadIdx.x;
            if (i < st.N) {
                if constexpr (KIND == 0) {  // pass-1 gather
                    float mm[9];
                    gather1_row<U, ALT>(st, c, i, mm);
#pragma unroll
                    for (int k = 0; k < 9; ++k) st.fsum[k * st.N + i] = mm[k];
                } else if (KIND == 1) {     // pass-1 per-particle update
                    float mm[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) mm[k] = st.fsum[k * st.N + i];
                    epi1_mixed(st, c, i, mm);
                } else {                    // pass 2
                    float acc[9];
                    gather2_row<HG, U, ALT>(st, c, i, acc);
                    epi2_mixed<HG>(st, c, i, acc);
                }
            }
        }
        __syncthreads();                // every thread has read the previous chunk's start
        if (threadIdx.x == 0)
            grab = (int64_t)gridDim.x * BATCH_CHUNK +
                   (int64_t)atomicAdd(&hdr->next[KIND], (unsigned long long)BATCH_CHUNK);
        __syncthreads();
        wb = grab;
    }
}

// the FP64 updates queued by every member in this step (persistent grid over
// the members' queues; the members' queue lengths are read in parallel, 1024
// members at a time, so empty queues cost nothing); clears each member's queue
// counter of the next step
__global__ void __launch_bounds__(128) k_batch_slow(const BatchHdr *hdr, BatchSlot *slots)
{
    __shared__ uint32_t cnt[1024];
    const int nspec = hdr->nspec;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int m0 = 0; m0 < nspec; m0 += 1024) {
        const int mn = min(1024, nspec - m0);
        for (int k = threadIdx.x; k < mn; k += blockDim.x) {
            const BatchSlot &sl = slots[m0 + k];
            cnt[k] = sl.s.slowq_n[sl.c.step_index & 1];
        }
        __syncthreads();
        for (int k = 0; k < mn; ++k) {
            const uint32_t n = cnt[k];
            if (n == 0) continue;
            const BatchSlot &sl = slots[m0 + k];
            for (uint32_t q = t; q < n; q += stride) epi1_slow(sl.s, sl.c, sl.s.slowq[q]);
        }
        __syncthreads();
    }
    for (uint32_t m = t; m < (uint32_t)nspec; m += stride) slots[m].s.slowq_n[(slots[m].c.step_index + 1) & 1] = 0u;
}

// end of a step: flip the ping-pong buffers and count the step, per slot
__global__ void k_batch_advance(BatchHdr *hdr, BatchSlot *slots)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) hdr->next[0] = hdr->next[1] = hdr->next[2] = 0ull;   // the kernels of this step are done
    if (k >= hdr->nspec) return;
    slots[k].c.ucur ^= 1;
    slots[k].c.dcur ^= 1;
    slots[k].c.step_index += 1;
}

BatchSlot make_batch_slot(const tlsph_ctx &ctx)
{
    BatchSlot b;
    b.s = ctx.s;
    b.c = make_mix_const(ctx, ctx.steps);
    b.blk0 = 0;
    return b;
}

// The kernel of a kind and variant (the pass-1 kernels do not depend on the
// hourglass flag and are instantiated once), its launch and its occupancy.
template <int KIND, bool HG>
struct BatchKernel {
    using fn = void (*)(BatchHdr *, const BatchSlot *);
    static fn get(int v)
    {
        if (KIND == 0) {
            switch (v) {
            case 1: return k_batch<0, false, 6, 4>;
            case 2: return k_batch<0, false, 10, 4>;
            case 3: return k_batch<0, false, 8, 2>;
            case BATCH_TABLE_VARIANT: return k_batch<0, false, 8, 4, true>;
            default: return k_batch<0, false, 8, 4>;
            }
        } else if (KIND == 1) {
            switch (v) {
            case 1: return k_batch<1, false, 4, 1>;
            case 2: return k_batch<1, false, 3, 1>;
            default: return k_batch<1, false, 5, 1>;
            }
        } else {
            switch (v) {
            case 1: return k_batch<2, HG, 6, 2>;
            case 2: return k_batch<2, HG, 4, 2>;
            case 3: return k_batch<2, HG, 8, 1>;
            case 4: return k_batch<2, HG, 5, 2, true>;
            default: return k_batch<2, HG, 5, 2>;
            }
        }
    }
};

template <bool HG>
static void batch_kernels(BatchHdr *hdr, BatchSlot *slots, const int *shape, const int *grid, cudaStream_t st)
{
    BatchKernel<0, HG>::get(shape[0])<<<grid[0], 128, 0, st>>>(hdr, slots);
    BatchKernel<1, HG>::get(shape[1])<<<grid[1], 128, 0, st>>>(hdr, slots);
    k_batch_slow<<<grid[3], 128, 0, st>>>(hdr, slots);
    BatchKernel<2, HG>::get(shape[2])<<<grid[2], 128, 0, st>>>(hdr, slots);
}

cudaError_t launch_batch_step(BatchHdr *hdr, BatchSlot *slots, int nspec, bool hg, const int *shape, const int *grid,
                              cudaStream_t st)
{
    if (hg) batch_kernels<true>(hdr, slots, shape, grid, st);
    else batch_kernels<false>(hdr, slots, shape, grid, st);
    k_batch_advance<<<(nspec + 127) / 128, 128, 0, st>>>(hdr, slots);
    return cudaGetLastError();
}

template <bool HG>
static void batch_occupancy(const int *shape, int *per)
{
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[0], BatchKernel<0, HG>::get(shape[0]), 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[1], BatchKernel<1, HG>::get(shape[1]), 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[2], BatchKernel<2, HG>::get(shape[2]), 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[3], k_batch_slow, 128, 0);
}

// persistent grid of each kernel kind (pass-1 gather, per-particle update,
// pass 2, FP64 updates) for a launch shape: SMs x resident blocks per SM
void batch_grid(bool hg, const int *shape, int *grid)
{
    int dev = 0, sms = 0, per[4] = { 0, 0, 0, 0 };
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (hg) batch_occupancy<true>(shape, per);
    else batch_occupancy<false>(shape, per);
    for (int k = 0; k < 4; ++k) grid[k] = std::max(1, sms) * std::max(1, per[k]);
}

}  // namespace tlsph
