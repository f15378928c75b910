// Host runtime behind the C ABI in include/tlsph.h: argument checks, arena
// carving, the set-up sequence (copy in, neighbour CSR, L^{-1}, initial
// state), stream-ordered stepping, state transfer and error reporting.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <numeric>
#include <vector>

#include "tlsph_internal.cuh"

using namespace tlsph;

namespace {

thread_local std::string g_create_error;

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

// Byte layout of one context's device memory.  Offsets are relative to the
// base and 256-byte aligned.  The neighbour-build scratch overlays the
// F / sd / sig / A block, which is only initialised after the build.
struct Layout {
    size_t X, vol, mass, inv_mass, youngs, mat, bcm, bcv, row_ptr, Linv, u0, u1, v, vh, F, sd, sig, A;
    size_t ep, epdot, dinit, por, e, D0, D1, force, fail, status, mats, col, diag, inscan;
    size_t xo, s0, linv32, r1, r2, fsum, ell_off, ell_w;
    size_t Fh, Fl, sdh, sdl, sigf, slowq, slowq_n;
    size_t scratch, cell_start, cell_cursor, cell_items, scan_tmp, xf;
    size_t perm, iperm, stX, stvol, stmat, stbcm, stbcv, stf0;   // order, its inverse + staged caller-order inputs
    size_t overlay_end, ell;
    size_t total;
    int64_t max_cells;
    size_t scan_elems;
};

struct Carver {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    }
};

// sliced-ELL capacity carved from a caller arena: the pairs plus half again
// for slice padding and one row of padding per slice; when a specimen needs
// more, the context keeps to the warp-per-row plans
int64_t ell_capacity(int64_t N, int64_t nnz_cap)
{
    return std::max<int64_t>(nnz_cap + nnz_cap / 2 + 128 * ((N + 31) / 32), 32);
}

// Lattice-line order (TLSPH_FLAG_LINE_ORDER): perm[k] = caller index of
// internal particle k, sorted by the rounded lattice coordinates of the two
// shorter bounding-box axes, then by the coordinate along the longest axis
// (quantised to 32 bits over its extent; ties keep the caller order).  A
// least-significant-digit radix sort (four 16-bit digits) of 64-bit keys.
std::vector<int32_t> line_order_perm(const double *X, const double *vol, int64_t N)
{
    std::vector<int32_t> perm((size_t)N);
    for (int64_t i = 0; i < N; ++i) perm[(size_t)i] = (int32_t)i;
    if (N < 2) return perm;
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], X[3 * i + k]);
            hi[k] = std::max(hi[k], X[3 * i + k]);
        }
    int L = 0;
    for (int k = 1; k < 3; ++k)
        if (hi[k] - lo[k] > hi[L] - lo[L]) L = k;
    const int a = (L + 1) % 3, b = (L + 2) % 3;
    std::vector<double> v(vol, vol + N);
    std::nth_element(v.begin(), v.begin() + N / 2, v.end());
    const double d = std::cbrt(std::max(v[(size_t)(N / 2)], 0.0));
    const double inv = d > 0.0 ? 1.0 / d : 0.0;
    const uint64_t nb = (uint64_t)std::llround((hi[b] - lo[b]) * inv) + 1;
    const double extL = hi[L] - lo[L];
    const double qL = extL > 0.0 ? 4294967295.0 / extL : 0.0;
    std::vector<uint64_t> key((size_t)N), key2((size_t)N);
    std::vector<int32_t> idx2((size_t)N);
    for (int64_t i = 0; i < N; ++i) {
        const uint64_t ka = (uint64_t)std::llround((X[3 * i + a] - lo[a]) * inv);
        const uint64_t kb = (uint64_t)std::llround((X[3 * i + b] - lo[b]) * inv);
        const double t = std::min(4294967295.0, std::max(0.0, std::floor((X[3 * i + L] - lo[L]) * qL)));
        key[(size_t)i] = ((ka * nb + kb) << 32) | (uint64_t)t;
    }
    std::vector<int64_t> count(65536);
    for (int pass = 0; pass < 4; ++pass) {
        const int sh = 16 * pass;
        std::fill(count.begin(), count.end(), 0);
        for (int64_t i = 0; i < N; ++i) ++count[(key[(size_t)i] >> sh) & 0xffff];
        int64_t sum = 0;
        for (auto &c : count) { const int64_t t = c; c = sum; sum += t; }
        for (int64_t i = 0; i < N; ++i) {     // stable: equal digits keep their order
            const int64_t dst = count[(key[(size_t)i] >> sh) & 0xffff]++;
            key2[(size_t)dst] = key[(size_t)i];
            idx2[(size_t)dst] = perm[(size_t)i];
        }
        key.swap(key2);
        perm.swap(idx2);
    }
    return perm;
}

Layout make_layout(int64_t N, int64_t nnz_cap, bool mixed)
{
    Layout L{};
    const size_t n = (size_t)N, d = sizeof(double);
    Carver c;
    L.X = c.take(3 * n * d);
    L.vol = c.take(n * d);
    L.mass = c.take(n * d);
    L.inv_mass = c.take(n * d);
    L.youngs = c.take(n * d);
    L.mat = c.take(n * sizeof(int32_t));
    L.bcm = c.take(n);
    L.bcv = c.take(3 * n * d);
    L.row_ptr = c.take((n + 1) * sizeof(int64_t));
    L.Linv = c.take(9 * n * d);
    L.u0 = c.take(3 * n * d);
    L.u1 = c.take(3 * n * d);
    L.v = c.take(3 * n * d);
    L.vh = c.take(3 * n * d);
    L.ep = c.take(n * d);
    L.epdot = c.take(n * d);
    L.dinit = c.take(n * d);
    L.por = c.take(n * d);
    L.e = c.take(n * d);
    L.D0 = c.take(n * d);
    L.D1 = c.take(n * d);
    L.force = c.take(3 * n * d);
    L.fail = c.take(n * sizeof(int32_t));
    L.status = c.take(sizeof(uint32_t));
    L.diag = c.take(DIAG_BLOCKS * TLSPH_DIAG_COUNT * sizeof(double));
    L.inscan = c.take(INSCAN_BLOCKS * sizeof(InputScanDev));
    L.perm = c.take(n * sizeof(int32_t));
    L.iperm = c.take(n * sizeof(int32_t));
    L.mats = c.take(TLSPH_MAX_MATERIALS * sizeof(DevMat));
    if (mixed) {
        L.xo = c.take(n * 16);
        L.s0 = c.take(n * 16);
        L.ell_off = c.take(((n + 31) / 32 + 1) * sizeof(int64_t));
        L.ell_w = c.take(((n + 31) / 32) * sizeof(int32_t));
        L.linv32 = c.take(9 * n * sizeof(float));
        L.r1 = c.take(n * 16);
        L.r2 = c.take(6 * ((n + 31) / 32 * 32) * 16);   // tiles of 32 particles
        L.fsum = c.take(9 * n * sizeof(float));
        const size_t f = sizeof(float);
        L.Fh = c.take(9 * n * f); L.Fl = c.take(9 * n * f);
        L.sdh = c.take(6 * n * f); L.sdl = c.take(6 * n * f);
        L.sigf = c.take(6 * n * f);
        L.slowq = c.take(n * sizeof(int32_t));
        L.slowq_n = c.take(2 * sizeof(uint32_t));
    }
    // overlay block: F, sd, sig, A  |  neighbour-build scratch
    const size_t ov = c.off;
    L.F = c.take(9 * n * d);
    L.sd = c.take(6 * n * d);
    L.sig = c.take(6 * n * d);
    L.A = c.take(9 * n * d);
    const size_t state_end = c.off;
    L.max_cells = 2 * N + 4096;
    L.scan_elems = scan_tmp_elems(std::max<int64_t>(L.max_cells + 1, N + 1));
    Carver s;
    s.off = ov;
    // caller-order inputs staged for the reordering gather, then the scratch
    L.stX = s.take(3 * n * d);
    L.stvol = s.take(n * d);
    L.stmat = s.take(n * sizeof(int32_t));
    L.stbcm = s.take(n);
    L.stbcv = s.take(3 * n * d);
    L.stf0 = s.take(n * d);
    L.cell_start = s.take((size_t)(L.max_cells + 1) * sizeof(int64_t));
    L.cell_cursor = s.take((size_t)L.max_cells * sizeof(int64_t));
    L.cell_items = s.take(n * sizeof(int32_t));
    L.scan_tmp = s.take(L.scan_elems * sizeof(int64_t));
    L.xf = s.take(n * 16);
    c.off = std::max(state_end, s.off);
    L.overlay_end = c.off;
    L.col = c.take((size_t)std::max<int64_t>(nnz_cap, 1) * sizeof(int32_t));
    if (mixed) L.ell = c.take((size_t)ell_capacity(N, nnz_cap) * sizeof(int32_t));
    L.total = c.off;
    return L;
}

template <class T>
T *at(void *base, size_t off) { return reinterpret_cast<T *>(static_cast<char *>(base) + off); }

int fail_ctx(tlsph_ctx *ctx, int code, const std::string &msg)
{
    ctx->err = msg;
    if (ctx->sticky == TLSPH_OK) ctx->sticky = code;
    return code;
}

int cuda_fail(tlsph_ctx *ctx, cudaError_t e, const char *where)
{
    return fail_ctx(ctx, TLSPH_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool valid_config(const tlsph_config *c, std::string &why)
{
    if (!c) { why = "config is NULL"; return false; }
    if (!(c->h > 0.0) || !isfinite(c->h)) { why = "h must be positive"; return false; }
    if (!(c->rc > 0.0) || !isfinite(c->rc)) { why = "rc must be positive"; return false; }
    if (c->rc > 2.0 * c->h * (1.0 + 1e-12)) { why = "rc must not exceed the kernel support 2h"; return false; }
    if (!(c->dt > 0.0) || !isfinite(c->dt)) { why = "dt must be positive"; return false; }
    if (!(c->hg_alpha >= 0.0) || !isfinite(c->hg_alpha)) { why = "hg_alpha must be >= 0"; return false; }
    if (c->precision != TLSPH_PRECISION_FP64 && c->precision != TLSPH_PRECISION_MIXED) {
        why = "precision must be TLSPH_PRECISION_FP64 or TLSPH_PRECISION_MIXED";
        return false;
    }
    if ((c->flags & ~(TLSPH_FLAG_SPATIAL_ORDER | TLSPH_FLAG_LINE_ORDER | TLSPH_FLAG_AUTO_ORDER | TLSPH_FLAG_WALL)) != 0) {
        why = "unknown flags";
        return false;
    }
    const int orders = ((c->flags & TLSPH_FLAG_SPATIAL_ORDER) != 0) + ((c->flags & TLSPH_FLAG_LINE_ORDER) != 0) +
                       ((c->flags & TLSPH_FLAG_AUTO_ORDER) != 0);
    if (orders > 1) {
        why = "TLSPH_FLAG_SPATIAL_ORDER, TLSPH_FLAG_LINE_ORDER and TLSPH_FLAG_AUTO_ORDER exclude each other";
        return false;
    }
    return true;
}

void bind_state(tlsph_ctx *ctx, void *base, const Layout &L)
{
    DevState &s = ctx->s;
    if (ctx->cfg.precision == TLSPH_PRECISION_MIXED) {
        s.xo = at<int4>(base, L.xo);
        s.s0 = at<float4>(base, L.s0);
        s.ell_off = at<int64_t>(base, L.ell_off);
        s.ell_w = at<int32_t>(base, L.ell_w);
        s.w1t = nullptr;
        s.w1t_off = nullptr;
        s.linv32 = at<float>(base, L.linv32);
        s.r1 = at<float4>(base, L.r1);
        s.r2 = at<float4>(base, L.r2);
        s.fsum = at<float>(base, L.fsum);
        s.Fh = at<float>(base, L.Fh); s.Fl = at<float>(base, L.Fl);
        s.sdh = at<float>(base, L.sdh); s.sdl = at<float>(base, L.sdl);
        s.sigf = at<float>(base, L.sigf);
        s.slowq = at<int32_t>(base, L.slowq);
        s.slowq_n = at<uint32_t>(base, L.slowq_n);
    } else {
        s.fsum = nullptr;
        s.xo = nullptr;
        s.s0 = s.r1 = s.r2 = nullptr;
        s.ell_off = nullptr;
        s.ell_w = nullptr;
        s.colE = nullptr;
        s.w1t = nullptr;
        s.w1t_off = nullptr;
        s.linv32 = nullptr;
    }
    s.N = ctx->N;
    s.X = at<double>(base, L.X);
    s.vol = at<double>(base, L.vol);
    s.mass = at<double>(base, L.mass);
    s.inv_mass = at<double>(base, L.inv_mass);
    s.youngs = at<double>(base, L.youngs);
    s.mat = at<int32_t>(base, L.mat);
    s.bcm = at<uint8_t>(base, L.bcm);
    s.bcv = at<double>(base, L.bcv);
    s.row_ptr = at<int64_t>(base, L.row_ptr);
    s.Linv = at<double>(base, L.Linv);
    s.u[0] = at<double>(base, L.u0);
    s.u[1] = at<double>(base, L.u1);
    s.v = at<double>(base, L.v);
    s.vh = at<double>(base, L.vh);
    s.F = at<double>(base, L.F);
    s.sd = at<double>(base, L.sd);
    s.sig = at<double>(base, L.sig);
    s.A = at<double>(base, L.A);
    s.ep = at<double>(base, L.ep);
    s.epdot = at<double>(base, L.epdot);
    s.dinit = at<double>(base, L.dinit);
    s.por = at<double>(base, L.por);
    s.e = at<double>(base, L.e);
    s.D[0] = at<double>(base, L.D0);
    s.D[1] = at<double>(base, L.D1);
    s.force = at<double>(base, L.force);
    s.fail = at<int32_t>(base, L.fail);
    s.status = at<uint32_t>(base, L.status);
    ctx->diag = at<double>(base, L.diag);
    s.mats = at<DevMat>(base, L.mats);
}

struct FieldInfo {
    void *ptr;
    size_t elem, count;
    bool writable, sym;   // sym: stored as 6 per particle, exchanged as 9
};

FieldInfo field_info(tlsph_ctx *ctx, int field)
{
    DevState &s = ctx->s;
    const size_t n = (size_t)ctx->N, d = sizeof(double);
    switch (field) {
    case TLSPH_FIELD_X: return { (void *)s.X, d, 3 * n, false, false };
    case TLSPH_FIELD_U: return { s.u[ctx->ucur], d, 3 * n, true, false };
    case TLSPH_FIELD_V: return { s.v, d, 3 * n, true, false };
    case TLSPH_FIELD_F: return { s.F, d, 9 * n, true, false };
    case TLSPH_FIELD_SIGMA: return { s.sig, d, 9 * n, true, true };
    case TLSPH_FIELD_STRESS_DEV: return { s.sd, d, 9 * n, true, true };
    case TLSPH_FIELD_EPSP: return { s.ep, d, n, true, false };
    case TLSPH_FIELD_EPSP_RATE: return { s.epdot, d, n, true, false };
    case TLSPH_FIELD_DINIT: return { s.dinit, d, n, true, false };
    case TLSPH_FIELD_DAMAGE: return { s.D[ctx->dcur], d, n, true, false };
    case TLSPH_FIELD_POROSITY: return { s.por, d, n, true, false };
    case TLSPH_FIELD_FAIL_STEP: return { s.fail, sizeof(int32_t), n, true, false };
    case TLSPH_FIELD_FORCE: return { s.force, d, 3 * n, true, false };
    case TLSPH_FIELD_A: return { s.A, d, 9 * n, false, false };
    case TLSPH_FIELD_LINV: return { (void *)s.Linv, d, 9 * n, false, false };
    case TLSPH_FIELD_NBR_ROWPTR: return { (void *)s.row_ptr, sizeof(int64_t), n + 1, false, false };
    case TLSPH_FIELD_NBR_COL: return { (void *)s.col, sizeof(int32_t), (size_t)ctx->nnz, false, false };
    case TLSPH_FIELD_STEP: return { &ctx->steps, sizeof(int64_t), 1, true, false };
    case TLSPH_FIELD_ENERGY: return { s.e, d, n, true, false };
    default: return { nullptr, 0, 0, false, false };
    }
}

// fold the recorded events into the accumulators and free the slots
cudaError_t prof_fold(tlsph_ctx *ctx)
{
    if (ctx->prof_used == 0) return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(ctx->prof_ev[ctx->prof_used - 1]);
    if (e != cudaSuccess) return e;
    for (int b = 0; b + 2 < ctx->prof_used; b += 3) {
        float a = 0.f, c = 0.f;
        cudaEventElapsedTime(&a, ctx->prof_ev[b], ctx->prof_ev[b + 1]);
        cudaEventElapsedTime(&c, ctx->prof_ev[b + 1], ctx->prof_ev[b + 2]);
        ctx->prof_ms[0] += a;
        ctx->prof_ms[1] += c;
    }
    ctx->prof_used = 0;
    return cudaSuccess;
}

}  // namespace

namespace tlsph {

void set_last_error_text(const std::string &msg) { g_create_error = msg; }

DevMat make_dev_mat(const tlsph_material &m)
{
    DevMat d{};
    d.rho0 = m.rho0;
    d.E = m.E;
    d.K = m.E / (3.0 * (1.0 - 2.0 * m.nu));
    d.G = m.E / (2.0 * (1.0 + m.nu));
    d.eos = m.eos;
    d.damage = m.damage;
    d.rho0c02 = m.rho0 * m.c0 * m.c0;
    d.S_alpha = m.S_alpha;
    d.Gamma0 = m.Gamma0;
    d.g0rho0 = m.Gamma0 * m.rho0;
    d.inv_rho0 = 1.0 / m.rho0;
    d.A = m.A;
    d.B = m.B;
    d.n = m.n;
    d.C = m.C;
    d.inv_epsdot0 = m.epsdot0 > 0.0 ? 1.0 / m.epsdot0 : 0.0;
    d.inv_Wcr = m.Wcr > 0.0 ? 1.0 / m.Wcr : 0.0;
    d.D1 = m.D1; d.D2 = m.D2; d.D3 = m.D3; d.D4 = m.D4; d.D5 = m.D5;
    d.q1 = m.q1; d.q2 = m.q2; d.q3 = m.q3;
    d.fN = m.fN; d.eN = m.eN; d.sN = m.sN; d.fc = m.fc; d.fF = m.fF; d.komega = m.komega;
    d.nucl_coef = m.sN > 0.0 ? m.fN / (m.sN * sqrt(2.0 * M_PI)) : 0.0;
    d.fstar_slope = (m.fF > m.fc) ? (1.0 / m.q1 - m.fc) / (m.fF - m.fc) : 0.0;
    d.Kf = (float)d.K; d.Gf = (float)d.G; d.Af = (float)d.A; d.Bf = (float)d.B; d.nf = (float)d.n;
    d.Cf = (float)d.C; d.inv_epsdot0f = (float)d.inv_epsdot0; d.rho0c02f = (float)d.rho0c02;
    d.S_alphaf = (float)d.S_alpha; d.Gamma0f = (float)d.Gamma0;
    d.q1f = (float)d.q1; d.q2f = (float)d.q2; d.q3f = (float)d.q3; d.fcf = (float)d.fc; d.fFf = (float)d.fF;
    d.fstar_slopef = (float)d.fstar_slope;
    d.g0rho0f = (float)d.g0rho0;
    d.inv_rho0f = (float)d.inv_rho0;
    return d;
}

// The per-slot weight table of pass-1 plan form 5 (library-owned memory;
// 4 bytes per slot): slice offsets from the slice widths on the host, the
// weights by k_w1t_fill.  Released again when a plan without it is set.
void release_w1t(tlsph_ctx *ctx)
{
    if (ctx->w1t_mem) cudaFree(ctx->w1t_mem);
    if (ctx->w1t_off_mem) cudaFree(ctx->w1t_off_mem);
    ctx->w1t_mem = ctx->w1t_off_mem = nullptr;
    ctx->s.w1t = nullptr;
    ctx->s.w1t_off = nullptr;
}

int ctx_weight_table(tlsph_ctx *ctx)
{
    if (ctx->s.w1t) return TLSPH_OK;
    if (ctx->cfg.precision != TLSPH_PRECISION_MIXED || !ctx->ell_ok) {
        ctx->err = "the weight table belongs to the sliced lists of a mixed-precision context";
        return TLSPH_ERR_ARG;
    }
    if (!ctx->owns_mem) {
        ctx->err = "pass-1 form 5 keeps a weight table in library-owned memory: not available with a caller arena";
        return TLSPH_ERR_ARG;
    }
    const int64_t ng = (ctx->N + 31) / 32;
    std::vector<int32_t> w((size_t)ng);
    std::vector<int64_t> off((size_t)ng + 1);
    cudaError_t e = cudaMemcpyAsync(w.data(), ctx->s.ell_w, (size_t)ng * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "weight table widths");
    off[0] = 0;
    for (int64_t g = 0; g < ng; ++g) {
        const int wv = w[(size_t)g];
        const int64_t W = wv < 0 ? (int64_t)((~wv) & 0xffffff) : (int64_t)wv;
        off[(size_t)g + 1] = off[(size_t)g] + 8 * ((W + 3) & ~(int64_t)3);
    }
    if (cudaMalloc(&ctx->w1t_off_mem, ((size_t)ng + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&ctx->w1t_mem, (size_t)std::max<int64_t>(off[(size_t)ng], 1) * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        release_w1t(ctx);
        ctx->err = "no device memory for the pass-1 weight table";
        return TLSPH_ERR_NOMEM;
    }
    e = cudaMemcpyAsync(ctx->w1t_off_mem, off.data(), ((size_t)ng + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                        ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "weight table offsets");
    ctx->s.w1t = static_cast<const float4 *>(ctx->w1t_mem);
    ctx->s.w1t_off = static_cast<const int64_t *>(ctx->w1t_off_mem);
    e = mixed_w1t_fill(ctx->s, (float)(ctx->s.pack.unit / ctx->cfg.h), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);     // also keeps `off` alive for its copy
    if (e != cudaSuccess) return cuda_fail(ctx, e, "weight table");
    return TLSPH_OK;
}

}  // namespace tlsph

extern "C" {

size_t tlsph_workspace_bytes(const tlsph_config *cfg, int64_t N, int64_t nnz_cap)
{
    std::string why;
    if (!valid_config(cfg, why) || N <= 0 || nnz_cap < 0) return 0;
    return make_layout(N, nnz_cap, cfg->precision == TLSPH_PRECISION_MIXED).total + ALIGN;
}

// TLSPH_FLAG_AUTO_ORDER: the context in the caller's order, unless fewer than
// nine in ten of its neighbour slices are aligned (mixed precision only; the
// FP64 path reads the CSR); then the context is built again in lattice-line
// order and kept if that aligns more slices, else built once more in the
// caller's order.
static int create_auto_order(const tlsph_config *cfg, int64_t N, const double *X, const double *vol,
                             const int32_t *mat_id, const uint8_t *bc_mask, const double *bc_vel,
                             const double *f0, void *arena, size_t arena_bytes, int64_t nnz_cap,
                             void *stream, tlsph_ctx **out)
{
    tlsph_config caller = *cfg;
    caller.flags &= ~TLSPH_FLAG_AUTO_ORDER;
    int r = tlsph_create(&caller, N, X, vol, mat_id, bc_mask, bc_vel, f0, arena, arena_bytes, nnz_cap, stream, out);
    if (r != TLSPH_OK || caller.precision != TLSPH_PRECISION_MIXED) return r;
    int64_t slices = 0, aligned = 0;
    if (tlsph_neighbor_layout(*out, &slices, &aligned, nullptr, nullptr) != TLSPH_OK || 10 * aligned >= 9 * slices)
        return TLSPH_OK;
    tlsph_destroy(*out);
    *out = nullptr;
    tlsph_config line = caller;
    line.flags |= TLSPH_FLAG_LINE_ORDER;
    r = tlsph_create(&line, N, X, vol, mat_id, bc_mask, bc_vel, f0, arena, arena_bytes, nnz_cap, stream, out);
    if (r == TLSPH_OK) {
        int64_t s2 = 0, a2 = 0;
        if (tlsph_neighbor_layout(*out, &s2, &a2, nullptr, nullptr) == TLSPH_OK && a2 > aligned) return TLSPH_OK;
        tlsph_destroy(*out);
        *out = nullptr;
    }
    return tlsph_create(&caller, N, X, vol, mat_id, bc_mask, bc_vel, f0, arena, arena_bytes, nnz_cap, stream, out);
}

int tlsph_create(const tlsph_config *cfg, int64_t N, const double *X, const double *vol,
                 const int32_t *mat_id, const uint8_t *bc_mask, const double *bc_vel,
                 const double *f0, void *arena, size_t arena_bytes, int64_t nnz_cap,
                 void *stream, tlsph_ctx **out)
{
    g_create_error.clear();
    std::string why;
    if (!out) { g_create_error = "out is NULL"; return TLSPH_ERR_ARG; }
    *out = nullptr;
    if (!valid_config(cfg, why)) { g_create_error = why; return TLSPH_ERR_ARG; }
    if (cfg->flags & TLSPH_FLAG_AUTO_ORDER)
        return create_auto_order(cfg, N, X, vol, mat_id, bc_mask, bc_vel, f0, arena, arena_bytes, nnz_cap, stream, out);
    if (N <= 0 || N > INT32_MAX) { g_create_error = "N must be in [1, 2^31)"; return TLSPH_ERR_ARG; }
    if (!X || !vol) { g_create_error = "X and vol are required"; return TLSPH_ERR_ARG; }
    if (arena && ((uintptr_t)arena % ALIGN) != 0) { g_create_error = "arena must be 256-byte aligned"; return TLSPH_ERR_ARG; }
    if (arena && nnz_cap <= 0) { g_create_error = "nnz_cap is required with an arena"; return TLSPH_ERR_ARG; }

    tlsph_ctx *ctx = new (std::nothrow) tlsph_ctx();
    if (!ctx) { g_create_error = "host allocation failed"; return TLSPH_ERR_NOMEM; }
    ctx->cfg = *cfg;
    ctx->N = N;
    ctx->stream = static_cast<cudaStream_t>(stream);
    cudaStream_t st = ctx->stream;
    auto bail = [&](int code, const std::string &msg) {
        g_create_error = msg;
        if (ctx->owns_mem && ctx->mem) cudaFree(ctx->mem);
        if (ctx->ell_mem) cudaFree(ctx->ell_mem);
        if (ctx->col_mem) cudaFree(ctx->col_mem);
        delete ctx;
        return code;
    };

    // ---- memory: arena (capacity nnz_cap) or library-owned (exact nnz after the count)
    const bool mixed = cfg->precision == TLSPH_PRECISION_MIXED;
    Layout L = make_layout(N, arena ? nnz_cap : 0, mixed);
    void *base = nullptr;
    if (arena) {
        if (arena_bytes < L.total) return bail(TLSPH_ERR_NOMEM, "arena too small: need " + std::to_string(L.total) + " bytes");
        base = arena;
        ctx->nnz_cap = nnz_cap;
    } else {
        cudaError_t e = cudaMalloc(&base, L.overlay_end);
        if (e != cudaSuccess) { cudaGetLastError(); return bail(TLSPH_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); }
        ctx->owns_mem = true;
        ctx->mem = base;
    }
    bind_state(ctx, base, L);
    DevState &s = ctx->s;

    // ---- copy inputs (straight from the caller's arrays; absent ones are zero)
    const size_t n = (size_t)N;
    cudaError_t e = cudaSuccess;
#define CK(x) do { if ((e = (x)) != cudaSuccess) { cudaGetLastError(); return bail(TLSPH_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e)); } } while (0)
    double *stX = at<double>(base, L.stX), *stvol = at<double>(base, L.stvol), *stbcv = at<double>(base, L.stbcv);
    double *stf0 = at<double>(base, L.stf0);
    int32_t *stmat = at<int32_t>(base, L.stmat);
    uint8_t *stbcm = at<uint8_t>(base, L.stbcm);
    CK(cudaMemcpyAsync(stX, X, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(stvol, vol, n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (mat_id) CK(cudaMemcpyAsync(stmat, mat_id, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    else CK(cudaMemsetAsync(stmat, 0, n * sizeof(int32_t), st));
    if (bc_mask) CK(cudaMemcpyAsync(stbcm, bc_mask, n, cudaMemcpyHostToDevice, st));
    else CK(cudaMemsetAsync(stbcm, 0, n, st));
    if (bc_vel) CK(cudaMemcpyAsync(stbcv, bc_vel, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    else CK(cudaMemsetAsync(stbcv, 0, 3 * n * sizeof(double), st));
    if (f0) CK(cudaMemcpyAsync(stf0, f0, n * sizeof(double), cudaMemcpyHostToDevice, st));
    else CK(cudaMemsetAsync(stf0, 0, n * sizeof(double), st));
    CK(cudaMemsetAsync(s.status, 0, sizeof(uint32_t), st));
    CK(cudaMemsetAsync((void *)s.mass, 0, n * sizeof(double), st));
    CK(cudaMemsetAsync((void *)s.inv_mass, 0, n * sizeof(double), st));
    CK(cudaMemsetAsync((void *)s.youngs, 0, n * sizeof(double), st));

    // ---- one pass over the staged inputs: validation, bounding box, materials
    // in use and the sum of the initial velocities (the bulk reference of the
    // mixed path), reduced on the device in a fixed order (depends on N only)
    InputScanDev scan{};
    InputScanDev *scan_dev = at<InputScanDev>(base, L.inscan);
    CK(launch_scan_inputs(stX, stvol, stmat, stbcv, N, scan_dev, st));
    CK(cudaMemcpyAsync(&scan, scan_dev, sizeof(scan), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (scan.bad & INSCAN_BAD_VOL) return bail(TLSPH_ERR_ARG, "vol must be positive and finite");
    if (scan.bad & INSCAN_BAD_X) return bail(TLSPH_ERR_ARG, "X must be finite");
    if (scan.bad & INSCAN_BAD_MAT) return bail(TLSPH_ERR_ARG, "mat_id out of range");
    double lo3[3], hi3[3], vsum[3];
    for (int k = 0; k < 3; ++k) { lo3[k] = scan.lo[k]; hi3[k] = scan.hi[k]; vsum[k] = scan.vsum[k]; }
    for (int k = 0; k < TLSPH_MAX_MATERIALS; ++k) ctx->mat_used[k] = (scan.mats >> k) & 1u;

    // ---- neighbour CSR
    const CellGrid grid = cell_grid_from_bounds(lo3, hi3, N, cfg->rc);         // internal order
    const CellGrid sgrid = cell_grid_from_bounds(lo3, hi3, N, cfg->rc, 2);     // neighbour search
    if (grid.ncells > L.max_cells || sgrid.ncells > L.max_cells) return bail(TLSPH_ERR_ARG, "cell grid exceeds its bound");
    Scratch sc{ at<int64_t>(base, L.cell_start), at<int64_t>(base, L.cell_cursor), at<int32_t>(base, L.cell_items),
                at<int64_t>(base, L.scan_tmp), L.scan_elems, at<float4>(base, L.xf) };
    // ---- internal order (brick-major cells, caller index inside a cell) and the gather into it
    const bool line_order = (cfg->flags & TLSPH_FLAG_LINE_ORDER) != 0;
    ctx->reordered = (cfg->flags & (TLSPH_FLAG_SPATIAL_ORDER | TLSPH_FLAG_LINE_ORDER)) != 0;
    ctx->perm_dev = at<int32_t>(base, L.perm);
    if (line_order) {
        const std::vector<int32_t> lp = line_order_perm(X, vol, N);
        CK(cudaMemcpyAsync(ctx->perm_dev, lp.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    } else {
        CK(build_order(stX, N, grid, sc, !ctx->reordered, ctx->perm_dev, st));
    }
    CK(launch_gather_inputs(ctx->perm_dev, N, stX, stvol, stmat, stbcm, stbcv, stf0, s, st));
    // host copies of the order and its inverse (kept empty in caller order: the identity)
    if (ctx->reordered) {
        ctx->perm.resize(n);
        ctx->inv.resize(n);
        CK(cudaMemcpyAsync(ctx->perm.data(), ctx->perm_dev, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (size_t k = 0; k < n; ++k) ctx->inv[ctx->perm[k]] = (int32_t)k;
    }

    const double rc2 = cfg->rc * cfg->rc;
    int64_t *row_ptr = const_cast<int64_t *>(s.row_ptr);
    CK(build_neighbors_count(s, sgrid, sc, rc2, row_ptr, st));
    int64_t nnz = 0;
    CK(cudaMemcpyAsync(&nnz, row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (nnz > INT32_MAX) return bail(TLSPH_ERR_ARG, "more than 2^31 - 1 neighbour pairs");
    if (arena) {
        if (nnz > nnz_cap)
            return bail(TLSPH_ERR_NOMEM, "neighbour capacity too small: need nnz_cap >= " + std::to_string(nnz));
        s.col = at<int32_t>(base, L.col);
    } else {
        // the columns in an allocation of their own, now that their count is known
        e = cudaMalloc(&ctx->col_mem, (size_t)std::max<int64_t>(nnz, 1) * sizeof(int32_t));
        if (e != cudaSuccess) { cudaGetLastError(); return bail(TLSPH_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); }
        s.col = static_cast<int32_t *>(ctx->col_mem);
        ctx->nnz_cap = nnz;
    }
    ctx->nnz = nnz;
    // inverse order on the device (caller index -> internal index) for the caller-order reads
    ctx->inv_dev = nullptr;
    if (ctx->reordered) {
        ctx->inv_dev = at<int32_t>(base, L.iperm);
        CK(cudaMemcpyAsync(ctx->inv_dev, ctx->inv.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    CK(build_neighbors_fill(s, sgrid, sc, rc2, row_ptr, const_cast<int32_t *>(s.col), st));

    // ---- mixed: fixed-point positions and the sliced neighbour lists, read by
    // the correction-matrix kernel of a mixed context as by its steps
    if (mixed) {
        // bulk reference velocity of the FP32 velocity mirror: the mean initial velocity
        for (int k = 0; k < 3; ++k) s.vref[k] = vsum[k] / (double)n;
        // fixed-point positions about the bounding-box centre, |coordinate| < 2^31 - 2^10 units; the
        // unit also keeps every neighbour difference (each component below rc) within int32, which a
        // body smaller than about two cutoffs would otherwise overflow
        FixPack pk{};
        double ext = cfg->rc;
        for (int k = 0; k < 3; ++k) {
            pk.center[k] = 0.5 * (lo3[k] + hi3[k]);
            ext = std::max(ext, std::max(hi3[k] - pk.center[k], pk.center[k] - lo3[k]));
        }
        const int e2 = ext > 0.0 ? (int)std::ceil(std::log2(ext / 2147482624.0)) : 0;
        pk.unit = std::ldexp(1.0, e2);
        pk.inv_unit = std::ldexp(1.0, -e2);
        s.pack = pk;
        CK(mixed_init_positions(s, pk, st));
        ctx->slow_grid = mixed_slow_grid();
        // sliced neighbour lists for the thread-per-row plans
        const int64_t ng = (N + 31) / 32;
        int64_t *ell_off = const_cast<int64_t *>(s.ell_off);
        CK(cudaMemsetAsync(ell_off + ng, 0, sizeof(int64_t), st));
        CK(mixed_ell_widths(s, ell_off, st));
        CK(scan_exclusive_i64(ell_off, ng + 1, sc.scan_tmp, st));
        int64_t ell_n = 0;
        CK(cudaMemcpyAsync(&ell_n, ell_off + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        ctx->ell_words = ell_n;
        int32_t *colE = nullptr;
        if (arena) {
            if (ell_n <= ell_capacity(N, nnz_cap)) colE = at<int32_t>(base, L.ell);
        } else {
            e = cudaMalloc(&ctx->ell_mem, (size_t)std::max<int64_t>(ell_n, 1) * sizeof(int32_t));
            if (e == cudaSuccess) colE = static_cast<int32_t *>(ctx->ell_mem);
            else cudaGetLastError();
        }
        if (colE) {
            CK(mixed_ell_fill(s, ell_off, colE, st));
            s.colE = colE;
            ctx->ell_ok = true;
        } else {
            ctx->ell_ok = false;   // warp-per-row plans only
            ctx->plan[0] = 3; ctx->plan[1] = 256; ctx->plan[2] = 0; ctx->plan[3] = 128;
        }
    }

    // ---- correction matrices
    CK(cudaMemsetAsync(s.status, 0, sizeof(uint32_t), st));
    // S0 (mixed only) goes to the force array, which init_state clears afterwards
    if (mixed && ctx->ell_ok)
        CK(mixed_shape_matrix(s, cfg->h, const_cast<double *>(s.Linv), s.force, s.status, st));
    else
        CK(shape_matrix(s, cfg->h, const_cast<double *>(s.Linv), mixed ? s.force : nullptr, s.status, mixed, st));
    uint32_t n_sing = 0;
    CK(cudaMemcpyAsync(&n_sing, s.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (n_sing) return bail(TLSPH_ERR_SINGULAR_L, std::to_string(n_sing) + " particles have a singular correction matrix");
    CK(cudaMemsetAsync(s.status, 0, sizeof(uint32_t), st));
    if (mixed) CK(mixed_init_static(s, s.force, st));

    // ---- initial state (overwrites the scratch overlay)
    CK(launch_init_state(s, st));
    if (mixed) {
        CK(mixed_import(*ctx, -1, st));
        CK(cudaMemsetAsync(s.slowq_n, 0, 2 * sizeof(uint32_t), st));
    }
    CK(cudaStreamSynchronize(st));
#undef CK
    ctx->need_predict = true;
    *out = ctx;
    return TLSPH_OK;
}

int tlsph_set_material(tlsph_ctx *ctx, int mat_id, const tlsph_material *m)
{
    if (!ctx) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    if (!m || mat_id < 0 || mat_id >= TLSPH_MAX_MATERIALS) { ctx->err = "bad material id or NULL material"; return TLSPH_ERR_ARG; }
    std::string why;
    if (!(m->rho0 > 0) || !(m->E > 0) || !(m->nu > -1.0 && m->nu < 0.5)) why = "need rho0 > 0, E > 0, -1 < nu < 0.5";
    else if (m->eos != 0 && m->eos != 1) why = "eos must be 0 or 1";
    else if (m->eos == 1 && !(m->c0 > 0)) why = "Mie-Grueneisen needs c0 > 0";
    else if (m->damage < 0 || m->damage > 3) why = "damage model out of range";
    else if (!(m->A >= 0) || !(m->B >= 0) || !(m->n > 0)) why = "need A >= 0, B >= 0, n > 0";
    else if (m->damage == TLSPH_DAMAGE_CL && !(m->Wcr > 0)) why = "Cockcroft-Latham needs Wcr > 0";
    else if (m->damage == TLSPH_DAMAGE_GTN && (!(m->q1 > 0) || !(m->sN > 0) || !(m->fF > m->fc) || !(m->fc >= 0)))
        why = "GTN needs q1 > 0, sN > 0, fF > fc >= 0";
    else if (m->damage == TLSPH_DAMAGE_GTN && !(m->A > 0)) why = "GTN needs A > 0";
    if (!why.empty()) { ctx->err = why; return TLSPH_ERR_ARG; }
    ctx->mats_host[mat_id] = make_dev_mat(*m);
    ctx->mat_set[mat_id] = true;
    cudaError_t e = cudaMemcpyAsync(const_cast<DevMat *>(ctx->s.mats) + mat_id, &ctx->mats_host[mat_id], sizeof(DevMat),
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_material copy");
    e = launch_material_fields(ctx->s, mat_id, ctx->dcur, ctx->steps == 0, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_material fields");
    // the copy source lives in ctx; wait so a later overwrite cannot race it
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_material sync");
    ctx->need_predict = true;
    return TLSPH_OK;
}

int tlsph_step(tlsph_ctx *ctx, int nsteps)
{
    if (!ctx) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    if (nsteps < 0) { ctx->err = "nsteps < 0"; return TLSPH_ERR_ARG; }
    for (int k = 0; k < TLSPH_MAX_MATERIALS; ++k)
        if (ctx->mat_used[k] && !ctx->mat_set[k]) {
            ctx->err = "material " + std::to_string(k) + " is used but not set";
            return TLSPH_ERR_STATE;
        }
    cudaError_t e;
    if (ctx->need_predict) {
        e = launch_predict(ctx->s, ctx->ucur, ctx->cfg.dt, (ctx->cfg.flags & TLSPH_FLAG_WALL) != 0, ctx->steps, ctx->stream);
        if (e == cudaSuccess && ctx->cfg.precision == TLSPH_PRECISION_MIXED)
            e = mixed_after_predict(ctx->s, ctx->dcur, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "predict");
        ctx->need_predict = false;
    }
    for (int k = 0; k < nsteps; ++k) {
        cudaEvent_t *ev = nullptr;
        if (ctx->prof) {
            if (ctx->prof_used + 3 > (int)ctx->prof_ev.size()) {
                e = prof_fold(ctx);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "profile fold");
            }
            ev = &ctx->prof_ev[ctx->prof_used];
            ctx->prof_used += 3;
            ctx->prof_steps += 1;
        }
        if (ctx->cfg.precision == TLSPH_PRECISION_MIXED)
            e = launch_step_mixed(*ctx, ctx->steps, ctx->stream, ev);
        else
            e = launch_step_fp64(ctx->s, ctx->cfg, ctx->ucur, ctx->dcur, ctx->steps, ctx->stream, ev);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "step launch");
        ctx->ucur ^= 1;
        ctx->dcur ^= 1;
        ctx->steps += 1;
    }
    return TLSPH_OK;
}

int tlsph_status_bits(tlsph_ctx *ctx, uint32_t *bits)
{
    if (!ctx || !bits) return TLSPH_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(bits, ctx->s.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
    return TLSPH_OK;
}

int tlsph_diagnostics(tlsph_ctx *ctx, double *out, int n)
{
    if (!ctx || !out || n != TLSPH_DIAG_COUNT) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    cudaError_t e = launch_diagnostics(ctx->s, ctx->dcur, ctx->diag, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, ctx->diag, TLSPH_DIAG_COUNT * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "diagnostics");
    return TLSPH_OK;
}

int tlsph_diagnostics_async(tlsph_ctx *ctx, double *out, int n)
{
    if (!ctx || !out || n != TLSPH_DIAG_COUNT) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    // the reductions reuse one partials buffer: stream order keeps each call's copy ahead of the next call
    cudaError_t e = launch_diagnostics(ctx->s, ctx->dcur, ctx->diag, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, ctx->diag, TLSPH_DIAG_COUNT * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "diagnostics");
    return TLSPH_OK;
}

int tlsph_sync(tlsph_ctx *ctx)
{
    if (!ctx) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    uint32_t bits = 0;
    int rc = tlsph_status_bits(ctx, &bits);
    if (rc != TLSPH_OK) return rc;
    if (bits) {
        ctx->err = "device status bits " + std::to_string(bits);
        return TLSPH_ERR_NUMERICS;
    }
    return TLSPH_OK;
}

int tlsph_set_guard(tlsph_ctx *ctx, double band)
{
    if (!ctx) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    if (!(band >= 1e-5) || !std::isfinite(band)) {
        ctx->err = "guard band must be finite and >= 1e-5 (below it the FP32 screen is not conservative)";
        return TLSPH_ERR_ARG;
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_guard sync");
    ctx->guard = band;
    return TLSPH_OK;
}

int tlsph_set_grip_ramp(tlsph_ctx *ctx, double tau)
{
    if (!ctx) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    if (!(tau >= 0.0) || !std::isfinite(tau)) {
        ctx->err = "grip ramp tau must be finite and >= 0";
        return TLSPH_ERR_ARG;
    }
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_grip_ramp sync");
    ctx->s.grip_ramp = tau;
    e = launch_apply_grip(ctx->s, (double)ctx->steps * ctx->cfg.dt, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_grip_ramp");
    ctx->need_predict = true;
    return TLSPH_OK;
}

int tlsph_neighbor_layout(const tlsph_ctx *ctx, int64_t *slices, int64_t *aligned_slices, int64_t *slots,
                          int64_t *words)
{
    if (!ctx) return TLSPH_ERR_ARG;
    if (!ctx->ell_ok) return TLSPH_ERR_STATE;
    // the per-slice widths, read back and counted here (not at creation)
    const int64_t ng = (ctx->N + 31) / 32;
    std::vector<int32_t> w((size_t)ng);
    cudaError_t e = cudaMemcpyAsync(w.data(), ctx->s.ell_w, (size_t)ng * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { cudaGetLastError(); return TLSPH_ERR_CUDA; }
    int64_t aligned = 0, nslots = 0;
    for (int32_t wv : w) {
        aligned += wv < 0;
        nslots += 32 * (int64_t)(wv < 0 ? ((~wv) & 0xffffff) : wv);
    }
    if (slices) *slices = ng;
    if (aligned_slices) *aligned_slices = aligned;
    if (slots) *slots = nslots;
    if (words) *words = ctx->ell_words;
    return TLSPH_OK;
}

int tlsph_info(const tlsph_ctx *ctx, int64_t *N, int64_t *nnz, int64_t *steps)
{
    if (!ctx) return TLSPH_ERR_ARG;
    if (N) *N = ctx->N;
    if (nnz) *nnz = ctx->nnz;
    if (steps) *steps = ctx->steps;
    return TLSPH_OK;
}

// neighbour CSR in caller indices (rows of caller particles, columns mapped
// back and sorted ascending) from the internal CSR
static cudaError_t caller_csr(tlsph_ctx *ctx, std::vector<int64_t> &rp, std::vector<int32_t> &col)
{
    const int64_t N = ctx->N, nnz = ctx->nnz;
    std::vector<int64_t> rpi(N + 1);
    std::vector<int32_t> ci(nnz);
    cudaError_t e = cudaMemcpyAsync(rpi.data(), ctx->s.row_ptr, (N + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(ci.data(), ctx->s.col, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return e;
    rp.assign(N + 1, 0);
    col.resize(nnz);
    for (int64_t i = 0; i < N; ++i) {
        const int32_t k = ctx->inv[i];
        rp[i + 1] = rp[i] + (rpi[k + 1] - rpi[k]);
    }
    for (int64_t i = 0; i < N; ++i) {
        const int32_t k = ctx->inv[i];
        int32_t *o = col.data() + rp[i];
        int64_t m = 0;
        for (int64_t p = rpi[k]; p < rpi[k + 1]; ++p) o[m++] = ctx->perm[ci[p]];
        std::sort(o, o + m);
    }
    return cudaSuccess;
}

int tlsph_get_state(tlsph_ctx *ctx, int field, void *dst, size_t bytes, int dst_on_device)
{
    if (!ctx) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    FieldInfo f = field_info(ctx, field);
    if (!f.ptr || !dst) { ctx->err = "unknown field or NULL dst"; return TLSPH_ERR_ARG; }
    if (bytes != f.elem * f.count) { ctx->err = "byte count does not match the field"; return TLSPH_ERR_ARG; }
    cudaStream_t st = ctx->stream;
    cudaError_t e;
    if (field == TLSPH_FIELD_STEP) {   // host-side counter
        e = dst_on_device ? cudaMemcpy(dst, &ctx->steps, sizeof(int64_t), cudaMemcpyHostToDevice) : cudaSuccess;
        if (!dst_on_device) memcpy(dst, &ctx->steps, sizeof(int64_t));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "get_state step");
        return TLSPH_OK;
    }
    if (ctx->cfg.precision == TLSPH_PRECISION_MIXED) {
        e = mixed_sync_to_fp64(*ctx, field, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "mixed export");
    }
    const int64_t N = ctx->N;
    if (field == TLSPH_FIELD_NBR_ROWPTR || field == TLSPH_FIELD_NBR_COL) {
        if (!ctx->reordered) {
            e = cudaMemcpyAsync(dst, f.ptr, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
        } else {
            std::vector<int64_t> rp;
            std::vector<int32_t> col;
            e = caller_csr(ctx, rp, col);
            const void *src = field == TLSPH_FIELD_NBR_ROWPTR ? (const void *)rp.data() : (const void *)col.data();
            if (e == cudaSuccess)
                e = cudaMemcpy(dst, src, bytes, dst_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "get_state");
        return TLSPH_OK;
    }
    // per-particle field: stored comps (6 for symmetric tensors) -> exchanged comps
    const int comps = (int)(f.count / (size_t)N);
    const int scomps = f.sym ? 6 : comps;
    const size_t sbytes = (size_t)N * scomps * f.elem;
    // a page-locked host destination is mapped into the device's address space:
    // the device writes the caller-order array there itself
    void *mapped = nullptr;
    if (!dst_on_device) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, dst) == cudaSuccess) {
            if (pa.type == cudaMemoryTypeHost && pa.devicePointer) mapped = pa.devicePointer;
        } else {
            cudaGetLastError();
        }
    }
    const bool plain = !f.sym && !ctx->reordered;
    if (dst_on_device || mapped) {
        void *d = dst_on_device ? dst : mapped;
        if (plain)
            e = cudaMemcpyAsync(d, f.ptr, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
        else
            e = launch_to_caller(f.ptr, d, ctx->inv_dev, N, comps, scomps, (int)f.elem, f.sym, st);
    } else {
        // pageable destination: copy into a host staging array, then into the
        // caller's order on the host (faster here than the driver's own
        // staging into pages the caller has not touched yet)
        std::vector<unsigned char> tmp(sbytes);
        e = cudaMemcpyAsync(tmp.data(), f.ptr, sbytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && plain) {
            memcpy(dst, tmp.data(), sbytes);
        } else if (e == cudaSuccess) {
            unsigned char *o = static_cast<unsigned char *>(dst);
            for (int64_t k = 0; k < N; ++k) {
                const int64_t i = ctx->reordered ? ctx->perm[k] : k;
                if (f.sym) {
                    const double *a = reinterpret_cast<const double *>(tmp.data()) + 6 * k;
                    double *m = reinterpret_cast<double *>(o) + 9 * i;
                    m[0] = a[0]; m[4] = a[1]; m[8] = a[2];
                    m[1] = m[3] = a[3]; m[5] = m[7] = a[4]; m[2] = m[6] = a[5];
                } else {
                    memcpy(o + (size_t)i * comps * f.elem, tmp.data() + (size_t)k * comps * f.elem, comps * f.elem);
                }
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "get_state");
    return TLSPH_OK;
}

int tlsph_set_state(tlsph_ctx *ctx, int field, const void *src, size_t bytes, int src_on_device)
{
    if (!ctx) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    FieldInfo f = field_info(ctx, field);
    if (!f.ptr || !src) { ctx->err = "unknown field or NULL src"; return TLSPH_ERR_ARG; }
    if (!f.writable) { ctx->err = "field is read only"; return TLSPH_ERR_ARG; }
    if (bytes != f.elem * f.count) { ctx->err = "byte count does not match the field"; return TLSPH_ERR_ARG; }
    cudaStream_t st = ctx->stream;
    cudaError_t e;
    if (field == TLSPH_FIELD_STEP) {   // host-side counter
        int64_t v = 0;
        e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && src_on_device) e = cudaMemcpy(&v, src, sizeof(int64_t), cudaMemcpyDeviceToHost);
        if (!src_on_device) memcpy(&v, src, sizeof(int64_t));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "set_state step");
        if (v < 0) { ctx->err = "step count must be >= 0"; return TLSPH_ERR_ARG; }
        ctx->steps = v;
        return TLSPH_OK;
    }
    if (ctx->cfg.precision == TLSPH_PRECISION_MIXED) {
        e = mixed_sync_to_fp64(*ctx, -1, st);   // bring every FP64 field up to date first
        if (e != cudaSuccess) return cuda_fail(ctx, e, "mixed export");
    }
    const int64_t N = ctx->N;
    const int comps = (int)(f.count / (size_t)N);
    const int scomps = f.sym ? 6 : comps;
    if (src_on_device) {
        if (f.sym || ctx->reordered)
            e = launch_permute(src, f.ptr, ctx->perm_dev, N, scomps, (int)f.elem, false, f.sym, st);
        else
            e = cudaMemcpyAsync(f.ptr, src, bytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    } else {
        std::vector<unsigned char> tmp((size_t)N * scomps * f.elem);
        const unsigned char *a = static_cast<const unsigned char *>(src);
        for (int64_t k = 0; k < N; ++k) {
            const int64_t i = ctx->reordered ? ctx->perm[k] : k;
            if (f.sym) {
                const double *m = reinterpret_cast<const double *>(a) + 9 * i;
                double *o = reinterpret_cast<double *>(tmp.data()) + 6 * k;
                o[0] = m[0]; o[1] = m[4]; o[2] = m[8];
                o[3] = 0.5 * (m[1] + m[3]); o[4] = 0.5 * (m[5] + m[7]); o[5] = 0.5 * (m[2] + m[6]);
            } else {
                memcpy(tmp.data() + (size_t)k * comps * f.elem, a + (size_t)i * comps * f.elem, comps * f.elem);
            }
        }
        e = cudaMemcpyAsync(f.ptr, tmp.data(), tmp.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess && ctx->cfg.precision == TLSPH_PRECISION_MIXED) {
        e = mixed_import(*ctx, field, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_state");
    ctx->need_predict = true;
    return TLSPH_OK;
}

const char *tlsph_last_error(const tlsph_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int tlsph_destroy(tlsph_ctx *ctx)
{
    if (!ctx) return TLSPH_ERR_ARG;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->owns_mem && ctx->mem) cudaFree(ctx->mem);
    if (ctx->ell_mem) cudaFree(ctx->ell_mem);
    if (ctx->w1t_mem) cudaFree(ctx->w1t_mem);
    if (ctx->w1t_off_mem) cudaFree(ctx->w1t_off_mem);
    if (ctx->col_mem) cudaFree(ctx->col_mem);
    for (auto &ev : ctx->prof_ev) cudaEventDestroy(ev);
    mixed_release(*ctx);
    delete ctx;
    return TLSPH_OK;
}

int tlsph_set_plan(tlsph_ctx *ctx, const int32_t *plan, int n)
{
    if (!ctx || !plan || n != 4) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    const int32_t v1 = plan[0], b1 = plan[1], v2 = plan[2], b2 = plan[3];
    const bool ok = v1 >= 0 && v1 <= 5 && v2 >= 0 && v2 <= 8 && b1 >= 32 && b1 <= 256 && b1 % 32 == 0 &&
                    b2 >= 32 && b2 <= 256 && b2 % 32 == 0 && !(v2 >= 4 && b2 > 128) && !(v1 == 5 && b1 > 128);
    if (!ok) { ctx->err = "plan out of range"; return TLSPH_ERR_ARG; }
    if (ctx->cfg.precision != TLSPH_PRECISION_MIXED && v1 == 5) {
        ctx->err = "pass-1 form 5 is a form of the mixed step";
        return TLSPH_ERR_ARG;
    }
    if (!ctx->ell_ok && (v1 == 1 || v1 == 2 || v1 >= 4 || v2 >= 1)) {
        ctx->err = "this context has no sliced neighbour lists: only the warp-per-row plans (0, 3 / 0) apply";
        return TLSPH_ERR_ARG;
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_plan sync");
    if (v1 == 5) {
        const int r = ctx_weight_table(ctx);
        if (r != TLSPH_OK) return r;
    } else {
        release_w1t(ctx);
    }
    for (int k = 0; k < 4; ++k) ctx->plan[k] = plan[k];
    return TLSPH_OK;
}

int tlsph_get_plan(const tlsph_ctx *ctx, int32_t *plan, int n)
{
    if (!ctx || !plan || n != 4) return TLSPH_ERR_ARG;
    for (int k = 0; k < 4; ++k) plan[k] = ctx->plan[k];
    return TLSPH_OK;
}

int tlsph_profile_enable(tlsph_ctx *ctx, int enable)
{
    if (!ctx) return TLSPH_ERR_ARG;
    if (ctx->sticky) return TLSPH_ERR_STATE;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "profile sync");
    if (enable && ctx->prof_ev.empty()) {
        ctx->prof_ev.resize(3 * 1024);
        for (auto &ev : ctx->prof_ev) {
            e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
        }
    }
    if (enable) {
        ctx->prof_used = 0;
        ctx->prof_ms[0] = ctx->prof_ms[1] = 0.0;
        ctx->prof_steps = 0;
    } else {
        e = prof_fold(ctx);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "profile fold");
    }
    ctx->prof = enable != 0;
    return TLSPH_OK;
}

int tlsph_profile_read(tlsph_ctx *ctx, double *ms, int n, int64_t *steps)
{
    if (!ctx || (n > 0 && !ms)) return TLSPH_ERR_ARG;
    cudaError_t e = prof_fold(ctx);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "profile fold");
    for (int k = 0; k < n; ++k) ms[k] = k < 2 ? ctx->prof_ms[k] : 0.0;
    if (steps) *steps = ctx->prof_steps;
    return TLSPH_OK;
}

int tlsph_material_point_batch(const tlsph_material *mat, double dt, int64_t n, const double *deps,
                               const double *J, double *state, void *stream)
{
    if (!mat || n < 0 || (n > 0 && (!deps || !J || !state)) || !(dt > 0)) return TLSPH_ERR_ARG;
    if (n == 0) return TLSPH_OK;
    // the material record travels as a kernel argument copy
    DevMat dm = make_dev_mat(*mat);
    cudaError_t e = launch_material_point_value(dm, dt, n, deps, J, state, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? TLSPH_OK : TLSPH_ERR_CUDA;
}

}  // extern "C"
