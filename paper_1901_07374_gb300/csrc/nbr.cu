// Set-up kernels: exclusive scan, neighbour sets fixed in the reference
// configuration (Sec. 1, Sec. 2.2: S_i = { j != i : |X_j - X_i| < rc },
// never rebuilt) and the correction matrix L_i with its inverse (Sec. 2.2,
// Eq. correction_matrix).
//
// Neighbour search: particles are binned into a uniform grid of cells at
// least rc wide (count, scan, scatter); each particle then tests the 27
// surrounding cells.  The distance predicate is evaluated in FP64 as
// ((dx*dx + dy*dy) + dz*dz) < rc*rc with every product and sum rounded
// separately (no fused multiply-add), so the pair set is exactly the one its
// definition gives in IEEE double.  Rows are sorted ascending afterwards.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "tlsph_device.cuh"
#include "tlsph_internal.cuh"

namespace tlsph {

// ---------------------------------------------------------------- scan
static constexpr int SCAN_THREADS = 512;
static constexpr int SCAN_TILE = 2 * SCAN_THREADS;

size_t scan_tmp_elems(int64_t n)
{
    size_t total = 0;
    int64_t m = n;
    while (m > SCAN_TILE) {
        m = (m + SCAN_TILE - 1) / SCAN_TILE;
        total += (size_t)m + 1;
    }
    return total + 1;
}

// exclusive scan of one tile per block; block totals to part[blockIdx.x]
__global__ void k_scan_tile(int64_t *data, int64_t n, int64_t *part)
{
    __shared__ int64_t sh[SCAN_TILE];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const int t = threadIdx.x;
    int64_t i0 = base + 2 * t, i1 = i0 + 1;
    sh[2 * t] = i0 < n ? data[i0] : 0;
    sh[2 * t + 1] = i1 < n ? data[i1] : 0;
    // up-sweep
    int off = 1;
    for (int d = SCAN_TILE >> 1; d > 0; d >>= 1) {
        __syncthreads();
        if (t < d) {
            int ai = off * (2 * t + 1) - 1, bi = off * (2 * t + 2) - 1;
            sh[bi] += sh[ai];
        }
        off <<= 1;
    }
    __syncthreads();
    if (t == 0) {
        if (part) part[blockIdx.x] = sh[SCAN_TILE - 1];
        sh[SCAN_TILE - 1] = 0;
    }
    // down-sweep
    for (int d = 1; d < SCAN_TILE; d <<= 1) {
        off >>= 1;
        __syncthreads();
        if (t < d) {
            int ai = off * (2 * t + 1) - 1, bi = off * (2 * t + 2) - 1;
            int64_t tmp = sh[ai];
            sh[ai] = sh[bi];
            sh[bi] += tmp;
        }
    }
    __syncthreads();
    if (i0 < n) data[i0] = sh[2 * t];
    if (i1 < n) data[i1] = sh[2 * t + 1];
}

__global__ void k_scan_add(int64_t *data, int64_t n, const int64_t *part)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const int64_t add = part[blockIdx.x];
    for (int k = threadIdx.x; k < SCAN_TILE; k += blockDim.x) {
        int64_t i = base + k;
        if (i < n) data[i] += add;
    }
}

cudaError_t scan_exclusive_i64(int64_t *data, int64_t n, int64_t *tmp, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        k_scan_tile<<<1, SCAN_THREADS, 0, st>>>(data, n, nullptr);
        return cudaGetLastError();
    }
    int64_t *part = tmp;
    k_scan_tile<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(data, n, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_exclusive_i64(part, nb, tmp + nb + 1, st);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nb, 256, 0, st>>>(data, n, part);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- cell grid
__device__ __forceinline__ int cell_coord(double x, double lo, double inv_cs, int nc)
{
    int c = (int)floor((x - lo) * inv_cs);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// The search visits the cells within `reach` of a particle's cell.  With the
// single-precision coordinates of the prefilter it also clips them to the
// ball of radius rcm about the particle (rc plus a margin that covers the
// FP32 rounding of the coordinates and of the cell boundaries): a (y, z) line
// of cells is skipped when its distance exceeds rcm, and the cells of a line
// are cut to those that meet the ball.  A pair within rc always lies in a
// visited cell, and each visited candidate still goes through the prefilter
// and the FP64 predicate, so the result is that of the unclipped search.
struct GridArgs {
    double lo0, lo1, lo2, inv_cs;
    int nc0, nc1, nc2, reach;
    float flo0, flo1, flo2, fcs, finv_cs, rcm2;   // the grid in the prefilter's centred FP32 frame
};

static GridArgs grid_args(const CellGrid &g)
{
    GridArgs a{ g.xmin[0], g.xmin[1], g.xmin[2], 1.0 / g.cs, g.nc[0], g.nc[1], g.nc[2], g.reach };
    a.flo0 = a.flo1 = a.flo2 = 0.0f;
    a.fcs = a.finv_cs = a.rcm2 = 0.0f;
    return a;
}

__device__ __forceinline__ void cell_of(const GridArgs &a, const double *x, int &cx, int &cy, int &cz)
{
    cx = cell_coord(x[0], a.lo0, a.inv_cs, a.nc0);
    cy = cell_coord(x[1], a.lo1, a.inv_cs, a.nc1);
    cz = cell_coord(x[2], a.lo2, a.inv_cs, a.nc2);
}

__global__ void k_cell_count(const double *X, int64_t N, GridArgs a, int64_t *cell_count)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int cx, cy, cz;
    cell_of(a, X + 3 * i, cx, cy, cz);
    atomicAdd((unsigned long long *)&cell_count[((int64_t)cz * a.nc1 + cy) * a.nc0 + cx], 1ull);
}

__global__ void k_cell_scatter(const double *X, int64_t N, GridArgs a, const int64_t *cell_start,
                               int64_t *cursor, int32_t *items)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int cx, cy, cz;
    cell_of(a, X + 3 * i, cx, cy, cz);
    int64_t c = ((int64_t)cz * a.nc1 + cy) * a.nc0 + cx;
    unsigned long long slot = atomicAdd((unsigned long long *)&cursor[c], 1ull);
    items[cell_start[c] + (int64_t)slot] = (int32_t)i;
}

// the neighbour predicate with every operation rounded on its own
__device__ __forceinline__ bool within(const double *xi, const double *xj, double rc2)
{
    double dx = __dsub_rn(xj[0], xi[0]);
    double dy = __dsub_rn(xj[1], xi[1]);
    double dz = __dsub_rn(xj[2], xi[2]);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < rc2;
}

// Single-precision prefilter of the FP64 predicate: xf holds X - centre
// rounded once to FP32 (error <= delta per coordinate), so the FP32 r^2 of a
// pair is within a margin of the exact one that the host bounds; a pair whose
// FP32 r^2 is below lo is a neighbour, above hi is not, and only the band in
// between is decided by the FP64 predicate itself, so the result is the FP64
// predicate's exactly.
struct Prefilter {
    double cx, cy, cz;
    float lo, hi;
};

__global__ void k_xf(const double *X, int64_t N, Prefilter p, float4 *xf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    xf[i] = make_float4((float)(X[3 * i] - p.cx), (float)(X[3 * i + 1] - p.cy), (float)(X[3 * i + 2] - p.cz), 0.0f);
}

// distance from c to the interval [lo, lo + w] (0 inside)
__device__ __forceinline__ float gap(float c, float lo, float w) { return fmaxf(fmaxf(lo - c, c - (lo + w)), 0.0f); }

// one thread per particle: count (out == nullptr) or write its neighbours
__global__ void k_nbr(const double *X, int64_t N, GridArgs a, const int64_t *cell_start,
                      const int32_t *items, double rc2, int64_t *count, const int64_t *row_ptr,
                      int32_t *out, const float4 *xf, Prefilter pf)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double xi[3] = { X[3 * i], X[3 * i + 1], X[3 * i + 2] };
    const float4 fi = xf ? xf[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    int cx, cy, cz;
    cell_of(a, xi, cx, cy, cz);
    int64_t n = 0;
    int64_t w = out ? row_ptr[i] : 0;
    const int R = a.reach;
    for (int z = max(cz - R, 0); z <= min(cz + R, a.nc2 - 1); ++z) {
        float dz2 = 0.0f;
        if (xf) {
            const float dz = gap(fi.z, fmaf((float)z, a.fcs, a.flo2), a.fcs);
            dz2 = dz * dz;
            if (dz2 > a.rcm2) continue;
        }
        for (int y = max(cy - R, 0); y <= min(cy + R, a.nc1 - 1); ++y) {
            int64_t rowc = ((int64_t)z * a.nc1 + y) * a.nc0;
            int x0 = max(cx - R, 0), x1 = min(cx + R, a.nc0 - 1);
            if (xf) {
                const float dy = gap(fi.y, fmaf((float)y, a.fcs, a.flo1), a.fcs);
                const float dyz2 = dz2 + dy * dy;
                if (dyz2 > a.rcm2) continue;
                const float rx = sqrtf(a.rcm2 - dyz2);
                x0 = max(x0, (int)floorf((fi.x - rx - a.flo0) * a.finv_cs));
                x1 = min(x1, (int)floorf((fi.x + rx - a.flo0) * a.finv_cs));
                if (x0 > x1) continue;
            }
            // cells x0..x1 of this (y, z) line are contiguous in the cell order
            int64_t b = cell_start[rowc + x0], e = cell_start[rowc + x1 + 1];
            for (int64_t k = b; k < e; ++k) {
                int32_t j = items[k];
                if (j == i) continue;
                bool nb;
                if (xf) {
                    const float4 fj = xf[j];
                    const float dx = fj.x - fi.x, dy = fj.y - fi.y, dz = fj.z - fi.z;
                    const float r2f = dx * dx + dy * dy + dz * dz;
                    nb = r2f < pf.lo ? true : (r2f > pf.hi ? false : within(xi, X + 3 * (int64_t)j, rc2));
                } else {
                    nb = within(xi, X + 3 * (int64_t)j, rc2);
                }
                if (nb) {
                    if (out) out[w + n] = j;
                    ++n;
                }
            }
        }
    }
    if (!out) count[i] = n;
}

// Rows sorted ascending, one warp per row: a bitonic network over E elements
// (E / 32 per lane, element e = k * 32 + lane, padded with INT_MAX); rows
// longer than 256 fall back to an insertion sort by lane 0.
template <int PER>
__device__ __forceinline__ void warp_bitonic(int32_t (&v)[PER], int lane)
{
    constexpr int E = 32 * PER;
#pragma unroll
    for (int size = 2; size <= E; size <<= 1) {
#pragma unroll
        for (int d = size >> 1; d > 0; d >>= 1) {
            if (d >= 32) {
                const int kd = d >> 5;
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    if (k & kd) continue;
                    const int e = k * 32 + lane;
                    const bool asc = (e & size) == 0;
                    const int32_t a = v[k], b = v[k | kd];
                    const int32_t lo = min(a, b), hi = max(a, b);
                    v[k] = asc ? lo : hi;
                    v[k | kd] = asc ? hi : lo;
                }
            } else {
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    const int e = k * 32 + lane;
                    const bool asc = (e & size) == 0;
                    const int32_t o = __shfl_xor_sync(0xffffffffu, v[k], d);
                    const bool keep_min = ((lane & d) == 0) == asc;
                    v[k] = keep_min ? min(v[k], o) : max(v[k], o);
                }
            }
        }
    }
}

template <int PER>
__device__ __forceinline__ void sort_row_warp(int32_t *c, int n, int lane)
{
    int32_t v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = k * 32 + lane;
        v[k] = e < n ? c[e] : INT_MAX;
    }
    warp_bitonic<PER>(v, lane);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = k * 32 + lane;
        if (e < n) c[e] = v[k];
    }
}

__global__ void k_sort_rows(const int64_t *row_ptr, int32_t *col, int64_t N)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;                       // whole warps: blockDim is a multiple of 32
    const int64_t b = row_ptr[i], e = row_ptr[i + 1];
    const int64_t n = e - b;
    if (n <= 64) sort_row_warp<2>(col + b, (int)n, lane);
    else if (n <= 128) sort_row_warp<4>(col + b, (int)n, lane);
    else if (n <= 256) sort_row_warp<8>(col + b, (int)n, lane);
    else if (lane == 0) {
        for (int64_t k = b + 1; k < e; ++k) {
            int32_t v = col[k];
            int64_t m = k - 1;
            while (m >= b && col[m] > v) { col[m + 1] = col[m]; --m; }
            col[m + 1] = v;
        }
    }
}

static unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// prefilter thresholds for the grid's box: the FP32 positions are centred on
// the box, so each coordinate carries at most delta = half extent x 2^-24;
// |r2f - r2| <= 4 sqrt(3) rc delta + 4 sqrt(3) delta^2 + 4 2^-24 rc^2 for a
// pair near the cutoff, widened by 4x
static Prefilter prefilter_for(const CellGrid &g, double rc2)
{
    Prefilter p{};
    double ext = 0.0, c[3];
    for (int k = 0; k < 3; ++k) {
        const double span = g.nc[k] * g.cs;
        c[k] = g.xmin[k] + 0.5 * span;
        ext = fmax(ext, 0.5 * span);
    }
    p.cx = c[0]; p.cy = c[1]; p.cz = c[2];
    const double rc = sqrt(rc2), delta = ext * 0x1p-24;
    const double margin = 4.0 * (6.93 * rc * delta + 6.93 * delta * delta + 4.0 * 0x1p-24 * rc2);
    p.lo = (float)((rc2 - margin) * (1.0 - 1e-6));
    p.hi = (float)((rc2 + margin) * (1.0 + 1e-6));
    if (!(p.lo > 0.0f)) p.lo = 0.0f;   // no certain neighbours: every pair below hi goes to FP64
    return p;
}

// the grid in the prefilter's frame, with the clipping radius: rc enlarged by
// 1e-4 of itself plus 32 units of FP32 rounding at the grid's extent (the
// coordinates, the cell boundaries and the clipped range are each within a
// few of those)
static GridArgs clip_args(const CellGrid &g, const Prefilter &p, double rc2)
{
    GridArgs a = grid_args(g);
    double ext = 0.0;
    for (int k = 0; k < 3; ++k) ext = fmax(ext, g.nc[k] * g.cs);
    const double rcm = sqrt(rc2) * (1.0 + 1e-4) + 32.0 * ext * 0x1p-24;
    a.flo0 = (float)(g.xmin[0] - p.cx);
    a.flo1 = (float)(g.xmin[1] - p.cy);
    a.flo2 = (float)(g.xmin[2] - p.cz);
    a.fcs = (float)g.cs;
    a.finv_cs = (float)(1.0 / g.cs);
    a.rcm2 = (float)(rcm * rcm);
    return a;
}

cudaError_t build_neighbors_count(const DevState &s, const CellGrid &g, const Scratch &sc, double rc2,
                                  int64_t *row_ptr, cudaStream_t st)
{
    cudaError_t e;
    const Prefilter pf = prefilter_for(g, rc2);
    const GridArgs a = clip_args(g, pf, rc2);
    if (sc.xf) {
        k_xf<<<blocks_for(s.N, 256), 256, 0, st>>>(s.X, s.N, pf, sc.xf);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // cell histogram -> cell_start (exclusive scan) -> scatter with a cursor
    if ((e = cudaMemsetAsync(sc.cell_start, 0, (g.ncells + 1) * sizeof(int64_t), st)) != cudaSuccess) return e;
    k_cell_count<<<blocks_for(s.N, 256), 256, 0, st>>>(s.X, s.N, a, sc.cell_start);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive_i64(sc.cell_start, g.ncells + 1, sc.scan_tmp, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sc.cell_cursor, 0, g.ncells * sizeof(int64_t), st)) != cudaSuccess) return e;
    k_cell_scatter<<<blocks_for(s.N, 256), 256, 0, st>>>(s.X, s.N, a, sc.cell_start, sc.cell_cursor,
                                                         sc.cell_items);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_nbr<<<blocks_for(s.N, 128), 128, 0, st>>>(s.X, s.N, a, sc.cell_start, sc.cell_items, rc2, row_ptr,
                                                 nullptr, nullptr, sc.xf, pf);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(row_ptr + s.N, 0, sizeof(int64_t), st)) != cudaSuccess) return e;
    return scan_exclusive_i64(row_ptr, s.N + 1, sc.scan_tmp, st);
}

cudaError_t build_neighbors_fill(const DevState &s, const CellGrid &g, const Scratch &sc, double rc2,
                                 const int64_t *row_ptr, int32_t *col, cudaStream_t st)
{
    const Prefilter pf = prefilter_for(g, rc2);
    const GridArgs a = clip_args(g, pf, rc2);
    k_nbr<<<blocks_for(s.N, 128), 128, 0, st>>>(s.X, s.N, a, sc.cell_start, sc.cell_items, rc2, nullptr,
                                                 row_ptr, col, sc.xf, pf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sort_rows<<<blocks_for(s.N * 32, 256), 256, 0, st>>>(row_ptr, col, s.N);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- particle order
// Internal particle order: cells of the neighbour grid grouped into bricks of
// 4 x 4 x 4 cells, bricks in row-major order, cells row-major inside a brick,
// particles of a cell by ascending caller index.  brick_rank is a dense
// bijection of the cells onto [0, ncells) (bricks at the far faces are
// clipped), so the counting sort needs no more buckets than the grid has
// cells.  Consecutive rows are then spatially compact, which keeps the
// neighbour gathers of a thread block inside a small region of L1/L2.
__device__ __forceinline__ int64_t brick_rank(int cx, int cy, int cz, int ncx, int ncy, int ncz)
{
    const int bx = cx >> 2, by = cy >> 2, bz = cz >> 2;
    const int lx = cx & 3, ly = cy & 3, lz = cz & 3;
    const int hz = min(4, ncz - 4 * bz), hy = min(4, ncy - 4 * by), wx = min(4, ncx - 4 * bx);
    return (int64_t)ncx * ncy * (4 * bz) + (int64_t)ncx * (4 * by) * hz + (int64_t)(4 * bx) * hy * hz +
           (int64_t)(lz * hy + ly) * wx + lx;
}

__global__ void k_order_count(const double *X, int64_t N, GridArgs a, int64_t *count)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int cx, cy, cz;
    cell_of(a, X + 3 * i, cx, cy, cz);
    atomicAdd((unsigned long long *)&count[brick_rank(cx, cy, cz, a.nc0, a.nc1, a.nc2)], 1ull);
}

__global__ void k_order_scatter(const double *X, int64_t N, GridArgs a, const int64_t *start, int64_t *cursor,
                                int32_t *perm)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int cx, cy, cz;
    cell_of(a, X + 3 * i, cx, cy, cz);
    const int64_t c = brick_rank(cx, cy, cz, a.nc0, a.nc1, a.nc2);
    unsigned long long slot = atomicAdd((unsigned long long *)&cursor[c], 1ull);
    perm[start[c] + (int64_t)slot] = (int32_t)i;
}

// ascending caller index inside each cell (cells are short)
__global__ void k_sort_segments(const int64_t *start, int32_t *v, int64_t nseg)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nseg) return;
    const int64_t b = start[c], e = start[c + 1];
    for (int64_t k = b + 1; k < e; ++k) {
        const int32_t x = v[k];
        int64_t m = k - 1;
        while (m >= b && v[m] > x) { v[m + 1] = v[m]; --m; }
        v[m + 1] = x;
    }
}

__global__ void k_identity(int32_t *perm, int64_t N)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) perm[i] = (int32_t)i;
}

// ---------------------------------------------------------------- input scan
// Every block takes a contiguous range of particles, every thread a strided
// part of it; the block reduction and the final one run in a fixed order, so
// the FP64 velocity sum depends on N only.
__device__ __forceinline__ void inscan_init(InputScanDev &a)
{
    for (int k = 0; k < 3; ++k) { a.lo[k] = INFINITY; a.hi[k] = -INFINITY; a.vsum[k] = 0.0; }
    a.mats = 0ull;
    a.bad = 0u;
    a.pad = 0u;
}
__device__ __forceinline__ void inscan_merge(InputScanDev &a, const InputScanDev &b)
{
    for (int k = 0; k < 3; ++k) {
        a.lo[k] = fmin(a.lo[k], b.lo[k]);
        a.hi[k] = fmax(a.hi[k], b.hi[k]);
        a.vsum[k] += b.vsum[k];
    }
    a.mats |= b.mats;
    a.bad |= b.bad;
}
__device__ __forceinline__ void inscan_warp(InputScanDev &a)
{
    for (int o = 16; o > 0; o >>= 1) {
        InputScanDev b;
        for (int k = 0; k < 3; ++k) {
            b.lo[k] = __shfl_xor_sync(0xffffffffu, a.lo[k], o);
            b.hi[k] = __shfl_xor_sync(0xffffffffu, a.hi[k], o);
            b.vsum[k] = __shfl_xor_sync(0xffffffffu, a.vsum[k], o);
        }
        b.mats = __shfl_xor_sync(0xffffffffu, a.mats, o);
        b.bad = __shfl_xor_sync(0xffffffffu, a.bad, o);
        inscan_merge(a, b);
    }
}
// block of 256 threads: the result in thread 0's a
__device__ __forceinline__ void inscan_block(InputScanDev &a, InputScanDev *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    inscan_warp(a);
    if (lane == 0) sh[wid] = a;
    __syncthreads();
    if (wid == 0) {
        if (lane < (int)(blockDim.x >> 5)) a = sh[lane];
        else inscan_init(a);
        inscan_warp(a);
    }
}

__global__ void __launch_bounds__(256) k_scan_inputs(const double *X, const double *vol, const int32_t *mat,
                                                     const double *bcv, int64_t N, InputScanDev *parts)
{
    __shared__ InputScanDev sh[8];
    const int64_t lo = (int64_t)blockIdx.x * N / gridDim.x, hi = (int64_t)(blockIdx.x + 1) * N / gridDim.x;
    InputScanDev a;
    inscan_init(a);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double vv = vol[i];
        if (!(vv > 0.0 && isfinite(vv))) a.bad |= INSCAN_BAD_VOL;
        for (int k = 0; k < 3; ++k) {
            const double c = X[3 * i + k];
            if (!isfinite(c)) a.bad |= INSCAN_BAD_X;
            a.lo[k] = fmin(a.lo[k], c);
            a.hi[k] = fmax(a.hi[k], c);
            a.vsum[k] += bcv[3 * i + k];
        }
        const int32_t m = mat[i];
        if (m >= 0 && m < TLSPH_MAX_MATERIALS) a.mats |= 1ull << m;
        else a.bad |= INSCAN_BAD_MAT;
    }
    inscan_block(a, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = a;
}

// one block of 256 threads over the per-block results, in their order
__global__ void __launch_bounds__(256) k_scan_inputs_final(InputScanDev *parts, int nblocks)
{
    __shared__ InputScanDev sh[8];
    InputScanDev a;
    if ((int)threadIdx.x < nblocks) a = parts[threadIdx.x];
    else inscan_init(a);
    inscan_block(a, sh);
    if (threadIdx.x == 0) parts[0] = a;
}

cudaError_t launch_scan_inputs(const double *X, const double *vol, const int32_t *mat, const double *bcv, int64_t N,
                               InputScanDev *parts, cudaStream_t st)
{
    static_assert(INSCAN_BLOCKS <= 256, "the final reduction takes one block of 256 threads");
    k_scan_inputs<<<INSCAN_BLOCKS, 256, 0, st>>>(X, vol, mat, bcv, N, parts);
    k_scan_inputs_final<<<1, 256, 0, st>>>(parts, INSCAN_BLOCKS);
    return cudaGetLastError();
}

cudaError_t build_order(const double *X_user, int64_t N, const CellGrid &g, const Scratch &sc, bool keep,
                        int32_t *perm, cudaStream_t st)
{
    cudaError_t e;
    if (keep) {
        k_identity<<<blocks_for(N, 256), 256, 0, st>>>(perm, N);
        return cudaGetLastError();
    }
    GridArgs a = grid_args(g);
    if ((e = cudaMemsetAsync(sc.cell_start, 0, (g.ncells + 1) * sizeof(int64_t), st)) != cudaSuccess) return e;
    k_order_count<<<blocks_for(N, 256), 256, 0, st>>>(X_user, N, a, sc.cell_start);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive_i64(sc.cell_start, g.ncells + 1, sc.scan_tmp, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sc.cell_cursor, 0, g.ncells * sizeof(int64_t), st)) != cudaSuccess) return e;
    k_order_scatter<<<blocks_for(N, 256), 256, 0, st>>>(X_user, N, a, sc.cell_start, sc.cell_cursor, perm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_sort_segments<<<blocks_for(g.ncells, 128), 128, 0, st>>>(sc.cell_start, perm, g.ncells);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- correction matrix
// One warp per particle: L_i = sum_j V_j (X_j - X_i) (x) grad W_i(X_ij), with
// grad W = W'(r) (X_j - X_i) / r, so L_i is symmetric; inverted by the
// adjugate.  A row whose |det L| <= 1e-12 |L|_F^3 is reported singular and
// gets L^{-1} = 0.
__global__ void k_shape(const double *X, const double *vol, const int64_t *row_ptr, const int32_t *col,
                        int64_t N, double inv_h, double dw_norm, double *Linv, double *S0, uint32_t *n_singular)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;
    const double xi = X[3 * i], yi = X[3 * i + 1], zi = X[3 * i + 2];
    double l[6] = { 0, 0, 0, 0, 0, 0 };
    double g[3] = { 0, 0, 0 };
    for (int64_t p = row_ptr[i] + lane; p < row_ptr[i + 1]; p += 32) {
        const int64_t j = col[p];
        const double dx = X[3 * j] - xi, dy = X[3 * j + 1] - yi, dz = X[3 * j + 2] - zi;
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double rinv = rsqrt(r2);
        const double c0 = vol[j] * spline_dw(r2 * rinv * inv_h) * rinv;
        g[0] += c0 * dx; g[1] += c0 * dy; g[2] += c0 * dz;
        const double c = dw_norm * c0;
        l[0] += c * dx * dx; l[1] += c * dy * dy; l[2] += c * dz * dz;
        l[3] += c * dx * dy; l[4] += c * dy * dz; l[5] += c * dz * dx;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) l[k] = warp_allsum(l[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = warp_allsum(g[k]);
    if (lane == 0 && S0) {
        S0[3 * i] = g[0]; S0[3 * i + 1] = g[1]; S0[3 * i + 2] = g[2];
    }
    if (lane == 0) {
        double L[9], c[9];
        sym_to_full(l, L);
        cof3(L, c);
        const double det = L[0] * c[0] + L[1] * c[1] + L[2] * c[2];
        double fn2 = 0.0;
        for (int k = 0; k < 9; ++k) fn2 += L[k] * L[k];
        const double fn = sqrt(fn2);
        const bool ok = isfinite(det) && fabs(det) > 1e-12 * fn * fn * fn;
        // L^{-1} = adj(L) / det = cof(L)^T / det
        for (int k = 0; k < 3; ++k)
            for (int m = 0; m < 3; ++m) Linv[9 * i + 3 * k + m] = ok ? c[3 * m + k] / det : 0.0;
        if (!ok) atomicAdd(n_singular, 1u);
    }
}

// The same sums for a mixed-precision context, whose pair terms are FP32 in
// every step: X_ij is the FP64 difference rounded once to FP32, the kernel
// weight is formed in FP32, each lane sums its few pairs in FP32 and the lane
// sums meet in FP64; the 3x3 inversion stays FP64.  L and S0 come out with
// FP32 rounding of the pair terms (the mixed path keeps L^{-1} and S0 as FP32
// copies), at about a tenth of the FP64 cost.
__global__ void k_shape_f32(const double *X, const double *vol, const int64_t *row_ptr, const int32_t *col,
                            int64_t N, float inv_h, double dw_norm, double *Linv, double *S0, uint32_t *n_singular)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;
    const double xi = X[3 * i], yi = X[3 * i + 1], zi = X[3 * i + 2];
    float lf[6] = { 0, 0, 0, 0, 0, 0 };
    float gf[3] = { 0, 0, 0 };
    for (int64_t p = row_ptr[i] + lane; p < row_ptr[i + 1]; p += 32) {
        const int64_t j = col[p];
        const float dx = (float)(X[3 * j] - xi), dy = (float)(X[3 * j + 1] - yi), dz = (float)(X[3 * j + 2] - zi);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float rinv = rsqrtf(r2);
        const float c0 = (float)vol[j] * spline_dw(r2 * rinv * inv_h) * rinv;
        gf[0] += c0 * dx; gf[1] += c0 * dy; gf[2] += c0 * dz;
        lf[0] += c0 * dx * dx; lf[1] += c0 * dy * dy; lf[2] += c0 * dz * dz;
        lf[3] += c0 * dx * dy; lf[4] += c0 * dy * dz; lf[5] += c0 * dz * dx;
    }
    double l[6], g[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) l[k] = dw_norm * warp_allsum((double)lf[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = warp_allsum((double)gf[k]);
    if (lane == 0 && S0) {
        S0[3 * i] = g[0]; S0[3 * i + 1] = g[1]; S0[3 * i + 2] = g[2];
    }
    if (lane == 0) {
        double L[9], c[9];
        sym_to_full(l, L);
        cof3(L, c);
        const double det = L[0] * c[0] + L[1] * c[1] + L[2] * c[2];
        double fn2 = 0.0;
        for (int k = 0; k < 9; ++k) fn2 += L[k] * L[k];
        const double fn = sqrt(fn2);
        const bool ok = isfinite(det) && fabs(det) > 1e-12 * fn * fn * fn;
        for (int k = 0; k < 3; ++k)
            for (int m = 0; m < 3; ++m) Linv[9 * i + 3 * k + m] = ok ? c[3 * m + k] / det : 0.0;
        if (!ok) atomicAdd(n_singular, 1u);
    }
}

cudaError_t shape_matrix(const DevState &s, double h, double *Linv, double *S0, uint32_t *n_singular,
                         bool fp32_terms, cudaStream_t st)
{
    const double dw_norm = 1.0 / (M_PI * h * h * h * h);
    if (fp32_terms)
        k_shape_f32<<<blocks_for(s.N * 32, 256), 256, 0, st>>>(s.X, s.vol, s.row_ptr, s.col, s.N, (float)(1.0 / h),
                                                               dw_norm, Linv, S0, n_singular);
    else
        k_shape<<<blocks_for(s.N * 32, 256), 256, 0, st>>>(s.X, s.vol, s.row_ptr, s.col, s.N, 1.0 / h, dw_norm, Linv,
                                                           S0, n_singular);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- neighbour build without allocation
// Scratch of tlsph_neighbors_noalloc: one file-scope device array, present
// on every GPU that loads the library until the process exits.  Sized for
// NOALLOC_MAX_N particles: cell starts and cursors for 2N + 4096 cells,
// the cell item list, scan partial sums and the bounding box.
static constexpr int64_t NOALLOC_MAX_N = 262144;
static constexpr size_t NOALLOC_SCRATCH_BYTES = 10u << 20;   // 10 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// bounding box of X (one block, deterministic min / max); a coordinate that
// is not finite (fmin / fmax would skip a NaN) makes every bound NaN, which
// the host rejects
__global__ void k_bounds(const double *X, int64_t N, double *out6)
{
    __shared__ double lo[3][256], hi[3][256];
    const int t = threadIdx.x;
    double l[3] = { INFINITY, INFINITY, INFINITY }, h[3] = { -INFINITY, -INFINITY, -INFINITY };
    int bad = 0;
    for (int64_t i = t; i < N; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            const double x = X[3 * i + k];
            bad |= !isfinite(x);
            l[k] = fmin(l[k], x);
            h[k] = fmax(h[k], x);
        }
    for (int k = 0; k < 3; ++k) { lo[k][t] = l[k]; hi[k][t] = h[k]; }
    bad = __syncthreads_or(bad);
    if (bad) {
        if (t == 0)
            for (int k = 0; k < 6; ++k) out6[k] = NAN;
        return;
    }
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int k = 0; k < 3; ++k) {
                lo[k][t] = fmin(lo[k][t], lo[k][t + w]);
                hi[k][t] = fmax(hi[k][t], hi[k][t + w]);
            }
        __syncthreads();
    }
    if (t == 0)
        for (int k = 0; k < 3; ++k) { out6[k] = lo[k][0]; out6[3 + k] = hi[k][0]; }
}

// the cell grid over a bounding box: cells a little wider than rc so rounding
// in the cell coordinate can never put two particles closer than rc two cells
// apart, widened until there are at most 2N + 4096 cells
CellGrid cell_grid_from_bounds(const double *lo, const double *hi, int64_t N, double rc, int div)
{
    CellGrid g{};
    double cs = rc / (double)div * (1.0 + 1e-6);
    const double cap = 2.0 * (double)N + 4096.0;
    for (;;) {
        double cells = 1.0;
        for (int k = 0; k < 3; ++k) cells *= floor((hi[k] - lo[k]) / cs) + 1.0;
        if (cells <= cap) break;
        cs *= 1.25;
    }
    for (int k = 0; k < 3; ++k) {
        g.xmin[k] = lo[k];
        g.nc[k] = (int32_t)(floor((hi[k] - lo[k]) / cs) + 1.0);
    }
    g.cs = cs;
    g.ncells = (int64_t)g.nc[0] * g.nc[1] * g.nc[2];
    g.reach = cs >= rc ? 1 : (int32_t)ceil(rc / cs);
    return g;
}

// device address of g_noalloc_scratch, looked up once per device with that
// device current
static std::mutex g_noalloc_mutex;
static void *g_noalloc_base[256];

static cudaError_t noalloc_scratch(void **base)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_base[dev] = p;
    }
    *base = g_noalloc_base[dev];
    return cudaSuccess;
}

}  // namespace tlsph

extern "C" int tlsph_neighbors_noalloc(const double *X, int64_t N, double rc, int64_t *row_ptr, int32_t *col,
                                       int64_t nnz_cap, int64_t *nnz_out, void *stream)
{
    using namespace tlsph;
    auto fail = [](int code, const std::string &msg) {
        set_last_error_text(msg);
        return code;
    };
    if (!X || !row_ptr || !nnz_out) return fail(TLSPH_ERR_ARG, "X, row_ptr and nnz_out are required");
    if (N <= 0) return fail(TLSPH_ERR_ARG, "N must be positive");
    if (N > NOALLOC_MAX_N)
        return fail(TLSPH_ERR_ARG, "tlsph_neighbors_noalloc handles at most " + std::to_string(NOALLOC_MAX_N) +
                                   " particles (its scratch is a fixed 10 MiB device array); got N = " +
                                   std::to_string(N));
    if (!(rc > 0.0) || !isfinite(rc)) return fail(TLSPH_ERR_ARG, "rc must be positive and finite");
    if (nnz_cap < 0 || (nnz_cap > 0 && !col)) return fail(TLSPH_ERR_ARG, "col is required when nnz_cap > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return fail(TLSPH_ERR_CUDA, std::string("scratch address: ") + cudaGetErrorString(e));

    // carve the scratch (256-byte aligned pieces)
    const int64_t max_cells = 2 * N + 4096;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = static_cast<char *>(base) + off;
        off = (off + bytes + 255) & ~(size_t)255;
        return p;
    };
    Scratch sc{};
    sc.cell_start = reinterpret_cast<int64_t *>(take((size_t)(max_cells + 1) * sizeof(int64_t)));
    sc.cell_cursor = reinterpret_cast<int64_t *>(take((size_t)max_cells * sizeof(int64_t)));
    sc.cell_items = reinterpret_cast<int32_t *>(take((size_t)N * sizeof(int32_t)));
    sc.scan_tmp_elems = scan_tmp_elems(max_cells + 1);
    sc.scan_tmp = reinterpret_cast<int64_t *>(take(sc.scan_tmp_elems * sizeof(int64_t)));
    double *bounds = reinterpret_cast<double *>(take(6 * sizeof(double)));
    if (off > NOALLOC_SCRATCH_BYTES) return fail(TLSPH_ERR_NOMEM, "scratch layout exceeds its array");

    double bb[6];
    k_bounds<<<1, 256, 0, st>>>(X, N, bounds);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(bb, bounds, sizeof bb, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(TLSPH_ERR_CUDA, std::string("bounds: ") + cudaGetErrorString(e));
    for (int k = 0; k < 6; ++k)
        if (!isfinite(bb[k])) return fail(TLSPH_ERR_ARG, "X must be finite");
    const CellGrid g = cell_grid_from_bounds(bb, bb + 3, N, rc, 2);
    if (g.ncells > max_cells) return fail(TLSPH_ERR_ARG, "cell grid exceeds its bound");

    DevState s{};
    s.N = N;
    s.X = X;
    const double rc2 = rc * rc;
    int64_t nnz = 0;
    if ((e = build_neighbors_count(s, g, sc, rc2, row_ptr, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&nnz, row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(TLSPH_ERR_CUDA, std::string("neighbour count: ") + cudaGetErrorString(e));
    *nnz_out = nnz;
    if (nnz > nnz_cap)
        return fail(TLSPH_ERR_NOMEM, "col capacity too small: need nnz_cap >= " + std::to_string(nnz));
    if ((e = build_neighbors_fill(s, g, sc, rc2, row_ptr, col, st)) != cudaSuccess)
        return fail(TLSPH_ERR_CUDA, std::string("neighbour fill: ") + cudaGetErrorString(e));
    return TLSPH_OK;
}
