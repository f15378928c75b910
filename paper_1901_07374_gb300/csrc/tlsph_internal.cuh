// Internal declarations of the TLSPH CUDA library: the context, the device
// material record and the launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tlsph.h"

namespace tlsph {

// Material constants as the kernels use them: the paper's symbols plus the
// derived moduli (K = E / (3 (1 - 2 nu)), G = E / (2 (1 + nu))) and the
// reciprocals the inner loops would otherwise divide by.
struct DevMat {
    double rho0, E, K, G;
    int32_t eos, damage;
    double rho0c02, S_alpha, Gamma0;
    double A, B, n, C, inv_epsdot0;
    double inv_Wcr;
    double D1, D2, D3, D4, D5;
    double q1, q2, q3, fN, eN, sN, fc, fF, komega;
    double nucl_coef;    // fN / (sN sqrt(2 pi))
    double fstar_slope;  // (1/q1 - fc) / (fF - fc)
    double g0rho0;       // Gamma0 rho0 (energy term of the Mie-Grueneisen EOS)
    double inv_rho0;
    // single-precision copies for the mixed path's elastic fast path
    float Kf, Gf, Af, Bf, nf, Cf, inv_epsdot0f, rho0c02f, S_alphaf, Gamma0f;
    float q1f, q2f, q3f, fcf, fFf, fstar_slopef;
    float g0rho0f, inv_rho0f;
};

// Fixed-point reference positions of the mixed path: X = center + unit * (x, y, z)
// with int32 x, y, z and unit a power of two chosen so that |x|, |y|, |z| < 2^31.
// A neighbour offset X_ij is then an exact integer difference, converted to
// FP32 in units of `unit`.
struct FixPack {
    double center[3];
    double unit, inv_unit;
};

// Device arrays of one context.  SoA per quantity; vectors and tensors of a
// particle are contiguous (3 or 6/9 doubles) so the epilogues read them with
// wide loads.  Symmetric tensors are stored as 6 values (xx, yy, zz, xy, yz, zx).
struct DevState {
    int64_t N;
    const double *X;        // N*3
    const double *vol;      // N
    const double *mass;     // N   rho0 V
    const double *inv_mass; // N   1 / (rho0 V)
    const double *youngs;   // N   Young modulus of the particle's material (hourglass stiffness)
    const int32_t *mat;     // N
    const uint8_t *bcm;     // N
    const double *bcv;      // N*3
    const int64_t *row_ptr; // N+1
    const int32_t *col;     // nnz
    const double *Linv;     // N*9
    double *u[2];           // N*3 ping-pong: u^n and the predicted u^{n+1}
    double *v;              // N*3 v^n
    double *vh;             // N*3 v^{n+1/2}
    double *F;              // N*9
    double *sd;             // N*6 unrotated deviator
    double *sig;            // N*6 Cauchy stress
    double *A;              // N*9
    double *ep, *epdot, *dinit, *por;  // N
    double *D[2];           // N ping-pong
    double *force;          // N*3
    int32_t *fail;          // N
    uint32_t *status;       // 1
    const DevMat *mats;     // TLSPH_MAX_MATERIALS
    // mixed-precision records (null in the FP64 path)
    int4 *xo;               // N   {fixed-point position x, y, z (FixPack), 0}
    float4 *s0;             // N   {sum_j V_j W'(r)/r (X_j - X_i), 0}  (static, FP64-accurate)
    float *linv32;          // N*9 L^{-1} rounded
    float4 *r1;             // N   pass-1 gather record {v^{n+1/2} - vref, V (1 - D)}
    float4 *r2;             // pass-2 gather record: 6 float4 per particle in tiles of 32 particles (r2_tile)
    float *fsum;            // 9 x N pass-1 pair sums (split launch plans)
    // mixed path: F and the stress deviator as compensated FP32 pairs (value =
    // hi + lo, SoA by component: component k of particle i at k N + i); the
    // FP64 arrays F, sd and sig are refreshed from these when read
    float *Fh, *Fl;         // 9 x N deformation gradient
    float *sdh, *sdl;       // 6 x N unrotated stress deviator
    float *sigf;            // 6 x N Cauchy stress
    int32_t *slowq;         // N     particles queued for the FP64 constitutive update this step
    uint32_t *slowq_n;      // 2     queue lengths, used alternately by even and odd steps
    const int32_t *colE;    // sliced neighbour lists (slices of 32 rows, explicit or aligned form)
    const int64_t *ell_off; // (N + 31) / 32 + 1 slice word offsets
    const int32_t *ell_w;   // (N + 31) / 32 slice widths: W (explicit) or ~W (aligned)
    const float4 *w1t;      // pass-1 weight W'(q)/r of every slot (groups of 4 slots), or NULL
    const int64_t *w1t_off; // (N + 31) / 32 + 1 slice offsets into w1t (float4 units), or NULL
    double vref[3];         // bulk reference velocity of the r1 mirror
    FixPack pack;
    double grip_ramp = 0.0;  // tau of the grip velocity ramp (Sec. 6); 0: constant prescribed velocities
    double *e = nullptr;     // N   specific internal energy (Eq. conservation3)
};

// The pass-2 record is tiled by 32 particles: component k (0..5) of particle j
// sits at r2[r2_tile(j) + 32 k].  A warp reading 32 consecutive particles
// still reads 512 contiguous bytes per component, and one address reaches all
// six components of a neighbour (the others are constant offsets from it).
__host__ __device__ __forceinline__ int64_t r2_tile(int64_t j) { return (j >> 5) * (6 * 32) + (j & 31); }
constexpr int R2_STRIDE = 32;

struct Scratch {            // neighbour-build scratch (set-up only)
    int64_t *cell_start;    // ncells + 1
    int64_t *cell_cursor;   // ncells
    int32_t *cell_items;    // N
    int64_t *scan_tmp;      // scan partial sums
    size_t scan_tmp_elems;
    float4 *xf = nullptr;   // N single-precision positions for the prefilter of the FP64 predicate (or null)
};

}  // namespace tlsph

struct tlsph_ctx {
    tlsph_config cfg;
    int64_t N = 0, nnz = 0, nnz_cap = 0, steps = 0;
    cudaStream_t stream = nullptr;
    bool owns_mem = false;
    void *mem = nullptr;
    tlsph::DevState s{};
    tlsph::DevMat mats_host[TLSPH_MAX_MATERIALS]{};
    bool mat_set[TLSPH_MAX_MATERIALS]{};
    bool mat_used[TLSPH_MAX_MATERIALS]{};
    int ucur = 0;   // u[ucur] = u^n, u[ucur ^ 1] = predicted u^{n+1}
    int dcur = 0;   // D[dcur] = D^n
    // mixed launch plan: pass-1 form, block, pass-2 form, block (the fastest on
    // GB300 for the 1M-particle bar; the autotuner may choose another)
    int32_t plan[4] = { 4, 64, 4, 128 };
    double guard = 1e-5;        // relative guard band of the mixed path's FP32 elastic screen (tlsph_set_guard)
    int slow_grid = 1;          // persistent grid of the mixed path's FP64-update kernel on the context's device
    bool need_predict = true;   // v^{n+1/2}, u^{n+1} must be recomputed before the next step
    bool mixed_dirty = false;   // FP32 mirrors must be refreshed from the FP64 state
    void *mixed = nullptr;      // mixed-precision state (mixed.cu)
    // profiling: 3 events per step (before pass 1, between, after pass 2)
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev;
    int prof_used = 0;
    double prof_ms[2] = { 0.0, 0.0 };
    int64_t prof_steps = 0;
    int sticky = TLSPH_OK;
    std::string err;
    // internal order: perm[k] = caller index of internal particle k, inv its inverse
    bool reordered = false;
    bool ell_ok = false;        // sliced neighbour lists built (thread-per-row plans allowed)
    int64_t ell_words = 0;      // 4-byte words of the sliced lists
    double *diag = nullptr;     // DIAG_BLOCKS x TLSPH_DIAG_COUNT partials; the first row holds the result
    void *ell_mem = nullptr;    // library-owned sliced-ELL columns
    void *w1t_mem = nullptr;    // library-owned pass-1 weight table (pass-1 plan form 5) and its offsets
    void *w1t_off_mem = nullptr;
    void *col_mem = nullptr;    // library-owned CSR columns
    int32_t *perm_dev = nullptr;
    int32_t *inv_dev = nullptr;   // device copy of inv when reordered, else null (identity)
    std::vector<int32_t> perm, inv;   // host copies of the order when reordered (empty in caller order)
};

namespace tlsph {

// nbr.cu (scan, neighbour grid, CSR, order, correction matrix)
size_t scan_tmp_elems(int64_t n);
cudaError_t scan_exclusive_i64(int64_t *data, int64_t n, int64_t *tmp, cudaStream_t st);
struct CellGrid {
    double xmin[3];
    double cs;
    int32_t nc[3];
    int64_t ncells;
    int32_t reach;          // cells to either side that a neighbour within rc can lie in
};
// cell edge rc / div (div 1: the internal order's grid; div 2: the neighbour
// search's), enlarged while the cells would exceed 2 N + 4096
CellGrid cell_grid_from_bounds(const double *lo, const double *hi, int64_t N, double rc, int div = 1);
cudaError_t build_neighbors_count(const DevState &s, const CellGrid &g, const Scratch &sc, double rc2,
                                  int64_t *row_ptr, cudaStream_t st);
cudaError_t build_neighbors_fill(const DevState &s, const CellGrid &g, const Scratch &sc, double rc2,
                                 const int64_t *row_ptr, int32_t *col, cudaStream_t st);
// S0: optional N*3 output of sum_j V_j W'(r)/r (X_j - X_i) (kernel-normalisation free)
// internal particle order (perm[k] = caller index of internal particle k);
// keep = identity
cudaError_t build_order(const double *X_user, int64_t N, const CellGrid &g, const Scratch &sc, bool keep,
                        int32_t *perm, cudaStream_t st);
// create-time scan of the staged caller-order inputs: bounding box, the
// materials in use, the sum of the initial velocities and validity flags;
// a deterministic reduction over INSCAN_BLOCKS blocks whose result lands in
// parts[0]
struct InputScanDev {
    double lo[3], hi[3], vsum[3];
    unsigned long long mats;   // bit m: material m in use
    unsigned int bad;          // INSCAN_BAD_* bits
    unsigned int pad;
};
constexpr unsigned INSCAN_BAD_VOL = 1u, INSCAN_BAD_X = 2u, INSCAN_BAD_MAT = 4u;
constexpr int INSCAN_BLOCKS = 152;
cudaError_t launch_scan_inputs(const double *X, const double *vol, const int32_t *mat, const double *bcv, int64_t N,
                               InputScanDev *parts, cudaStream_t st);
// fp32_terms: FP32 pair terms summed in FP64 across lanes (mixed contexts)
cudaError_t shape_matrix(const DevState &s, double h, double *Linv, double *S0, uint32_t *n_singular,
                         bool fp32_terms, cudaStream_t st);

// step64.cu
// deterministic reductions of the diagnostics (tlsph_diagnostics) over a
// fixed grid of DIAG_BLOCKS blocks; the result lands in partials[0 .. TLSPH_DIAG_COUNT)
constexpr int DIAG_BLOCKS = 152;
cudaError_t launch_diagnostics(const DevState &s, int dcur, double *partials, cudaStream_t st);
cudaError_t launch_init_state(const DevState &s, cudaStream_t st);
cudaError_t launch_material_fields(const DevState &s, int mat_id, int dcur, bool gtn_damage, cudaStream_t st);
// half kick and drift of the first step after a state change; steps = steps done (the
// half-step velocity holds at (steps + 1/2) dt)
cudaError_t launch_predict(const DevState &s, int ucur, double dt, bool wall, int64_t steps, cudaStream_t st);
// prescribed particles' velocities at time t (grip ramp switched on)
cudaError_t launch_apply_grip(const DevState &s, double t, cudaStream_t st);

// rigid wall on z = 0: put a particle that drifted below it back on the plane
// and remove the velocity component into it
__host__ __device__ inline void wall_contact(double Xz, double &uz, double &vz)
{
    if (Xz + uz < 0.0) {
        uz = -Xz;
        if (vz < 0.0) vz = 0.0;
    }
}
// ev: null, or 3 events recorded before pass 1, between the passes and after pass 2
cudaError_t launch_step_fp64(const DevState &s, const tlsph_config &cfg, int ucur, int dcur,
                             int64_t step_index, cudaStream_t st, cudaEvent_t *ev);
cudaError_t launch_material_point_value(const DevMat &m, double dt, int64_t n, const double *deps,
                                        const double *J, double *state, cudaStream_t st);
cudaError_t launch_export_sym(const double *src6, double *dst9, int64_t N, cudaStream_t st);
cudaError_t launch_import_sym(const double *src9, double *dst6, int64_t N, cudaStream_t st);
// staged caller-order inputs -> internal arrays (dst[k] = src[perm[k]])
cudaError_t launch_gather_inputs(const int32_t *perm, int64_t N, const double *X, const double *vol,
                                 const int32_t *mat, const uint8_t *bcm, const double *bcv, const double *f0,
                                 const DevState &s, cudaStream_t st);
// per-particle field transfer between internal and caller order on the device:
// out: dst[perm[k]] = src[k]; in: dst[k] = src[perm[k]] (comps per particle,
// elem bytes 1/4/8; sym = 6 stored <-> 9 exchanged)
// caller-order copy of a per-particle field: dst element e (caller particle
// i = e / comps) from internal particle inv[i] (inv null: identity); sym
// expands the 6 stored components of a symmetric tensor to 9; coalesced
// writes, so dst may be device memory or mapped page-locked host memory
cudaError_t launch_to_caller(const void *src, void *dst, const int32_t *inv, int64_t N, int comps, int scomps,
                             int elem, bool sym, cudaStream_t st);
cudaError_t launch_permute(const void *src, void *dst, const int32_t *perm, int64_t N, int comps, int elem,
                           bool out, bool sym, cudaStream_t st);

DevMat make_dev_mat(const tlsph_material &m);

// text returned by tlsph_last_error(NULL) on the calling thread
void set_last_error_text(const std::string &msg);

// mixed.cu -- step constants of the mixed path (defined there)
struct MixConst {
    double dt, half_dt;
    float dt_dw, inv_h, dw_norm, w_norm, hg_coef;   // dt_dw = dt x W' normalisation; inv_h = unit / h
    float inv_unit_f;                               // 1 / unit (a power of two)
    float yield_keep;                               // 1 - guard band of the FP32 elastic screen
    float hg_w;                                     // -alpha/2 x W normalisation / unit (hourglass force factor)
    double inv_unit;
    double vref0, vref1, vref2;
    int64_t N;
    int64_t step_index;
    int ucur, dcur;
    int wall;
};

// one context in a batch table (device memory)
struct BatchSlot {
    DevState s;
    MixConst c;
    int64_t blk0;      // first work block of this context
};
struct BatchHdr {
    int nspec;
    int64_t total_blk;
    const int64_t *blk0;    // nspec first work blocks, ascending (device, after the slots)
    unsigned long long next[3];   // work-block counters of the three persistent kernels (zero between steps)
};
BatchSlot make_batch_slot(const tlsph_ctx &ctx);
// build the per-slot pass-1 weight table of a mixed context if it has none
// (library-owned memory only); a TLSPH_* code
int ctx_weight_table(tlsph_ctx *ctx);
// free it (its members and the state's pointers)
void release_w1t(tlsph_ctx *ctx);
// launch shape of the batch kernels: a variant index per kernel kind (pass-1
// gather, per-particle update, pass 2), each variant a register cap (resident
// blocks of 128 per SM) and a number of pairs in flight
constexpr int BATCH_KINDS = 3;
extern const int BATCH_VARIANTS[BATCH_KINDS];
// the pass-1 gather variant that reads the members' per-slot weight tables
constexpr int BATCH_TABLE_VARIANT = 4;
// grid: the persistent grid of each of the four kernel kinds (batch_grid)
cudaError_t launch_batch_step(BatchHdr *hdr, BatchSlot *slots, int nspec, bool hg, const int *shape, const int *grid,
                              cudaStream_t st);
void batch_grid(bool hg, const int *shape, int *grid);

// fixed-point positions xo (before the sliced lists and the correction matrices)
cudaError_t mixed_init_positions(const DevState &s, const FixPack &pk, cudaStream_t st);
// FP32 copies of S0 and L^{-1}
cudaError_t mixed_init_static(const DevState &s, const double *S0, cudaStream_t st);
// L^{-1} and S0 of a mixed context over its sliced lists (xo and the lists built)
cudaError_t mixed_shape_matrix(const DevState &s, double h, double *Linv, double *S0, uint32_t *n_singular,
                               cudaStream_t st);
cudaError_t mixed_ell_widths(const DevState &s, int64_t *ell_off, cudaStream_t st);
cudaError_t mixed_ell_fill(const DevState &s, const int64_t *ell_off, int32_t *colE, cudaStream_t st);
cudaError_t mixed_w1t_fill(const DevState &s, float inv_h, cudaStream_t st);
cudaError_t mixed_after_predict(const DevState &s, int dcur, cudaStream_t st);
// FP64 arrays -> compensated mixed state for one field (TLSPH_FIELD_F,
// _STRESS_DEV, _SIGMA) or all of them (-1)
cudaError_t mixed_import(const tlsph_ctx &ctx, int field, cudaStream_t st);
cudaError_t launch_step_mixed(tlsph_ctx &ctx, int64_t step_index, cudaStream_t st, cudaEvent_t *ev);
// persistent grid of the FP64-update kernel on the current device
int mixed_slow_grid();
// compensated mixed state -> FP64 arrays for one field or all (-1)
cudaError_t mixed_sync_to_fp64(tlsph_ctx &ctx, int field, cudaStream_t st);
int mixed_kernels_per_step(const tlsph_ctx &ctx);
void mixed_release(tlsph_ctx &ctx);

}  // namespace tlsph
