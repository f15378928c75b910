/*
 * tlsph.h -- C ABI of the GB300 (sm_103a) damage-weighted Total-Lagrangian
 * SPH step of de Vaucorbeil & Hutchinson, "A damage and failure implementation
 * for the simulation of ductile solids with Total-Lagrangian Smooth Particle
 * Hydrodynamics" (arXiv 1901.07374).
 *
 * The library advances a body of N particles through the explicit time step
 * the paper builds:
 *   - neighbour sets S_i fixed in the reference configuration (Sec. 1, 2.2),
 *   - the correction matrix L_i and the corrected kernel gradient
 *     (Sec. 2.2, Eq. correction_matrix),
 *   - the damage-weighted velocity gradient and deformation gradient
 *     (Sec. 3.1, Eqs. Crack_approx_Fdot, Crack_approx_F),
 *   - the constitutive update: equation of state (Sec. 4, Eq. pH),
 *     Johnson-Cook flow stress and radial return (Sec. 4, Eq.
 *     JC_viscoplastic_model, Algorithm 1), GTN porous plasticity (Sec. 5.4,
 *     Algorithm 2),
 *   - Cockcroft-Latham, Johnson-Cook and GTN damage with failure
 *     (Sec. 5.1-5.4); a fully damaged particle keeps no stress and rests
 *     (Sec. 3.1),
 *   - the damage-weighted nodal forces (Sec. 3.1, equation after
 *     Crack_approx_F) with hourglass control (Sec. 2 names the scheme
 *     without a formula; here a spring along each current bond of stiffness
 *     hg_alpha (E_i + E_j)/2 V_i V_j W(X_ij) / X_ij^2 on the mean of the two
 *     particles' projected position errors, scaled by (1 - D_i)(1 - D_j)),
 *   - velocity-Verlet integration.
 *
 * Units are SI.  Every floating-point array crossing this ABI is IEEE double,
 * row-major, particle-major (particle i's 3-vector at [3i, 3i+3), its 3x3
 * tensor at [9i, 9i+9) with T[9i + 3k + l] = T_kl).
 *
 * Ownership: inputs are copied at tlsph_create; the caller keeps its arrays.
 * Device memory is either a caller-owned arena (carved, never freed by the
 * library) or, when no arena is given, allocated and freed by the library.
 *
 * Errors: every entry point returns a tlsph_status.  Nothing aborts or
 * throws across the ABI.  An error inside a context is sticky: later calls on
 * that context return TLSPH_ERR_STATE until tlsph_destroy.  A text
 * description is available from tlsph_last_error.
 *
 * Threading: a context is used from one host thread at a time.  Distinct
 * contexts may be used concurrently.
 */
#ifndef TLSPH_H
#define TLSPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tlsph_ctx tlsph_ctx;

typedef enum {
    TLSPH_OK = 0,
    TLSPH_ERR_ARG = -1,         /* a null pointer, size or value out of range */
    TLSPH_ERR_SINGULAR_L = -2,  /* a correction matrix L_i is singular (e.g. a particle with no neighbours) */
    TLSPH_ERR_NUMERICS = -3,    /* device status: non-finite state, det F <= 0, or an iteration cap reached */
    TLSPH_ERR_NOMEM = -4,       /* arena too small / allocation failed / neighbour capacity exceeded */
    TLSPH_ERR_CUDA = -5,        /* a CUDA runtime call failed */
    TLSPH_ERR_STATE = -6        /* the context holds an earlier error, or a call out of order */
} tlsph_status;

/* device status bits reported through tlsph_sync / tlsph_status_bits */
#define TLSPH_ST_POLAR_CAP   1u   /* polar decomposition hit its iteration cap */
#define TLSPH_ST_NEWTON_CAP  2u   /* a GTN Newton solve hit its iteration cap */
#define TLSPH_ST_BAD_J       4u   /* det F^{n+1} <= 0 or non-finite */
#define TLSPH_ST_NONFINITE   8u   /* a non-finite stress or force */

/* arithmetic of the per-pair work */
#define TLSPH_PRECISION_FP64  0   /* everything in FP64 */
#define TLSPH_PRECISION_MIXED 1   /* FP32 pair gathers and sums, FP64 state, guards and constitutive update */

typedef struct {
    double h;          /* smoothing length [m]; the cubic-spline kernel has support 2h */
    double rc;         /* neighbour cutoff [m]: S_i = { j != i : |X_j - X_i| < rc } (normally 2h) */
    double dt;         /* time step [s], fixed for the run */
    double hg_alpha;   /* hourglass-control coefficient (0 disables it) */
    int32_t precision; /* TLSPH_PRECISION_FP64 or TLSPH_PRECISION_MIXED */
    int32_t flags;     /* 0 or an OR of at most one of TLSPH_FLAG_SPATIAL_ORDER, TLSPH_FLAG_LINE_ORDER,
                          TLSPH_FLAG_AUTO_ORDER and of TLSPH_FLAG_WALL */
} tlsph_config;

/* Store particles in a spatially compact internal order (cells of the
 * neighbour grid grouped into 4x4x4-cell bricks, caller index inside a
 * cell).  Every field crossing the ABI stays in the caller's order.  Off by
 * default: for particles generated lattice-row by lattice-row the caller's
 * order is faster, because the k-th neighbours of consecutive rows are then
 * consecutive particles and a warp's gathers coalesce; the brick order helps
 * inputs in arbitrary order. */
#define TLSPH_FLAG_SPATIAL_ORDER 1

/* Store particles in lattice-line order along the specimen's longest
 * bounding-box axis L: sorted by (round((X_a - min_a) / d),
 * round((X_b - min_b) / d), X_L) with a, b the two shorter axes and d the
 * cube root of the median particle volume.  For particles on a (jittered)
 * simple cubic lattice of spacing d every lattice line along L becomes
 * contiguous, so the 32 rows of a warp share their neighbourhood shape and
 * their neighbour index offsets: the mixed path's neighbour lists are then
 * aligned slices with almost no padding slots.  Every field crossing the ABI
 * stays in the caller's order; results differ from the caller's order only by
 * the order of the sums over j.  Not combinable with TLSPH_FLAG_SPATIAL_ORDER
 * or TLSPH_FLAG_AUTO_ORDER (TLSPH_ERR_ARG). */
#define TLSPH_FLAG_LINE_ORDER 4

/* Choose the internal order at creation (mixed precision; an FP64 context
 * keeps the caller's order): the caller's order when at least nine in ten of
 * the mixed path's 32-row neighbour slices come out aligned
 * (tlsph_neighbor_layout), otherwise TLSPH_FLAG_LINE_ORDER if that aligns
 * more of them.  The choice costs one more creation (and the line sort) only
 * for inputs whose order leaves their slices explicit, e.g. bodies whose
 * lattice lines change length across the cross-section.  Not combinable with
 * the other order flags (TLSPH_ERR_ARG). */
#define TLSPH_FLAG_AUTO_ORDER 8

/* A rigid frictionless wall on the plane z = 0 (current configuration): a
 * particle that would drift below it is put back on the plane and its
 * velocity may not point into it (a kinematic contact; the paper has none).
 * Used by the Taylor-impact workload. */
#define TLSPH_FLAG_WALL 2

/* damage models */
#define TLSPH_DAMAGE_NONE 0
#define TLSPH_DAMAGE_CL   1   /* Cockcroft-Latham (Sec. 5.1) + linear evolution (Sec. 5.3) */
#define TLSPH_DAMAGE_JC   2   /* Johnson-Cook (Sec. 5.2) + linear evolution (Sec. 5.3) */
#define TLSPH_DAMAGE_GTN  3   /* Gurson-Tvergaard-Needleman (Sec. 5.4, Algorithm 2) */

/* A material (Sec. 4 and 5).  Field meaning follows the paper's symbols. */
typedef struct {
    double rho0, E, nu;       /* reference density, Young modulus, Poisson ratio */
    int32_t eos;              /* 0: linear sigma_m = K (J - 1); 1: Mie-Grueneisen (Eq. pH) */
    double c0, S_alpha, Gamma0;               /* Mie-Grueneisen constants (eos = 1) */
    double A, B, n, C, epsdot0;               /* Johnson-Cook flow stress (Eq. JC_viscoplastic_model), T* = 0 */
    int32_t damage;                           /* TLSPH_DAMAGE_* */
    double Wcr;                               /* Cockcroft-Latham critical plastic work [Pa] */
    double D1, D2, D3, D4, D5;                /* Johnson-Cook damage constants */
    double q1, q2, q3, fN, eN, sN, fc, fF, komega; /* GTN constants */
} tlsph_material;

#define TLSPH_MAX_MATERIALS 64

/* Fields of tlsph_get_state / tlsph_set_state (element type and count). */
typedef enum {
    TLSPH_FIELD_X = 0,          /* f64 N*3  reference positions (read only) */
    TLSPH_FIELD_U = 1,          /* f64 N*3  displacement u^n */
    TLSPH_FIELD_V = 2,          /* f64 N*3  velocity v^n */
    TLSPH_FIELD_F = 3,          /* f64 N*9  deformation gradient F^n */
    TLSPH_FIELD_SIGMA = 4,      /* f64 N*9  Cauchy stress (current frame; the next step's internal-energy
                                                update starts from it) */
    TLSPH_FIELD_STRESS_DEV = 5, /* f64 N*9  unrotated deviatoric stress (the constitutive state) */
    TLSPH_FIELD_EPSP = 6,       /* f64 N    equivalent plastic strain (matrix strain for GTN) */
    TLSPH_FIELD_EPSP_RATE = 7,  /* f64 N    plastic strain rate of the last step */
    TLSPH_FIELD_DINIT = 8,      /* f64 N    damage initiation variable D_init */
    TLSPH_FIELD_DAMAGE = 9,     /* f64 N    damage D */
    TLSPH_FIELD_POROSITY = 10,  /* f64 N    GTN void volume fraction f */
    TLSPH_FIELD_FAIL_STEP = 11, /* i32 N    step at which the particle failed, -1 while intact */
    TLSPH_FIELD_FORCE = 12,     /* f64 N*3  nodal force f^n */
    TLSPH_FIELD_A = 13,         /* f64 N*9  A_i = P_i L_i^{-T} (read only) */
    TLSPH_FIELD_LINV = 14,      /* f64 N*9  L_i^{-1} (read only) */
    TLSPH_FIELD_NBR_ROWPTR = 15,/* i64 N+1  neighbour CSR row pointers (read only) */
    TLSPH_FIELD_NBR_COL = 16,   /* i32 nnz  neighbour CSR columns, rows ascending (read only) */
    TLSPH_FIELD_STEP = 17,      /* i64 1    number of completed steps (failure steps count from it) */
    TLSPH_FIELD_ENERGY = 18,    /* f64 N    specific internal energy e (J/kg; Sec. 2.1, Eq. conservation3) */
    TLSPH_FIELD_COUNT = 19
} tlsph_field;

/* Bytes of device memory a context needs for N particles and up to nnz_cap
 * neighbour pairs; 0 if the arguments are invalid. */
size_t tlsph_workspace_bytes(const tlsph_config *cfg, int64_t N, int64_t nnz_cap);

/* Create a context: copies the inputs to the device, builds the neighbour
 * CSR (cell binning on the GPU, rows sorted ascending), computes L_i^{-1}
 * and sets the initial state (u = 0, F = I, no stress, v = bc_vel, f = f0).
 *   X       host, N*3 reference positions
 *   vol     host, N reference volumes (> 0)
 *   mat_id  host, N material indices in [0, TLSPH_MAX_MATERIALS), or NULL (all 0)
 *   bc_mask host, N bytes, 1 = velocity prescribed to bc_vel every step, or NULL
 *   bc_vel  host, N*3 prescribed velocities; also the initial velocity of
 *           unconstrained particles when bc_mask[i] == 0 (may be NULL: zero)
 *   f0      host, N initial porosity (GTN), or NULL (zero)
 *   arena   device memory owned by the caller, 256-byte aligned, or NULL for
 *           library-owned memory; arena_bytes its size
 *   nnz_cap neighbour capacity when an arena is given (use
 *           tlsph_workspace_bytes to size the arena); ignored otherwise
 *   stream  cudaStream_t every launch of this context is ordered on (NULL:
 *           the legacy default stream)
 * Blocks until the set-up is done.  Returns TLSPH_ERR_SINGULAR_L if some L_i
 * is singular, TLSPH_ERR_NOMEM if the arena or nnz_cap is too small (the
 * needed pair count is in tlsph_last_error(NULL)); no context is created on
 * error (an arena's contents are then unspecified: the inputs are validated
 * on the device after their upload). */
int tlsph_create(const tlsph_config *cfg, int64_t N, const double *X, const double *vol,
                 const int32_t *mat_id, const uint8_t *bc_mask, const double *bc_vel,
                 const double *f0, void *arena, size_t arena_bytes, int64_t nnz_cap,
                 void *stream, tlsph_ctx **out);

/* Set material `mat_id` (Sec. 4-5 constants).  Every material referenced by
 * mat_id must be set before the first tlsph_step.  Setting a GTN material
 * before the first step also sets D = q1 f*(f0) on its particles. */
int tlsph_set_material(tlsph_ctx *ctx, int mat_id, const tlsph_material *mat);

/* Enqueue nsteps time steps on the context's stream (asynchronous; errors of
 * the device work are reported by tlsph_sync). */
int tlsph_step(tlsph_ctx *ctx, int nsteps);

/* Wait for the context's stream; returns TLSPH_ERR_NUMERICS if the device
 * status word has any TLSPH_ST_* bit set (the bits stay readable through
 * tlsph_status_bits), TLSPH_ERR_CUDA on a CUDA error. */
int tlsph_sync(tlsph_ctx *ctx);

/* Device status bits accumulated since create (synchronises). */
int tlsph_status_bits(tlsph_ctx *ctx, uint32_t *bits);

/* N, nnz and the number of completed steps. */
int tlsph_info(const tlsph_ctx *ctx, int64_t *N, int64_t *nnz, int64_t *steps);

/* Copy a field (tlsph_field) at the current step boundary into dst (host
 * memory, or device memory if dst_on_device), `bytes` must equal the field's
 * size.  A page-locked host dst (cudaHostAlloc, cudaHostRegister, a pinned
 * torch tensor) is written by the device directly; a pageable one through a
 * host staging copy.  Synchronises the context's stream. */
int tlsph_get_state(tlsph_ctx *ctx, int field, void *dst, size_t bytes, int dst_on_device);

/* Overwrite a writable field (U, V, F, SIGMA, STRESS_DEV, EPSP, EPSP_RATE,
 * DINIT, DAMAGE, POROSITY, ENERGY, FAIL_STEP, FORCE, STEP) from src; the
 * half-step velocity and the predicted displacement are recomputed from U, V
 * and FORCE.  Used for checkpoint/resume (all of these fields together are a
 * resumable state: the internal-energy update of the next step starts from
 * SIGMA) and for tests that start from a chosen state. */
int tlsph_set_state(tlsph_ctx *ctx, int field, const void *src, size_t bytes, int src_on_device);

/* Last error text of ctx, or of the calling thread's last failed
 * tlsph_create or tlsph_neighbors_noalloc when ctx is NULL.  Valid until the
 * next call on ctx. */
const char *tlsph_last_error(const tlsph_ctx *ctx);

/* Diagnostics of the state at the current step boundary (no counterpart in
 * the paper; conservation checks and monitoring): out[0..2] momentum
 * sum_i m_i v_i, out[3..5] force sum sum_i f_i, out[6] kinetic energy
 * sum_i m_i |v_i|^2 / 2, out[7] number of failed particles, out[8] largest D,
 * out[9] largest equivalent plastic strain, out[10] internal energy
 * sum_i m_i e_i (Eq. conservation3; with out[6] the energy balance); SI units, FP64, host array of n =
 * TLSPH_DIAG_COUNT doubles.  The sums are deterministic (fixed blocking and
 * order).  Synchronises the context's stream.  TLSPH_ERR_ARG for n !=
 * TLSPH_DIAG_COUNT or NULL out. */
#define TLSPH_DIAG_COUNT 11
int tlsph_diagnostics(tlsph_ctx *ctx, double *out, int n);

/* The same reductions without waiting: they and the copy of the
 * TLSPH_DIAG_COUNT doubles into out are queued on the context's stream
 * behind the work already queued there (so they describe the state after the
 * steps queued before the call), and out holds them once the stream has
 * passed that point (tlsph_sync, or an event recorded on the stream after the
 * call).  out: host memory that stays valid until then, page-locked for the
 * copy not to wait; several calls may be in flight, each into its own out.
 * TLSPH_ERR_ARG for n != TLSPH_DIAG_COUNT or NULL out. */
int tlsph_diagnostics_async(tlsph_ctx *ctx, double *out, int n);

/* Release the context (and its device memory when the library owns it). */
int tlsph_destroy(tlsph_ctx *ctx);

/* Launch plan of the mixed-precision step: plan[0] pass-1 form (0 warp per
 * 32 rows; 1 thread per row; 2 thread-per-row gather + per-particle kernel;
 * 3 warp-per-32-rows gather + per-particle kernel; 4 as 2 with four pairs in
 * flight per thread; 5 as 4 with the kernel weight W'(q)/r of every slot read
 * from a table the library builds when the form is set, 4 bytes per slot of
 * the sliced lists, and frees when another form is set: the same bits as 4,
 * TLSPH_ERR_ARG for a context in a caller arena, TLSPH_ERR_NOMEM if the table
 * does not fit; block size at most 128), plan[1] its block size, plan[2]
 * pass-2 form (0 warp
 * per 32 rows; 1 thread per row, two pairs in flight; 2 thread-per-row
 * gather + per-particle kernel; 3 thread per row, one pair in flight; 4 as
 * 1 with registers capped for six resident blocks; 5 as 3 with registers
 * capped for eight resident blocks; 6 as 1 capped for seven resident blocks;
 * 7 as 1 capped for five resident blocks; 8 as 7 with rows 0 and 1 of the
 * stress term formed by packed FP32x2 operations; block size at most 128 for
 * 4 to 8),
 * plan[3] its block size (multiples of 32 up to 256).  Every plan computes
 * the same method; sums over a row are grouped differently, so results
 * differ only by FP32 rounding.  n must be 4.  TLSPH_ERR_ARG for a plan out
 * of range.  A new mixed context starts with (4, 64, 4, 128).  The FP64 path
 * ignores the plan. */
int tlsph_set_plan(tlsph_ctx *ctx, const int32_t *plan, int n);
int tlsph_get_plan(const tlsph_ctx *ctx, int32_t *plan, int n);

/* Guard band of the mixed path's FP32 elastic screen (Algorithm 1, Sec. 4:
 * the decision sigma_eq <= sigma_f; the band has no counterpart in the
 * paper).  A particle takes the FP32 elastic branch only when, in FP32,
 * sigma_eq^2 <= sigma_f^2 (1 - band); every other particle runs the FP64
 * constitutive update.  band >= 1e-5 (default 1e-5) keeps the screen
 * conservative; band >= 1 sends every particle through the FP64 update.
 * TLSPH_ERR_ARG for band < 1e-5 or non-finite.  Applies to the context's
 * own steps and, through the batch table, to batched steps after the next
 * tlsph_batch_set.  The FP64 path ignores it. */
int tlsph_set_guard(tlsph_ctx *ctx, double band);


/* Grip velocity ramp (Sec. 6: the end rows move at v_max (1 - e^{-t}), with
 * v_max in mm/ms and t in ms).  With tau > 0 every prescribed velocity
 * (bc_mask set) holds as bc_vel (1 - exp(-t / tau)) at the time t of the
 * velocity it constrains: t_n + dt/2 for the half-step velocity, t_{n+1} for
 * the step's end, t_n = n dt with n the context's step count.  tau = 0
 * (default) keeps bc_vel constant.  On the call the prescribed particles'
 * velocities are set to their ramped value at the current time (zero at
 * step 0), and the next step starts from them.  Fully damaged particles stay
 * at rest.  TLSPH_ERR_ARG for tau < 0 or non-finite.  Batches pick the ramp
 * up at the next tlsph_batch_set. */
int tlsph_set_grip_ramp(tlsph_ctx *ctx, double tau);

/* Form of the mixed path's sliced neighbour lists (the thread-per-row plans
 * read the fixed neighbour sets of Sec. 2.2 through them; the paper has no
 * counterpart of the layout).  A slice is the 32 consecutive rows of one warp.
 * An "aligned" slice stores the union of its rows' neighbour index offsets
 * j - i once plus one bit per row and offset; an "explicit" slice stores
 * every row's neighbour indices, padded to the slice's longest row.  Writes
 * the number of slices, of aligned slices, of slots (32 x slice width,
 * summed) and of 4-byte words the lists occupy; each pointer may be NULL.
 * Reads the slice widths back from the device (synchronises the context's
 * stream).
 * TLSPH_ERR_STATE if the context has no sliced lists (FP64 precision, or
 * a caller arena too small for them). */
int tlsph_neighbor_layout(const tlsph_ctx *ctx, int64_t *slices, int64_t *aligned_slices, int64_t *slots,
                          int64_t *words);

/* ---- Batched stepping (many specimens advanced together) ----------------
 * A batch advances every member context with one launch per kernel kind and
 * step over all members (a persistent grid striding over every member's
 * blocks of rows), optionally replayed from a captured CUDA graph.  Members
 * must be mixed-precision contexts (TLSPH_PRECISION_MIXED) that all use
 * hourglass control or all do not.  A member's rows are computed by the
 * same kernels whatever else is in the batch, so its result alone in a batch
 * and in any mix is identical bit for bit; against the context's own
 * tlsph_step launches it agrees to FP32 rounding.  The member set can change
 * between calls (continuous batching) without recapturing the graph. */
typedef struct tlsph_batch tlsph_batch;

/* capacity: most members at once; stream: the caller's cudaStream_t the
 * batch's work is ordered with (the launches themselves run on a stream the
 * batch owns, so a CUDA graph can be captured even when `stream` is the
 * legacy default stream) */
int tlsph_batch_create(int capacity, void *stream, tlsph_batch **out);

/* Replace the member set (n <= capacity contexts, no repeats).  Waits for
 * each member's own stream.  A member stepped or modified outside the batch
 * must be set again before the next tlsph_batch_step. */
int tlsph_batch_set(tlsph_batch *b, tlsph_ctx *const *ctxs, int n);

/* Enqueue nsteps steps of every member on the batch stream (use_graph != 0:
 * capture one step as a CUDA graph on first use and replay it).  Later work
 * on a member's own stream (tlsph_get_state, tlsph_sync) is ordered after it. */
int tlsph_batch_step(tlsph_batch *b, int nsteps, int use_graph);

int tlsph_batch_sync(tlsph_batch *b);
const char *tlsph_batch_last_error(const tlsph_batch *b);

/* Launch shape of the batch's kernels (no paper counterpart; a performance
 * setting): shape[k] selects a variant for kernel kind
 * k = 0 (pass-1 gather), 1 (per-particle update), 2 (pass 2); a variant
 * fixes how many blocks of 128 threads the kernel's registers are capped for
 * and how many neighbour pairs a thread has in flight (and, for one pass-2
 * variant, packed FP32x2 stress rows as in pass-2 plan form 8; pass-1 variant
 * 4 reads each member's per-slot weight table as pass-1 plan form 5 does,
 * building the tables members lack: TLSPH_ERR_ARG for a member in a caller
 * arena, and a member whose table is released by its own tlsph_set_plan
 * stops tlsph_batch_step with TLSPH_ERR_STATE until tlsph_batch_set).  n must
 * be 3 (the
 * number of kinds).  Setting a different shape waits for the batch's
 * launches in flight and re-captures its graph at the next tlsph_batch_step.
 * Every variant computes the same method; the results of two variants agree
 * to FP32 rounding (the compiler may fuse multiply-adds differently under
 * another register cap), and with any one shape a member's result does not
 * depend on the other members.  TLSPH_ERR_ARG for an index out of
 * range.  tlsph_batch_get_shape writes the current variant of each kind into
 * shape and the number of variants of each kind into variants (either may be
 * NULL). */
int tlsph_batch_set_shape(tlsph_batch *b, const int32_t *shape, int n);
int tlsph_batch_get_shape(const tlsph_batch *b, int32_t *shape, int32_t *variants, int n);
int tlsph_batch_destroy(tlsph_batch *b);

/* Per-kernel device time of the step (CUDA events recorded around each
 * launch on the context's stream).  enable != 0 clears the accumulators and
 * starts recording; 0 stops.  Hot-path kernels: 0 = pass 1 (velocity
 * gradient + constitutive update), 1 = pass 2 (forces + integration). */
int tlsph_profile_enable(tlsph_ctx *ctx, int enable);

/* Accumulated device milliseconds of kernel k into ms[k] for k < n and the
 * number of profiled steps (synchronises). */
int tlsph_profile_read(tlsph_ctx *ctx, double *ms, int n, int64_t *steps);

/* Material-point update (the constitutive step of one particle, Sec. 4-5,
 * Algorithms 1-2, with the damage update) applied to n independent points on
 * the device.  All pointers are DEVICE memory:
 *   deps   n*9 strain increments in the unrotated frame (symmetric)
 *   J      n   det F^{n+1}
 *   state  n*16 in/out: [0,9) unrotated deviator, 9 sigma_m, 10 eps_p,
 *          11 eps_p rate, 12 D_init, 13 D, 14 f, 15 failed (0/1)
 * Asynchronous on `stream`. */
int tlsph_material_point_batch(const tlsph_material *mat, double dt, int64_t n,
                               const double *deps, const double *J, double *state,
                               void *stream);

/* Neighbour CSR of N reference positions without allocating any memory.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory -- code running under a host framework that owns
 * all device memory through its own pool, loops that must not take the
 * device-wide synchronisation a cudaMalloc/cudaFree implies, or plugins with
 * no allocator of their own.  It computes the same rows as tlsph_create
 * (S_i = { j != i : |X_j - X_i| < rc } with the same FP64 predicate, rows
 * ascending) but takes device inputs and outputs and keeps its scratch in a
 * fixed 10 MiB device array inside the library, which every GPU that loads
 * the library holds until the process exits.
 *   X        device, N*3 reference positions
 *   N        1 <= N <= 262144 (larger N is rejected with TLSPH_ERR_ARG)
 *   rc       cutoff (> 0)
 *   row_ptr  device, N+1 int64 output
 *   col      device, nnz_cap int32 output (may be NULL when nnz_cap == 0)
 *   nnz_out  host, receives the number of pairs
 *   stream   cudaStream_t for every launch (NULL: legacy default stream)
 * Returns TLSPH_ERR_NOMEM, with row_ptr and *nnz_out filled but col not
 * written, when nnz_cap is smaller than the pair count (call again with a
 * larger col).  It synchronises the stream twice (to read the bounding box
 * and the pair count); the column fill is still in flight on `stream` when
 * it returns.  The first call on a device looks up the scratch address on
 * that device (make it before any stream capture).  All calls share the one
 * scratch array and leave their contents in it: calls whose work overlaps on
 * the GPU (different streams, or another thread) race and must be
 * serialised by the caller.  Nothing is allocated, freed or pinned. */
int tlsph_neighbors_noalloc(const double *X, int64_t N, double rc, int64_t *row_ptr, int32_t *col,
                            int64_t nnz_cap, int64_t *nnz_out, void *stream);

/* ---- FMA-rate microbenchmark (no counterpart in the paper) -------------
 * Measures the current device's fused multiply-add rate, FP32 (fp64 = 0) or
 * FP64 (fp64 != 0): every resident thread of an SM-filling grid runs 8
 * independent FMA chains of 64 x iters FMAs (1 <= iters <= 2^20), timed with
 * CUDA events on a private stream after a warm-up launch.  Writes FMAs per
 * second to *fma_per_s (host).  It allocates and frees a small device sink.
 * TLSPH_ERR_ARG for a bad argument, TLSPH_ERR_CUDA if a CUDA call fails. */
int tlsph_fma_peak(int fp64, int iters, double *fma_per_s);

#ifdef __cplusplus
}
#endif

#endif /* TLSPH_H */
