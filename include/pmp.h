/*
 * pmp.h -- C ABI of the particle-mesh-particle (PMP) library for NVIDIA GB300
 * (sm_103a).
 *
 * The library implements the five-step particle-mesh-particle cycle of He,
 * Wibking, Vijayan, Krumholz & Li, "A novel algorithm for GPU-accelerated
 * particle-mesh interactions implemented in the Quokka code"
 * (arXiv:2509.18261), Sec. 2.2, for the two interaction kinds of Sec. 3:
 * supernova feedback (Sec. 3.2.1) and sink accretion (Sec. 3.1.1).
 *
 * Memory.  Every pointer handed to a pmp_* call is a DEVICE pointer owned by
 * the caller (for example the storage of a torch tensor), except where a
 * comment says "host".  The library borrows device pointers only for the work
 * it enqueues and never frees them.  It allocates device memory only in
 * pmp_create (a few hundred bytes for status words), pmp_batch_create and
 * pmp_batch_set_particles (a batch's tables), and frees it in pmp_destroy /
 * pmp_batch_destroy.  Scratch memory of a pass is the caller's: pmp_workspace_size
 * gives its size, pmp_gather writes the pass's plan into it (each particle's
 * kernel cells, found once), and pmp_deposit, pmp_apply_limited and
 * pmp_backward read it.
 *
 * Streams.  Work is enqueued on the context's stream (pmp_create /
 * pmp_set_stream) and returns immediately, except where a comment says the
 * call synchronises.
 *
 * Errors.  Argument errors are detected on the host: the call returns a
 * non-zero pmp_status and enqueues nothing.  Errors found while kernels run
 * (a particle outside the box, a non-finite or non-positive input) set a
 * sticky device status word; the affected particle or cell is skipped, no
 * kernel traps, and pmp_get_error reads and clears the word.
 *
 * Mesh layout (pmp_mesh).  Five FP64 fields (rho, p_x, p_y, p_z, E) of a box
 * of n[0] x n[1] x n[2] valid cells with ng ghost cells on every side.
 * Field f, cell (i, j, k), -ng <= i < n[0] + ng (likewise j, k), lives at
 *   data[f * field_stride + ((k + ng) * (n[1] + 2 ng) + (j + ng)) * (n[0] + 2 ng) + (i + ng)].
 * field_stride >= (n[0] + 2 ng)(n[1] + 2 ng)(n[2] + 2 ng); a multiple of 32
 * keeps every field 256-byte aligned.  Cells are cubes of side dx; positions
 * are in cell units, the centre of cell i at i + 1/2.
 *
 * The STATE mesh holds the conserved quantities U; only its valid cells are
 * read or written (ghost cells are never touched; on a periodic axis the
 * kernel wraps).  The BUFFER mesh holds Delta U^buf (Step 1, Eq.
 * delta_u_buf); it must have the state's n and periodic flags and
 * ng >= ceil(r_K), and must not overlap the state.
 *
 * Particles (pmp_particles).  Structure-of-arrays FP64, count entries each.
 *   x, y, z  position in cell units, 0 <= x < n[0] (likewise y, z).
 *   m        feedback: ejecta mass M_ej; sink: sink mass m_s.
 *   px..pz   feedback: ejecta momentum M_ej v_ej; sink: sink momentum.
 *   e        feedback: supernova energy E_sn; sink: unused (may be NULL).
 * Step 4 (sinks) updates m and p in place.
 *
 * Gathered rows.  pmp_gather writes a [rows][count] FP64 array (row r of
 * particle s at gathered[r * count + s]); rows = pmp_gathered_rows(kind):
 *   feedback (12): M_snr, V_snr, v_COM x, y, z, n_H, R_M, |p_radial|,
 *                  q = M_ej/V_snr, e = (E_sn + E_kin)/V_snr, |p_radial|/V_snr,
 *                  regime (0 EJ, 1 ST, 2 MC)                     (Sec. 3.2.1)
 *   sink (8):      rho_inf, v_inf, c_inf, mdot_BH, r_acc (cell units), sum w,
 *                  K = mdot_BH dt / V / sum w, kernel cell count  (Sec. 3.1.1)
 *   mass (6):      V_K = sum omega V, then m, p_x, p_y, p_z, e divided by V_K
 *
 * Numerics.  All arithmetic is FP64 in one fixed order per quantity, so the
 * sorted deposit is bit-for-bit reproducible across runs and launch shapes.
 * Products are rounded on their own except in four places, where a product
 * and the addition it feeds are fused (one rounding): the supernova gather
 * sums, the sum of the sink kernel weights, the momentum and energy rows of
 * Eq. du, and the Step-4 sums.  exp and log are the library's own (Cody &
 * Waite reduction plus a Taylor / atanh series).
 */
#ifndef PMP_H
#define PMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pmp_ctx pmp_ctx;
typedef struct CUstream_st *pmp_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    PMP_OK = 0,
    PMP_ERR_ARG = 1,              /* invalid argument (host check; nothing enqueued) */
    PMP_ERR_GHOST_TOO_THIN = 2,   /* buffer ng < ceil(r_K), or ng > n on some axis */
    PMP_ERR_PARTICLE_OUTSIDE = 3, /* device: a position outside [0, n) */
    PMP_ERR_NONFINITE = 4,        /* device: NaN/Inf or a non-positive mass/density */
    PMP_ERR_TIMEOUT = 5,          /* device: a bounded wait gave up */
    PMP_ERR_WORKSPACE = 6,        /* workspace missing or smaller than pmp_workspace_size */
    PMP_ERR_CUDA = 7              /* a CUDA runtime call failed */
} pmp_status;

/* Interaction kinds.  MASS is the particle-mesh (PM / PIC) deposit of Sec. 2.2,
 * which needs Steps 1, 2 and 5 only: no limiter and no particle update.  A
 * MASS particle spreads its mass, momentum and energy content (m, p, e) over
 * its kernel cells in proportion to the covered fraction omega of the
 * supernova kernel (r_K, subsample), Delta U_c = omega_c (m, p, e) / V_K with
 * V_K = sum_c omega_c V, so sum_c Delta U_c V = (m, p, e).  (The paper names
 * no assignment function for this use.)  `e` may be NULL (no energy). */
typedef enum { PMP_KIND_FEEDBACK = 0, PMP_KIND_SINK = 1, PMP_KIND_MASS = 2 } pmp_kind;

/* Step-1 accumulation strategy.
 * ATOMIC:  FP64 atomic additions (Sec. 2.2, Step 1); per cell the sum equals
 *          the sorted one up to the order of additions.  For sinks every
 *          pair's change is -a (1, p/rho, E/rho) with its cell's factors, so
 *          the deposit adds only -a per pair into a one-field scratch and a
 *          second pass adds (sum -a)(1, p/rho, E/rho) to each buffer cell
 *          (fused multiply-adds): the same sum up to the order of additions
 *          and the rounding of one product per value.
 * SORTED:  (cell, particle) pairs sorted by cell, then each cell summed in
 *          particle-index order; deterministic.
 * ROUNDED: the paper's reproducible atomics (App. A.1).  Each atomic
 *          addition to a buffer value also adds eps |new value| (eps = 2^-52)
 *          to an error bound E of that value; after the last particle every
 *          buffer value v (ghost cells included) loses the low
 *          N_bit = ceil(log2(E / |v|)) + 52 + M bits of its significand
 *          (N_bit clamped to [0, 52]; truncation toward zero; v = 0 or E = 0
 *          unchanged).  Two runs that add in different orders then agree bit
 *          for bit except with probability about 2^-M per value that several
 *          particles reach.  M is the context's (pmp_set_rounding_margin,
 *          28 by default).  E lives in the workspace. */
typedef enum { PMP_MODE_ATOMIC = 0, PMP_MODE_SORTED = 1, PMP_MODE_ROUNDED = 2 } pmp_mode;

typedef struct {
    int32_t n[3];        /* valid cells per axis, >= 1 */
    int32_t ng;          /* ghost cells on each side, >= 0 */
    int32_t periodic[3]; /* 1 = axis wraps; 0 = kernel cut at the domain face */
    int32_t reserved;    /* set to 0 */
    double dx;           /* cell size (physical units); V = dx^3 */
    int64_t field_stride;/* doubles between consecutive fields */
    double *data;        /* device, [5][field_stride] */
} pmp_mesh;

typedef struct {
    int64_t count;
    const double *x, *y, *z; /* device */
    double *m;               /* device */
    double *px, *py, *pz;    /* device */
    const double *e;         /* device; feedback only */
} pmp_particles;

/* Parameters of one interaction kind.  Units are the caller's (code units). */
typedef struct {
    int32_t kind;      /* pmp_kind */
    int32_t subsample; /* feedback: sub-points per axis (1..8) for the covered
                          fraction omega of a kernel cell (Sec. 3.2.1) */
    double r_K;        /* kernel radius in cells, 1 <= r_K <= 6 (Sec. 2.1) */
    double dt;         /* sink: time step (Eq. accretion_function) */
    double G;          /* sink: gravitational constant (Eq. rbh, Eq. truelove) */
    double gamma;      /* adiabatic index, > 1 */
    double lambda_bh;  /* sink: lambda of Eq. mdot (e^1.5 / 4 in the paper) */
    double J;          /* sink: Jeans number of Eq. truelove (0.25) */
    double cap;        /* sink: largest removed fraction of a cell's mass (0.25) */
    double rho_min;    /* sink: density floor */
    double A_sf;       /* feedback: M_sf = A_sf n_H^-0.26 */
    double A_p;        /* feedback: P_snr = A_p n_H^-0.17 (Eq. psnr) */
    double mu_H;       /* feedback: mass per H nucleus */
    double RM_ej;      /* feedback: EJ if R_M <= RM_ej (0.027) */
    double RM_st;      /* feedback: ST if RM_ej < R_M <= RM_st (1), else MC */
    double eps_K;      /* feedback: kinetic fraction of Eq. dp (0.28) */
} pmp_params;

/* Creates a context for one interaction kind; validates params (returns
 * PMP_ERR_ARG on a bad value) and allocates its device status words on the
 * current device.  *out is set to NULL on failure. */
pmp_status pmp_create(pmp_ctx **out, const pmp_params *params, pmp_stream stream);

/* Frees the context (synchronises its stream first).  NULL is ignored. */
void pmp_destroy(pmp_ctx *ctx);

/* Changes the stream later calls enqueue on. */
pmp_status pmp_set_stream(pmp_ctx *ctx, pmp_stream stream);

/* Sets the safety margin M of the ROUNDED deposit (App. A.1; 0 <= M <= 104,
 * else PMP_ERR_ARG).  Host only; applies to later pmp_deposit calls. */
pmp_status pmp_set_rounding_margin(pmp_ctx *ctx, int32_t M);

/* Number of gathered rows for a kind (12 feedback, 8 sink, 6 mass); 0 if unknown. */
int32_t pmp_gathered_rows(int32_t kind);

/* Bytes of device workspace one pass needs for `n_particles` particles of
 * the context's kind on a mesh with the buffer's n, with the deposit
 * strategy `mode` (ROUNDED adds 5 x field_stride doubles for the error
 * bound, ATOMIC for sinks field_stride doubles for the deposit's scratch, so
 * these depend on the buffer's field_stride too).  Host only, no device
 * work. */
pmp_status pmp_workspace_size(const pmp_ctx *ctx, const pmp_mesh *buffer, int64_t n_particles, int32_t mode,
                              size_t *bytes);

/* Step 1, preparation: Delta U^buf = 0 on every cell of the buffer, ghosts
 * included (Sec. 2.2, Step 1: "all cells initialized to zero"). */
pmp_status pmp_zero_buffer(pmp_ctx *ctx, pmp_mesh *buffer);

/* Particle side of Step 1: the per-particle quantities the deposition
 * function needs, summed over the particle's kernel cells in a fixed order
 * (z slowest, x fastest): M_snr, V_snr, v_COM, n_H, R_M and |p_radial| for
 * feedback (Sec. 3.2.1); rho_inf, v_inf, c_inf, r_BH -> mdot_BH (Eq. mdot),
 * r_acc and sum w (Eq. kernel, Eq. kernel_wgt) for sinks (Sec. 3.1.1).
 * gathered: device, [rows][count]; particles outside the box get zero rows
 * and set PMP_ERR_PARTICLE_OUTSIDE.
 * Also records the pass's plan in `workspace` (device, 256-byte aligned, at
 * least pmp_workspace_size bytes for `mode`): each particle's kernel cells
 * with their covered fractions, and for sinks the per-cell quantities of the
 * state.  The plan stays valid until the particles' positions or the state
 * change or pmp_gather runs again with this context. */
pmp_status pmp_gather(pmp_ctx *ctx, const pmp_mesh *state, const pmp_particles *particles, double *gathered,
                      int32_t mode, void *workspace, size_t workspace_bytes);

/* Step 1 (Eq. delta_u_buf): every particle adds its deposition function
 * Delta U^s (Eq. du for feedback; Eq. accretion_function for sinks, the
 * removal entering with a minus sign) to every kernel cell of the buffer,
 * ghost zones included, on top of what the buffer holds.  `workspace` must
 * hold the plan of the preceding pmp_gather on these particles with the same
 * `mode` (else PMP_ERR_WORKSPACE).  ATOMIC uses FP64 atomics; SORTED
 * synchronises the stream once to read the pair count; ROUNDED zeroes its
 * error bound, adds with atomics and then rounds every buffer value, so the
 * buffer should start from zero (pmp_zero_buffer).  Kernel cells with
 * omega = 0 receive nothing. */
pmp_status pmp_deposit(pmp_ctx *ctx, const pmp_mesh *state, const pmp_particles *particles, const double *gathered,
                       pmp_mesh *buffer, int32_t mode, void *workspace, size_t workspace_bytes);

/* pmp_gather followed by pmp_deposit (same arguments, same results: the
 * gathered rows, the plan in `workspace` and Step 1 into `buffer`).  For
 * sinks in the ATOMIC mode plan, gather and deposit run as one kernel: a
 * warp plans, gathers and deposits 32 consecutive sinks before it takes the
 * next, so the FP64 work of gather and deposit overlaps the plan's integer
 * work and the deposit re-reads cells the gather has just read (the
 * per-cell records are written first, the scratch is spread after).  The
 * buffer sums then differ from those of the two separate calls only by the
 * order of the atomic additions.  Other kinds and modes run the two calls
 * one after the other. */
pmp_status pmp_gather_deposit(pmp_ctx *ctx, const pmp_mesh *state, const pmp_particles *particles, double *gathered,
                              pmp_mesh *buffer, int32_t mode, void *workspace, size_t workspace_bytes);

/* Step 2 on one GPU (Sec. 2.2, Step 2): each ghost cell of the buffer is added
 * to the valid cell that owns it (periodic axes only); a valid cell with
 * several images sums them in the fixed order of App. A.2 taken as the
 * lexicographic order of the image offset (oz, oy, ox) in {-1,0,1}^3:
 * ((B_c + B_img1) + B_img2) + ...  Ghost cells are left as they were.
 * Needs ng <= n on every periodic axis. */
pmp_status pmp_fold_ghosts(pmp_ctx *ctx, pmp_mesh *buffer);

/* Steps 3-5 (Sec. 2.2): the cell-wise limiter eta = f_lim(U, Delta U^sum)/
 * Delta U^sum, then for sinks Step 4 -- u_s := u_s - sum_c eta_c Delta U^s_c V,
 * with Delta U^s recomputed and eta of a ghost image taken from its owner --
 * and finally Step 5, U := U + eta Delta U^sum on every valid cell.
 * Feedback: the momentum limiter of Eq. lambda, eta = (1, l, l, l, 1);
 *   `particles` and `gathered` may be NULL (Step 4 is skipped, Sec. 3.2.1).
 * Sink: the accretion limiter of Sec. 3.1.1 with the 25% cap (params.cap),
 *   the Truelove floor and the density floor rho_min; the same eta for all
 *   fields; `particles`/`gathered` are those of pmp_gather.
 * eta_out: optional device array, one FP64 per valid cell (x fastest): the
 *   momentum eta (feedback) or the common eta (sink).
 * workspace: sinks need the one pmp_gather filled for this pass (its plan and
 *   per-cell quantities).  Feedback does not read it (NULL is accepted): one
 *   pass over the cells settles most of them with an FP32 pre-test of the
 *   constraint and runs the FP64 limiter on the rest, with the same results
 *   as the FP64 limiter on every cell.
 * Order of work (sinks): eta is computed and the state updated in one pass
 *   over the cells, then Step 4 runs; Step 4 reads eta and the pre-update
 *   per-cell quantities kept in the workspace, so the result is that of the
 *   order the paper states (Step 4 before Step 5).  Step 4 sums a sink's
 *   kernel cells in canonical order, except after pmp_gather_deposit in the
 *   ATOMIC mode: that deposit stores each pair's removal a in the workspace,
 *   and Step 4 adds eta a over the cells in an order of its own (32 partial
 *   sums per sink, then their sum), like the ATOMIC buffer sums. */
pmp_status pmp_apply_limited(pmp_ctx *ctx, pmp_mesh *state, const pmp_mesh *buffer, pmp_particles *particles,
                             const double *gathered, double *eta_out, void *workspace, size_t workspace_bytes);

/* Adjoint of one feedback pass (gather, deposit, fold, limited apply) with
 * respect to the particle inputs, for a loss L whose gradient with respect to
 * the updated state is gU (device, a [5][field_stride] array laid out like
 * the state; ghosts ignored).  The limited apply is differentiated with eta
 * held fixed, and cells where the limiter is active (eta < 1) pass no
 * gradient.  The kernel cell set and omega are piecewise constant in
 * position and contribute no derivative.  Weights are recomputed, not
 * stored.  g_out: device [8][count] = dL/d(m, e, px, py, pz, x, y, z).
 * `state_in` is the state BEFORE the apply; `buffer` the folded buffer;
 * `gathered` and `workspace` from the pass's pmp_gather.  Feedback contexts
 * only. */
pmp_status pmp_backward(pmp_ctx *ctx, const pmp_mesh *state_in, const pmp_mesh *buffer, const pmp_particles *particles,
                        const double *gathered, const double *gU, double *g_out, void *workspace,
                        size_t workspace_bytes);

/* Auxiliary conserved fields under accretion (Sec. 3.1.1, the extensions
 * beyond minimal hydrodynamics): the dual-energy internal energy density and
 * species (passive scalar) densities change at fixed specific value, as the
 * paper prescribes (internal energy per unit mass in place of e_sp + v^2/2;
 * Delta rho_sp = (rho_sp / rho) Delta rho).  Every pair's change of a field X
 * is -a X/rho with the cell's X/rho, so the summed change is
 * (X/rho) Delta rho^sum and the limited update is
 *   X := X + eta ((X / rho) Delta rho^sum)
 * with eta the cell's accretion limiter; X/rho is thus kept, to rounding.
 * For a SINK context, after pmp_fold_ghosts and BEFORE pmp_apply_limited of
 * the same pass (rho must be the pre-update density).  extra: device,
 * n_extra fields of extra_stride doubles each, laid out like the state's
 * cells (only valid cells are read or written). */
pmp_status pmp_apply_extra(pmp_ctx *ctx, const pmp_mesh *state, const pmp_mesh *buffer, double *extra, int32_t n_extra,
                           int64_t extra_stride);

/* Sink creation (Sec. 3.1.2), for a SINK context after its accretion pass,
 * with that pass's summed buffer retained (Sec. 3.1, item 2).  A valid cell
 * becomes a new sink when (a) rho > rho_Tr (Eq. truelove with the cell's own
 * c_s), (b) rho is strictly larger than at every other cell whose centre
 * lies within r_K (periodic images on periodic axes), and (c) the buffer is
 * zero in every field at the cell, i.e. no sink's kernel reaches it (the
 * paper's way of keeping new sinks out of r_K of existing ones).  All three
 * are tested on the state as it was before any creation.  The qualifying
 * cells, in cell order (z slowest, x fastest), give sinks 0, 1, ...: at the
 * cell centre, with m_s = (rho - rho_Tr) V and p_s = m_s v (v = p / rho of
 * the cell); the cell keeps its velocity and specific energy: rho := rho_Tr,
 * p := rho_Tr v, E := rho_Tr E / rho.
 * x..pz: device arrays of `capacity` entries receiving the new sinks; only
 * the first `capacity` qualifying cells are created, the others are left
 * as they are.  *count (device int64) receives the number of qualifying
 * cells.  workspace: device, 256-byte aligned, at least
 * pmp_create_sinks_workspace_size bytes.  Enqueued on the context's stream. */
pmp_status pmp_create_sinks_workspace_size(const pmp_ctx *ctx, const pmp_mesh *state, size_t *bytes);
pmp_status pmp_create_sinks(pmp_ctx *ctx, pmp_mesh *state, const pmp_mesh *buffer, int64_t capacity, double *x,
                            double *y, double *z, double *m, double *px, double *py, double *pz, int64_t *count,
                            void *workspace, size_t workspace_bytes);

/* Synchronises the context's stream, then returns the first device error
 * since the last call (PMP_OK if none) in *code and the index of the
 * offending particle or cell in *index (-1 if none), and clears them. */
pmp_status pmp_get_error(pmp_ctx *ctx, int32_t *code, int64_t *index);

/* Synchronises the stream and reads the counters of the last
 * pmp_apply_limited (host array of 2): cells with eta < 1, and feedback cells
 * for which Eq. lambda had no root in [0, 1] (lambda set to 0). */
pmp_status pmp_limiter_counts(pmp_ctx *ctx, int64_t *counts);

/* Per-kernel timing.  When enabled, every kernel the context launches is
 * bracketed by two CUDA events recorded on the context's stream.
 * pmp_timing_read synchronises the stream, sums the bracketed durations per
 * kernel name into `out` (host array of `max` entries; *n receives the number
 * of distinct names, which may exceed max), and forgets the recorded events. */
typedef struct {
    char name[24];    /* e.g. "plan", "gather", "deposit", "fold", "apply" */
    int64_t launches; /* launches summed */
    double ms;        /* total duration, milliseconds */
} pmp_kernel_time;

pmp_status pmp_timing_enable(pmp_ctx *ctx, int32_t on);
pmp_status pmp_timing_read(pmp_ctx *ctx, pmp_kernel_time *out, int32_t max, int32_t *n);

/* ------------------------------------------------------------------------ */
/* Batched form: one pass over many uneven patches of one level             */
/* ------------------------------------------------------------------------ */

/* The patches of a batch tile a periodic domain as a rectilinear grid (every
 * patch in a row of the grid has the row's extent across it), like the boxes
 * of one AMR level in the paper's distributed setting (Sec. 2.2, Step 2).
 * Each patch keeps its state and buffer, laid out like a pmp_mesh with the
 * batch's ng, at `offset` of two caller-owned device arenas.  Its ghost cells
 * are never filled by the caller: the state's are read from the neighbour
 * patches, and the buffer's are summed into the neighbours' valid cells.
 *
 * neighbour[t]: the patch displaced by the t-th offset o = (ox, oy, oz) of
 * {-1,0,1}^3 without (0,0,0), listed with oz slowest and ox fastest.  A
 * ghost cell (i, j, k) of patch p is the valid cell of q = neighbour[o] at
 * i + n_q (i < 0), i - n_p (i >= n_p), i (otherwise), likewise j and k, with
 * o_a the sign of each case.  The summed buffer of a valid cell is
 * ((B_c + B_img1) + B_img2) + ... over its ghost images in lexicographic
 * order of the image offset (oz, oy, ox) (App. A.2); the image at offset o
 * lies in neighbour[-o]. */
typedef struct pmp_batch pmp_batch;

typedef struct {
    int32_t n[3];          /* valid cells per axis, >= ng */
    int32_t neighbour[26]; /* patch index per offset, see above */
    int64_t offset;        /* arena index of (field 0, padded cell 0) */
    int64_t field_stride;  /* doubles between fields, >= padded cell count */
} pmp_patch;

/* How pmp_cycle_batched runs a pass.
 * PERSISTENT: one cooperative launch of (SMs x resident blocks) blocks that
 *   take work items from a queue per phase, with a grid-wide barrier between
 *   phases whose waits end with PMP_ERR_TIMEOUT after a few seconds.
 * PER_PATCH:  every phase launched once per patch (the plain form).
 * GRAPH:      PERSISTENT captured once into a CUDA graph (per set of argument
 *   pointers) and replayed; the first call captures on the context's stream,
 *   which must not be capturing already. */
typedef enum { PMP_BATCH_PERSISTENT = 0, PMP_BATCH_PER_PATCH = 1, PMP_BATCH_GRAPH = 2 } pmp_batch_launch;

/* Step-1 strategy of a patch.
 * OWNER_CUBE, OWNER_ROWS: each buffer cell of the patch (ghosts included) is
 *   written once, as the sum of the patch's particles' contributions in
 *   particle-index order; tiles of 8 x 8 x 8 cells, or of full padded rows x
 *   8 x 4.  Deterministic: bit-for-bit the sum of the sorted mode.
 * ATOMIC: the patch's buffer is zeroed, then FP64 atomic additions. */
typedef enum {
    PMP_STRATEGY_OWNER_CUBE = 0,
    PMP_STRATEGY_OWNER_ROWS = 1,
    PMP_STRATEGY_ATOMIC = 2
} pmp_strategy;

/* Autotuner bins: 4 patch-size bins (padded cells < 16384, < 65536,
 * < 262144, larger) x 5 occupancy bins (no particles; particles per 1000
 * valid cells < 1, < 10, < 100, larger); bin = size * 5 + occupancy. */
#define PMP_BATCH_BINS 20

/* Creates a batch of n_patches patches (host array `patches`) with ng ghost
 * cells and cell size dx for the context's interaction kind, in arenas of
 * arena_len doubles.  Checks: ng >= ceil(r_K) (else PMP_ERR_GHOST_TOO_THIN);
 * every n >= ng; every patch inside the arena and disjoint from the others;
 * neighbour entries in range, of matching extent across their offset, and
 * reciprocal (the neighbour at -o of the neighbour at o is the patch).
 * Allocates the batch's device tables; synchronous.  Particle ranges start
 * empty; the strategy starts as OWNER_CUBE for every patch. */
pmp_status pmp_batch_create(pmp_ctx *ctx, const pmp_patch *patches, int32_t n_patches, int32_t ng, double dx,
                            int64_t arena_len, pmp_batch **out);

/* Particle ranges: host array first[n_patches + 1], first[0] = 0,
 * non-decreasing; patch p owns particles [first[p], first[p + 1]) of the
 * particle arrays handed to pmp_cycle_batched, positions in that patch's
 * cell units (0 <= x < n[0], likewise y, z).  Synchronises the context's
 * stream; (re)allocates the per-particle tables. */
pmp_status pmp_batch_set_particles(pmp_batch *batch, const int64_t *first);

/* Sets one pmp_strategy for every patch (synchronises the stream). */
pmp_status pmp_batch_set_strategy(pmp_batch *batch, int32_t strategy);

/* Copies the strategy of every patch into per_patch (host, n_patches). */
pmp_status pmp_batch_strategies(const pmp_batch *batch, int32_t *per_patch);

/* Autotuner: for each bin holding patches, times the Step-1 deposit of those
 * patches with every allowed strategy (OWNER_CUBE and OWNER_ROWS; ATOMIC too
 * unless `deterministic`), best of `reps` runs, and keeps the fastest for the
 * bin.  Runs the gather first; writes `gathered` and garbage into `buffer`;
 * leaves `state` and the particles unchanged.  bin_choice (host, optional,
 * PMP_BATCH_BINS entries) receives the chosen strategy per bin, -1 for empty
 * bins.  Synchronous. */
pmp_status pmp_batch_autotune(pmp_batch *batch, const double *state, double *buffer, pmp_particles *particles,
                              double *gathered, int32_t deterministic, int32_t reps, int32_t *bin_choice);

/* One pass (Steps 1-5 of Sec. 2.2; Step 4 for sinks) over every patch of the
 * batch: gather, deposit into `buffer` (every padded cell of every patch is
 * written), ghost summation across patches, limiter and update of the valid
 * cells of `state`.  Afterwards `buffer` holds the deposits in ghost cells
 * and the summed Delta U in valid cells, as the single-box calls leave it.
 * particles: count = first[n_patches]; gathered: [rows][count]; eta_out
 * (optional) one FP64 per valid cell, patch after patch, x fastest.  The
 * limiter counters (pmp_limiter_counts) and device errors (pmp_get_error)
 * are the context's.  `launch` is a pmp_batch_launch.  Enqueues on the
 * context's stream (GRAPH: captures on the first call). */
pmp_status pmp_cycle_batched(pmp_batch *batch, double *state, double *buffer, pmp_particles *particles,
                             double *gathered, double *eta_out, int32_t launch);

/* Persistent grid size (blocks) and item counts (host int64[3]: zeroing,
 * deposit, apply items) of the batch's current plan. */
pmp_status pmp_batch_info(const pmp_batch *batch, int32_t *grid, int64_t *items);

/* Fault injection for tests (no paper counterpart): the grid barriers of the
 * persistent launch (PMP_LAUNCH_PERSISTENT and PMP_LAUNCH_GRAPH) wait for
 * `arrivals` more blocks than the grid has, which never arrive.  Each wait is
 * bounded in time, so the pass ends after about 4 s: the waiting blocks set
 * PMP_ERR_TIMEOUT (first index -1, read with pmp_get_error) and the abort
 * word, every block returns, and the context stays usable.  0, the default,
 * restores normal operation.  arrivals must be 0 or 1 (else PMP_ERR_ARG).
 * Synchronises the context's stream; drops a captured graph. */
pmp_status pmp_batch_hold_barriers(pmp_batch *batch, int32_t arrivals);

/* Frees a batch's device tables (after its work has finished). */
void pmp_batch_destroy(pmp_batch *batch);

/* ------------------------------------------------------------------------ */
/* The batched form on several ranks (Sec. 2.2, Step 2 across ranks)        */
/* ------------------------------------------------------------------------ */

/* Assigns the patches of one level to n_ranks ranks along a space-filling
 * curve (Sec. 2.2 distributes boxes this way): patches ordered by the Morton
 * (Z-order) code of pos[p] (host, [n][3], each 0 <= v < 2^20: the patch's
 * place in the super-grid), ties by index, then cut into runs of consecutive
 * patches of about equal total cost (cost[p] >= 1, e.g. valid cells plus a
 * weight per particle); rank_of (host, n entries) receives the rank of each
 * patch.  Each cut falls at the patch boundary nearest to k / n_ranks of the
 * total cost; no rank is skipped, and with at least as many patches as ranks
 * every rank gets one (a patch costlier than a rank's share then moves the
 * later cuts along the curve).  Host only; PMP_ERR_ARG on a bad argument. */
pmp_status pmp_partition_sfc(int32_t n_patches, const int32_t *pos, const int64_t *cost, int32_t n_ranks,
                             int32_t *rank_of);

/* What one rank holds and exchanges in a pass.  Its local patches are its
 * owned patches (in global index order), one proxy per patch of another rank
 * that neighbours an owned patch (global index order), and one zero patch
 * (extents the largest of all patches) whose cells must stay zero.  A proxy
 * carries, each pass, the neighbour's valid state cells that lie in an owned
 * patch's ghost zone (exchange STATE, before the pass), the neighbour's
 * buffer ghost cells that lie on owned cells (GHOST, after Step 1: the images
 * App. A.2 adds, so the owned cells' sums have the one-rank order), and for
 * sinks the neighbour's folded sums next to owned patches (FOLDED, after
 * GHOST: Step 4 of an owned sink reads eta there).  Proxies and the zero patch
 * have the zero patch as every neighbour.  Local patches lie patch after
 * patch in a local arena, field strides rounded up to 32 doubles.
 * A region is a box of cells of one local patch, lo <= c < hi per axis in its
 * padded coordinates (-ng .. n + ng); a message to or from one peer is the
 * concatenation of its regions, each [5][volume] doubles (field slowest, x
 * fastest).  The messages of one exchange lie peer after peer (increasing
 * rank) in one buffer; `offset` is the region's first double there.  The
 * regions a rank sends to a peer are, in order, those the peer receives from
 * it.  pmp_plan_* is host code (no GPU needed). */
enum { PMP_XCH_STATE = 0, PMP_XCH_GHOST = 1, PMP_XCH_FOLDED = 2 };

typedef struct {
    int32_t peer;   /* the other rank */
    int32_t patch;  /* local patch index on this rank */
    int32_t lo[3], hi[3];
    int64_t offset; /* first double of the region in the exchange's buffer */
} pmp_region;

typedef struct pmp_plan pmp_plan;

/* Plan of rank `rank` for the global patches (neighbour tables as for
 * pmp_batch_create; offsets and strides ignored) with ng ghost cells and the
 * partition rank_of (host, n entries). */
pmp_status pmp_plan_create(const pmp_patch *patches, int32_t n_patches, int32_t ng, const int32_t *rank_of,
                           int32_t n_ranks, int32_t rank, pmp_plan **out);

/* The rank's local patches: counts, and (each optional, n_local entries) the
 * patches (extents, local neighbour table, local arena offsets and strides)
 * and their global indices (-1 for the zero patch); the local arena length. */
pmp_status pmp_plan_local(const pmp_plan *plan, int32_t *n_owned, int32_t *n_local, pmp_patch *local,
                          int32_t *global_id, int64_t *arena_len);

/* The regions of exchange `kind` that the rank sends (send = 1) or receives
 * (send = 0); *n receives their number, at most `max` are written to out. */
pmp_status pmp_plan_regions(const pmp_plan *plan, int32_t kind, int32_t send, pmp_region *out, int32_t max,
                            int32_t *n);

void pmp_plan_destroy(pmp_plan *plan);

/* A batch of a rank's local patches: patches [0, n_owned) are worked on (the
 * neighbour tables of these are checked as pmp_batch_create checks them,
 * except that a neighbour that is not owned need not list the patch back);
 * the others are proxies and the zero patch, only read.  Particles belong to
 * owned patches (pmp_batch_set_particles: empty ranges for the others). */
pmp_status pmp_batch_create_partial(pmp_ctx *ctx, const pmp_patch *patches, int32_t n_patches, int32_t n_owned,
                                    int32_t ng, double dx, int64_t arena_len, pmp_batch **out);

/* Parts of pmp_cycle_batched, for a pass whose exchanges run between them:
 * PMP_BATCH_PART_DEPOSIT is Step 1 (gather and deposit), PMP_BATCH_PART_FINISH
 * Steps 2-5 (the ghost sum, Step 4 for sinks, limiter and update).  Between
 * the two the caller unpacks the GHOST (and for sinks FOLDED) exchanges into
 * the buffer.  launch: PERSISTENT or PER_PATCH (PMP_ERR_ARG for GRAPH).
 * Arguments and results otherwise as pmp_cycle_batched, for owned patches. */
enum { PMP_BATCH_PART_ALL = 0, PMP_BATCH_PART_DEPOSIT = 1, PMP_BATCH_PART_FINISH = 2 };
pmp_status pmp_cycle_batched_part(pmp_batch *batch, double *state, double *buffer, pmp_particles *particles,
                                  double *gathered, double *eta_out, int32_t launch, int32_t part);

/* Region lists on the device for packing and unpacking (slot 0..5, a list per
 * slot; allocates device memory, synchronises the context's stream).  The
 * regions' patches are local patches of the batch. */
pmp_status pmp_batch_set_regions(pmp_batch *batch, int32_t slot, const pmp_region *regions, int32_t n);

/* Packs the slot's regions of `arena` (a state or buffer arena of the batch)
 * into msg (device, indexed by the regions' offsets).  folded = 1 packs the
 * folded sums (App. A.2 order, as Step 2 forms them) of the buffer `arena`
 * at valid cells of owned patches instead of the stored values.  Enqueued on
 * the context's stream. */
pmp_status pmp_batch_pack(pmp_batch *batch, int32_t slot, const double *arena, double *msg, int32_t folded);

/* Writes the slot's regions of msg into `arena`.  Enqueued on the context's
 * stream. */
pmp_status pmp_batch_unpack(pmp_batch *batch, int32_t slot, const double *msg, double *arena);

/* Size of the fixed device scratch of pmp_deposit_noalloc: 64 MiB, held on
 * every GPU that loads the library until the process exits. */
#define PMP_NOALLOC_SCRATCH_BYTES (64u << 20)

/* Step 1 for supernova feedback without any device allocation.  The paper
 * has no counterpart; this entry point exists for callers that cannot call
 * cudaMalloc (code running inside another framework's memory pool, plugins
 * handed only pre-allocated buffers, processes whose device footprint must
 * not grow after start-up).  It does what pmp_gather + pmp_deposit (ATOMIC)
 * do with a feedback context -- `gathered` receives the 12 feedback rows and
 * `buffer` accumulates the deposit on top of what it holds -- but it takes no
 * context and no workspace: its plan lives in a static device array of
 * PMP_NOALLOC_SCRATCH_BYTES compiled into the library.  That limits the
 * particle count to about 99,000 at r_K = 2 (each particle needs 28 + 8 C
 * bytes, C the kernel-cell bound: 81 at r_K = 2, 461 at r_K = 4); larger
 * counts return PMP_ERR_WORKSPACE and enqueue nothing.  params->kind must be
 * PMP_KIND_FEEDBACK.  The meshes are checked as pmp_deposit checks them
 * (PMP_ERR_ARG for a misaligned or NULL data pointer, a periodic flag other
 * than 0 or 1, a non-finite dx, meshes of different boxes, or a state that
 * overlaps the buffer; PMP_ERR_GHOST_TOO_THIN for buffer ng < ceil(r_K)).
 * Every call looks up the scratch's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing), so a call after a device
 * reset or on another device uses that device's copy; make the first call
 * on a device before any stream capture.  Every call shares the one scratch array, which
 * keeps the last call's contents: calls whose work overlaps on the GPU (two
 * streams, or two threads) race and corrupt each other; serialise them.
 * Particles outside the box are skipped; no device errors are reported (there
 * is no context to hold them).  Calls no cudaMalloc, cudaFree or allocating
 * library routine; enqueues on `stream` and returns. */
pmp_status pmp_deposit_noalloc(const pmp_params *params, const pmp_mesh *state, const pmp_particles *particles,
                               double *gathered, pmp_mesh *buffer, pmp_stream stream);

/* ------------------------------------------------------------------------ */
/* Measurement kernels (no paper counterpart)                               */
/* ------------------------------------------------------------------------ */

/* The peaks the particle kernels are measured against, taken on the GPU the
 * library runs on.  Both enqueue one launch on `stream` and return; the
 * caller times it (CUDA events on that stream).
 * pmp_probe_fp64: `blocks` blocks of pmp_probe_threads() threads, each running
 *   pmp_probe_chains() independent chains of `iters` FP64 fused multiply-adds
 *   (2 flops each); out (device) receives one double per thread, so it needs
 *   blocks * pmp_probe_threads() entries.
 * pmp_probe_atomic: n_adds FP64 atomicAdd of 1.0 spread over n_targets
 *   doubles of `target` (device), addition t to index (t * 2654435761) mod
 *   n_targets; grid-stride over `blocks` blocks.
 * PMP_ERR_ARG for NULL pointers or non-positive sizes. */
int32_t pmp_probe_threads(void);
int32_t pmp_probe_chains(void);
pmp_status pmp_probe_fp64(double *out, int32_t blocks, int32_t iters, pmp_stream stream);
pmp_status pmp_probe_atomic(double *target, int64_t n_targets, int64_t n_adds, int32_t blocks, pmp_stream stream);

/* The library's correctly rounded FP64 quotient and square root, computed
 * from integer and FP32 instructions by digit recurrence (no paper
 * counterpart: the kernels use them for the divisions and square roots of the
 * formulas of Sec. 3.1-3.2, whose results they equal bit for bit).  For
 * i < n: quot[i] = a[i] / b[i] and root[i] = sqrt(a[i]), rounded to nearest
 * even as IEEE 754 binary64 prescribes (zero, subnormal, infinite and NaN
 * operands included).  All four arrays are device memory of n doubles, owned
 * by the caller; one launch is enqueued on `stream`.  PMP_ERR_ARG for n < 0 or
 * a NULL array with n > 0; PMP_ERR_CUDA if the launch fails. */
pmp_status pmp_exact_math(const double *a, const double *b, int64_t n, double *quot, double *root,
                          pmp_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* PMP_H */
