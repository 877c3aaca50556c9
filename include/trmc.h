/*
 * trmc.h -- C ABI of libtrmc, a GB300 (sm_103a) implementation of the
 * collision step of the recursive Time Relaxed Monte Carlo method (TRMC-R)
 * together with the free transport and the cell sort around it.
 *
 * Paper: S. Trazzi, L. Pareschi, B. Wennberg, "Adaptive and Recursive Time
 * Relaxed Monte Carlo methods for rarefied gas dynamics", arXiv:1009.2768.
 *
 * Conventions shared by every entry point
 *  - Pointers named *_dev and every pointer inside trmc_state are CUDA device
 *    pointers owned by the caller; the library never frees them.  Other
 *    pointers are host pointers, read before the call returns.
 *  - Every call is asynchronous on the given stream (a cudaStream_t passed as
 *    void*, NULL = legacy default stream) and returns a trmc_status.  Argument
 *    errors are found on the host and returned at once with nothing launched.
 *  - Errors found by a kernel (a cell larger than the workspace, a particle
 *    that moved more than one cell in a transport step) set a device status
 *    word; trmc_check() reads it (synchronising the stream) and clears it.
 *  - One trmc_ctx per host thread; a context holds the library's workspace
 *    (device scratch) and must not be used by two streams at once.
 *  - Particle arrays are structure-of-arrays, sorted by cell: cell c owns the
 *    particles [cell_start[c], cell_start[c+1]).  They are double in
 *    TRMC_FP64 contexts and float in TRMC_FP32_MIXED contexts.
 *  - Results depend only on (seed, problem id, cell index within the problem,
 *    step, particle order within the cell), never on launch shape or on
 *    which other cells share the call: every per-cell sum runs over the same
 *    256 virtual lanes and 8 virtual warps, combined in a fixed tree, whatever
 *    the CTA size, so even the rounding of the FP64 sums is the same.
 */
#ifndef TRMC_H
#define TRMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum trmc_status {
    TRMC_OK = 0,
    TRMC_ERR_ARG = 1,       /* invalid argument (found on the host)            */
    TRMC_ERR_CUDA = 2,      /* a CUDA call failed                              */
    TRMC_ERR_NOMEM = 3,     /* device allocation failed                        */
    TRMC_ERR_CAPACITY = 4,  /* a cell did not fit in the workspace             */
    TRMC_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up              */
    TRMC_ERR_STATE = 6      /* state inconsistent (e.g. particle moved > 1 cell) */
} trmc_status;

typedef enum trmc_precision {
    TRMC_FP64 = 0,          /* velocities and all arithmetic in double          */
    TRMC_FP32_MIXED = 1     /* float velocities and collisions; moments, bounds,
                               level probabilities and the renormalisation in double */
} trmc_precision;

/* Tree truncation (Sec. 4.1 fixed order m, Sec. 4.3 adaptive TRMC-RAD,
 * Sec. 4.4 shape-dependent TRMC-WB). */
typedef enum trmc_trunc {
    TRMC_TRUNC_FIXED = 0,     /* m = params.m_fixed                              */
    TRMC_TRUNC_RAD = 1,       /* m per cell in state.m_max, adapted each step     */
    TRMC_TRUNC_UNLIMITED = 2, /* m = params.m_cap (depth limited only by N)       */
    TRMC_TRUNC_WB = 3         /* split to params.m_cap; an output whose collision tree has
                                 length L > params.m_fixed (= m_max) is resampled from the
                                 Maxwellian instead (Alg. 4.6), L per params.wb_length */
} trmc_trunc;

/* Length of a collision tree of k = j + h + 1 collisions (Sec. 4.4): Eq. def:1
 * L = k, Eq. def:2 L = 1 + min(L_j, L_h), Eq. def:3 L = 1 + (L_j + L_h) / 2,
 * with L = 0 for an original particle.  The trees are the ones the step's
 * plan builds; their lengths are known before any collision is performed. */
typedef enum trmc_length { TRMC_LEN_K = 1, TRMC_LEN_MIN = 2, TRMC_LEN_MEAN = 3 } trmc_length;

typedef enum trmc_indicator { TRMC_IND_PXX = 0, TRMC_IND_M4 = 1 } trmc_indicator;

typedef enum trmc_init_kind {
    TRMC_INIT_MAXWELL = 0,    /* Maxwellian M(rho,u,T), Eq. Max                     */
    TRMC_INIT_BIMAXWELL = 1,  /* T_par along x, T_perp along y and z                */
    TRMC_INIT_BKW = 2         /* BKW solution for Maxwell molecules, shape K        */
} trmc_init_kind;

#define TRMC_MCAP 64            /* deepest collision tree supported                 */
#define TRMC_INIT_COLS 9        /* kind, ux, uy, uz, T (or T_par), T_perp, K, x_lo, x_hi */
#define TRMC_MOM_COLS 10        /* N, rho, ux, uy, uz, T, P_xx, M_4, E, max|v|^2     */
#define TRMC_REPORT_LEN (16 + 3 * (TRMC_MCAP + 2))

/* Per-cell physical parameters (device array, optional).  rho_c = N_c * rho_scale. */
typedef struct trmc_cell_param {
    double eps;        /* Knudsen number, Eq. BE-r                          */
    double dt;         /* time step (written by trmc_transport in CFL mode)  */
    double rho_scale;  /* particle mass / cell volume                        */
    double alpha;      /* VHS exponent: B = |q|^alpha (0 Maxwell, 1 hard sphere) */
} trmc_cell_param;

/* The particle state.  All pointers are device pointers owned by the caller. */
typedef struct trmc_state {
    void *vx, *vy, *vz;           /* [capacity] velocities                        */
    void *x;                      /* [capacity] positions; NULL if space-homogeneous */
    void *vx_alt, *vy_alt, *vz_alt, *x_alt;  /* [capacity] sort targets (transport) */
    int64_t *cell_start;          /* [n_cells+1]                                  */
    int64_t *cell_start_alt;      /* [n_cells+1] sort target (transport)          */
    int32_t *m_max;               /* [n_cells] TRMC-RAD tree depth; NULL unless RAD */
    trmc_cell_param *cell_param;  /* [n_cells] or NULL (then the params scalars)   */
    const uint64_t *cell_key;     /* [n_cells] (problem << 32 | cell in problem) or NULL */
    double *cell_vmax2;           /* [n_cells] max |v|^2 after the last collide, or NULL */
    uint64_t *step_dev;           /* NULL, or a device step counter: trmc_collide then keys its
                                     draws with *step_dev (ignoring its step argument) and adds 1 to
                                     it when done, so a captured CUDA graph advances on replay */
    int32_t *cell_order;          /* [n_cells] or NULL: the order in which cells are handed to
                                     CTAs (e.g. largest first); results do not depend on it.  With
                                     cell_cost also set, trmc_collide rewrites it before each launch:
                                     longest cells first, by the times the previous launch measured */
    double *cell_carry;           /* [n_cells][4] or NULL: momentum (3) and sum |v|^2 that rounding
                                     the thermalised velocities to the storage precision left over;
                                     the next step's renormalisation target adds it back, so
                                     sum(stored) + carry is conserved to FP64 round-off */
    uint32_t *cell_cost;          /* [n_cells] or NULL: trmc_collide writes the time each cell took
                                     (SM clock cycles / 16, saturated); start it at zero */
    int64_t capacity;             /* length of each particle array                */
    int32_t n_cells;
    uint32_t problem_id;          /* used when cell_key is NULL                   */
} trmc_state;

/* Collision-step parameters (host struct, read at call time). */
typedef struct trmc_collide_params {
    double dt, eps, alpha, rho_scale;  /* for cells without a trmc_cell_param      */
    double delta1, delta2;             /* TRMC-RAD thresholds (Sec. 4.3)            */
    int32_t trunc;                     /* trmc_trunc                                */
    int32_t m_fixed;                   /* order for TRMC_TRUNC_FIXED; m_max >= 0 for TRMC_TRUNC_WB */
    int32_t m_min, m_cap;              /* TRMC-RAD bounds, 1 <= m_min <= m_cap <= TRMC_MCAP */
    int32_t indicator;                 /* trmc_indicator for TRMC-RAD               */
    int32_t wb_length;                 /* trmc_length for TRMC_TRUNC_WB, else 0       */
} trmc_collide_params;

typedef enum trmc_bc {
    TRMC_BC_SPECULAR = 0,   /* both ends are specular walls: x -> 2 x_wall - x, v_x -> -v_x          */
    TRMC_BC_RESERVOIR = 1   /* both ends are reservoirs (inflow / outflow), see trmc_transport      */
} trmc_bc;

/* One 1D problem for trmc_transport: cells [cell_begin, cell_begin+n_cells).
 * Specular walls: the n_cells cells of equal width cover [x_lo, x_hi].
 * Reservoirs: the first and the last cell are ghost cells just outside
 * [x_lo, x_hi) (one cell width each), the n_cells - 2 cells between cover
 * [x_lo, x_hi); res_lo / res_hi give the reservoir density, mean x velocity
 * and temperature beyond x_lo / x_hi, particle_mass the mass of one particle. */
typedef struct trmc_domain {
    int32_t cell_begin, n_cells;
    double x_lo, x_hi;
    int32_t bc;                       /* trmc_bc */
    int32_t reserved;                 /* must be 0 */
    double res_lo[3], res_hi[3];      /* reservoir (rho, u_x, T); unused for walls */
    double particle_mass;             /* unused for walls */
} trmc_domain;

/* Step statistics, accumulated with integer atomics (device struct, optional). */
typedef struct trmc_stats {
    unsigned long long collisions;   /* real binary collisions                       */
    unsigned long long dummy;        /* VHS dummy (rejected) collisions              */
    unsigned long long maxwell;      /* particles resampled from the Maxwellian       */
    unsigned long long exceed;       /* pairs with |q|^alpha above the bound Sigma    */
    unsigned long long passes;       /* TRMC-RAD passes (1 per cell without a redo)   */
    unsigned long long feas;         /* tree-depth reductions for lack of leaves      */
    unsigned long long cells;        /* cells processed                               */
    unsigned long long capacity_skips; /* cells skipped: larger than the workspace     */
    unsigned long long changed;      /* particles whose velocity was rewritten         */
    unsigned long long particles;    /* particles in the processed cells               */
    unsigned long long wb_rejected;  /* TRMC-WB: outputs resampled for a too-long tree  */
} trmc_stats;

typedef struct trmc_ctx trmc_ctx;

/* Create a context on the current CUDA device.  workspace_bytes sizes the
 * device scratch used by cells whose working set does not fit in shared
 * memory (0 = a default of 1 GiB).  seed keys every random draw. */
trmc_status trmc_create(trmc_ctx **out, int32_t precision, uint64_t seed, size_t workspace_bytes);
trmc_status trmc_destroy(trmc_ctx *ctx);
/* Text of the last error of this context (static storage, never NULL). */
const char *trmc_last_error(const trmc_ctx *ctx);
/* Synchronise the stream, then return and clear the device status word. */
trmc_status trmc_check(trmc_ctx *ctx, void *stream);

/* Launch shape of the collision kernel: CTA size (a multiple of 32 in
 * [32, 512]; above 256 every launch runs the kernel built for cells too large
 * for shared memory, which stages the others whole all the same) and the
 * number of CTAs resident per SM the shared-memory budget is split for
 * (1..16).  Defaults 128 and 4.  Results do not depend on it; only speed does
 * (the autotuner in the binding sweeps it). */
trmc_status trmc_set_collide_launch(trmc_ctx *ctx, int32_t threads, int32_t ctas_per_sm);

/* Work schedule of the collision kernel inside a cell.  The paper has no
 * counterpart (its trees run one collision at a time); results do not depend
 * on it, only speed does (the autotuner in the binding sweeps it).
 *  - warp_particles: a tree level of at most this many particles (two per
 *    collision) runs in one warp, with warp-level synchronisation only; the
 *    larger ones are spread over the CTA.  Even, in [2, 8192], or 0 for the
 *    default (64 in FP64 contexts, 256 in FP32-mixed ones).
 *  - records_per_thread: the input-independent part of every collision (its
 *    draw, threshold and direction, its input and product slots) is computed
 *    up front, by the whole CTA, for the levels of at most this many
 *    collisions per thread (and for every level one warp takes); a level then
 *    only loads, collides and stores.  In [1, 16], or 0 for the default (4); larger
 *    values need more shared memory per cell (32 B a collision in FP32-mixed
 *    contexts, 48 B in FP64), and a cell without room for them computes in
 *    place.
 * Returns TRMC_ERR_ARG for values outside those ranges. */
trmc_status trmc_set_collide_schedule(trmc_ctx *ctx, int32_t warp_particles, int32_t records_per_thread);

/* Launch shape of the transport's counting sort (the count and scatter
 * kernels, one CTA per old cell): threads per CTA, a multiple of 32 in
 * [32, 256], or 0 (the default) for a size picked from the mean cell size
 * (64 up to 1024 particles, 128 up to 4096, else 256).  The paper has no
 * counterpart; results do not depend on it (the sort is stable whatever the
 * CTA size), only speed does. */
trmc_status trmc_set_transport_launch(trmc_ctx *ctx, int32_t threads);

/* Sample initial velocities (and positions, if state->x != NULL) for every
 * particle of every cell, from the synthetic closed-form laws listed in
 * trmc_init_kind.  cell_init_dev: [n_cells][TRMC_INIT_COLS] doubles on the
 * device (kind, ux, uy, uz, T or T_par, T_perp, K, x_lo, x_hi).  Also fills
 * cell_vmax2 when present.  Draws use Philox tag INIT at step 0. */
trmc_status trmc_init_cells(trmc_ctx *ctx, trmc_state *state, const double *cell_init_dev, void *stream);

/* One homogeneous collision step in every cell (Sec. 3.1 splitting, Eq. WST,
 * Alg. 4.2-4.4, conservative Maxwellian resampling, TRMC-RAD of Sec. 4.3,
 * TRMC-WB of Sec. 4.4).
 * The cell's mass, momentum and energy are conserved to round-off.
 * step keys the random draws.  report_dev (optional) receives
 * [n_cells][TRMC_REPORT_LEN] int64 per-cell plan records; stats_dev
 * (optional) accumulates trmc_stats. */
trmc_status trmc_collide(trmc_ctx *ctx, trmc_state *state, const trmc_collide_params *params,
                         uint64_t step, int64_t *report_dev, trmc_stats *stats_dev, void *stream);

/* Free transport x += v_x dt, boundaries, then a stable regrouping of the
 * particles by cell (operator splitting, Sec. 3.1).  domains_dev:
 * [n_domains] trmc_domain on the device.  If cfl > 0, dt_dev[d] receives
 * cfl * dx / max|v| over domain d (from state->cell_vmax2, which must be
 * present) and, when state->cell_param is present, cell_param[c].dt is set
 * for every cell of the domain; otherwise dt_dev[d] is read.  Requires
 * dt * max|v_x| <= dx (a particle moves at most one cell).
 * Reservoir domains: particles that end outside [x_lo, x_hi) are deleted
 * (outflow, and ghost particles that did not enter); the survivors keep
 * their order; each ghost cell is then refilled with Iround(rho dx / mass)
 * particles of the reservoir's Maxwellian, uniform in the ghost cell
 * (Philox tag RESERVOIR, keyed by step).  The particle count changes: it is
 * state->cell_start[n_cells] on the device; a count above state->capacity
 * is reported as TRMC_ERR_CAPACITY by trmc_check (the overflow is dropped).
 * step keys the reservoir draws (ignored when state->step_dev is set).
 * The sorted particles land in the *_alt arrays and the state's pointers
 * are swapped, so on return state->vx etc. name the sorted arrays. */
trmc_status trmc_transport(trmc_ctx *ctx, trmc_state *state, const trmc_domain *domains_dev,
                           int32_t n_domains, double cfl, double *dt_dev, uint64_t step, void *stream);

/* Per-cell moments [n_cells][TRMC_MOM_COLS] doubles on the device:
 * N, rho = N rho_scale, u (3), T, P_xx, M_4 = <|v|^4>, E = <|v|^2>/2, max |v|^2
 * (Sec. 2 and Sec. 5.1 definitions, per unit mass). */
trmc_status trmc_moments(trmc_ctx *ctx, const trmc_state *state, double *out_dev, void *stream);

/* ---- a collision step that allocates nothing -----------------------------
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory at the point where they advance the gas, such as an
 * application running the step where cudaMalloc is forbidden or would
 * synchronise the device, or a plug-in that is handed particle arrays but no
 * allocator.  trmc_collide_static computes exactly what trmc_collide computes
 * (same kernel, same draws), needs no trmc_ctx, and calls no cudaMalloc,
 * cudaFree or other allocating routine.  Its scratch is one file-scope device
 * array of TRMC_STATIC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits.
 *  - max_cell_particles: the caller's bound on the largest cell.  The scratch
 *    is split into one overflow slab per CTA sized for such a cell; if not
 *    even one slab fits, the call returns TRMC_ERR_CAPACITY and launches
 *    nothing.  A cell that still does not fit (larger than the bound) is left
 *    unchanged and reported through status_dev as (TRMC_ERR_CAPACITY, cell).
 *  - The parameters are checked exactly as trmc_collide checks them
 *    (TRMC_ERR_ARG for the same invalid states and parameters).
 *  - status_dev (optional, device int[2]): receives device-detected errors
 *    (code, first cell), as trmc_check() would report them; the caller clears it.
 *    Without it the call cannot report device-detected errors at all: they go
 *    to the scratch's own status word, which the next call clears unread.
 *  - The first call on a device looks up the scratch's device address and
 *    sets the kernel's shared-memory limit; make that first call before any
 *    stream capture.
 *  - All calls share the scratch: calls that overlap on the GPU (different
 *    streams, or two host threads) race and must not be issued.
 *  - Every call clears the scratch's status word and work counter first. */
#define TRMC_STATIC_SCRATCH_BYTES (32u << 20)
trmc_status trmc_collide_static(trmc_state *state, const trmc_collide_params *params, int32_t precision,
                                uint64_t seed, uint64_t step, int32_t max_cell_particles,
                                int *status_dev, void *stream);

/* ---- self-test of the FP64 angle and logarithm evaluations -----------------
 * The paper has no counterpart: a check of the library's own evaluations of
 * sin/cos(2 pi u) and ln u for the 53-bit uniforms of the draws (table plus
 * series, used by the collisions and the Maxwellian resampling of FP64
 * contexts) and of its square root, against CUDA's sincospi, log and sqrt.
 * For each 64-bit word w of words_dev[n] (device), out_dev[n][8] (device)
 * receives: sin, cos of 2 pi u (library), the same from sincospi, ln u'
 * (library) and log(u') from CUDA, sqrt(x) (library) and sqrt(x) from CUDA,
 * with u = (w >> 11) 2^-53, u' = ((w >> 11) + 1) 2^-53 and x the double with
 * the low 52 bits of w as fraction and 1 + (w >> 53) mod 2045 as biased
 * exponent.  Asynchronous on the stream; TRMC_ERR_ARG for a negative n or NULL
 * arrays. */
trmc_status trmc_fp64_selftest(const uint64_t *words_dev, int32_t n, double *out_dev, void *stream);

/* ---- self-test of the split's integer Iround --------------------------------
 * The paper has no counterpart: a check of the library's integer evaluation of
 * the split count of Alg. 4.2, Iround(q R) = floor(x) + [u < x - floor(x)] with
 * x = q R rounded as one FP64 multiply and u = K 2^-53, which the collision
 * step uses in place of FP64 arithmetic.  For i < n: q_dev[i] in [0, 1],
 * R_dev[i] in [1, 2^31), K_dev[i] < 2^53 (all device); out_dev[i] (device)
 * receives the count.  Asynchronous on the stream; TRMC_ERR_ARG for a
 * negative n or NULL arrays. */
trmc_status trmc_split_selftest(const double *q_dev, const int32_t *R_dev, const uint64_t *K_dev, int32_t n,
                                int32_t *out_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TRMC_H */
