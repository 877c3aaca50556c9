/*
 * trmc_oracle.h -- plain, slow FP64 CPU oracle of the recursive Time Relaxed
 * Monte Carlo (TRMC-R) collision step, the free transport and the cell sort.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against an independent, obviously correct statement of the method.  Only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no source with the CUDA library (its own Philox, its
 * own permutation, its own everything) and nothing in the product links it.
 *
 * Paper: S. Trazzi, L. Pareschi, B. Wennberg, "Adaptive and Recursive Time
 * Relaxed Monte Carlo methods for rarefied gas dynamics" (arXiv:1009.2768).
 * Each function cites the section / equation / algorithm it follows.  Where
 * the paper is silent or garbled, the reading taken is stated at the use.
 *
 * Parity status: every function here is pinned by tests under tests/
 * (test_oracle_*.py) against numpy's Philox, closed forms (BKW moments, the
 * truncated Wild-sum factors), exact conservation, brute-force enumeration
 * and the Maxwellian / Bird-like limits.
 */
#ifndef TRMC_ORACLE_H
#define TRMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MCAP 64          /* largest tree depth the oracle supports */

/* Philox counter tags (the fourth counter word carries step, pass and tag). */
enum { ORC_TAG_INIT = 1, ORC_TAG_SPLIT = 2, ORC_TAG_PARITY = 3, ORC_TAG_KSEL = 4,
       ORC_TAG_PERM0 = 5, ORC_TAG_PERMK = 6, ORC_TAG_COLL = 7, ORC_TAG_MAXW = 8,
       ORC_TAG_RESERVOIR = 9 };

/* --- random numbers (Salmon et al., SC'11, Philox4x64-10) --------------- */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
void orc_draw(uint64_t seed, uint64_t problem, uint64_t index, uint64_t aux,
              uint64_t cell, uint64_t step, uint32_t pass, uint32_t tag, uint64_t out[4]);
double orc_u01(uint64_t w);         /* [0,1), 53 bits        */
double orc_u01_open(uint64_t w);    /* (0,1], 53 bits        */
uint32_t orc_below(uint64_t w, uint32_t n);   /* integer in [0,n) */

/* --- pseudo-random permutation of [0,n): key order (n <= 32), else an
 *     alternating Feistel network (8 or 6 rounds) on 2^b >= n with cycle
 *     walking ---------------------------------------------------------------- */
typedef struct { uint64_t n; int b; uint64_t key[4]; } orc_prp;
void orc_prp_init(orc_prp *p, uint64_t n, const uint64_t key[4]);
uint64_t orc_prp_fwd(const orc_prp *p, uint64_t x);
uint64_t orc_prp_inv(const orc_prp *p, uint64_t y);
void orc_prp_tables(uint64_t n, const uint64_t *keys, int64_t K, int32_t *out);

/* --- collision step ------------------------------------------------------ */
enum { ORC_TRUNC_FIXED = 0, ORC_TRUNC_RAD = 1, ORC_TRUNC_UNLIMITED = 2, ORC_TRUNC_WB = 3 };
/* Tree-length definitions of Sec. 4.4: Eq. def:1 (L = k), def:2 (1 + min), def:3 (1 + mean). */
enum { ORC_LEN_K = 1, ORC_LEN_MIN = 2, ORC_LEN_MEAN = 3 };
enum { ORC_IND_PXX = 0, ORC_IND_M4 = 1 };

typedef struct {
    double dt, eps, alpha, rho_scale;   /* rho_c = N_c * rho_scale */
    double delta1, delta2;              /* adaptive thresholds (Sec. 4.3) */
    int32_t trunc, m_fixed, m_min, m_cap, indicator;
    int32_t wb_length;                  /* TRMC-WB: ORC_LEN_*; m_fixed is then m_max */
    uint64_t seed;
} orc_collide_params;

typedef struct { double eps, dt, rho_scale, alpha; } orc_cell_param;

/* Per-cell report, int64 fields in this order (the CUDA library fills a
 * record of the same layout so the two can be compared field by field). */
enum {
    ORC_R_N = 0, ORC_R_PASSES, ORC_R_MFIRST, ORC_R_MLAST, ORC_R_MNEXT, ORC_R_RFINAL,
    ORC_R_N0, ORC_R_LEAVES, ORC_R_COLL, ORC_R_DUMMY, ORC_R_EXCEED, ORC_R_FEAS,
    ORC_R_PDROP, ORC_R_PSURP, ORC_R_MEFF0, ORC_R_WBREJ,
    ORC_R_NK = 16,                    /* pass-0 split quotas N_0..N_{MCAP+1}   */
    ORC_R_CK = 16 + ORC_MCAP + 2,     /* pass-0 collisions per level C_0..C_MCAP+1 */
    ORC_R_DK = 16 + 2 * (ORC_MCAP + 2),
    ORC_R_LEN = 16 + 3 * (ORC_MCAP + 2)
};

/* Length of one collision tree given as the list `path` of Algorithm 4.5:
 * path[0] = k, then for every node with k > 0, in pre-order, the sizes (j, h)
 * of its two subtrees (j + h = k - 1).  def is ORC_LEN_*.  Returns -1 if the
 * list is malformed. */
double orc_tree_length(const int32_t *path, int64_t len, int def);

/* One cell: v* are the cell's N particles (updated in place). */
int orc_collide_cell(double *vx, double *vy, double *vz, int64_t n,
                     uint64_t problem, uint64_t cell, uint64_t step,
                     int32_t *m_state, const orc_collide_params *prm,
                     const orc_cell_param *cp, int64_t *report);

/* All cells of a state; cell c holds [cell_start[c], cell_start[c+1]).
 * cell_key (nullable) gives (problem << 32 | local cell) per cell, else
 * (problem_id, c).  cell_param (nullable) overrides eps/dt/rho_scale/alpha. */
/* Returns 0, 1 for inconsistent parameters, 2 for a cell whose velocities or
 * energy sum are not finite. */
int orc_collide(double *vx, double *vy, double *vz, const int64_t *cell_start,
                int32_t n_cells, const uint64_t *cell_key, uint64_t problem_id,
                uint64_t step, int32_t *m_state, const orc_collide_params *prm,
                const orc_cell_param *cell_param, int64_t *reports, int n_threads);

/* --- transport + stable cell sort (operator splitting, Sec. 3.1) -------- */
enum { ORC_BC_SPECULAR = 0, ORC_BC_RESERVOIR = 1 };
typedef struct {
    int32_t cell_begin, n_cells;     /* cells [cell_begin, cell_begin+n_cells); with
                                        reservoirs the first and last are ghost cells */
    double x_lo, x_hi;               /* walls, or the reservoirs' faces               */
    int32_t bc, reserved;
    double res_lo[3], res_hi[3];     /* reservoir rho, u_x, T                         */
    double particle_mass;
} orc_domain;

/* Returns the new particle count, -1 if it would exceed capacity, or -2 for a
 * non-finite position, velocity or time step. */
int64_t orc_transport(double *x, double *vx, double *vy, double *vz,
                      int64_t *cell_start, int32_t n_cells_total,
                      const orc_domain *dom, int32_t n_dom, const double *dt_dom,
                      const uint64_t *cell_key, uint64_t problem_id, uint64_t seed, uint64_t step,
                      double *x_out, double *vx_out, double *vy_out, double *vz_out, int64_t capacity,
                      int64_t *cell_start_out);
/* CFL time step per domain: cfl * dx / max |v| over the domain's particles. */
void orc_cfl_dt(const double *vx, const double *vy, const double *vz,
                const int64_t *cell_start, const orc_domain *dom, int32_t n_dom,
                double cfl, double *dt_out);

/* --- initial data --------------------------------------------------------- */
enum { ORC_INIT_MAXWELL = 0, ORC_INIT_BIMAXWELL = 1, ORC_INIT_BKW = 2 };
/* cell_init rows: kind, ux, uy, uz, T (or T_par), T_perp, K0, x_lo, x_hi  */
#define ORC_INIT_COLS 9
int orc_init_cells(const double *cell_init, const int64_t *cell_start, int32_t n_cells,
                   const uint64_t *cell_key, uint64_t problem_id, uint64_t seed,
                   double *vx, double *vy, double *vz, double *x);

/* --- moments: per cell N, rho, Ux, Uy, Uz, T, Pxx, M4, E, max|v|^2 -------- */
#define ORC_MOM_COLS 10
void orc_moments(const double *vx, const double *vy, const double *vz,
                 const int64_t *cell_start, int32_t n_cells, const double *rho_scale,
                 double *out);

#ifdef __cplusplus
}
#endif
#endif
