/*
 * collide.c -- oracle of the TRMC-R homogeneous collision step in one cell.
 * TEST INFRASTRUCTURE ONLY (see trmc_oracle.h).
 *
 * Follows Sec. 3.2 (truncated Wild sum, Eq. WST), Algorithm 4.2 (split into
 * collision sets with Iround), Algorithms 4.3/4.4 (recursive collision trees
 * for Maxwell / VHS molecules, binary collision Eq. Maxwell_coll with sigma
 * from Eq. n3d), the conservative Maxwellian resampling (end of Sec. 4.2) and
 * the adaptive truncation TRMC-RAD (Sec. 4.3) and the shape-dependent
 * truncation TRMC-WB (Sec. 4.4, Eqs. def:1-3, Algorithms 4.5/4.6).
 *
 * Algorithm 4.3 processes the levels n = m..1 and, whenever a level-n
 * collision needs a sample of f_k (k = 1..n-1), either takes a stored sibling
 * of an earlier level-k collision or creates a new level-k collision.  We take
 * the level-synchronous reading of it: the number of level-k collisions is
 * fixed from the top down by the demand of the levels above (plus the level's
 * own quota), each level-n collision picks k uniformly in {0..n-1} (Alg. 4.1),
 * and the 2C_k products of level k are assigned to the level-k demands and to
 * the level's own final outputs by a uniformly random permutation (the
 * "stored particle with a random choice").  Every original particle is used
 * once: as an uncollided level-0 particle, as a leaf of a tree, or as a member
 * of the thermalised set N_{m+1}.  The readings taken where the paper is
 * silent are marked READING below.
 */
#include "trmc_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define MC ORC_MCAP
static const double TWO_PI = 6.283185307179586;

typedef struct { double x, y, z; } vec3;

typedef struct {
    uint64_t seed, problem, cell, step;
} keyctx;

static void draw(const keyctx *k, uint64_t index, uint64_t aux, uint32_t pass,
                 uint32_t tag, uint64_t out[4])
{
    orc_draw(k->seed, k->problem, index, aux, k->cell, k->step, pass, tag, out);
}

/* ---- one pass of the tree plan ------------------------------------------ */
typedef struct {
    int lo, m_eff;
    int64_t Nq[MC + 2];      /* quotas from the split (Alg. 4.2)           */
    int64_t Nn[MC + 2];      /* quotas after the odd-count rule             */
    int64_t D[MC + 2];       /* demand for level-k samples (consumer slots) */
    int64_t C[MC + 2];       /* collisions at level n                      */
    int64_t out[MC + 2];     /* final outputs of level n                   */
    int32_t *label[MC + 1];  /* label[n][c] = k of collision c (sorted)    */
    int64_t *slot[2][MC + 1];/* consumer slot of side s of collision c    */
    int64_t n0, leaves, R;
    int64_t pdrop, psurp, feas;
} plan_t;

static void plan_free(plan_t *pl)
{
    for (int n = 0; n <= MC; ++n) {
        free(pl->label[n]); pl->label[n] = NULL;
        free(pl->slot[0][n]); pl->slot[0][n] = NULL;
        free(pl->slot[1][n]); pl->slot[1][n] = NULL;
    }
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Algorithm 4.2.  omega_n / lambda_n = (1-tau) tau^n / tau^n = q, so every
 * level takes Iround(q * remaining).  Iround uses one uniform per level
 * (READING: the paper does not say how its rounding is randomised).  The
 * loop stops as soon as nobody is left (READING of "until N_n > 0 and n < m":
 * repeat while particles remain and n < m).  lo > 0 is the continuation
 * pass of the adaptive method, which splits only levels lo..m. */
static int split(const keyctx *k, uint32_t pass, double q, int64_t n_total,
                 int lo, int m, int64_t *Nq)
{
    memset(Nq, 0, sizeof(int64_t) * (MC + 2));
    int64_t rem = n_total;
    for (int n = lo; n <= m; ++n) {
        double x = q * (double)rem;
        double fl = floor(x);
        uint64_t w[4];
        draw(k, (uint64_t)n, 0, pass, ORC_TAG_SPLIT, w);
        int64_t cnt = (int64_t)fl + ((orc_u01(w[0]) < x - fl) ? 1 : 0);
        Nq[n] = cnt;
        rem -= cnt;
        if (rem == 0) return n;
    }
    Nq[m + 1] = rem;
    return m;
}

/* Tree plan for levels m_eff..1 (top down), then the leaf feasibility check.
 * n_total participants, of which Nq[0] stay uncollided (pass 0 only). */
static void build_plan(plan_t *pl, const keyctx *k, uint32_t pass, int64_t n_total)
{
    int m_top = pl->m_eff;
    pl->feas = 0;
    for (;;) {
        memset(pl->D, 0, sizeof pl->D);
        memset(pl->C, 0, sizeof pl->C);
        memset(pl->out, 0, sizeof pl->out);
        memcpy(pl->Nn, pl->Nq, sizeof pl->Nn);
        for (int n = m_top + 1; n <= MC; ++n) pl->Nn[n] = 0;
        pl->pdrop = pl->psurp = 0;
        plan_free(pl);
        for (int n = m_top; n >= 1; --n) {
            int64_t T = pl->Nn[n] + pl->D[n];
            /* READING: an odd number of wanted level-n samples leaves one
             * product of the last pair over.  A fair coin either sends one
             * quota particle of this level to the thermalised set or keeps
             * the surplus product as an extra level-n output. */
            if (T & 1) {
                uint64_t w[4];
                draw(k, (uint64_t)n, 0, pass, ORC_TAG_PARITY, w);
                if (pl->Nn[n] >= 1 && orc_u01(w[0]) < 0.5) { pl->Nn[n] -= 1; T -= 1; pl->pdrop++; }
                else { T += 1; pl->psurp++; }
            }
            int64_t Cn = T / 2;
            pl->C[n] = Cn;
            /* Each collision draws k uniformly in {0..n-1} (Alg. 4.1 / 4.3).
             * The labels are then given to collisions 0..C_n-1 in sorted
             * order: only the multiset matters, because the inputs are
             * matched to products by an independent uniform permutation. */
            int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(Cn > 0 ? Cn : 1));
            for (int64_t c = 0; c < Cn; ++c) {
                uint64_t w[4];
                draw(k, (uint64_t)(c >> 2), (uint64_t)n, pass, ORC_TAG_KSEL, w);
                lab[c] = (int32_t)orc_below(w[c & 3], (uint32_t)n);
            }
            qsort(lab, (size_t)Cn, sizeof(int32_t), cmp_i32);
            pl->label[n] = lab;
            /* Consumer slots: side 0 of every collision, then side 1. */
            for (int s = 0; s < 2; ++s) {
                int64_t *sl = (int64_t *)malloc(sizeof(int64_t) * (size_t)(Cn > 0 ? Cn : 1));
                for (int64_t c = 0; c < Cn; ++c) {
                    int a = (s == 0) ? lab[c] : (n - 1 - lab[c]);
                    sl[c] = pl->D[a]++;
                }
                pl->slot[s][n] = sl;
            }
            pl->out[n] = 2 * Cn - pl->D[n];
        }
        /* Feasibility (the tree length is bounded by N, end of Sec. 4.1):
         * the trees need D_0 leaves but only the non-level-0 particles can
         * serve.  READING: take the missing leaves from level 0, else drop
         * the top level into the thermalised set and plan again. */
        int64_t n0 = pl->Nq[0];
        int64_t A = n_total - n0;
        if (pl->D[0] <= A) { pl->n0 = n0; pl->leaves = pl->D[0]; pl->R = A - pl->D[0]; break; }
        int64_t deficit = pl->D[0] - A;
        if (deficit <= n0) { pl->n0 = n0 - deficit; pl->leaves = pl->D[0]; pl->R = 0; break; }
        pl->feas++;
        m_top--;
    }
    pl->m_eff = m_top;
}

/* Binary collision, Eq. Maxwell_coll with sigma uniform on S^2 (Eq. n3d,
 * cos(theta) = 2 xi_1 - 1).  For VHS (alpha > 0) the pair collides if
 * Sigma * xi < |v_i - v_j|^alpha (Alg. 4.4), else it is a dummy collision
 * and both leave unchanged. */
static void binary_collision(vec3 a, vec3 b, const uint64_t w[4], double alpha, double Sigma,
                             vec3 *oa, vec3 *ob, int *accepted, int *exceeded)
{
    double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    double g = sqrt(dx * dx + dy * dy + dz * dz);
    *exceeded = 0;
    if (alpha != 0.0) {
        double ga = (alpha == 1.0) ? g : pow(g, alpha);
        if (ga > Sigma) *exceeded = 1;
        double xi = orc_u01(w[0]);
        if (!(xi * Sigma < ga)) { *oa = a; *ob = b; *accepted = 0; return; }
    }
    double ct = 2.0 * orc_u01(w[1]) - 1.0;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double phi = TWO_PI * orc_u01(w[2]);
    double sx = cos(phi) * st, sy = sin(phi) * st, sz = ct;
    double h = 0.5 * g;
    double cx = 0.5 * (a.x + b.x), cy = 0.5 * (a.y + b.y), cz = 0.5 * (a.z + b.z);
    oa->x = cx + h * sx; oa->y = cy + h * sy; oa->z = cz + h * sz;
    ob->x = cx - h * sx; ob->y = cy - h * sy; ob->z = cz - h * sz;
    *accepted = 1;
}

/* ---- tree lengths (Sec. 4.4) --------------------------------------------- */
/* Length of a tree of root size k = j + h + 1 from the lengths of its two
 * subtrees: Eq. def:1 counts the collisions, Eq. def:2 takes 1 + the shorter
 * subtree, Eq. def:3 1 + their mean.  A sample of f_0 (an original particle)
 * has length 0. */
static double tree_len(int def, double Lj, double Lh)
{
    if (def == ORC_LEN_K) return 1.0 + Lj + Lh;
    if (def == ORC_LEN_MIN) return 1.0 + (Lj < Lh ? Lj : Lh);
    return 1.0 + 0.5 * (Lj + Lh);
}

/* Algorithm 4.5 read back: the list holds k, then (j, h) of every node in
 * pre-order; the length is evaluated recursively from the leaves. */
static double path_len(const int32_t *path, int64_t len, int64_t *idx, int32_t k, int def)
{
    if (k == 0) return 0.0;
    if (*idx + 2 > len) return -1.0;
    int32_t j = path[*idx], h = path[*idx + 1];
    *idx += 2;
    if (j < 0 || h < 0 || j + h + 1 != k) return -1.0;
    double Lj = path_len(path, len, idx, j, def);
    if (Lj < 0.0) return -1.0;
    double Lh = path_len(path, len, idx, h, def);
    if (Lh < 0.0) return -1.0;
    return tree_len(def, Lj, Lh);
}

double orc_tree_length(const int32_t *path, int64_t len, int def)
{
    if (len < 1 || path[0] < 0 || def < ORC_LEN_K || def > ORC_LEN_MEAN) return -1.0;
    int64_t idx = 1;
    double L = path_len(path, len, &idx, path[0], def);
    return (L >= 0.0 && idx == len) ? L : -1.0;
}

typedef struct {
    int64_t coll, dummy, exceed;
    int64_t wbrej;           /* TRMC-WB: outputs whose tree was too long       */
    /* what the collisions changed: sum over this pass's leaves of
     * (output - original) for v, |v|^2 and the adaptive indicator */
    double dP[3], dE, dS;
} counters_t;

/* Execute one planned pass.  part[i] (i < n_total) are the participating
 * particle slots; vin holds their (original) velocities, vfin receives the
 * outputs.  On return pool[0..R-1] lists the thermalised slots in rank order
 * and is_pool/is_level0 flags are updated. */
static double indicator(vec3 v, const double U[3], int ind);

static void run_pass(const plan_t *pl, const keyctx *k, uint32_t pass,
                     const int64_t *part, int64_t n_total, const vec3 *vin, vec3 *vfin,
                     int64_t *pool, double alpha, double Sigma, const double U[3], int ind,
                     int wb_def, int wb_mmax, counters_t *cnt)
{
    int m = pl->m_eff;
    /* Roles: a uniform permutation of the participants (READING: the paper
     * takes particles "with a random choice"); ranks [0,n0) stay uncollided,
     * the next D_0 are the leaves, the rest are thermalised. */
    uint64_t key[4];
    draw(k, 0, 0, pass, ORC_TAG_PERM0, key);
    orc_prp perm;
    orc_prp_init(&perm, (uint64_t)n_total, key);
    int64_t *leaf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(pl->leaves > 0 ? pl->leaves : 1));
    for (int64_t i = 0; i < n_total; ++i) {
        int64_t r = (int64_t)orc_prp_fwd(&perm, (uint64_t)i);
        if (r < pl->n0) continue;
        r -= pl->n0;
        if (r < pl->leaves) leaf[r] = part[i];
        else pool[r - pl->leaves] = part[i];
    }
    /* Products of each level and the permutation that feeds them to the
     * level's consumers (slot t < D_k) or to its outputs (t >= D_k). */
    vec3 *prod[MC + 1];
    int64_t *feeder[MC + 1];
    int64_t *outp[MC + 1];
    double *Lc[MC + 1];      /* TRMC-WB: length of the tree of collision c of level n */
    for (int n = 0; n <= MC; ++n) { prod[n] = NULL; feeder[n] = NULL; outp[n] = NULL; Lc[n] = NULL; }
    for (int n = 1; n <= m; ++n) {
        int64_t P = 2 * pl->C[n];
        prod[n] = (vec3 *)malloc(sizeof(vec3) * (size_t)(P > 0 ? P : 1));
        if (wb_def) Lc[n] = (double *)malloc(sizeof(double) * (size_t)(pl->C[n] > 0 ? pl->C[n] : 1));
        feeder[n] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(pl->D[n] > 0 ? pl->D[n] : 1));
        outp[n] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(pl->out[n] > 0 ? pl->out[n] : 1));
        uint64_t kk[4];
        draw(k, 0, (uint64_t)n, pass, ORC_TAG_PERMK, kk);
        orc_prp pk;
        orc_prp_init(&pk, (uint64_t)P, kk);
        for (int64_t p = 0; p < P; ++p) {
            int64_t t = (int64_t)orc_prp_fwd(&pk, (uint64_t)p);
            if (t < pl->D[n]) feeder[n][t] = p;
            else outp[n][t - pl->D[n]] = p;
        }
    }
    /* Collision waves, level 1 first: every input of a level-n collision
     * is either a leaf (k = 0) or a product of a lower level.  For TRMC-WB
     * the length of each collision's tree follows from its inputs' trees
     * (both products of a collision share the tree). */
    for (int n = 1; n <= m; ++n) {
        for (int64_t c = 0; c < pl->C[n]; ++c) {
            vec3 in[2];
            double Lin[2];
            for (int s = 0; s < 2; ++s) {
                int a = (s == 0) ? pl->label[n][c] : (n - 1 - pl->label[n][c]);
                int64_t sl = pl->slot[s][n][c];
                if (a == 0) { in[s] = vin[leaf[sl]]; Lin[s] = 0.0; }
                else {
                    in[s] = prod[a][feeder[a][sl]];
                    Lin[s] = wb_def ? Lc[a][feeder[a][sl] >> 1] : 0.0;
                }
            }
            if (wb_def) Lc[n][c] = tree_len(wb_def, Lin[0], Lin[1]);
            uint64_t w[4];
            draw(k, (uint64_t)c, (uint64_t)n, pass, ORC_TAG_COLL, w);
            int acc, exc;
            binary_collision(in[0], in[1], w, alpha, Sigma, &prod[n][2 * c], &prod[n][2 * c + 1], &acc, &exc);
            if (alpha != 0.0) { if (acc) cnt->coll++; else cnt->dummy++; }
            else cnt->coll++;
            cnt->exceed += exc;
        }
    }
    /* TRMC-WB (Algorithm 4.6): an output whose tree is longer than m_max is
     * not kept; the particle it would replace joins the thermalised set,
     * after the set's own members, in output order.  READING: the trees are
     * the ones the plan actually built (the plan is fixed before any
     * collision, so the lengths are known "without performing collisions").
     * A lone rejected output with no thermalised set is kept: the only
     * Maxwellian sample with its momentum and energy is the output itself. */
    int64_t nrej = 0;
    unsigned char *rej = NULL;
    if (wb_def) {
        rej = (unsigned char *)calloc((size_t)(pl->leaves > 0 ? pl->leaves : 1), 1);
        int64_t jj = 0;
        for (int n = 1; n <= m; ++n)
            for (int64_t o = 0; o < pl->out[n]; ++o, ++jj)
                if (Lc[n][outp[n][o] >> 1] > (double)wb_mmax) { rej[jj] = 1; nrej++; }
        if (pl->R == 0 && nrej == 1) { memset(rej, 0, (size_t)(pl->leaves > 0 ? pl->leaves : 1)); nrej = 0; }
    }
    cnt->wbrej += nrej;
    /* Output j (levels 1..m in order, then by rank) replaces leaf j. */
    int64_t j = 0, r = 0;
    for (int n = 1; n <= m; ++n)
        for (int64_t o = 0; o < pl->out[n]; ++o) {
            if (rej && rej[j]) { pool[pl->R + r++] = leaf[j++]; continue; }
            vec3 nv = prod[n][outp[n][o]], ov = vin[leaf[j]];
            cnt->dP[0] += nv.x - ov.x; cnt->dP[1] += nv.y - ov.y; cnt->dP[2] += nv.z - ov.z;
            cnt->dE += (nv.x * nv.x + nv.y * nv.y + nv.z * nv.z) - (ov.x * ov.x + ov.y * ov.y + ov.z * ov.z);
            cnt->dS += indicator(nv, U, ind) - indicator(ov, U, ind);
            vfin[leaf[j++]] = nv;
        }
    for (int n = 0; n <= MC; ++n) { free(prod[n]); free(feeder[n]); free(outp[n]); free(Lc[n]); }
    free(rej);
    free(leaf);
}

/* RAD indicator of one velocity: P_xx term or |v|^4 (Sec. 4.3, Sec. 5). */
static double indicator(vec3 v, const double U[3], int ind)
{
    if (ind == ORC_IND_M4) { double e = v.x * v.x + v.y * v.y + v.z * v.z; return e * e; }
    double d = v.x - U[0];
    return d * d;
}

int orc_collide_cell(double *vx, double *vy, double *vz, int64_t n,
                     uint64_t problem, uint64_t cell, uint64_t step,
                     int32_t *m_state, const orc_collide_params *prm,
                     const orc_cell_param *cp, int64_t *report)
{
    if (report) memset(report, 0, sizeof(int64_t) * ORC_R_LEN);
    if (report) report[ORC_R_N] = n;
    double dt = cp ? cp->dt : prm->dt, eps = cp ? cp->eps : prm->eps;
    double alpha = cp ? cp->alpha : prm->alpha, rho_scale = cp ? cp->rho_scale : prm->rho_scale;
    int m0;
    if (prm->trunc == ORC_TRUNC_FIXED) m0 = prm->m_fixed;
    else if (prm->trunc == ORC_TRUNC_RAD) m0 = *m_state;
    else m0 = prm->m_cap;
    if (m0 < 1) m0 = 1;
    if (m0 > prm->m_cap) m0 = prm->m_cap;
    if (n < 2) {
        if (report) { report[ORC_R_MNEXT] = (prm->trunc == ORC_TRUNC_RAD) ? m0 : 0; report[ORC_R_N0] = n; }
        return 0;
    }
    keyctx k = { prm->seed, problem, cell, step };

    /* Moments (Sec. 2): momentum, energy, mean velocity. */
    vec3 *vin = (vec3 *)malloc(sizeof(vec3) * (size_t)n);
    vec3 *vfin = (vec3 *)malloc(sizeof(vec3) * (size_t)n);
    double P[3] = { 0, 0, 0 }, E = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        vin[i].x = vx[i]; vin[i].y = vy[i]; vin[i].z = vz[i];
        vfin[i] = vin[i];
        P[0] += vx[i]; P[1] += vy[i]; P[2] += vz[i];
        E += vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
    }
    double U[3] = { P[0] / (double)n, P[1] / (double)n, P[2] / (double)n };
    /* VHS bound Sigma = sigma(2 dv), dv = max_i |v_i - mean| (Sec. 4.2);
     * sigma(g) = g^alpha with 4 pi K = 1, so mu = rho * Sigma (READING of
     * mu >= 4 pi rho sigma_bar, Sec. 3.2, and mu = 4 pi Sigma, Sec. 4.2). */
    double Sigma = 1.0;
    if (alpha != 0.0) {
        double d2 = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double a = vin[i].x - U[0], b = vin[i].y - U[1], c = vin[i].z - U[2];
            double s = a * a + b * b + c * c;
            if (s > d2) d2 = s;
        }
        double g = 2.0 * sqrt(d2);
        Sigma = (alpha == 1.0) ? g : pow(g, alpha);
    }
    double rho = (double)n * rho_scale;
    double mu = rho * Sigma;
    double q = exp(-(mu * dt) / eps);    /* e^{-mu dt/eps}, Eq. WST */
    double S_pre = 0.0;
    for (int64_t i = 0; i < n; ++i) S_pre += indicator(vin[i], U, prm->indicator);
    S_pre /= (double)n;

    /* Passes: pass 0 splits all N over levels 0..m; an adaptive rejection
     * continues with levels m+1..2m on the thermalised set (Sec. 4.3). */
    int64_t *part = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *pool = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) part[i] = i;
    int64_t n_part = n;
    counters_t cnt = { 0, 0, 0, 0, { 0.0, 0.0, 0.0 }, 0.0, 0.0 };
    const int wb_def = (prm->trunc == ORC_TRUNC_WB) ? prm->wb_length : 0;
    int m = m0, lo = 0, m_next = m0;
    uint32_t pass = 0;
    int64_t R = 0, leaves_total = 0;
    plan_t pl;
    memset(&pl, 0, sizeof pl);
    for (;;) {
        pl.lo = lo;
        pl.m_eff = split(&k, pass, q, n_part, lo, m, pl.Nq);
        if (lo > 0) pl.Nq[0] = 0;
        build_plan(&pl, &k, pass, n_part);
        if (report && pass == 0) {
            report[ORC_R_N0] = pl.n0;
            report[ORC_R_MEFF0] = pl.m_eff;
            for (int i = 0; i <= MC + 1; ++i) {
                report[ORC_R_NK + i] = pl.Nq[i];
                report[ORC_R_CK + i] = pl.C[i];
                report[ORC_R_DK + i] = pl.D[i];
            }
        }
        if (report) {
            report[ORC_R_FEAS] += pl.feas;
            report[ORC_R_PDROP] += pl.pdrop;
            report[ORC_R_PSURP] += pl.psurp;
        }
        run_pass(&pl, &k, pass, part, n_part, vin, vfin, pool, alpha, Sigma, U, prm->indicator,
                 wb_def, prm->m_fixed, &cnt);
        leaves_total += pl.leaves;
        R = pl.R + cnt.wbrej;
        plan_free(&pl);
        if (prm->trunc != ORC_TRUNC_RAD) { m_next = m; break; }

        /* TRMC-RAD test (Sec. 4.3): E1 = |S^{n+1,m} - S^n| / |S^n| with the
         * thermalised part taken from the analytic Maxwellian it will be
         * sampled from (last paragraph of Sec. 4.3).  The change of the
         * indicator sum is formed from the particles that changed: the
         * collisions' dS, minus the thermalised set's original sum, plus its
         * analytic Maxwellian sum. */
        double Pp[3] = { 0, 0, 0 }, Ep = 0.0, Sp = 0.0;
        for (int64_t t = 0; t < R; ++t) {
            vec3 v = vin[pool[t]];
            Pp[0] += v.x; Pp[1] += v.y; Pp[2] += v.z;
            Ep += v.x * v.x + v.y * v.y + v.z * v.z;
            Sp += indicator(v, U, prm->indicator);
        }
        double Sth = 0.0;
        if (R == 1) {
            Sth = indicator(vin[pool[0]], U, prm->indicator);
        } else if (R >= 2) {
            double Pt[3] = { Pp[0] - cnt.dP[0], Pp[1] - cnt.dP[1], Pp[2] - cnt.dP[2] };
            double Et = Ep - cnt.dE;
            double et = Et - (Pt[0] * Pt[0] + Pt[1] * Pt[1] + Pt[2] * Pt[2]) / (double)R;
            if (et < 0.0) et = 0.0;
            double ub[3] = { Pt[0] / (double)R, Pt[1] / (double)R, Pt[2] / (double)R };
            if (prm->indicator == ORC_IND_M4) {
                double Tp = et / (3.0 * (double)R);
                double u2 = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
                Sth = (double)R * (u2 * u2 + 10.0 * u2 * Tp + 15.0 * Tp * Tp);
            } else {
                double d = ub[0] - U[0];
                Sth = et / 3.0 + (double)R * d * d;
            }
        }
        double dS_total = cnt.dS + (Sth - Sp);
        double E1 = (S_pre != 0.0) ? fabs(dS_total) / fabs((double)n * S_pre) : 0.0;
        if (E1 > prm->delta2 && R > 0 && 2 * m <= prm->m_cap) {
            /* Reject: keep what was computed, continue with 2m. */
            for (int64_t t = 0; t < R; ++t) part[t] = pool[t];
            n_part = R;
            lo = m + 1;
            m = 2 * m;
            pass++;
            continue;
        }
        if (E1 < prm->delta1) m_next = (m / 2 > prm->m_min) ? m / 2 : prm->m_min;
        else m_next = m;
        break;
    }

    /* Thermalised particles: Maxwellian samples (Box-Muller) renormalised so
     * that the cell's momentum and energy are exactly those before the step
     * (READING of the conservative sampling cited at the end of Sec. 4.2:
     * v = P_t/R + s (z - zbar), s fixing the kinetic energy). */
    if (R >= 2) {
        /* target: what the thermalised set carried, corrected by what the
         * collisions' round-off changed (sums over changed particles only) */
        double Pt[3] = { 0, 0, 0 }, Et = 0.0;
        for (int64_t t = 0; t < R; ++t) {
            vec3 v = vin[pool[t]];
            Pt[0] += v.x; Pt[1] += v.y; Pt[2] += v.z;
            Et += v.x * v.x + v.y * v.y + v.z * v.z;
        }
        Pt[0] -= cnt.dP[0]; Pt[1] -= cnt.dP[1]; Pt[2] -= cnt.dP[2];
        Et -= cnt.dE;
        vec3 *z = (vec3 *)malloc(sizeof(vec3) * (size_t)R);
        double zs[3] = { 0, 0, 0 };
        for (int64_t t = 0; t < R; ++t) {
            uint64_t w[4];
            draw(&k, (uint64_t)t, 0, 0, ORC_TAG_MAXW, w);
            double r1 = sqrt(-2.0 * log(orc_u01_open(w[0])));
            double a1 = TWO_PI * orc_u01(w[1]);
            double r2 = sqrt(-2.0 * log(orc_u01_open(w[2])));
            double a2 = TWO_PI * orc_u01(w[3]);
            z[t].x = r1 * cos(a1); z[t].y = r1 * sin(a1); z[t].z = r2 * cos(a2);
            zs[0] += z[t].x; zs[1] += z[t].y; zs[2] += z[t].z;
        }
        double zb[3] = { zs[0] / (double)R, zs[1] / (double)R, zs[2] / (double)R };
        double ez = 0.0;
        for (int64_t t = 0; t < R; ++t) {
            double a = z[t].x - zb[0], b = z[t].y - zb[1], c = z[t].z - zb[2];
            ez += a * a + b * b + c * c;
        }
        double et = Et - (Pt[0] * Pt[0] + Pt[1] * Pt[1] + Pt[2] * Pt[2]) / (double)R;
        if (et < 0.0) et = 0.0;
        double s = (ez > 0.0) ? sqrt(et / ez) : 0.0;
        double ub[3] = { Pt[0] / (double)R, Pt[1] / (double)R, Pt[2] / (double)R };
        for (int64_t t = 0; t < R; ++t) {
            vec3 v;
            v.x = ub[0] + s * (z[t].x - zb[0]);
            v.y = ub[1] + s * (z[t].y - zb[1]);
            v.z = ub[2] + s * (z[t].z - zb[2]);
            vfin[pool[t]] = v;
        }
        free(z);
    }
    /* R == 1: the lone thermalised particle keeps its velocity, which is
     * the only choice with the prescribed momentum and energy. */

    for (int64_t i = 0; i < n; ++i) { vx[i] = vfin[i].x; vy[i] = vfin[i].y; vz[i] = vfin[i].z; }
    if (prm->trunc == ORC_TRUNC_RAD) *m_state = m_next;
    if (report) {
        report[ORC_R_PASSES] = (int64_t)pass + 1;
        report[ORC_R_MFIRST] = m0;
        report[ORC_R_MLAST] = m;
        report[ORC_R_MNEXT] = m_next;
        report[ORC_R_RFINAL] = R;
        report[ORC_R_LEAVES] = leaves_total;
        report[ORC_R_COLL] = cnt.coll;
        report[ORC_R_DUMMY] = cnt.dummy;
        report[ORC_R_EXCEED] = cnt.exceed;
        report[ORC_R_WBREJ] = cnt.wbrej;
    }
    free(vin); free(vfin); free(part); free(pool);
    return 0;
}

/* ---- many cells, optionally on several host threads ----------------------- */
typedef struct {
    double *vx, *vy, *vz;
    const int64_t *cell_start;
    int32_t n_cells;
    const uint64_t *cell_key;
    uint64_t problem_id, step;
    int32_t *m_state;
    const orc_collide_params *prm;
    const orc_cell_param *cell_param;
    int64_t *reports;
    int tid, nth;
} job_t;

static void *collide_worker(void *arg)
{
    job_t *j = (job_t *)arg;
    for (int32_t c = j->tid; c < j->n_cells; c += j->nth) {
        int64_t b = j->cell_start[c], e = j->cell_start[c + 1];
        uint64_t prob = j->problem_id, lc = (uint64_t)c;
        if (j->cell_key) { prob = j->cell_key[c] >> 32; lc = j->cell_key[c] & 0xFFFFFFFFULL; }
        orc_collide_cell(j->vx + b, j->vy + b, j->vz + b, e - b, prob, lc, j->step,
                         j->m_state ? j->m_state + c : NULL, j->prm,
                         j->cell_param ? j->cell_param + c : NULL,
                         j->reports ? j->reports + (int64_t)c * ORC_R_LEN : NULL);
    }
    return NULL;
}

int orc_collide(double *vx, double *vy, double *vz, const int64_t *cell_start,
                int32_t n_cells, const uint64_t *cell_key, uint64_t problem_id,
                uint64_t step, int32_t *m_state, const orc_collide_params *prm,
                const orc_cell_param *cell_param, int64_t *reports, int n_threads)
{
    if (prm->trunc == ORC_TRUNC_RAD && !m_state) return 1;
    if (prm->m_cap < 1 || prm->m_cap > MC) return 1;
    if (prm->trunc == ORC_TRUNC_WB &&
        (prm->wb_length < ORC_LEN_K || prm->wb_length > ORC_LEN_MEAN || prm->m_fixed < 0)) return 1;
    /* the method is defined for finite velocities whose energy sums are finite */
    for (int32_t c = 0; c < n_cells; ++c) {
        double e = 0.0;
        for (int64_t i = cell_start[c]; i < cell_start[c + 1]; ++i) e += vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
        if (!isfinite(e)) return 2;
    }
    if (n_threads < 1) n_threads = 1;
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * (size_t)n_threads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int t = 0; t < n_threads; ++t) {
        job_t j = { vx, vy, vz, cell_start, n_cells, cell_key, problem_id, step, m_state,
                    prm, cell_param, reports, t, n_threads };
        jobs[t] = j;
    }
    if (n_threads == 1) collide_worker(&jobs[0]);
    else {
        for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, collide_worker, &jobs[t]);
        for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    }
    free(jobs); free(th);
    return 0;
}
