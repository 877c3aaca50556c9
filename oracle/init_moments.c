/*
 * init_moments.c -- oracle of the initial-data sampler and of the cell
 * moments.  TEST INFRASTRUCTURE ONLY (see trmc_oracle.h).
 *
 * Moments follow Sec. 2 (rho, u, T, E) and Sec. 5.1 (M_4 = int f |v|^4,
 * P_xx = int f (v_1 - u_1)^2), per unit mass in each cell.
 *
 * Initial data are synthetic closed forms (no dataset is involved):
 *  - Maxwellian M(rho,u,T), Eq. Max;
 *  - bi-Maxwellian with temperature T_par along x and T_perp along y, z;
 *  - the BKW solution for Maxwell molecules at shape K: a mixture of
 *    sqrt(K) chi_3 (weight (5K-3)/(2K)) and sqrt(K) chi_5 (weight 3(1-K)/(2K))
 *    radial laws with isotropic direction (unit density and temperature).
 * Normal deviates come from Box-Muller on Philox draws with tag INIT.
 */
#include "trmc_oracle.h"
#include <math.h>

static const double TWO_PI = 6.283185307179586;

int orc_init_cells(const double *cell_init, const int64_t *cell_start, int32_t n_cells,
                   const uint64_t *cell_key, uint64_t problem_id, uint64_t seed,
                   double *vx, double *vy, double *vz, double *x)
{
    for (int32_t c = 0; c < n_cells; ++c) {
        const double *ci = cell_init + (int64_t)c * ORC_INIT_COLS;
        int kind = (int)ci[0];
        uint64_t prob = problem_id, lc = (uint64_t)c;
        if (cell_key) { prob = cell_key[c] >> 32; lc = cell_key[c] & 0xFFFFFFFFULL; }
        for (int64_t i = cell_start[c]; i < cell_start[c + 1]; ++i) {
            uint64_t li = (uint64_t)(i - cell_start[c]);
            uint64_t w[4], w2[4];
            orc_draw(seed, prob, li, 0, lc, 0, 0, ORC_TAG_INIT, w);
            orc_draw(seed, prob, li, 1, lc, 0, 0, ORC_TAG_INIT, w2);
            double r1 = sqrt(-2.0 * log(orc_u01_open(w[0]))), a1 = TWO_PI * orc_u01(w[1]);
            double r2 = sqrt(-2.0 * log(orc_u01_open(w[2]))), a2 = TWO_PI * orc_u01(w[3]);
            double z0 = r1 * cos(a1), z1 = r1 * sin(a1), z2 = r2 * cos(a2);
            double v0, v1, v2;
            if (kind == ORC_INIT_MAXWELL) {
                double s = sqrt(ci[4]);
                v0 = ci[1] + s * z0; v1 = ci[2] + s * z1; v2 = ci[3] + s * z2;
            } else if (kind == ORC_INIT_BIMAXWELL) {
                double sp = sqrt(ci[4]), st = sqrt(ci[5]);
                v0 = ci[1] + sp * z0; v1 = ci[2] + st * z1; v2 = ci[3] + st * z2;
            } else {
                double K = ci[6], sk = sqrt(K);
                double wg = (5.0 * K - 3.0) / (2.0 * K);
                double zz = (z0 * z0 + z1 * z1) + z2 * z2;
                double f = 1.0;
                if (!(orc_u01(w2[3]) < wg)) {
                    double r3 = sqrt(-2.0 * log(orc_u01_open(w2[1]))), a3 = TWO_PI * orc_u01(w2[2]);
                    double z3 = r3 * cos(a3), z4 = r3 * sin(a3);
                    f = sqrt((zz + z3 * z3 + z4 * z4) / zz);
                }
                v0 = ci[1] + sk * f * z0; v1 = ci[2] + sk * f * z1; v2 = ci[3] + sk * f * z2;
            }
            vx[i] = v0; vy[i] = v1; vz[i] = v2;
            if (x) x[i] = ci[7] + (ci[8] - ci[7]) * orc_u01(w2[0]);
        }
    }
    return 0;
}

void orc_moments(const double *vx, const double *vy, const double *vz,
                 const int64_t *cell_start, int32_t n_cells, const double *rho_scale,
                 double *out)
{
    for (int32_t c = 0; c < n_cells; ++c) {
        double *o = out + (int64_t)c * ORC_MOM_COLS;
        int64_t b = cell_start[c], e = cell_start[c + 1], n = e - b;
        for (int j = 0; j < ORC_MOM_COLS; ++j) o[j] = 0.0;
        o[0] = (double)n;
        if (n == 0) continue;
        double P[3] = { 0, 0, 0 }, E = 0.0, M4 = 0.0, vm = 0.0;
        for (int64_t i = b; i < e; ++i) {
            double s = (vx[i] * vx[i] + vy[i] * vy[i]) + vz[i] * vz[i];
            P[0] += vx[i]; P[1] += vy[i]; P[2] += vz[i];
            E += s; M4 += s * s;
            if (s > vm) vm = s;
        }
        double U[3] = { P[0] / (double)n, P[1] / (double)n, P[2] / (double)n };
        double th = 0.0, pxx = 0.0;
        for (int64_t i = b; i < e; ++i) {
            double a = vx[i] - U[0], bb = vy[i] - U[1], cc = vz[i] - U[2];
            th += a * a + bb * bb + cc * cc;
            pxx += a * a;
        }
        o[1] = (double)n * (rho_scale ? rho_scale[c] : 1.0);
        o[2] = U[0]; o[3] = U[1]; o[4] = U[2];
        o[5] = th / (3.0 * (double)n);
        o[6] = pxx / (double)n;
        o[7] = M4 / (double)n;
        o[8] = 0.5 * E / (double)n;
        o[9] = vm;
    }
}
