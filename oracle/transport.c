/*
 * transport.c -- oracle of the free-transport step and the cell sort.
 * TEST INFRASTRUCTURE ONLY (see trmc_oracle.h).
 *
 * Sec. 3.1 splits each time step into a purely convective step (Q = 0) and
 * a space-homogeneous collision step.  The convective step moves every
 * particle along x by v_x dt (1D in space, 3D in velocity, as in the
 * stationary-shock test of Sec. 5.2).  READING: the paper gives no boundary
 * detail.  Walls are specular (x -> 2 x_wall - x, v_x -> -v_x).  Reservoirs
 * (the inflow / outflow of the stationary shock, whose end states are fixed
 * by the Rankine-Hugoniot relations of Sec. 5.2) are ghost cells of one cell
 * width just outside [x_lo, x_hi): every particle that ends outside
 * [x_lo, x_hi) is removed, and each ghost cell is then refilled with
 * Iround(rho dx / mass) particles of its reservoir's Maxwellian (Eq. Max),
 * uniform in the cell.  The particles are regrouped by cell with a stable
 * counting sort, which is the plain definition: count per cell, exclusive
 * prefix sum, scatter in input order.
 */
#include "trmc_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double TWO_PI = 6.283185307179586;

void orc_cfl_dt(const double *vx, const double *vy, const double *vz,
                const int64_t *cell_start, const orc_domain *dom, int32_t n_dom,
                double cfl, double *dt_out)
{
    for (int32_t d = 0; d < n_dom; ++d) {
        double s2 = 0.0;
        int64_t b = cell_start[dom[d].cell_begin];
        int64_t e = cell_start[dom[d].cell_begin + dom[d].n_cells];
        for (int64_t i = b; i < e; ++i) {
            double s = (vx[i] * vx[i] + vy[i] * vy[i]) + vz[i] * vz[i];
            if (s > s2) s2 = s;
        }
        int nint = dom[d].bc == ORC_BC_RESERVOIR ? dom[d].n_cells - 2 : dom[d].n_cells;
        double dx = (dom[d].x_hi - dom[d].x_lo) / (double)nint;
        dt_out[d] = (s2 > 0.0) ? cfl * dx / sqrt(s2) : 0.0;
    }
}

int64_t orc_transport(double *x, double *vx, double *vy, double *vz,
                      int64_t *cell_start, int32_t n_cells_total,
                      const orc_domain *dom, int32_t n_dom, const double *dt_dom,
                      const uint64_t *cell_key, uint64_t problem_id, uint64_t seed, uint64_t step,
                      double *x_out, double *vx_out, double *vy_out, double *vz_out, int64_t capacity,
                      int64_t *cell_start_out)
{
    int64_t np = cell_start[n_cells_total];
    /* positions and velocities must be finite: a cell index is taken from them */
    for (int64_t i = 0; i < np; ++i)
        if (!isfinite(x[i]) || !isfinite(vx[i]) || !isfinite(vy[i]) || !isfinite(vz[i])) return -2;
    for (int32_t d = 0; d < n_dom; ++d)
        if (!isfinite(dt_dom[d])) return -2;
    int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));   /* -1: removed */
    int64_t *refill = (int64_t *)calloc((size_t)(n_cells_total > 0 ? n_cells_total : 1), sizeof(int64_t));
    /* cells that belong to no domain keep their particles */
    for (int32_t c = 0; c < n_cells_total; ++c)
        for (int64_t i = cell_start[c]; i < cell_start[c + 1]; ++i) key[i] = c;
    for (int32_t d = 0; d < n_dom; ++d) {
        const orc_domain *D = &dom[d];
        double dt = dt_dom[d];
        double lo = D->x_lo, hi = D->x_hi;
        int res = D->bc == ORC_BC_RESERVOIR;
        int nint = res ? D->n_cells - 2 : D->n_cells;
        double dx = (hi - lo) / (double)nint;
        int64_t b = cell_start[D->cell_begin], e = cell_start[D->cell_begin + D->n_cells];
        for (int64_t i = b; i < e; ++i) {
            double xn = x[i] + vx[i] * dt;
            if (res) {
                if (xn < lo || xn >= hi) { key[i] = -1; continue; }
            } else if (xn < lo) { xn = 2.0 * lo - xn; vx[i] = -vx[i]; }
            else if (xn > hi) { xn = 2.0 * hi - xn; vx[i] = -vx[i]; }
            x[i] = xn;
            double f = floor((xn - lo) / dx);
            int64_t c = (f < 0.0) ? 0 : (int64_t)f;
            if (c > nint - 1) c = nint - 1;
            key[i] = D->cell_begin + (res ? 1 : 0) + c;
        }
        if (res) {
            for (int side = 0; side < 2; ++side) {
                int32_t g = side == 0 ? D->cell_begin : D->cell_begin + D->n_cells - 1;
                const double *r = side == 0 ? D->res_lo : D->res_hi;
                uint64_t prob = problem_id, lc = (uint64_t)g;
                if (cell_key) { prob = cell_key[g] >> 32; lc = cell_key[g] & 0xFFFFFFFFULL; }
                uint64_t w[4];
                orc_draw(seed, prob, 0xFFFFFFFFULL, 2, lc, step, 0, ORC_TAG_RESERVOIR, w);
                double want = r[0] * dx / D->particle_mass;
                double fl = floor(want);
                refill[g] = (int64_t)fl + ((orc_u01(w[0]) < want - fl) ? 1 : 0);
            }
        }
    }
    /* stable counting sort of the kept particles, ghost cells sized for the refill */
    memset(cell_start_out, 0, sizeof(int64_t) * (size_t)(n_cells_total + 1));
    for (int64_t i = 0; i < np; ++i)
        if (key[i] >= 0) cell_start_out[key[i] + 1]++;
    for (int32_t c = 0; c < n_cells_total; ++c) cell_start_out[c + 1] += refill[c];
    for (int32_t c = 0; c < n_cells_total; ++c) cell_start_out[c + 1] += cell_start_out[c];
    int64_t total = cell_start_out[n_cells_total];
    if (total > capacity) { free(key); free(refill); return -1; }
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cells_total > 0 ? n_cells_total : 1));
    for (int32_t c = 0; c < n_cells_total; ++c) fill[c] = cell_start_out[c];
    for (int64_t i = 0; i < np; ++i) {
        if (key[i] < 0) continue;
        int64_t j = fill[key[i]]++;
        x_out[j] = x[i]; vx_out[j] = vx[i]; vy_out[j] = vy[i]; vz_out[j] = vz[i];
    }
    /* refill the ghost cells from the reservoirs' Maxwellians */
    for (int32_t d = 0; d < n_dom; ++d) {
        const orc_domain *D = &dom[d];
        if (D->bc != ORC_BC_RESERVOIR) continue;
        double dx = (D->x_hi - D->x_lo) / (double)(D->n_cells - 2);
        for (int side = 0; side < 2; ++side) {
            int32_t g = side == 0 ? D->cell_begin : D->cell_begin + D->n_cells - 1;
            const double *r = side == 0 ? D->res_lo : D->res_hi;
            double x0 = side == 0 ? D->x_lo - dx : D->x_hi;
            double sT = sqrt(r[2]);
            uint64_t prob = problem_id, lc = (uint64_t)g;
            if (cell_key) { prob = cell_key[g] >> 32; lc = cell_key[g] & 0xFFFFFFFFULL; }
            for (int64_t j = 0; j < refill[g]; ++j) {
                uint64_t w[4], w2[4];
                orc_draw(seed, prob, (uint64_t)j, 0, lc, step, 0, ORC_TAG_RESERVOIR, w);
                orc_draw(seed, prob, (uint64_t)j, 1, lc, step, 0, ORC_TAG_RESERVOIR, w2);
                double r1 = sqrt(-2.0 * log(orc_u01_open(w[0]))), a1 = TWO_PI * orc_u01(w[1]);
                double r2 = sqrt(-2.0 * log(orc_u01_open(w[2]))), a2 = TWO_PI * orc_u01(w[3]);
                int64_t k = fill[g]++;
                vx_out[k] = r[1] + sT * (r1 * cos(a1));
                vy_out[k] = sT * (r1 * sin(a1));
                vz_out[k] = sT * (r2 * cos(a2));
                x_out[k] = x0 + dx * orc_u01(w2[0]);
            }
        }
    }
    free(fill);
    free(key);
    free(refill);
    return total;
}
