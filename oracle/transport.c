/*
 * transport.c -- oracle of the free-transport step and the cell sort.
 * TEST INFRASTRUCTURE ONLY (see trmc_oracle.h).
 *
 * Sec. 3.1 splits each time step into a purely convective step (Q = 0) and
 * a space-homogeneous collision step.  The convective step moves every
 * particle along x by v_x dt (1D in space, 3D in velocity, as in the
 * stationary-shock test of Sec. 5.2).  READING: the paper gives no boundary
 * detail; walls are specular (x -> 2 x_wall - x, v_x -> -v_x).  The particles
 * are then regrouped by cell with a stable counting sort, which is the plain
 * definition: count per cell, exclusive prefix sum, scatter in input order.
 */
#include "trmc_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

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
        double dx = (dom[d].x_hi - dom[d].x_lo) / (double)dom[d].n_cells;
        dt_out[d] = (s2 > 0.0) ? cfl * dx / sqrt(s2) : 0.0;
    }
}

int orc_transport(double *x, double *vx, double *vy, double *vz,
                  int64_t *cell_start, int32_t n_cells_total,
                  const orc_domain *dom, int32_t n_dom, const double *dt_dom,
                  double *x_out, double *vx_out, double *vy_out, double *vz_out,
                  int64_t *cell_start_out)
{
    int64_t np = cell_start[n_cells_total];
    int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));
    /* cells that belong to no domain keep their particles */
    for (int32_t c = 0; c < n_cells_total; ++c)
        for (int64_t i = cell_start[c]; i < cell_start[c + 1]; ++i) key[i] = c;
    for (int32_t d = 0; d < n_dom; ++d) {
        const orc_domain *D = &dom[d];
        double dt = dt_dom[d];
        double lo = D->x_lo, hi = D->x_hi;
        double dx = (hi - lo) / (double)D->n_cells;
        int64_t b = cell_start[D->cell_begin], e = cell_start[D->cell_begin + D->n_cells];
        for (int64_t i = b; i < e; ++i) {
            double xn = x[i] + vx[i] * dt;
            if (xn < lo) { xn = 2.0 * lo - xn; vx[i] = -vx[i]; }
            else if (xn > hi) { xn = 2.0 * hi - xn; vx[i] = -vx[i]; }
            x[i] = xn;
            double f = floor((xn - lo) / dx);
            int64_t c = (f < 0.0) ? 0 : (int64_t)f;
            if (c > D->n_cells - 1) c = D->n_cells - 1;
            key[i] = D->cell_begin + c;
        }
    }
    /* stable counting sort by key */
    memset(cell_start_out, 0, sizeof(int64_t) * (size_t)(n_cells_total + 1));
    for (int64_t i = 0; i < np; ++i) cell_start_out[key[i] + 1]++;
    for (int32_t c = 0; c < n_cells_total; ++c) cell_start_out[c + 1] += cell_start_out[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cells_total > 0 ? n_cells_total : 1));
    for (int32_t c = 0; c < n_cells_total; ++c) fill[c] = cell_start_out[c];
    for (int64_t i = 0; i < np; ++i) {
        int64_t j = fill[key[i]]++;
        x_out[j] = x[i]; vx_out[j] = vx[i]; vy_out[j] = vy[i]; vz_out[j] = vz[i];
    }
    free(fill);
    free(key);
    return 0;
}
