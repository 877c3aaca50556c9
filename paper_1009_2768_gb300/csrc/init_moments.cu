// init_moments.cu -- initial-data sampler and per-cell moments on sm_103a.
//
// Moments follow Sec. 2 (rho, u, T, E) and Sec. 5.1 (M_4 = <|v|^4>,
// P_xx = <(v_1 - u_1)^2>), per unit mass, one CTA per cell with FP64 block
// reductions.  The sampler draws the synthetic closed-form initial data of
// the workloads (Maxwellian Eq. Max, bi-Maxwellian, BKW mixture of
// sqrt(K) chi_3 and sqrt(K) chi_5 radial laws) from Philox tag INIT.
#include "internal.h"
#include "trmc_device.cuh"

namespace trmc {
namespace {

constexpr double kTwoPi = 6.283185307179586;

template <typename Real>
__global__ void __launch_bounds__(256) init_kernel(const double *ci_all, const int64_t *cs, const uint64_t *cell_key,
                                                   uint32_t problem_id, uint64_t seed, Real *vx, Real *vy, Real *vz,
                                                   Real *x, double *cell_vmax2)
{
    __shared__ double red[kRedScratch];
    const int c = blockIdx.x;
    const double *ci = ci_all + size_t(c) * TRMC_INIT_COLS;
    const int kind = int(ci[0]);
    CellRng rng{seed, problem_id, uint64_t(c), 0};
    if (cell_key) { rng.problem = cell_key[c] >> 32; rng.cell = cell_key[c] & 0xFFFFFFFFull; }
    const int64_t b = cs[c], e = cs[c + 1];
    double vm = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        const uint64_t li = uint64_t(i - b);
        const U64x4 w = rng.draw(li, 0, 0, TAG_INIT);
        const U64x4 w2 = rng.draw(li, 1, 0, TAG_INIT);
        const double r1 = sqrt(-2.0 * log(u01_open(w.w[0]))), a1 = kTwoPi * u01(w.w[1]);
        const double r2 = sqrt(-2.0 * log(u01_open(w.w[2]))), a2 = kTwoPi * u01(w.w[3]);
        const double z0 = r1 * cos(a1), z1 = r1 * sin(a1), z2 = r2 * cos(a2);
        double v0, v1, v2;
        if (kind == TRMC_INIT_MAXWELL) {
            const double s = sqrt(ci[4]);
            v0 = ci[1] + s * z0; v1 = ci[2] + s * z1; v2 = ci[3] + s * z2;
        } else if (kind == TRMC_INIT_BIMAXWELL) {
            const double sp = sqrt(ci[4]), st = sqrt(ci[5]);
            v0 = ci[1] + sp * z0; v1 = ci[2] + st * z1; v2 = ci[3] + st * z2;
        } else {
            const double K = ci[6], sk = sqrt(K);
            const double wg = (5.0 * K - 3.0) / (2.0 * K);
            const double zz = (z0 * z0 + z1 * z1) + z2 * z2;
            double f = 1.0;
            if (!(u01(w2.w[3]) < wg)) {
                const double r3 = sqrt(-2.0 * log(u01_open(w2.w[1]))), a3 = kTwoPi * u01(w2.w[2]);
                const double z3 = r3 * cos(a3), z4 = r3 * sin(a3);
                f = sqrt((zz + z3 * z3 + z4 * z4) / zz);
            }
            v0 = ci[1] + sk * f * z0; v1 = ci[2] + sk * f * z1; v2 = ci[3] + sk * f * z2;
        }
        const Real rv0 = Real(v0), rv1 = Real(v1), rv2 = Real(v2);
        vx[i] = rv0; vy[i] = rv1; vz[i] = rv2;
        if (x) x[i] = Real(ci[7] + (ci[8] - ci[7]) * u01(w2.w[0]));
        const double d0 = rv0, d1 = rv1, d2 = rv2;
        vm = fmax(vm, __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
    }
    if (cell_vmax2) {
        vm = block_max(vm, red);
        if (threadIdx.x == 0) cell_vmax2[c] = vm;
    }
}

template <typename Real>
__global__ void __launch_bounds__(256) moments_kernel(const Real *vx, const Real *vy, const Real *vz, const int64_t *cs,
                                                      const trmc_cell_param *cp, double *out)
{
    __shared__ double red[kRedScratch];
    const int c = blockIdx.x;
    const int64_t b = cs[c], e = cs[c + 1], n = e - b;
    double *o = out + size_t(c) * TRMC_MOM_COLS;
    if (n == 0) {
        if (threadIdx.x < TRMC_MOM_COLS) o[threadIdx.x] = 0.0;
        return;
    }
    double s[5] = {0, 0, 0, 0, 0};
    double vm = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        const double x = vx[i], y = vy[i], z = vz[i];
        const double q = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
        s[0] += x; s[1] += y; s[2] += z; s[3] += q; s[4] += q * q;
        vm = fmax(vm, q);
    }
    block_sum<5>(s, red);
    vm = block_max(vm, red);
    const double U0 = s[0] / double(n), U1 = s[1] / double(n), U2 = s[2] / double(n);
    double t[2] = {0, 0};
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        const double a = double(vx[i]) - U0, bb = double(vy[i]) - U1, cc = double(vz[i]) - U2;
        t[0] += a * a + bb * bb + cc * cc;
        t[1] += a * a;
    }
    block_sum<2>(t, red);
    if (threadIdx.x == 0) {
        o[0] = double(n);
        o[1] = double(n) * (cp ? cp[c].rho_scale : 1.0);
        o[2] = U0; o[3] = U1; o[4] = U2;
        o[5] = t[0] / (3.0 * double(n));
        o[6] = t[1] / double(n);
        o[7] = s[4] / double(n);
        o[8] = 0.5 * s[3] / double(n);
        o[9] = vm;
    }
}

}  // namespace

trmc_status launch_init(trmc_ctx *ctx, trmc_state *st, const double *cell_init, cudaStream_t s)
{
    if (st->n_cells == 0) return TRMC_OK;
    if (ctx->precision == TRMC_FP64)
        init_kernel<double><<<st->n_cells, 256, 0, s>>>(cell_init, st->cell_start, st->cell_key, st->problem_id, ctx->seed,
                                                        static_cast<double *>(st->vx), static_cast<double *>(st->vy),
                                                        static_cast<double *>(st->vz), static_cast<double *>(st->x),
                                                        st->cell_vmax2);
    else
        init_kernel<float><<<st->n_cells, 256, 0, s>>>(cell_init, st->cell_start, st->cell_key, st->problem_id, ctx->seed,
                                                       static_cast<float *>(st->vx), static_cast<float *>(st->vy),
                                                       static_cast<float *>(st->vz), static_cast<float *>(st->x),
                                                       st->cell_vmax2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TRMC_OK : cuda_error(ctx, e, "init launch");
}

trmc_status launch_moments(trmc_ctx *ctx, const trmc_state *st, double *out, cudaStream_t s)
{
    if (st->n_cells == 0) return TRMC_OK;
    if (ctx->precision == TRMC_FP64)
        moments_kernel<double><<<st->n_cells, 256, 0, s>>>(static_cast<const double *>(st->vx),
                                                           static_cast<const double *>(st->vy),
                                                           static_cast<const double *>(st->vz), st->cell_start,
                                                           st->cell_param, out);
    else
        moments_kernel<float><<<st->n_cells, 256, 0, s>>>(static_cast<const float *>(st->vx),
                                                          static_cast<const float *>(st->vy),
                                                          static_cast<const float *>(st->vz), st->cell_start,
                                                          st->cell_param, out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TRMC_OK : cuda_error(ctx, e, "moments launch");
}

}  // namespace trmc
