// transport.cu -- free transport and stable cell regrouping on sm_103a.
//
// The convective half of the splitting (Sec. 3.1): x <- x + v_x dt with
// specular walls at both ends of each 1D domain, then the particles are
// regrouped by cell, keeping their order within a cell (the order feeds
// the collision step's random roles).  Because dt * max|v_x| <= dx, a
// particle moves at most one cell, so the regrouping is a banded counting
// sort: each old cell counts its particles going to the cell on the left,
// staying, and going right (kernel 1); one scan turns those counts into the
// new cell starts (kernel 2); each old cell then scatters its particles
// with block-wide stable ranks from warp ballots (kernel 3).  Positions and
// cells are recomputed identically in kernels 1 and 3.  In FP64 contexts
// the position update uses explicitly rounded operations (no contraction),
// so cells are bit-identical to the CPU oracle's.
#include <utility>

#include "internal.h"
#include "trmc_device.cuh"

namespace trmc {
namespace {

constexpr int kTT = 256;   // threads per CTA

// Position update and new cell (relative to the domain's first cell), double.
struct Mover64 {
    double lo, hi, dx, dt;
    int nc;
    __device__ __forceinline__ int move(double &x, double &vx) const
    {
        double xn = __dadd_rn(x, __dmul_rn(vx, dt));
        if (xn < lo) { xn = __dsub_rn(__dmul_rn(2.0, lo), xn); vx = -vx; }
        else if (xn > hi) { xn = __dsub_rn(__dmul_rn(2.0, hi), xn); vx = -vx; }
        x = xn;
        const double f = floor(__ddiv_rn(__dsub_rn(xn, lo), dx));
        int c = (f < 0.0) ? 0 : (f > double(nc - 1) ? nc - 1 : int(f));
        return c;
    }
};
struct Mover32 {
    float lo, hi, inv_dx, dt;
    int nc;
    __device__ __forceinline__ int move(float &x, float &vx) const
    {
        float xn = x + vx * dt;
        if (xn < lo) { xn = 2.0f * lo - xn; vx = -vx; }
        else if (xn > hi) { xn = 2.0f * hi - xn; vx = -vx; }
        x = xn;
        const float f = floorf((xn - lo) * inv_dx);
        int c = (f < 0.0f) ? 0 : (f > float(nc - 1) ? nc - 1 : int(f));
        return c;
    }
};
template <typename Real> struct MoverT;
template <> struct MoverT<double> { using type = Mover64; };
template <> struct MoverT<float> { using type = Mover32; };

struct CellDom {
    int d;          // domain index or -1
    int first;      // domain's first cell
};

__device__ __forceinline__ bool domain_ok(const trmc_domain &D, int nc_total)
{
    return D.n_cells >= 1 && D.cell_begin >= 0 && D.cell_begin <= nc_total - D.n_cells && D.x_hi > D.x_lo;
}

// Domain of cell c (first valid match); malformed domains are ignored and
// reported, so their cells keep their particles and no write leaves the state.
__device__ __forceinline__ CellDom find_domain(const trmc_domain *doms, int nd, int c, int nc_total, int *status)
{
    for (int d = 0; d < nd; ++d) {
        const trmc_domain D = doms[d];
        if (!domain_ok(D, nc_total)) {
            if (atomicCAS(status, 0, TRMC_ERR_ARG) == 0) status[1] = d;
            continue;
        }
        if (c >= D.cell_begin && c < D.cell_begin + D.n_cells) return CellDom{d, D.cell_begin};
    }
    return CellDom{-1, 0};
}

template <typename Real>
__device__ __forceinline__ typename MoverT<Real>::type make_mover(const trmc_domain &D, double dt);
template <>
__device__ __forceinline__ Mover64 make_mover<double>(const trmc_domain &D, double dt)
{
    Mover64 m;
    m.lo = D.x_lo; m.hi = D.x_hi; m.nc = D.n_cells; m.dt = dt;
    m.dx = __ddiv_rn(__dsub_rn(D.x_hi, D.x_lo), double(D.n_cells));
    return m;
}
template <>
__device__ __forceinline__ Mover32 make_mover<float>(const trmc_domain &D, double dt)
{
    Mover32 m;
    m.lo = float(D.x_lo); m.hi = float(D.x_hi); m.nc = D.n_cells; m.dt = float(dt);
    m.inv_dx = float(double(D.n_cells) / (D.x_hi - D.x_lo));
    return m;
}

// Kernel 0: CFL time step per domain from the per-cell max |v|^2.
__global__ void cfl_kernel(const trmc_domain *doms, int nd, int nc_total, const double *cell_vmax2, double cfl,
                           double *dt, trmc_cell_param *cell_param)
{
    __shared__ double red[kRedScratch];
    const int d = blockIdx.x;
    if (d >= nd) return;
    const trmc_domain D = doms[d];
    if (!domain_ok(D, nc_total)) {
        if (threadIdx.x == 0) dt[d] = 0.0;
        return;
    }
    double vm = 0.0;
    for (int c = threadIdx.x; c < D.n_cells; c += blockDim.x) vm = fmax(vm, cell_vmax2[D.cell_begin + c]);
    vm = block_max(vm, red);
    const double dx = __ddiv_rn(__dsub_rn(D.x_hi, D.x_lo), double(D.n_cells));
    const double h = (vm > 0.0) ? __ddiv_rn(__dmul_rn(cfl, dx), __dsqrt_rn(vm)) : 0.0;
    if (threadIdx.x == 0) dt[d] = h;
    if (cell_param)
        for (int c = threadIdx.x; c < D.n_cells; c += blockDim.x) cell_param[D.cell_begin + c].dt = h;
}

// Kernel 1: per old cell, how many particles go left / stay / go right.
template <typename Real>
__global__ void __launch_bounds__(kTT) count_kernel(const Real *x, const Real *vx, const int64_t *cs,
                                                    const trmc_domain *doms, int nd, int nc_total, const double *dt,
                                                    int64_t *counts, int *status)
{
    __shared__ CellDom sd;
    __shared__ unsigned long long tot[3];
    const int c = blockIdx.x;
    if (threadIdx.x == 0) { sd = find_domain(doms, nd, c, nc_total, status); tot[0] = tot[1] = tot[2] = 0; }
    __syncthreads();
    const int64_t b = cs[c], e = cs[c + 1];
    unsigned long long n3[3] = {0, 0, 0};
    if (sd.d < 0) {
        n3[1] = (unsigned long long)(e - b);
        if (threadIdx.x == 0) { counts[3 * c] = 0; counts[3 * c + 1] = e - b; counts[3 * c + 2] = 0; }
        return;
    }
    const auto mv = make_mover<Real>(doms[sd.d], dt[sd.d]);
    const int local = c - sd.first;
    bool bad = false;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        Real xi = x[i], vi = vx[i];
        int d = mv.move(xi, vi) - local;
        if (d < -1 || d > 1) { bad = true; d = d < 0 ? -1 : 1; }
        n3[d + 1]++;
    }
    if (bad) { if (atomicCAS(status, 0, TRMC_ERR_STATE) == 0) status[1] = c; }
    for (int j = 0; j < 3; ++j) {
        unsigned long long v = n3[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&tot[j], v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        counts[3 * c] = (int64_t)tot[0];
        counts[3 * c + 1] = (int64_t)tot[1];
        counts[3 * c + 2] = (int64_t)tot[2];
    }
}

// Kernel 2: new cell starts (single CTA, exclusive scan of the new counts).
__global__ void __launch_bounds__(1024) scan_kernel(const int64_t *counts, int nc, int64_t *new_start)
{
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nc; base += blockDim.x) {
        const int c = base + threadIdx.x;
        int64_t v = 0;
        if (c < nc) {
            v = counts[3 * c + 1];
            if (c > 0) v += counts[3 * (c - 1) + 2];
            if (c + 1 < nc) v += counts[3 * (c + 1)];
        }
        int64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = (lane < int(blockDim.x >> 5)) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int64_t before = carry + (warp > 0 ? wsum[warp - 1] : 0);
        if (c < nc) new_start[c] = before + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) new_start[nc] = carry;
}

// Kernel 3: stable scatter of one old cell into the new order.
template <typename Real>
__global__ void __launch_bounds__(kTT) scatter_kernel(const Real *x, const Real *vx, const Real *vy, const Real *vz,
                                                      const int64_t *cs, const trmc_domain *doms, int nd,
                                                      const double *dt, const int64_t *counts,
                                                      const int64_t *new_start, int nc_total,
                                                      Real *xo, Real *vxo, Real *vyo, Real *vzo, int *status)
{
    __shared__ CellDom sd;
    __shared__ int64_t dest[3];
    __shared__ int wcnt[3][kTT / 32];
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        sd = find_domain(doms, nd, c, nc_total, status);
        // where this cell's movers land in the new order (stable: particles from
        // the left neighbour first, then stayers, then those from the right)
        dest[2] = (c + 1 < nc_total) ? new_start[c + 1] : 0;                        // going right
        dest[1] = new_start[c] + (c > 0 ? counts[3 * (c - 1) + 2] : 0);            // staying
        dest[0] = (c > 0) ? new_start[c - 1] + (c > 1 ? counts[3 * (c - 2) + 2] : 0) + counts[3 * (c - 1) + 1] : 0;
    }
    __syncthreads();
    const int64_t b = cs[c], e = cs[c + 1];
    typename MoverT<Real>::type mv;
    int local = 0;
    if (sd.d >= 0) { mv = make_mover<Real>(doms[sd.d], dt[sd.d]); local = c - sd.first; }
    for (int64_t chunk = b; chunk < e; chunk += blockDim.x) {
        const int64_t i = chunk + threadIdx.x;
        const bool live = i < e;
        Real xi = 0, vi = 0, yi = 0, zi = 0;
        int d = 0;
        if (live) {
            xi = x[i]; vi = vx[i]; yi = vy[i]; zi = vz[i];
            if (sd.d >= 0) {
                d = mv.move(xi, vi) - local;
                d = d < -1 ? -1 : (d > 1 ? 1 : d);
            }
        }
        unsigned bal[3];
#pragma unroll
        for (int g = 0; g < 3; ++g) bal[g] = __ballot_sync(0xffffffffu, live && d == g - 1);
        if (lane == 0) {
#pragma unroll
            for (int g = 0; g < 3; ++g) wcnt[g][warp] = __popc(bal[g]);
        }
        __syncthreads();
        if (live) {
            const int g = d + 1;
            int64_t pos = dest[g];
            for (int w = 0; w < warp; ++w) pos += wcnt[g][w];
            pos += __popc(bal[g] & ((1u << lane) - 1u));
            xo[pos] = xi; vxo[pos] = vi; vyo[pos] = yi; vzo[pos] = zi;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            int64_t t = 0;
            for (int w = 0; w < nw; ++w) t += wcnt[threadIdx.x][w];
            dest[threadIdx.x] += t;
        }
        __syncthreads();
    }
}

template <typename Real>
trmc_status launch_t(trmc_ctx *ctx, trmc_state *st, const trmc_domain *doms, int32_t nd, double cfl,
                     double *dt, cudaStream_t s)
{
    const int nc = st->n_cells;
    if (ctx->tr_cells < nc) {
        if (ctx->tr_counts) cudaFree(ctx->tr_counts);
        ctx->tr_counts = nullptr;
        ctx->tr_cells = 0;
        cudaError_t e = cudaMalloc(&ctx->tr_counts, sizeof(int64_t) * 3 * size_t(nc));
        if (e != cudaSuccess) return set_error(ctx, TRMC_ERR_NOMEM, "transport scratch allocation failed");
        ctx->tr_cells = nc;
    }
    if (cfl > 0.0) {
        cfl_kernel<<<nd, 256, 0, s>>>(doms, nd, nc, st->cell_vmax2, cfl, dt, st->cell_param);
    }
    const Real *x = static_cast<const Real *>(st->x), *vx = static_cast<const Real *>(st->vx);
    count_kernel<Real><<<nc, kTT, 0, s>>>(x, vx, st->cell_start, doms, nd, nc, dt, ctx->tr_counts, ctx->status);
    scan_kernel<<<1, 1024, 0, s>>>(ctx->tr_counts, nc, st->cell_start_alt);
    scatter_kernel<Real><<<nc, kTT, 0, s>>>(x, vx, static_cast<const Real *>(st->vy), static_cast<const Real *>(st->vz),
                                            st->cell_start, doms, nd, dt, ctx->tr_counts, st->cell_start_alt, nc,
                                            static_cast<Real *>(st->x_alt), static_cast<Real *>(st->vx_alt),
                                            static_cast<Real *>(st->vy_alt), static_cast<Real *>(st->vz_alt),
                                            ctx->status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "transport launch");
    std::swap(st->x, st->x_alt);
    std::swap(st->vx, st->vx_alt);
    std::swap(st->vy, st->vy_alt);
    std::swap(st->vz, st->vz_alt);
    std::swap(st->cell_start, st->cell_start_alt);
    return TRMC_OK;
}

}  // namespace

trmc_status launch_transport(trmc_ctx *ctx, trmc_state *st, const trmc_domain *doms, int32_t nd, double cfl,
                             double *dt, cudaStream_t s)
{
    if (ctx->precision == TRMC_FP64) return launch_t<double>(ctx, st, doms, nd, cfl, dt, s);
    return launch_t<float>(ctx, st, doms, nd, cfl, dt, s);
}

}  // namespace trmc
