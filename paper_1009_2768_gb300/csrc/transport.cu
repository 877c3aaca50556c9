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
// Reservoir domains (inflow / outflow, Sec. 5.2): the first and last cell
// are ghost cells outside [x_lo, x_hi).  A particle that ends outside
// [x_lo, x_hi) is dropped; a ghost cell's "stay" count slot carries the
// number of particles its reservoir refills it with (kernel 4), so the scan
// and the scatter need no special case.
#include <utility>

#include "internal.h"
#include "trmc_device.cuh"

namespace trmc {
namespace {

constexpr int kTT = 256;   // threads per CTA (at most; the count and scatter launch fewer for small cells)
constexpr double kTwoPi = 6.283185307179586;

// GB300 has 2 FP64 lanes per SM and clock, so the FP64 mover keeps FP64
// instructions to the four roundings the method defines (x + v_x dt, and
// (x - lo) / dx as a product with the rounded reciprocal); comparisons and the
// floor use integer operations on the bit patterns.
//
// Order-preserving integer image of a double (-0.0 maps to +0.0's image).
__device__ __forceinline__ long long okey(double d)
{
    long long b = __double_as_longlong(d);
    if (b == (long long)0x8000000000000000ull) b = 0;
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll);
}

// floor(q) for 0 <= q < 2^20 from the bit pattern.  Returns false where q is
// within 2^-29 of an integer (or outside that range): there the product may
// round to the other side of the integer than the correctly rounded quotient
// it stands for, and the caller divides instead.
__device__ __forceinline__ bool bits_floor(double q, int &fl)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(q);
    if (b >> 63) return false;
    const int e = int(b >> 52) - 1023;
    if (e >= 20 || e < -52) return false;
    const unsigned long long mant = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
    unsigned long long frac;                       // fraction of q in units of 2^-52
    if (e >= 0) {
        fl = int(mant >> (52 - e));
        frac = (mant & ((1ull << (52 - e)) - 1ull)) << e;
    } else {
        fl = 0;
        frac = mant >> (-e);
    }
    const unsigned long long top = frac >> (52 - 29);
    return top != 0ull && top != (1ull << 29) - 1ull;
}

// Position update and new cell (relative to the domain's first cell, -1 if
// the particle leaves through a reservoir face), double.
struct Mover64 {
    double lo, hi, dx, inv_dx, dt;
    long long klo, khi;   // okey(lo), okey(hi)
    int nc, res;          // interior cells; reservoir domain (ghost cell first)
    __device__ __forceinline__ int move(double &x, double &vx) const
    {
        double xn = __dadd_rn(x, __dmul_rn(vx, dt));
        const long long k = okey(xn);
        if (res) {
            if (k < klo || k >= khi) return -1;
        } else if (k < klo) { xn = __dsub_rn(__dmul_rn(2.0, lo), xn); vx = -vx; }
        else if (k > khi) { xn = __dsub_rn(__dmul_rn(2.0, hi), xn); vx = -vx; }
        x = xn;
        // floor of the correctly rounded quotient (xn - lo) / dx: the product
        // with the rounded reciprocal is within |q| * 3.4e-16 of it, so their
        // floors agree unless the product lies within 2^-29 of an integer
        const double a = __dsub_rn(xn, lo);
        int c;
        if (!bits_floor(__dmul_rn(a, inv_dx), c)) {
            const double f = floor(__ddiv_rn(a, dx));
            c = (f < 0.0) ? 0 : (f > double(nc - 1) ? nc - 1 : int(f));
        }
        if (c > nc - 1) c = nc - 1;
        return c + res;
    }
};
struct Mover32 {
    float lo, hi, inv_dx, dt;
    int nc, res;
    __device__ __forceinline__ int move(float &x, float &vx) const
    {
        float xn = x + vx * dt;
        if (res) {
            if (xn < lo || xn >= hi) return -1;
        } else if (xn < lo) { xn = 2.0f * lo - xn; vx = -vx; }
        else if (xn > hi) { xn = 2.0f * hi - xn; vx = -vx; }
        x = xn;
        const float f = floorf((xn - lo) * inv_dx);
        int c = (f < 0.0f) ? 0 : (f > float(nc - 1) ? nc - 1 : int(f));
        return c + res;
    }
};
template <typename Real> struct MoverT;
template <> struct MoverT<double> { using type = Mover64; };
template <> struct MoverT<float> { using type = Mover32; };

struct CellDom {
    int d;          // domain index or -1
    int first;      // domain's first cell
};

// 16-byte vectors of particle data: four floats or two doubles.  Arrays whose
// base is 16-byte aligned and whose capacity is a multiple of the vector
// width are read one vector per thread (element g V + j of vector g): a
// cell's range then covers whole vectors, with the elements before its start
// and from its end on masked off, and no read leaves the allocation.
template <typename Real> struct Vec16;
template <> struct Vec16<float> {
    static constexpr int V = 4;
    float4 v;
    __device__ __forceinline__ float operator[](int j) const { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }
};
template <> struct Vec16<double> {
    static constexpr int V = 2;
    double2 v;
    __device__ __forceinline__ double operator[](int j) const { return j == 0 ? v.x : v.y; }
};
template <typename Real>
__device__ __forceinline__ Vec16<Real> load16(const Real *a, int64_t g)
{
    Vec16<Real> r;
    if constexpr (sizeof(Real) == 4) r.v = reinterpret_cast<const float4 *>(a)[g];
    else r.v = reinterpret_cast<const double2 *>(a)[g];
    return r;
}

__device__ __forceinline__ bool domain_ok(const trmc_domain &D, int nc_total)
{
    const bool res = D.bc == TRMC_BC_RESERVOIR;
    return D.n_cells >= (res ? 3 : 1) && D.cell_begin >= 0 && D.cell_begin <= nc_total - D.n_cells &&
           D.x_hi > D.x_lo && (D.bc == TRMC_BC_SPECULAR || (res && D.particle_mass > 0.0));
}
__device__ __forceinline__ int interior_cells(const trmc_domain &D)
{
    return D.bc == TRMC_BC_RESERVOIR ? D.n_cells - 2 : D.n_cells;
}

template <typename Real>
__device__ __forceinline__ typename MoverT<Real>::type make_mover(const trmc_domain &D, double dt);
template <>
__device__ __forceinline__ Mover64 make_mover<double>(const trmc_domain &D, double dt)
{
    Mover64 m;
    m.lo = D.x_lo; m.hi = D.x_hi; m.nc = interior_cells(D); m.dt = dt; m.res = D.bc == TRMC_BC_RESERVOIR;
    m.dx = __ddiv_rn(__dsub_rn(D.x_hi, D.x_lo), double(m.nc));
    m.inv_dx = __ddiv_rn(1.0, m.dx);
    m.klo = okey(m.lo); m.khi = okey(m.hi);
    return m;
}
template <>
__device__ __forceinline__ Mover32 make_mover<float>(const trmc_domain &D, double dt)
{
    Mover32 m;
    m.lo = float(D.x_lo); m.hi = float(D.x_hi); m.nc = interior_cells(D); m.dt = float(dt);
    m.res = D.bc == TRMC_BC_RESERVOIR;
    m.inv_dx = float(double(m.nc) / (D.x_hi - D.x_lo));
    return m;
}

// A domain's cells and mover, set up once per transport call by kernel 0, so
// that the per-cell kernels find their domain among a few integers and need
// no FP64 division (GB300: 2 FP64 lanes per SM and clock, ~400 cycles each).
struct DomMove {
    Mover64 m64;
    Mover32 m32;
    int first, n_cells, ok;
};

// Kernel 0: per domain, the CFL time step from the per-cell max |v|^2 (cfl > 0;
// otherwise dt holds the caller's steps) and the domain's mover.
__global__ void cfl_kernel(const trmc_domain *doms, int nd, int nc_total, const double *cell_vmax2, double cfl,
                           double *dt, trmc_cell_param *cell_param, DomMove *dm, int *status)
{
    __shared__ double red[kRedScratch];
    const int d = blockIdx.x;
    if (d >= nd) return;
    const trmc_domain D = doms[d];
    if (!domain_ok(D, nc_total)) {
        if (threadIdx.x == 0) {
            if (cfl > 0.0) dt[d] = 0.0;
            dm[d].ok = 0; dm[d].first = D.cell_begin; dm[d].n_cells = D.n_cells;
            if (atomicCAS(status, 0, TRMC_ERR_ARG) == 0) status[1] = d;
        }
        return;
    }
    if (cfl <= 0.0) {
        if (threadIdx.x == 0) {
            const double h = dt[d];
            dm[d].m64 = make_mover<double>(D, h); dm[d].m32 = make_mover<float>(D, h);
            dm[d].first = D.cell_begin; dm[d].n_cells = D.n_cells; dm[d].ok = 1;
        }
        return;
    }
    __shared__ double sh_h;
    // maximum on the bit patterns of the non-negative values: no FP64 instruction
    // per cell; the step itself is computed once, by thread 0
    long long vb = 0;
    for (int c0 = threadIdx.x; c0 < D.n_cells; c0 += 4 * blockDim.x) {
        long long t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = c0 + u * int(blockDim.x);
            t[u] = c < D.n_cells ? __double_as_longlong(cell_vmax2[D.cell_begin + c]) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) vb = max(vb, t[u]);
    }
    const double vm = block_max_nonneg(__longlong_as_double(vb), red);
    if (threadIdx.x == 0) {
        const double dx = __ddiv_rn(__dsub_rn(D.x_hi, D.x_lo), double(interior_cells(D)));
        const double h = (vm > 0.0) ? __ddiv_rn(__dmul_rn(cfl, dx), __dsqrt_rn(vm)) : 0.0;
        dt[d] = h;
        sh_h = h;
        dm[d].m64 = make_mover<double>(D, h); dm[d].m32 = make_mover<float>(D, h);
        dm[d].first = D.cell_begin; dm[d].n_cells = D.n_cells; dm[d].ok = 1;
    }
    __syncthreads();
    const double h = sh_h;
    if (cell_param)
        for (int c = threadIdx.x; c < D.n_cells; c += blockDim.x) cell_param[D.cell_begin + c].dt = h;
}

// Kernel 1: per old cell, how many particles go left / stay / go right.
// Particles a ghost cell is refilled with: Iround(rho dx / mass), one
// uniform (Philox tag RESERVOIR, reserved index).
__device__ __forceinline__ int64_t refill_count(const trmc_domain &D, int c, const uint64_t *cell_key,
                                                uint32_t problem_id, uint64_t seed, uint64_t step)
{
    const bool lo_side = c == D.cell_begin;
    const double *r = lo_side ? D.res_lo : D.res_hi;
    const double dx = __ddiv_rn(__dsub_rn(D.x_hi, D.x_lo), double(D.n_cells - 2));
    CellRng rng{seed, problem_id, uint64_t(c), step};
    if (cell_key) { rng.problem = cell_key[c] >> 32; rng.cell = cell_key[c] & 0xFFFFFFFFull; }
    const double want = __ddiv_rn(__dmul_rn(r[0], dx), D.particle_mass);
    const double fl = floor(want);
    const U64x4 w = rng.draw(0xFFFFFFFFull, 2, 0, TAG_RESERVOIR);
    return int64_t(fl) + ((u01(w.w[0]) < __dsub_rn(want, fl)) ? 1 : 0);
}

// Domain of cell c among the set-up records (first valid match), -1 if none.
__device__ __forceinline__ int find_dom(const DomMove *dm, int nd, int c)
{
    for (int d = 0; d < nd; ++d)
        if (dm[d].ok && c >= dm[d].first && c < dm[d].first + dm[d].n_cells) return d;
    return -1;
}
template <typename Real> __device__ __forceinline__ typename MoverT<Real>::type mover_of(const DomMove &m);
template <> __device__ __forceinline__ Mover64 mover_of<double>(const DomMove &m) { return m.m64; }
template <> __device__ __forceinline__ Mover32 mover_of<float>(const DomMove &m) { return m.m32; }

template <typename Real, bool Vec>
__global__ void __launch_bounds__(kTT) count_kernel(const Real *x, const Real *vx, const int64_t *cs,
                                                    const trmc_domain *doms, const DomMove *dm, int nd,
                                                    int64_t *counts, int *status, const uint64_t *cell_key,
                                                    uint32_t problem_id, uint64_t seed, uint64_t step,
                                                    const uint64_t *step_dev, double *cell_vmax2)
{
    __shared__ int sdom;
    __shared__ unsigned long long tot[3];
    const int c = blockIdx.x;
    if (threadIdx.x == 0) {
        sdom = find_dom(dm, nd, c);
        tot[0] = tot[1] = tot[2] = 0;
    }
    __syncthreads();
    const int dd = sdom;
    const int64_t b = cs[c], e = cs[c + 1];
    unsigned long long n3[3] = {0, 0, 0};
    if (dd < 0) {
        n3[1] = (unsigned long long)(e - b);
        if (threadIdx.x == 0) { counts[3 * c] = 0; counts[3 * c + 1] = e - b; counts[3 * c + 2] = 0; }
        return;
    }
    const auto mv = mover_of<Real>(dm[dd]);
    const int local = c - dm[dd].first;
    const bool ghost = mv.res && (local == 0 || local == dm[dd].n_cells - 1);
    bool bad = false;
    auto count = [&](Real xi, Real vi) {
        const int nl = mv.move(xi, vi);
        if (nl < 0) return;                         // left through a reservoir face
        int d = nl - local;
        if (d < -1 || d > 1 || (ghost && d == 0)) { bad = true; d = d < 0 ? -1 : 1; }
        n3[d + 1]++;
    };
    if constexpr (Vec) {
        // one 16-byte vector of x and of v_x per thread and step
        constexpr int V = Vec16<Real>::V;
        constexpr int U = 4;                        // vectors issued together
        const int64_t g0 = b / V, g1 = (e + V - 1) / V;
        for (int64_t q0 = g0 + threadIdx.x; q0 < g1; q0 += U * blockDim.x) {
            Vec16<Real> xs[U], vs[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t g = q0 + int64_t(u) * blockDim.x;
                if (g < g1) { xs[u] = load16(x, g); vs[u] = load16(vx, g); }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t g = q0 + int64_t(u) * blockDim.x;
                if (g >= g1) continue;
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const int64_t i = g * V + j;
                    if (i >= b && i < e) count(xs[u][j], vs[u][j]);
                }
            }
        }
    } else {
        constexpr int U = 4;                        // loads issued together
        for (int64_t i0 = b + threadIdx.x; i0 < e; i0 += U * blockDim.x) {
            Real xs[U], vs[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + int64_t(u) * blockDim.x;
                if (i < e) { xs[u] = x[i]; vs[u] = vx[i]; }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (i0 + int64_t(u) * blockDim.x < e) count(xs[u], vs[u]);
        }
    }
    if (ghost && threadIdx.x == 0) {                // the refill takes the "stay" slot
        n3[1] = (unsigned long long)refill_count(doms[dd], c, cell_key, problem_id, seed, step_dev ? *step_dev : step);
        if (cell_vmax2) cell_vmax2[c] = 0.0;        // the refill kernel takes the maximum over its CTAs
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
__global__ void __launch_bounds__(1024) scan_kernel(const int64_t *counts, int nc, int64_t *new_start,
                                                    int64_t capacity, int *status)
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
    if (threadIdx.x == 0) {
        new_start[nc] = carry;
        if (carry > capacity && atomicCAS(status, 0, TRMC_ERR_CAPACITY) == 0) status[1] = -1;
    }
}

// Kernel 4: refill the ghost cells of reservoir domains from their
// Maxwellians (kRefillCTAs CTAs per ghost cell, so that the two ghost cells of
// a domain occupy every SM: a ghost cell takes thousands of particles, each a
// chain of FP64 transcendentals, and GB300 has 2 FP64 lanes per SM), uniform
// positions in the cell.  The ghost cell's max |v|^2 (zeroed by kernel 1) is the maximum
// over the CTAs, taken on the bit patterns of the non-negative values.
constexpr int kRefillCTAs = 76;
template <typename Real>
__global__ void __launch_bounds__(kTT) refill_kernel(const trmc_domain *doms, int nd, int nc_total,
                                                     const int64_t *new_start, const uint64_t *cell_key,
                                                     uint32_t problem_id, uint64_t seed, uint64_t step,
                                                     const uint64_t *step_dev, Real *xo, Real *vxo, Real *vyo,
                                                     Real *vzo, int64_t capacity, double *cell_vmax2)
{
    __shared__ double red[kRedScratch];
    const int part = blockIdx.x % kRefillCTAs, gc = blockIdx.x / kRefillCTAs;
    const int d = gc >> 1, side = gc & 1;
    if (d >= nd) return;
    const trmc_domain D = doms[d];
    if (D.bc != TRMC_BC_RESERVOIR || !domain_ok(D, nc_total)) return;
    const int g = side == 0 ? D.cell_begin : D.cell_begin + D.n_cells - 1;
    const double *r = side == 0 ? D.res_lo : D.res_hi;
    const double dx = __ddiv_rn(__dsub_rn(D.x_hi, D.x_lo), double(D.n_cells - 2));
    const double x0 = side == 0 ? __dsub_rn(D.x_lo, dx) : D.x_hi;
    const double sT = sqrt(r[2]);
    const uint64_t stp = step_dev ? *step_dev : step;
    CellRng rng{seed, problem_id, uint64_t(g), stp};
    if (cell_key) { rng.problem = cell_key[g] >> 32; rng.cell = cell_key[g] & 0xFFFFFFFFull; }
    const int64_t b = new_start[g], n = new_start[g + 1] - b;
    double vm = 0.0;
    for (int64_t j = int64_t(part) * blockDim.x + threadIdx.x; j < n; j += int64_t(kRefillCTAs) * blockDim.x) {
        const U64x4 w = rng.draw(uint64_t(j), 0, 0, TAG_RESERVOIR);
        const U64x4 w2 = rng.draw(uint64_t(j), 1, 0, TAG_RESERVOIR);
        const double r1 = sqrt(-2.0 * log(u01_open(w.w[0]))), a1 = kTwoPi * u01(w.w[1]);
        const double r2 = sqrt(-2.0 * log(u01_open(w.w[2]))), a2 = kTwoPi * u01(w.w[3]);
        const Real v0 = Real(r[1] + sT * (r1 * cos(a1))), v1 = Real(sT * (r1 * sin(a1))), v2 = Real(sT * (r2 * cos(a2)));
        const Real xx = Real(__dadd_rn(x0, __dmul_rn(dx, u01(w2.w[0]))));
        if (b + j < capacity) { xo[b + j] = xx; vxo[b + j] = v0; vyo[b + j] = v1; vzo[b + j] = v2; }
        const double e0 = v0, e1 = v1, e2 = v2;
        vm = fmax(vm, __dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2)));
    }
    vm = block_max(vm, red);
    if (threadIdx.x == 0 && cell_vmax2 && vm > 0.0)
        atomicMax(reinterpret_cast<unsigned long long *>(cell_vmax2 + g), (unsigned long long)__double_as_longlong(vm));
}

// Kernel 3: stable scatter of one old cell into the new order.
template <typename Real>
__global__ void __launch_bounds__(kTT) scatter_kernel(const Real *x, const Real *vx, const Real *vy, const Real *vz,
                                                      const int64_t *cs, const DomMove *dm, int nd,
                                                      const int64_t *counts,
                                                      const int64_t *new_start, int nc_total,
                                                      Real *xo, Real *vxo, Real *vyo, Real *vzo, int *status,
                                                      int64_t capacity)
{
    __shared__ CellDom sd;
    __shared__ int64_t dest[3];
    __shared__ int wcnt[3][kTT / 32];
    __shared__ typename MoverT<Real>::type smv;
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        const int d = find_dom(dm, nd, c);
        sd = CellDom{d, d >= 0 ? dm[d].first : 0};
        if (d >= 0) smv = mover_of<Real>(dm[d]);
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
    if (sd.d >= 0) { mv = smv; local = c - sd.first; }
    // the next chunk's loads are issued before this chunk's barriers
    Real nx = 0, nv = 0, ny = 0, nz = 0;
    if (b + threadIdx.x < e) { nx = x[b + threadIdx.x]; nv = vx[b + threadIdx.x]; ny = vy[b + threadIdx.x]; nz = vz[b + threadIdx.x]; }
    for (int64_t chunk = b; chunk < e; chunk += blockDim.x) {
        const int64_t i = chunk + threadIdx.x;
        bool live = i < e;
        Real xi = nx, vi = nv, yi = ny, zi = nz;
        {
            const int64_t in = i + blockDim.x;
            if (in < e) { nx = x[in]; nv = vx[in]; ny = vy[in]; nz = vz[in]; }
        }
        int d = 0;
        if (live) {
            if (sd.d >= 0) {
                const int nl = mv.move(xi, vi);
                if (nl < 0) live = false;           // left through a reservoir face
                d = nl - local;
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
            if (pos < capacity) { xo[pos] = xi; vxo[pos] = vi; vyo[pos] = yi; vzo[pos] = zi; }
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
                     double *dt, uint64_t step, cudaStream_t s)
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
    if (ctx->tr_ndom < nd) {
        if (ctx->tr_dom) cudaFree(ctx->tr_dom);
        ctx->tr_dom = nullptr;
        ctx->tr_ndom = 0;
        cudaError_t e = cudaMalloc(&ctx->tr_dom, sizeof(DomMove) * size_t(nd));
        if (e != cudaSuccess) return set_error(ctx, TRMC_ERR_NOMEM, "transport scratch allocation failed");
        ctx->tr_ndom = nd;
    }
    DomMove *dm = static_cast<DomMove *>(ctx->tr_dom);
    cfl_kernel<<<nd, 512, 0, s>>>(doms, nd, nc, st->cell_vmax2, cfl, dt, st->cell_param, dm, ctx->status);
    const Real *x = static_cast<const Real *>(st->x), *vx = static_cast<const Real *>(st->vx);
    // one CTA per old cell, sized to the cells (measured on GB300: 64 threads
    // for cells of about 500 particles move them 11 % faster than 256, which
    // suit cells of thousands); the order the scatter writes does not depend on it
    const int64_t per_cell = st->capacity / (nc > 0 ? nc : 1);
    const int tt = ctx->transport_threads ? ctx->transport_threads
                                          : per_cell <= 1024 ? 64 : per_cell <= 4096 ? 128 : kTT;
    // 16-byte vector loads (four floats) in the count kernel where x and v_x
    // start on a 16-byte boundary and the capacity is a whole number of
    // vectors.  Measured on GB300: as fast as one float per thread on the
    // stationary shock; with doubles (two per vector) 4 % slower on the shock
    // tubes, so FP64 contexts read one double per thread
    auto a16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const bool vec = sizeof(Real) == 4 && a16(st->x) && a16(st->vx) && st->capacity % Vec16<Real>::V == 0;
    const Real *vy = static_cast<const Real *>(st->vy), *vz = static_cast<const Real *>(st->vz);
    Real *xo = static_cast<Real *>(st->x_alt), *vxo = static_cast<Real *>(st->vx_alt);
    Real *vyo = static_cast<Real *>(st->vy_alt), *vzo = static_cast<Real *>(st->vz_alt);
    if (vec)
        count_kernel<Real, true><<<nc, tt, 0, s>>>(x, vx, st->cell_start, doms, dm, nd, ctx->tr_counts, ctx->status,
                                                    st->cell_key, st->problem_id, ctx->seed, step, st->step_dev,
                                                    st->cell_vmax2);
    else
        count_kernel<Real, false><<<nc, tt, 0, s>>>(x, vx, st->cell_start, doms, dm, nd, ctx->tr_counts, ctx->status,
                                                     st->cell_key, st->problem_id, ctx->seed, step, st->step_dev,
                                                     st->cell_vmax2);
    scan_kernel<<<1, 1024, 0, s>>>(ctx->tr_counts, nc, st->cell_start_alt, st->capacity, ctx->status);
    // (the scatter reads one particle per thread: its writes, in the new order,
    // are then coalesced across the warp; with a vector per thread they were
    // four times as scattered and the scatter 50 % slower on the stationary
    // shock)
    scatter_kernel<Real><<<nc, tt, 0, s>>>(x, vx, vy, vz, st->cell_start, dm, nd, ctx->tr_counts,
                                                   st->cell_start_alt, nc, xo, vxo, vyo, vzo, ctx->status,
                                                   st->capacity);
    refill_kernel<Real><<<2 * nd * kRefillCTAs, kTT, 0, s>>>(doms, nd, nc, st->cell_start_alt, st->cell_key, st->problem_id, ctx->seed,
                                               step, st->step_dev, static_cast<Real *>(st->x_alt),
                                               static_cast<Real *>(st->vx_alt), static_cast<Real *>(st->vy_alt),
                                               static_cast<Real *>(st->vz_alt), st->capacity, st->cell_vmax2);
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
                             double *dt, uint64_t step, cudaStream_t s)
{
    if (ctx->precision == TRMC_FP64) return launch_t<double>(ctx, st, doms, nd, cfl, dt, step, s);
    return launch_t<float>(ctx, st, doms, nd, cfl, dt, step, s);
}

}  // namespace trmc
