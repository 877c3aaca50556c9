// collide.cu -- the TRMC-R collision step on sm_103a.
//
// One CTA handles one cell at a time (persistent CTAs, cells taken from a
// ticket counter).  The cell's velocities are staged in shared memory when
// they fit, otherwise in a per-CTA slab of the context's device workspace.
// Per cell, in order:
//   1. moments (FP64 block reductions): momentum, energy, mean, VHS bound
//      Sigma = (2 max|v - u|)^alpha, mu = rho Sigma, q = exp(-mu dt / eps);
//   2. split into collision sets N_0..N_m, N_{m+1} with Iround (Alg. 4.2);
//   3. tree plan, top level first: per level n, C_n = ceil((N_n + D_n)/2)
//      collisions (odd counts: fair coin between dropping one quota particle
//      and keeping a surplus output), each taking k uniform in {0..n-1}
//      (Alg. 4.1/4.3); the label histogram of level n fixes the demand D_k
//      on the levels below; leaves that cannot be served lower the depth;
//   4. roles: a pseudo-random permutation of the cell's particles picks the
//      uncollided, the leaves and the thermalised set (the "random choice");
//   5. collision waves, level 1 first, all collisions of a level in
//      parallel (Eq. Maxwell_coll, sigma from Eq. n3d, VHS acceptance of
//      Alg. 4.4); products go to their consumers or outputs through a
//      per-level permutation (the store of siblings, Sec. 4.1);
//   6. outputs replace the leaves; TRMC-RAD (Sec. 4.3) tests the relative
//      change of the indicator with the analytic Maxwellian part and, if
//      it is too large, continues the split with levels m+1..2m on the
//      thermalised set, keeping every collision already done;
//      TRMC-WB (Sec. 4.4) instead splits to m_cap, carries the length of
//      every product's tree through the waves (Eqs. def:1-3) and sends an
//      output whose tree is longer than m_max to the thermalised set;
//   7. the thermalised particles are resampled from the local Maxwellian
//      and renormalised to the exact momentum and energy they carried;
//   8. changed particles are written back (coalesced, predicated).
// FP64 contexts compute everything in double and match the CPU oracle draw
// for draw; FP32-mixed contexts store velocities and collide in float while
// moments, Sigma, q and the renormalisation stay in double.
#include <algorithm>
#include <cfloat>

#include "internal.h"
#include "trmc_device.cuh"

namespace trmc {
namespace {

constexpr int NLEV = kMC + 2;
// Levels with at most warp_level collisions are "deep": they run in one warp or
// in dependency order from precomputed records, the others by the whole CTA.
// Measured on GB300: 32 for FP64 (its collisions are slow; spread them over the
// CTA), 128 for FP32.
// Both are defaults of the context's schedule (trmc_set_collide_schedule).
constexpr int kWarpLevel64 = 32, kWarpLevel32 = 128;
constexpr int kRecordPerThread = 4;
constexpr int kPreLabels = 16;     // labels per level drawn ahead of the plan, at least
constexpr int kMaxPre = 64;        // and at most

struct Args {
    void *vx, *vy, *vz;
    const int64_t *cell_start;
    int32_t n_cells;
    int32_t *m_max;
    const trmc_cell_param *cell_param;
    const uint64_t *cell_key;
    double *cell_vmax2;
    double *cell_carry;
    uint64_t *step_dev;
    const int32_t *cell_order;
    uint32_t *cell_cost;
    uint32_t problem_id;
    uint64_t seed, step;
    trmc_collide_params prm;
    int64_t *report;
    trmc_stats *stats;
    int *status;
    unsigned int *tickets;           // [0] next cell, [1] CTAs done, [2] largest cell so far
    volatile unsigned int *n_max_host;   // NULL, or host-mapped: the last launch's largest cell
    char *slabs;
    size_t slab_bytes;
    int smem_bytes;
    int warp_level;                  // collisions of the largest level one warp takes alone
    int rec_per_thread;              // records precomputed for levels of up to this many collisions a thread
    const BigEntry *big;             // NULL, or the pre-pass's sums of this launch's large cells
    uint64_t big_stamp;              // this launch's number in big[].stamp
};

template <typename Real>
struct Sh {
    int32_t Nq[NLEV], D[NLEV], C[NLEV], O[NLEV], IB[NLEV];
    int32_t Pn[kMC + 1];
    uint64_t uSK[NLEV];              // split uniforms of the levels, u = uSK 2^-53
    U64x4 keys[NLEV];
    double red[kRedScratch];
    uint8_t lab[NLEV][kMaxPre];      // labels of the first npre[lv] collisions of each level; after
                                     // the plan, the dealing table of a level of at most 32 products
    uint8_t npre[NLEV];
    int32_t dbase[NLEV + 1], ndraws; // first draw of each level in the level-draw phase, their number
    int32_t cell, n, m, lo, m_eff, pass, n0, D0, R, npart, m_next, Dge1;
    int32_t n0_prev, D0_prev;
    int32_t scan[33], nrej;
    uint32_t coin[3];                // parity coin of level lv: bit lv (uP[lv] < 1/2)
    int32_t cand[4], cand_ok[4], cand_next;
    int32_t feas, pdrop_tot, psurp_tot, skip, cont, m_top, m_first, n0_first;
    double q, Sigma, U[3], P[3], E, S_pre, dP[3], dE, dS, Pp[3], Ep, Sp, carry[4], Pt[3], Et, msc[4];
    double alpha, dt, eps, rho_scale;
    uint64_t problem, lcell;
    U64x4 keyP0;                     // key of the pass's role permutation
    // Velocities being changed: with `full` every particle staged, Vc[slot];
    // otherwise only the changed ones (pass-0 ranks from n0 on), compact,
    // Vc[rank - n0].  [3][nVc]
    Real *Vc;
    int32_t nVc, full;
    uint32_t *flags;                 // staged whole: the changed slots (the write-back is coalesced)
    int32_t *inv0;                   // pass 0: slot of each rank (the ranks from n0 on are filled)
    int32_t *posA[2];                // passes >= 1: position in Vc of each rank (ping-pong between passes)
    int32_t *Mt, *St;
    Real *IBuf, *OBuf;
    double *ILBuf, *OLBuf;           // TRMC-WB: tree length of every consumer slot / output
    // the recorded levels (the deep ones and those of at most a few collisions
    // per thread) in ascending order, the offset of their collisions in the
    // per-collision records, and the records:
    // exclusive label prefix per level (triangular rows), input and output
    // locations, acceptance threshold xi*Sigma and scattering direction
    int32_t WL[NLEV], WB[NLEV + 1], nWL;
    // the tail: deep levels above the highest level of more than warp_level
    // collisions (LB); its records from index tail0 run in dependency order:
    // prodOf maps a tail consumer slot (from IB[LB + 1]) to the record that
    // fills it, done holds the round in which a record ran (0: not yet)
    int32_t LB, tail0, ntail, tailbase;
    int32_t *prodOf, *done;
    int32_t *LP;
    int2 *psrc, *pdst;
    Real *prnd;
    int32_t *ext;                    // TRMC-WB: slots of rejected outputs, appended to the pool
    char *smem_rest, *slab_rest;
    char *slab_hi;                   // end of the slab bytes this cell wrote (discarded after it)
    size_t smem_rest_cap, slab_rest_cap;
    char *pass_smem, *pass_slab;
    size_t pass_smem_cap, pass_slab_cap;
};

__device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~size_t(15); }
__device__ __forceinline__ int tri(int n) { return (n * (n - 1)) >> 1; }

// Bump allocator over two arenas: shared memory first, then the slab.
__device__ __forceinline__ void *take(char *&smem, size_t &scap, char *&slab, size_t &gcap, size_t bytes)
{
    bytes = al16(bytes);
    if (bytes <= scap) { void *p = smem; smem += bytes; scap -= bytes; return p; }
    if (bytes <= gcap) { void *p = slab; slab += bytes; gcap -= bytes; return p; }
    return nullptr;
}

// Exclusive prefix count of a per-thread flag over the CTA, in thread order;
// returns the CTA total.  Every thread of the CTA must call it.
__device__ __forceinline__ int block_flag_scan(bool flag, int &excl, int32_t *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) scratch[warp] = __popc(b);
    __syncthreads();
    if (warp == 0) {
        int v = lane < nw ? scratch[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane < nw) scratch[lane] = v;
    }
    __syncthreads();
    excl = (warp ? scratch[warp - 1] : 0) + __popc(b & ((1u << lane) - 1u));
    const int total = scratch[nw - 1];
    __syncthreads();
    return total;
}

// a < RN(sqrt(g2)) for a >= 0, g2 >= 0, given a2 = fl(a a), decided on the
// squares and exactly as the comparison with the correctly rounded square
// root: more than 4 units apart in the last place (the bit patterns of
// non-negative doubles order like their values), a^2 and g2 are on the sides
// they show, and a is more than an ulp away from sqrt(g2); only nearer than
// that is the square root taken.  Hard-sphere acceptance (Alg. 4.4) then costs
// one FP64 multiply instead of a square root for every rejected collision.
__device__ __forceinline__ bool lt_sqrt(double a, double a2, double g2)
{
    const long long d = __double_as_longlong(a2) - __double_as_longlong(g2);
    if (d < -4) return true;
    if (d > 4) return false;
    return a < sqrt(g2);
}

// ---- Iround of the split in integer arithmetic -------------------------------
// Alg. 4.2 gives level n the count Iround(q R), R the particles not yet
// placed, and the FP64 reference evaluates it as x = fl(q R) (round to
// nearest, ties to even), then floor(x) + [u < x - floor(x)] with the level's
// uniform u = K 2^-53.  The same value from the bits of q: the exact product
// M R of q's 53-bit significand and R (at most 84 bits), rounded to 53 bits
// like the FP64 multiply, then the integer part and the fraction compared
// with K, all exact.  q is a probability (0 <= q <= 1) and 1 <= R < 2^31.
// This keeps the sequential split off GB300's FP64 pipe (2 lanes/clk/SM).
__device__ __forceinline__ int iround_q(uint64_t qb, uint32_t R, uint64_t K)
{
    const uint32_t E = uint32_t(qb >> 52) & 0x7FFu;
    if (E == 0) return (qb != 0 && K == 0) ? 1 : 0;      // q = 0, or subnormal: 0 <= x < 2^-53
    if (E >= 1023) return int(R);                          // q = 1: x = R
    const uint64_t M = (qb & ((1ull << 52) - 1ull)) | (1ull << 52);
    const uint64_t lo = M * uint64_t(R), hi = __umul64hi(M, uint64_t(R));
    const int L = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);   // bits of M R
    int s = L - 53;                                        // bits rounded off, 0..31
    uint64_t X = lo;
    if (s > 0) {
        X = (lo >> s) | (hi << (64 - s));
        const uint64_t dropped = lo & ((1ull << s) - 1ull), half = 1ull << (s - 1);
        if (dropped > half || (dropped == half && (X & 1ull))) {
            if (++X == (1ull << 53)) { X = 1ull << 52; ++s; }
        }
    }
    const int d = 1075 - int(E) - s;                       // x = X 2^-d, d >= 22
    const uint64_t fl = d < 64 ? (X >> d) : 0ull;
    const uint64_t Fr = d < 64 ? (X & ((1ull << d) - 1ull)) : X;   // x - floor(x) = Fr 2^-d
    bool up;
    if (d <= 53) up = K < (Fr << (53 - d));                // K 2^-53 < Fr 2^-d
    else if (Fr == 0) up = false;
    else up = (d - 53 >= 64) ? (K == 0) : (K <= ((Fr - 1ull) >> (d - 53)));   // K 2^(d-53) <= Fr - 1
    return int(fl) + (up ? 1 : 0);
}

// ---- FP64 angles and logarithms of the 53-bit uniforms ----------------------
// GB300 issues FP64 at 2 lanes per SM and clock, and every FP64 instruction of
// a collision or a Maxwellian sample counts.  These evaluate sin/cos(2 pi u)
// and ln u for the draws' uniforms from correctly rounded tables
// (fp64_tables.inc, written by gen_tables.py) with short series, in about 18
// and 14 FP64 instructions, to within 2 ulp (checked against sincospi and log
// by trmc_fp64_selftest).
#include "fp64_tables.inc"

__device__ __forceinline__ double exact_small(uint64_t v)       // v < 2^52, exactly
{
    return __longlong_as_double((long long)(0x4330000000000000ull | v)) - 4503599627370496.0;
}

// u = k 2^-53, 0 <= k < 2^53: the top 8 bits of k pick a = 2 pi i / 256, the
// other 45 give t = 2 pi (u - i / 256) in [0, 2 pi / 256); the addition
// formulas combine sin a, cos a with the Taylor series of sin t and cos t - 1
// (the first omitted terms, t^9 / 9! and t^10 / 10!, are below 1e-20).  All of
// it runs in 64-bit fixed point on the integer units (t, sin t and 1 - cos t
// scaled by 2^64, the table by 2^62; every product keeps its high 64 bits), so
// the only FP64 instructions are the two conversions at the end.  Absolute
// error below 2^-59 before the conversions, which round to nearest.
__device__ __forceinline__ void sincos_2pi(uint64_t k, double &s, double &c)
{
    const int i = int(k >> 45);
    const uint64_t T = __umul64hi((k & ((1ull << 45) - 1ull)) << 16, kQ2Pi59);   // t 2^64
    const uint64_t T2 = __umul64hi(T, T);                                          // t^2 2^64
    // sin t = t - t^3 (1/6 - t^2 (1/120 - t^2 / 5040))
    uint64_t p = kQInv120 - __umul64hi(T2, kQInv5040);
    p = kQInv6 - __umul64hi(T2, p);
    const long long SN = (long long)(T - __umul64hi(__umul64hi(T2, T), p));
    // 1 - cos t = t^2 (1/2 - t^2 (1/24 - t^2 (1/720 - t^2 / 40320)))
    uint64_t q = kQInv720 - __umul64hi(T2, kQInv40320);
    q = kQInv24 - __umul64hi(T2, q);
    q = (1ull << 63) - __umul64hi(T2, q);
    const long long CM = (long long)__umul64hi(T2, q);
    const long long S = kSinCos256Q62[i][0], C = kSinCos256Q62[i][1];
    s = double(S - __mul64hi(S, CM) + __mul64hi(C, SN)) * 0x1p-62;
    c = double(C - __mul64hi(C, CM) - __mul64hi(S, SN)) * 0x1p-62;
}

// Square root of a double x >= 0 on the integer units: x = m 2^E with E even
// and m < 2^54, z = m 2^-54 in [1/4, 1); 1/sqrt(z) is seeded by the float unit's
// reciprocal square root (about 22 bits) and refined by two Newton steps
// y (3 - z y^2) / 2 in 64-bit fixed point; sqrt(z) = z y is rounded to 53
// bits and given the exponent 26 + E / 2.  Within 0.51 ulp (faithful; checked
// against sqrt by trmc_fp64_selftest).  Zero, subnormal, infinite and NaN
// inputs go to sqrt.
__device__ __forceinline__ double sqrt_pos(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ef = int(b >> 52);                     // sign bit clear for x >= 0
    if (ef == 0 || ef >= 0x7FF) return sqrt(x);
    int E = ef - 1075;
    unsigned long long m = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
    if (E & 1) { m <<= 1; E -= 1; }
    const unsigned long long X = m << 10;           // z 2^64, in [2^62, 2^64)
    const float y0 = rsqrtf(__uint2float_rn(unsigned(X >> 40)) * 0x1p-24f);
    const unsigned yb = __float_as_uint(y0);         // y0 in (1, 2]
    unsigned long long Y = (unsigned long long)((yb & 0x7FFFFFu) | 0x800000u) << (39 + int(yb >> 23) - 127);
#pragma unroll
    for (int it = 0; it < 2; ++it) {                // Y = y 2^62
        const unsigned long long zy2 = __umul64hi(X, __umul64hi(Y, Y));        // z y^2 2^60
        Y = __umul64hi(Y, ((3ull << 60) - zy2) << 2) << 1;
    }
    const unsigned long long S = __umul64hi(X, Y);   // sqrt(z) 2^62
    const unsigned long long bits = ((unsigned long long)(1023 + 26 + (E >> 1) - 1) << 52) + ((S + 256ull) >> 9);
    return __longlong_as_double((long long)bits);
}

// ln u, u = k 2^-53, 1 <= k <= 2^53: u = 2^(e - 52) (m / 2) with m in [1, 2),
// m = T_j (1 + t) with T_j = 1 + j / 128 from the top 7 fraction bits and
// t in [0, 1/128); ln u = (e - 52) ln 2 + ln(T_j / 2) + ln(1 + t), all terms
// of one sign but the small last one, with ln(1 + t) by its series to t^8.
// For u >= 1 - 1/128 the series of ln(1 - d) in the exact d = 1 - u keeps
// the relative accuracy.
__device__ __forceinline__ double log_u53(uint64_t k)
{
    if (k >= (1ull << 53) - (1ull << 46)) {
        const double d = exact_small((1ull << 53) - k) * 0x1p-53;
        const double p = fma(d, fma(d, fma(d, fma(d, fma(d, fma(d, 1.0 / 8.0, 1.0 / 7.0), 1.0 / 6.0), 1.0 / 5.0),
                                                 1.0 / 4.0), 1.0 / 3.0), 0.5);
        return -fma(d * d, p, d);
    }
    const int e = 63 - __clzll((long long)k);
    const uint64_t frac = (k << (52 - e)) & ((1ull << 52) - 1ull);
    const int j = int(frac >> 45);
    const double t = exact_small(frac & ((1ull << 45) - 1ull)) * kLnT128[j][1];
    const double p = fma(t, fma(t, fma(t, fma(t, fma(t, fma(t, -1.0 / 8.0, 1.0 / 7.0), -1.0 / 6.0), 1.0 / 5.0),
                                             -1.0 / 4.0), 1.0 / 3.0), -0.5);
    const double l1 = fma(t * t, p, t);
    const double ne = double(e - 52);
    return fma(ne, kLn2[0], fma(ne, kLn2[1], kLnT128[j][0] + l1));
}

template <typename Real> struct Math;
template <> struct Math<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt_pos(x); }
    static __device__ __forceinline__ double pow_(double x, double a) { return pow(x, a); }
    static __device__ __forceinline__ double uni(uint64_t w) { return u01(w); }
    // sin / cos of 2 pi u from the 53-bit uniform's bits, in fixed point
    // (sincos_2pi above; within 2 ulp of CUDA's sincospi(2u))
    static __device__ __forceinline__ void angle(uint64_t w, double &s, double &c) { sincos_2pi(w >> 11, s, c); }
    static __device__ __forceinline__ void normals(const U64x4 &w, double &z0, double &z1, double &z2)
    {
        const double r1 = sqrt(-2.0 * log_u53((w.w[0] >> 11) + 1));
        const double r2 = sqrt(-2.0 * log_u53((w.w[2] >> 11) + 1));
        double s1, c1, s2, c2;
        sincos_2pi(w.w[1] >> 11, s1, c1);
        sincos_2pi(w.w[3] >> 11, s2, c2);
        z0 = r1 * c1;
        z1 = r1 * s1;
        z2 = r2 * c2;
    }
};
template <> struct Math<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float pow_(float x, float a) { return powf(x, a); }
    static __device__ __forceinline__ float uni(uint64_t w) { return u01f(w); }
    static __device__ __forceinline__ void angle(uint64_t w, float &s, float &c) { sincospif(2.0f * u01f(w), &s, &c); }
    static __device__ __forceinline__ void normals(const U64x4 &w, float &z0, float &z1, float &z2)
    {
        const float r1 = sqrtf(-2.0f * logf(u01f_open(w.w[0])));
        const float r2 = sqrtf(-2.0f * logf(u01f_open(w.w[2])));
        float s1, c1, s2, c2;
        sincospif(2.0f * u01f(w.w[1]), &s1, &c1);
        sincospif(2.0f * u01f(w.w[3]), &s2, &c2);
        z0 = r1 * c1;
        z1 = r1 * s1;
        z2 = r2 * c2;
        (void)s2;
    }
};

// Per-thread partial sums of particle quantities.  In FP64 contexts they are
// plain double sums.  In FP32-mixed contexts they are compensated float sums
// (TwoSum, with squares split exactly by an FMA), about 48 significant bits,
// so no per-particle work lands on GB300's FP64 pipe (2 lanes/clk/SM); the
// partials are combined in FP64 across the warp and the block.
template <typename Real> struct Sum;
template <> struct Sum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ void add_sq3(double x, double y, double z) { s += x * x + y * y + z * z; }
    __device__ __forceinline__ double get() const { return s; }
};
template <> struct Sum<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = hi + x, bp = t - hi;
        lo += (hi - (t - bp)) + (x - bp);
        hi = t;
    }
    __device__ __forceinline__ void add_sq(float x)
    {
        const float p = x * x;
        add(p);
        lo += fmaf(x, x, -p);
    }
    __device__ __forceinline__ void sub_sq(float x)
    {
        const float p = x * x;
        add(-p);
        lo -= fmaf(x, x, -p);
    }
    __device__ __forceinline__ void add_sq3(float x, float y, float z) { add_sq(x); add_sq(y); add_sq(z); }
    __device__ __forceinline__ void sub_sq3(float x, float y, float z) { sub_sq(x); sub_sq(y); sub_sq(z); }
    __device__ __forceinline__ double get() const { return double(hi) + double(lo); }
};

// ---- canonical sums ---------------------------------------------------------
// A per-cell sum over an index range [0, N) (particles, leaves, thermalised
// ranks) is defined independently of the CTA size: 256 virtual lanes, lane v
// adding the terms of indices v, v + 256, v + 512, ... in increasing order;
// 8 virtual warps of 32 consecutive lanes, each reduced by a xor butterfly
// (offsets 16, 8, 4, 2, 1); the 8 warp totals added as
// ((w0 + w1) + (w2 + w3)) + ((w4 + w5) + (w6 + w7)).  A CTA of bs threads
// (bs in {32, 64, 128, 256}) runs virtual warps warp, warp + bs/32, ... one
// after the other, so every total, and every decision taken from it (the
// bound Sigma, q, the split), has the same bits for every launch shape.
constexpr int kVW = 8;

// Reduce the first K partial sums of virtual warp vw (every lane of the warp
// calls it, K <= 16) and store the totals at scratch[vw * K + j].  In FP64
// the values are reduce-scattered: at each of the first log2(P) butterfly
// steps (P = K rounded up to a power of two) a lane keeps half of its values
// and adds its partner's copies of them, P - 1 + log2(32/P) FP64 adds instead
// of 5K (GB300 issues FP64 at 2 lanes/clk/SM).  Each total is the value a
// plain xor butterfly gives (a + b = b + a at every step).
template <int K, int N>
__device__ __forceinline__ void vw_put(const Sum<double> (&v)[N], double *scratch, int vw)
{
    static_assert(K >= 1 && K <= 16 && K <= N, "vw_put handles 1..16 values");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int P = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : 16, G = 32 / P;
    const int lane = threadIdx.x & 31;
    double t[P];
#pragma unroll
    for (int i = 0; i < P; ++i) t[i] = i < K ? v[i].s : 0.0;
    int idx = 0;
#pragma unroll
    for (int h = P / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double send = up ? t[i] : t[i + h], keep = up ? t[i + h] : t[i];
            t[i] = keep + __shfl_xor_sync(FULL, send, o);
        }
        if (up) idx += h;
    }
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) t[0] += __shfl_xor_sync(FULL, t[0], o);
    if ((lane & (G - 1)) == 0 && idx < K) scratch[vw * K + idx] = t[0];
}

// The same for compensated float partials, added as float pairs (ff_add is
// symmetric in its operands, so the butterfly is canonical too).
template <int K, int N>
__device__ __forceinline__ void vw_put(const Sum<float> (&v)[N], double *scratch, int vw)
{
    static_assert(K >= 1 && K <= 16 && K <= N, "vw_put handles 1..16 values");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int P = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : 16, G = 32 / P;
    const int lane = threadIdx.x & 31;
    float th[P], tl[P];
#pragma unroll
    for (int i = 0; i < P; ++i) { th[i] = i < K ? v[i].hi : 0.0f; tl[i] = i < K ? v[i].lo : 0.0f; }
    int idx = 0;
#pragma unroll
    for (int h = P / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float sh_ = up ? th[i] : th[i + h], sl_ = up ? tl[i] : tl[i + h];
            float kh = up ? th[i + h] : th[i], kl = up ? tl[i + h] : tl[i];
            ff_add(kh, kl, __shfl_xor_sync(FULL, sh_, o), __shfl_xor_sync(FULL, sl_, o));
            th[i] = kh; tl[i] = kl;
        }
        if (up) idx += h;
    }
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1)
        ff_add(th[0], tl[0], __shfl_xor_sync(FULL, th[0], o), __shfl_xor_sync(FULL, tl[0], o));
    if ((lane & (G - 1)) == 0 && idx < K) reinterpret_cast<float2 *>(scratch)[vw * K + idx] = make_float2(th[0], tl[0]);
}

// The 8 virtual-warp totals of K values (stored by vw_put) combined in the
// fixed tree; every thread gets the totals and, with a divisor (K <= 8), the
// totals divided by it.  Every thread of the CTA must call it.
template <typename Real, int K>
__device__ __forceinline__ void vw_total(double *scratch, double (&out)[K], double div = 0.0, double *quot = nullptr)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (warp == 0 && lane < K) {
        double s;
        if constexpr (sizeof(Real) == 8) {
            const double *g = scratch + lane;
            s = ((g[0] + g[K]) + (g[2 * K] + g[3 * K])) + ((g[4 * K] + g[5 * K]) + (g[6 * K] + g[7 * K]));
        } else {
            const float2 *g = reinterpret_cast<const float2 *>(scratch) + lane;
            float h[4], l[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                h[p] = g[2 * p * K].x; l[p] = g[2 * p * K].y;
                ff_add(h[p], l[p], g[(2 * p + 1) * K].x, g[(2 * p + 1) * K].y);
            }
            ff_add(h[0], l[0], h[1], l[1]);
            ff_add(h[2], l[2], h[3], l[3]);
            ff_add(h[0], l[0], h[2], l[2]);
            s = double(h[0]) + double(l[0]);
        }
        scratch[256 + lane] = s;
        if (quot && K <= 8) scratch[264 + lane] = s / div;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < K; ++j) out[j] = scratch[256 + j];
    if (quot && K <= 8) {
#pragma unroll
        for (int j = 0; j < K; ++j) quot[j] = scratch[264 + j];
    }
}

// One canonical sum (stored by vw_put<1>) and one maximum of non-negative
// values (as an ordered integer key, order-free) over the CTA.
template <typename Real>
__device__ __forceinline__ void vw_total_max(double *scratch, long long key, double &sum, long long &mkey)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(FULL, key, o));
    long long *rk = reinterpret_cast<long long *>(scratch);
    if (lane == 0) rk[32 + warp] = key;
    double s[1];
    vw_total<Real, 1>(scratch, s);            // its first barrier also publishes the keys
    sum = s[0];
    long long m = rk[32];
    for (int w = 1; w < nw; ++w) m = max(m, rk[32 + w]);
    mkey = m;
    __syncthreads();
}

// |v|^2 and the adaptive indicator in the working precision
template <typename Real>
__device__ __forceinline__ Real indicator_r(Real x, Real y, Real z, Real Ux, int ind)
{
    if (ind == TRMC_IND_M4) {
        const Real e = x * x + y * y + z * z;
        return e * e;
    }
    const Real d = x - Ux;
    return d * d;
}

__device__ __forceinline__ double indicator(double x, double y, double z, const double U[3], int ind)
{
    if (ind == TRMC_IND_M4) {
        const double e = x * x + y * y + z * z;
        return e * e;
    }
    const double d = x - U[0];
    return d * d;
}

__device__ __forceinline__ void raise_status(int *status, int code, int cell)
{
    if (atomicCAS(status, 0, code) == 0) status[1] = cell;
}

// One cell, by the whole CTA; returns the thread's collision counts
// (collisions, dummy, exceed).
// Mode kWhole: the cell is staged whole, in shared memory, or in the CTA's
// slab when it does not fit.  Mode kDual: a cell that fits in shared memory is
// staged whole, a larger one compact (only the particles that change).  The
// two modes are separate kernels: the compact path costs the whole path a few
// per cent in registers and code size, so a launch takes it only when it has
// a cell too large for shared memory.
// TV: the truncation the instantiation serves -- TRMC-RAD with the P_xx or
// the M4 indicator (Sec. 4.3), TRMC-WB (Sec. 4.4), or a fixed or unlimited
// depth -- so that a kernel carries none of the other truncations' code in
// its hot loops: on GB300 the smaller code runs 5-10 % faster (fewer
// instruction-cache misses).
enum { kWhole = 0, kDual = 1 };
enum { kPlain = 0, kRadPxx = 1, kRadM4 = 2, kWb = 3 };
struct Counts { int c[3]; };

template <typename Real, int Mode, int TV>
__device__ __forceinline__ Counts process_cell(const Args &a, uint64_t step, Sh<Real> &sh, unsigned char *dsm,
                                               char *slab, int cell)
{
    const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31;
    constexpr bool kRad = TV == kRadPxx || TV == kRadM4;
    constexpr int kInd = TV == kRadM4 ? TRMC_IND_M4 : TRMC_IND_PXX;
    int cnt[3] = {0, 0, 0};
    Real *gx = static_cast<Real *>(a.vx), *gy = static_cast<Real *>(a.vy), *gz = static_cast<Real *>(a.vz);
    const int64_t base = a.cell_start[cell];
    const int n = int(a.cell_start[cell + 1] - base);
    // the input-independent part of a level's collisions (draw, threshold,
    // direction) is computed up front for every level of at most rec_max
    // collisions, a few per thread: there it takes latency off the level's
    // wave; bigger levels keep every thread busy and compute it in place
    const int rec_max = max(a.warp_level, a.rec_per_thread * bs);
    const trmc_collide_params &prm = a.prm;

    if (tid == 0) {
        sh.cell = cell;
        sh.n = n;
        if (a.cell_param) {
            const trmc_cell_param cp = a.cell_param[cell];
            sh.eps = cp.eps; sh.dt = cp.dt; sh.rho_scale = cp.rho_scale; sh.alpha = cp.alpha;
        } else {
            sh.eps = prm.eps; sh.dt = prm.dt; sh.rho_scale = prm.rho_scale; sh.alpha = prm.alpha;
        }
        if (a.cell_key) { sh.problem = a.cell_key[cell] >> 32; sh.lcell = a.cell_key[cell] & 0xFFFFFFFFull; }
        else { sh.problem = a.problem_id; sh.lcell = uint64_t(cell); }
        int m0 = prm.trunc == TRMC_TRUNC_FIXED ? prm.m_fixed
                 : kRad ? a.m_max[cell] : prm.m_cap;
        if (m0 < 1) m0 = 1;
        if (m0 > prm.m_cap) m0 = prm.m_cap;
        sh.m = m0; sh.m_next = m0; sh.m_first = m0; sh.lo = 0; sh.pass = 0; sh.npart = n; sh.skip = 0;
        sh.feas = sh.pdrop_tot = sh.psurp_tot = 0;
        sh.n0_prev = 0; sh.D0_prev = 0; sh.nrej = 0;
        sh.dP[0] = sh.dP[1] = sh.dP[2] = 0.0; sh.dE = 0.0; sh.dS = 0.0;
        for (int j = 0; j < 4; ++j) sh.carry[j] = a.cell_carry ? a.cell_carry[4 * int64_t(cell) + j] : 0.0;
        // persistent layout: a cell whose particles fit in shared memory with
        // the slot table is staged whole (Vc, then inv0); a larger one keeps
        // only inv0 and stages the particles that change once pass 0 has
        // planned (the later passes' position tables follow when needed)
        char *smem = reinterpret_cast<char *>(dsm);
        size_t scap = size_t(a.smem_bytes);
        char *gs = slab;
        size_t gcap = a.slab_bytes;
        const size_t pv = al16(3 * size_t(n) * sizeof(Real)), pb = al16(4 * size_t(n));
        const size_t pf = al16(4 * size_t((n + 31) / 32));
        sh.Vc = nullptr; sh.nVc = 0; sh.flags = nullptr; sh.full = 1;
        char *p = nullptr;
        if (pv + pf + pb <= scap) { p = smem; smem += pv + pf + pb; scap -= pv + pf + pb; }
        else if (Mode == kWhole) {
            if (pv + pf + pb <= gcap) { p = gs; gs += pv + pf + pb; gcap -= pv + pf + pb; }
            else sh.skip = 1;
        } else {
            sh.full = 0;
            if (pb <= scap) { p = smem; smem += pb; scap -= pb; }
            else if (pb <= gcap) { p = gs; gs += pb; gcap -= pb; }
            else sh.skip = 1;
        }
        if (p && sh.full) {
            sh.nVc = n;
            sh.Vc = reinterpret_cast<Real *>(p);
            sh.flags = reinterpret_cast<uint32_t *>(p + pv);
            p += pv + pf;
        }
        sh.inv0 = reinterpret_cast<int32_t *>(p);
        sh.smem_rest = smem; sh.smem_rest_cap = scap; sh.slab_rest = gs; sh.slab_rest_cap = gcap;
        sh.slab_hi = gs;
    }
    __syncthreads();
    if (n < 2 || sh.skip) {
        if (tid == 0) {
            if (sh.skip) {
                raise_status(a.status, TRMC_ERR_CAPACITY, cell);
                if (a.stats) atomicAdd(&a.stats->capacity_skips, 1ull);
            }
            if (a.report) {
                int64_t *r = a.report + int64_t(cell) * TRMC_REPORT_LEN;
                for (int j = 0; j < TRMC_REPORT_LEN; ++j) r[j] = 0;
                r[0] = n;
                r[4] = kRad ? sh.m : 0;
                r[6] = n;
            }
        }
        if (a.cell_vmax2 && !sh.skip) {
            double vm = 0.0;
            for (int i = tid; i < n; i += bs) {
                const double x = double(gx[base + i]), y = double(gy[base + i]), z = double(gz[base + i]);
                vm = fmax(vm, __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
            }
            vm = block_max_nonneg(vm, sh.red);
            if (tid == 0) a.cell_vmax2[cell] = vm;
        }
        return Counts{{cnt[0], cnt[1], cnt[2]}};
    }
    // the cell's random stream, rebuilt at each draw from shared memory (four
    // 64-bit values held across the whole cell would cost registers)
    auto rng = [&]() { return CellRng{a.seed, sh.problem, sh.lcell, step}; };

    // ---- 1. stage + moments -------------------------------------------------
    // (the indicator sums only for TRMC-RAD; the speed bound only for VHS; on
    // GB300 every FP64 instruction counts, so maxima of non-negative doubles
    // are taken on their bit patterns)
    {
        const bool rad = kRad;
        const bool need_m4 = rad && kInd == TRMC_IND_M4, need_pxx = rad && kInd == TRMC_IND_PXX;
        const bool need_d2 = sh.alpha != 0.0;
        // the particles are read from global memory and, for a cell staged
        // whole, stored in shared memory (a larger cell stages the changed ones
        // once the plan names them); the sums run over the canonical virtual
        // warps (for 256 threads one per warp)
        const int nw = bs >> 5, warp = tid >> 5;
        const bool full = Mode == kWhole || sh.full;
        Real *Vx = sh.Vc, *Vy = sh.Vc + n, *Vz = sh.Vc + 2 * n;
        constexpr int U = 4;      // loads issued together, ahead of the sums they feed
        // a large cell not staged whole: its virtual warps' partial sums, when
        // the pre-pass of this launch made them (the same values), else here
        const BigEntry *pre = nullptr;
        if (Mode == kDual && !full && a.big && n >= kBigCell) {
            const BigEntry *e = a.big + cell % kBigSlots;
            if (e->cell == cell && e->stamp == a.big_stamp) pre = e;
        }
        if (pre)
            for (int j = tid; j < kVW * (need_m4 ? 5 : 4); j += bs) sh.red[j] = pre->part[j];
        for (int vw = warp; !pre && vw < kVW; vw += nw) {
            Sum<Real> acc[5];
            for (int i0 = 32 * vw + lane; i0 < n; i0 += U * 32 * kVW) {
                Real x[U], y[U], z[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * 32 * kVW;
                    if (i < n) { x[u] = gx[base + i]; y[u] = gy[base + i]; z[u] = gz[base + i]; }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * 32 * kVW;
                    if (i < n) {
                        if (full) { Vx[i] = x[u]; Vy[i] = y[u]; Vz[i] = z[u]; }
                        acc[0].add(x[u]); acc[1].add(y[u]); acc[2].add(z[u]);
                        acc[3].add_sq3(x[u], y[u], z[u]);
                        if (need_m4) {
                            const Real e = x[u] * x[u] + y[u] * y[u] + z[u] * z[u];
                            acc[4].add(e * e);
                        }
                    }
                }
            }
            if (need_m4) vw_put<5>(acc, sh.red, vw);
            else vw_put<4>(acc, sh.red, vw);
        }
        if (full)
            for (int w = tid; w < (n + 31) >> 5; w += bs) sh.flags[w] = 0u;     // change flags, set after the plan
        // totals, and the mean velocity (warp 0 divides, once per cell)
        double s[5] = {0, 0, 0, 0, 0}, su[5];
        if (need_m4) {
            vw_total<Real, 5>(sh.red, s, double(n), su);
        } else {
            double s4[4], su4[4];
            vw_total<Real, 4>(sh.red, s4, double(n), su4);
            for (int j = 0; j < 4; ++j) { s[j] = s4[j]; su[j] = su4[j]; }
            su[4] = 0.0;
        }
        const double U0 = su[0], U1 = su[1], U2 = su[2];
        const Real u0 = Real(U0), u1 = Real(U1), u2 = Real(U2);
        Real d2 = 0;
        long long d2b = 0;
        double t[1] = {0.0};
        double dmax = 0.0;
        if (need_d2 || need_pxx) {
            // a second pass over the cell: from shared memory, or, for a cell
            // not staged whole, from L2 (it was just read)
            for (int vw = warp; vw < kVW; vw += nw) {
                Sum<Real> pxx[1];
                auto dev = [&](Real x, Real y, Real z) {
                    const Real ax = x - u0, ay = y - u1, az = z - u2;
                    if (need_d2) {
                        const Real q = ax * ax + ay * ay + az * az;
                        if constexpr (sizeof(Real) == 8) d2b = max(d2b, __double_as_longlong(q));
                        else d2 = fmaxf(d2, q);
                    }
                    if (need_pxx) pxx[0].add(ax * ax);
                };
                if (full) {
                    for (int i = 32 * vw + lane; i < n; i += 32 * kVW) dev(Vx[i], Vy[i], Vz[i]);
                } else {
                    constexpr int U = 2;
                    for (int i0 = 32 * vw + lane; i0 < n; i0 += U * 32 * kVW) {
                        Real x[U], y[U], z[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int i = i0 + u * 32 * kVW;
                            if (i < n) { x[u] = gx[base + i]; y[u] = gy[base + i]; z[u] = gz[base + i]; }
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            if (i0 + u * 32 * kVW < n) dev(x[u], y[u], z[u]);
                    }
                }
                vw_put<1>(pxx, sh.red, vw);
            }
            if constexpr (sizeof(Real) == 4) d2b = (long long)__float_as_int(d2);
            long long mk;
            vw_total_max<Real>(sh.red, d2b, t[0], mk);
            if constexpr (sizeof(Real) == 8) dmax = __longlong_as_double(mk);
            else dmax = double(__int_as_float(int(mk)));
        }
        if (tid == 0) {
            sh.P[0] = s[0]; sh.P[1] = s[1]; sh.P[2] = s[2]; sh.E = s[3];
            sh.U[0] = U0; sh.U[1] = U1; sh.U[2] = U2;
            double Sigma = 1.0;
            if (sh.alpha != 0.0) {
                const double g = 2.0 * sqrt(dmax);
                Sigma = (sh.alpha == 1.0) ? g : pow(g, sh.alpha);
            }
            sh.Sigma = Sigma;
            const double rho = double(n) * sh.rho_scale;
            const double mu = rho * Sigma;
            sh.q = exp(-(mu * sh.dt) / sh.eps);
            sh.S_pre = need_m4 ? su[4] : t[0] / double(n);
        }
        __syncthreads();
    }

    // ---- pass loop (pass 0, then TRMC-RAD continuations) --------------------
    for (;;) {
        const int pass = sh.pass, warp = tid >> 5, npart = sh.npart;
        // the roles write, for each rank from n0 on, the particle's slot
        // (pass 0) or its position in Vc (later passes, from the previous
        // pass's table: the participants of a continuation are the previous
        // pass's thermalised set, ranks poolp.. of that pass)
        int32_t *inv = pass == 0 ? sh.inv0 : sh.posA[pass & 1];
        const int32_t *invp = sh.posA[(pass + 1) & 1];
        const int poolp = sh.n0_prev + sh.D0_prev;
        auto role_of = [&](int i) -> int {
            return pass == 0 ? i : pass == 1 ? (Mode == kWhole || sh.full ? sh.inv0[poolp + i] : poolp - sh.n0_prev + i)
                                             : invp[poolp + i];
        };

        // One attempt of the tree plan (warp 0) on depth sh.m_top, then, if the
        // trees find enough leaves, the layout of the pass's buffers; otherwise
        // sh.cont is set and sh.m_top holds the next depth to try.  The plan
        // lives in registers: lane j holds levels j and j + 32 (quota, demand,
        // collisions, outputs); level 64, the deepest possible, never receives
        // demand and is held by every lane.
        auto plan_attempt = [&]() {
            if (sh.skip) return;
            constexpr unsigned FULL = 0xffffffffu;
            const int m_top = sh.m_top;
            const int jA = lane, jB = lane + 32;
            const int nA = jA <= m_top ? sh.Nq[jA] : 0, nB = jB <= m_top ? sh.Nq[jB] : 0;
            const int n64 = m_top >= 64 ? sh.Nq[64] : 0;
            int dA = 0, dB = 0, cA = 0, cB = 0, oA = 0, oB = 0, c64 = 0, o64 = 0, pdrop = 0, psurp = 0;
            const uint32_t coin0 = sh.coin[0], coin1 = sh.coin[1], coin2 = sh.coin[2];
            // highest level in 1..top with a quota or a demand (0: none); levels
            // without either have no collision and are skipped
            auto next_level = [&](int top) -> int {
                if (top >= 64 && n64 > 0) return 64;
                const unsigned bB = __ballot_sync(FULL, jB <= top && nB + dB > 0);
                if (bB) return 63 - __clz(bB);
                const unsigned bA = __ballot_sync(FULL, jA >= 1 && jA <= top && nA + dA > 0);
                return bA ? 31 - __clz(bA) : 0;
            };
            for (int lv = next_level(m_top); lv >= 1; lv = next_level(lv - 1)) {
                int nl = n64, dl = 0;
                if (lv < 64) {
                    nl = __shfl_sync(FULL, lv >= 32 ? nB : nA, lv & 31);
                    dl = __shfl_sync(FULL, lv >= 32 ? dB : dA, lv & 31);
                }
                int T = nl + dl;
                if (T & 1) {
                    const uint32_t cw = lv < 32 ? coin0 : lv < 64 ? coin1 : coin2;
                    if (nl >= 1 && ((cw >> (lv & 31)) & 1u)) { T -= 1; ++pdrop; }
                    else { T += 1; ++psurp; }
                }
                const int Cn = T >> 1;
                int32_t *row = sh.Mt + tri(lv), *srow = sh.St + tri(lv);
                // slot bases of this level's consumers: the demand of the levels above
                if (jA < lv) srow[jA] = dA;
                if (jB < lv) srow[jB] = dB;
                // r: collisions labelled k = j; s: collisions whose second input
                // is of level j (k = lv - 1 - j)
                int rA = 0, rB = 0, sA = 0, sB = 0;
                if (lv == 1) {
                    // every level-1 collision has k = 0: no labels needed
                    if (lane == 0) { rA = Cn; sA = Cn; row[0] = Cn; }
                } else if (Cn <= kPreLabels) {
                    const uint64_t L0 = *reinterpret_cast<const uint64_t *>(&sh.lab[lv][0]);
                    const uint64_t L1 = *reinterpret_cast<const uint64_t *>(&sh.lab[lv][8]);
                    for (int c = 0; c < Cn; ++c) {
                        const int k = int(((c < 8 ? L0 : L1) >> (8 * (c & 7))) & 0xFFu), j = lv - 1 - k;
                        rA += k == jA; rB += k == jB;
                        sA += j == jA; sB += j == jB;
                    }
                    if (jA < lv) row[jA] = rA;
                    if (jB < lv) row[jB] = rB;
                } else {
                    // label histogram: the predrawn labels (lanes with equal labels
                    // add once), then draws for the collisions beyond them
                    if (jA < lv) row[jA] = 0;
                    if (jB < lv) row[jB] = 0;
                    __syncwarp();
                    const int np = sh.npre[lv], cpre = Cn < np ? Cn : np;
                    const int k0 = lane < cpre ? int(sh.lab[lv][lane]) : -1;
                    const int k1 = lane + 32 < cpre ? int(sh.lab[lv][lane + 32]) : -1;
                    const unsigned g0 = __match_any_sync(FULL, k0), g1 = __match_any_sync(FULL, k1);
                    if (k0 >= 0 && __ffs(g0) - 1 == lane) atomicAdd(&row[k0], __popc(g0));
                    if (k1 >= 0 && __ffs(g1) - 1 == lane) atomicAdd(&row[k1], __popc(g1));
                    for (int g = (np >> 2) + lane; g < (Cn + 3) >> 2; g += 32) {
                        const U64x4 w = rng().draw(uint64_t(g), uint64_t(lv), uint32_t(pass), TAG_KSEL);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (4 * g + j < Cn) atomicAdd(&row[below(w.w[j], uint32_t(lv))], 1);
                    }
                    __syncwarp();
                    if (jA < lv) { rA = row[jA]; sA = row[lv - 1 - jA]; }
                    if (jB < lv) { rB = row[jB]; sB = row[lv - 1 - jB]; }
                }
                dA += rA + sA;
                dB += rB + sB;
                if (lv == 64) { c64 = Cn; o64 = 2 * Cn - dl; }
                else if (lane == (lv & 31)) {
                    if (lv < 32) { cA = Cn; oA = 2 * Cn - dl; }
                    else { cB = Cn; oB = 2 * Cn - dl; }
                }
            }
            // leaf feasibility (Sec. 4.1: a tree cannot be longer than the cell)
            const int d0 = __shfl_sync(FULL, dA, 0);
            const int n0q = sh.Nq[0], A = npart - n0q;
            int n0 = n0q, R = 0;
            if (d0 <= A) {
                R = A - d0;
            } else if (d0 - A <= n0q) {
                n0 = n0q - (d0 - A);
            } else {
                // Lowering the depth by one level at a time (the rule) gives the
                // same plan again while the removed top level is empty, so go
                // straight below the highest level with a quota; the number of
                // one-level reductions is still counted.
                const unsigned qB = __ballot_sync(FULL, jB <= m_top && nB > 0);
                const unsigned qA = __ballot_sync(FULL, jA >= 1 && jA <= m_top && nA > 0);
                const int h = n64 > 0 ? 64 : qB ? 63 - __clz(qB) : qA ? 31 - __clz(qA) : 0;
                const int nt = (h >= 1 ? h : 1) - 1;
                if (lane == 0) { sh.feas += m_top - nt; sh.m_top = nt; sh.cont = 1; }
                __syncwarp();
                return;
            }
            // layout of the pass: output offsets O and consumer-slot offsets IB
            // of every level (prefix sums over levels 1..m)
            const int m = m_top;
            const bool inA = jA >= 1 && jA <= m, inB = jB <= m;
            int pO = inA ? oA : 0, qO = inB ? oB : 0, pI = inA ? dA : 0, qI = inB ? dB : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t0 = __shfl_up_sync(FULL, pO, o), t1 = __shfl_up_sync(FULL, qO, o);
                const int t2 = __shfl_up_sync(FULL, pI, o), t3 = __shfl_up_sync(FULL, qI, o);
                if (lane >= o) { pO += t0; qO += t1; pI += t2; qI += t3; }
            }
            qO += __shfl_sync(FULL, pO, 31);
            qI += __shfl_sync(FULL, pI, 31);
            const int O63 = __shfl_sync(FULL, qO, 31), I63 = __shfl_sync(FULL, qI, 31);
            const int Otot = O63 + (m >= 64 ? o64 : 0), Dge1 = I63;     // D of level 64 is 0
            if (jA < m + 1) { sh.O[jA + 1] = pO; sh.IB[jA + 1] = pI; }
            if (jB < m + 1) { sh.O[jB + 1] = qO; sh.IB[jB + 1] = qI; }
            if (lane == 0 && m >= 64) { sh.O[65] = Otot; sh.IB[65] = Dge1; }
            sh.D[jA] = dA; sh.D[jB] = dB; sh.C[jA] = cA; sh.C[jB] = cB;
            if (lane == 0) { sh.D[64] = 0; sh.D[65] = 0; sh.C[64] = c64; sh.C[65] = 0; }
            // recorded levels (at most rec_max collisions) in ascending order with
            // the offsets of their collisions in the per-collision records
            const bool wA = inA && cA > 0 && cA <= rec_max;
            const bool wB = inB && cB > 0 && cB <= rec_max;
            const bool w64 = m >= 64 && c64 > 0 && c64 <= rec_max;
            const unsigned bwA = __ballot_sync(FULL, wA), bwB = __ballot_sync(FULL, wB);
            const unsigned ltm = (1u << lane) - 1u;
            const int iA = __popc(bwA & ltm), iB = __popc(bwA) + __popc(bwB & ltm);
            const int nWL = __popc(bwA) + __popc(bwB) + (w64 ? 1 : 0);
            int eA = wA ? cA : 0, eB = wB ? cB : 0;
            const int ownA = eA, ownB = eB;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t0 = __shfl_up_sync(FULL, eA, o), t1 = __shfl_up_sync(FULL, eB, o);
                if (lane >= o) { eA += t0; eB += t1; }
            }
            eB += __shfl_sync(FULL, eA, 31);
            const int W63 = __shfl_sync(FULL, eB, 31), W = W63 + (w64 ? c64 : 0);
            if (wA) { sh.WL[iA] = jA; sh.WB[iA] = eA - ownA; }
            if (wB) { sh.WL[iB] = jB; sh.WB[iB] = eB - ownB; }
            // the tail: deep levels above the highest level of more than
            // warp_level collisions (LB)
            const unsigned lbB = __ballot_sync(FULL, inB && cB > a.warp_level);
            const unsigned lbA = __ballot_sync(FULL, inA && cA > a.warp_level);
            const int LB = (m >= 64 && c64 > a.warp_level) ? 64 : lbB ? 63 - __clz(lbB) : lbA ? 31 - __clz(lbA) : 0;
            const int jt = __popc(__ballot_sync(FULL, wA && jA <= LB)) + __popc(__ballot_sync(FULL, wB && jB <= LB));
            const int WBjt = __reduce_add_sync(FULL, unsigned((wA && jA <= LB ? cA : 0) + (wB && jB <= LB ? cB : 0)));
            const int IBlb = __reduce_add_sync(FULL, unsigned((jA >= 1 && jA <= LB ? dA : 0) + (jB <= LB ? dB : 0)));
            // invariants of a consistent plan; a violation would index the
            // buffers out of range, so the cell is left unchanged instead
            const bool bad = (inA && (oA < 0 || cA < 0)) || (inB && (oB < 0 || cB < 0));
            const bool ok = n0 >= 0 && d0 >= 0 && R >= 0 && n0 + d0 + R == npart && Otot == d0 &&
                            !__any_sync(FULL, bad) && (m < 64 || (o64 >= 0 && c64 >= 0));
            if (lane == 0) {
                sh.cont = 0;
                sh.n0 = n0; sh.D0 = d0; sh.R = R;
                sh.pdrop_tot += pdrop;
                sh.psurp_tot += psurp;
                sh.m_eff = m;
                sh.Dge1 = Dge1;
                if (w64) { sh.WL[nWL - 1] = 64; sh.WB[nWL - 1] = W63; }
                sh.WB[nWL] = W;
                // the arenas' bump pointers in registers while the buffers are laid out
                char *ps = sh.pass_smem, *pg = sh.pass_slab;
                size_t pcs = sh.pass_smem_cap, pcg = sh.pass_slab_cap;
                if (Mode == kDual && !sh.full && pass == 0) {
                    // persistent from here on: the changed particles' velocities;
                    // later passes lay out after them
                    sh.nVc = npart - n0;
                    sh.Vc = static_cast<Real *>(take(ps, pcs, pg, pcg, 3 * size_t(sh.nVc + 1) * sizeof(Real)));
                    if (!sh.Vc) sh.skip = 1;
                    sh.posA[0] = sh.posA[1] = nullptr;
                    sh.smem_rest = ps; sh.smem_rest_cap = pcs; sh.slab_rest = pg; sh.slab_rest_cap = pcg;
                }
                sh.IBuf = static_cast<Real *>(take(ps, pcs, pg, pcg,
                                                   3 * size_t(Dge1 + 1) * sizeof(Real)));
                sh.OBuf = static_cast<Real *>(take(ps, pcs, pg, pcg,
                                                   3 * size_t(d0 + 1) * sizeof(Real)));
                if (!sh.IBuf || !sh.OBuf) sh.skip = 1;
                sh.ILBuf = sh.OLBuf = nullptr; sh.ext = nullptr;
                if (TV == kWb) {
                    sh.ILBuf = static_cast<double *>(take(ps, pcs, pg, pcg,
                                                          8 * size_t(Dge1 + 1)));
                    sh.OLBuf = static_cast<double *>(take(ps, pcs, pg, pcg,
                                                          8 * size_t(d0 + 1)));
                    sh.ext = static_cast<int32_t *>(take(ps, pcs, pg, pcg,
                                                         4 * size_t(d0 + 1)));
                    if (!sh.ILBuf || !sh.OLBuf || !sh.ext) sh.skip = 1;
                }
                // records of the recorded levels' collisions; without room for
                // them the waves compute everything in place (same results)
                int nwl = nWL;
                if (W > 0) {
                    char *s0 = ps, *g0 = pg;
                    const size_t sc0 = pcs, gc0 = pcg;
                    sh.LP = static_cast<int32_t *>(take(ps, pcs, pg, pcg,
                                                        4 * size_t(tri(m + 1) + 1)));
                    sh.psrc = static_cast<int2 *>(take(ps, pcs, pg, pcg, 8 * size_t(W)));
                    sh.pdst = static_cast<int2 *>(take(ps, pcs, pg, pcg, 8 * size_t(W)));
                    sh.prnd = static_cast<Real *>(take(ps, pcs, pg, pcg,
                                                       4 * size_t(W) * sizeof(Real)));
                    if (!sh.LP || !sh.psrc || !sh.pdst || !sh.prnd) {
                        ps = s0; pg = g0; pcs = sc0; pcg = gc0;
                        nwl = 0;
                    }
                }
                sh.nWL = nwl;
                sh.LB = LB;
                // the tail runs in dependency order when there is room for its maps
                sh.ntail = 0;
                const int nt = W - WBjt, nslots = Dge1 - IBlb;
                if (nwl > 0 && nwl - jt >= 2 && nt > 0) {
                    char *s0 = ps, *g0 = pg;
                    const size_t sc0 = pcs, gc0 = pcg;
                    sh.prodOf = static_cast<int32_t *>(take(ps, pcs, pg,
                                                            pcg, 4 * size_t(nslots + 1)));
                    sh.done = static_cast<int32_t *>(take(ps, pcs, pg,
                                                          pcg, 4 * size_t(nt)));
                    if (sh.prodOf && sh.done) {
                        sh.ntail = nt; sh.tail0 = WBjt; sh.tailbase = IBlb;
                    } else {
                        ps = s0; pg = g0; pcs = sc0; pcg = gc0;
                    }
                }
                sh.pass_smem = ps; sh.pass_slab = pg; sh.pass_smem_cap = pcs; sh.pass_slab_cap = pcg;
                if (pg > sh.slab_hi) sh.slab_hi = pg;
                if (!ok) sh.skip = 2;
                if (pass == 0) sh.n0_first = n0;
            }
            if (a.report && pass == 0) {
                int64_t *r = a.report + int64_t(cell) * TRMC_REPORT_LEN;
                if (lane == 0) { r[6] = n0; r[14] = m; }
                for (int j = lane; j < NLEV; j += 32) r[16 + j] = sh.Nq[j];
                r[16 + NLEV + jA] = cA; r[16 + NLEV + jB] = cB;
                r[16 + 2 * NLEV + jA] = dA; r[16 + 2 * NLEV + jB] = dB;
                if (lane == 0) {
                    r[16 + NLEV + 64] = c64; r[16 + NLEV + 65] = 0;
                    r[16 + 2 * NLEV + 64] = 0; r[16 + 2 * NLEV + 65] = 0;
                }
            }
            __syncwarp();
        };
        // 2. Split (Alg. 4.2): one uniform per level, drawn by the whole CTA,
        //    then the recurrence in integer arithmetic that reproduces the FP64
        //    Iround bit for bit (iround_q).
        {
            const int lo = sh.lo, m = sh.m;
            for (int t = tid; t <= m - lo; t += bs)
                sh.uSK[lo + t] = rng().draw(uint64_t(lo + t), 0, uint32_t(pass), TAG_SPLIT).w[0] >> 11;
            for (int j = tid; j < NLEV; j += bs) sh.Nq[j] = 0;
            if (tid < 3) sh.coin[tid] = 0u;
            if (tid == bs - 1) sh.keyP0 = rng().draw(0, 0, uint32_t(pass), TAG_PERM0);
        }
        __syncthreads();
        int m_split;
        {
            // Warp 0 runs the recurrence speculatively: lane j evaluates level
            // lv + j with the current remainder; the levels before the first
            // non-zero count get none, and only there does the remainder change.
            // A split whose counts are mostly zero (small q) takes a few rounds.
            if (warp == 0) {
                constexpr unsigned FULL = 0xffffffffu;
                const uint64_t qb = uint64_t(__double_as_longlong(sh.q));
                const int m = sh.m;
                // q as a 0.64 fixed-point number Q (exact for q >= 2^-12, else
                // truncated, which R Q can be off by less than 2^31 units)
                const uint32_t qE = uint32_t(qb >> 52) & 0x7FFu;
                const uint64_t qM = (qb & ((1ull << 52) - 1ull)) | (1ull << 52);
                uint64_t Q = 0, Qslack = 0;
                const bool qfix = qE >= 1011 - 63 && qE < 1023;
                if (qfix) {
                    if (qE >= 1011) Q = qM << (qE - 1011);
                    else { Q = qM >> (1011 - qE); Qslack = 1ull << 32; }
                }
                int rem = npart, lv = sh.lo, ms = m, htop = 0;
                while (lv <= m) {
                    const int l = lv + lane;
                    int c = 0;
                    if (l <= m) {
                        const uint64_t K = sh.uSK[l];
                        bool known = false;
                        if (qfix) {
                            // x = R Q 2^-64 exactly: integer part hi, fraction lo 2^-64.
                            // Farther than an ulp of x from an integer and from u, the
                            // FP64 product decides the same way as the exact one.
                            const uint32_t r32 = uint32_t(rem);
                            const uint64_t a0 = uint64_t(uint32_t(Q)) * r32, b0 = uint64_t(uint32_t(Q >> 32)) * r32;
                            const uint64_t mid = (a0 >> 32) + (b0 & 0xFFFFFFFFull);
                            const uint64_t lo = (mid << 32) | (a0 & 0xFFFFFFFFull), hi = (b0 >> 32) + (mid >> 32);
                            const int bl = hi ? 64 - __clzll((long long)hi) : 0;
                            const uint64_t marg = (1ull << (bl + 11)) + Qslack, u = K << 11;
                            const uint64_t du = lo > u ? lo - u : u - lo;
                            if (lo > marg && lo < 0ull - marg && du > marg) { c = int(hi) + (u < lo ? 1 : 0); known = true; }
                        }
                        if (!known) c = iround_q(qb, uint32_t(rem), K);
                    }
                    const unsigned nz = __ballot_sync(FULL, c != 0);
                    if (nz == 0) { lv += 32; continue; }
                    const int f = __ffs(nz) - 1;
                    const int cf = __shfl_sync(FULL, c, f);
                    if (lane == 0) sh.Nq[lv + f] = cf;
                    htop = lv + f;
                    rem -= cf;
                    if (rem == 0) { ms = lv + f; break; }
                    lv += f + 1;
                }
                __syncwarp();
                // the level draws: parity coin and product key of every level from 1
                // to the highest with a quota (none above it has collisions), and
                // labels of levels >= 2: at least kPreLabels and about as many more
                // as half the level's quota (its collisions), up to kMaxPre
                {
                    auto ndraw = [&](int l, int &np) -> int {
                        np = 0;
                        if (l > htop) return 0;
                        if (l == 1) return 2;
                        int g = kPreLabels / 4 + ((sh.Nq[l] + 7) >> 3);
                        if (g > kMaxPre / 4) g = kMaxPre / 4;
                        np = 4 * g;
                        return 2 + g;
                    };
                    int npA, npB;
                    const int cA_ = ndraw(lane + 1, npA), cB_ = ndraw(lane + 33, npB);
                    int pA = cA_, pB = cB_;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t0 = __shfl_up_sync(FULL, pA, o), t1 = __shfl_up_sync(FULL, pB, o);
                        if (lane >= o) { pA += t0; pB += t1; }
                    }
                    pB += __shfl_sync(FULL, pA, 31);
                    sh.dbase[lane + 1] = pA - cA_;
                    sh.dbase[lane + 33] = pB - cB_;
                    sh.npre[lane + 1] = uint8_t(npA);
                    sh.npre[lane + 33] = uint8_t(npB);
                    if (lane == 31) { sh.dbase[65] = pB; sh.ndraws = pB; }
                }
                if (lane == 0) {
                    if (rem > 0) sh.Nq[m + 1] = rem;
                    sh.m_eff = ms;
                    sh.m_top = ms;
                    sh.pass_smem = sh.smem_rest; sh.pass_smem_cap = sh.smem_rest_cap;
                    sh.pass_slab = sh.slab_rest; sh.pass_slab_cap = sh.slab_rest_cap;
                    const size_t T = size_t(tri(ms + 1));
                    sh.Mt = static_cast<int32_t *>(take(sh.pass_smem, sh.pass_smem_cap, sh.pass_slab, sh.pass_slab_cap, 4 * (T + 1)));
                    sh.St = static_cast<int32_t *>(take(sh.pass_smem, sh.pass_smem_cap, sh.pass_slab, sh.pass_slab_cap, 4 * (T + 1)));
                    if (!sh.Mt || !sh.St) sh.skip = 1;
                    if (sh.pass_slab > sh.slab_hi) sh.slab_hi = sh.pass_slab;
                }
            }
            __syncthreads();
            m_split = sh.m_eff;
        }
        // 3. The other draws of levels 1..m_eff: the parity coin (odd counts,
        //    Alg. 4.3), the key of the level's product permutation and its first
        //    npre labels k (Alg. 4.1), four per draw.
        {
            const int ndr = sh.ndraws;
            for (int t = tid; t < ndr; t += bs) {
                int a_ = 1, b_ = m_split;                 // level: the last with dbase <= t
                while (a_ < b_) {
                    const int mid = (a_ + b_ + 1) >> 1;
                    if (sh.dbase[mid] <= t) a_ = mid; else b_ = mid - 1;
                }
                const int lv = a_, kind = t - sh.dbase[lv];
                const uint64_t idx = kind == 0 ? uint64_t(lv) : kind == 1 ? 0ull : uint64_t(kind - 2);
                const uint64_t aux = kind == 0 ? 0ull : uint64_t(lv);
                const uint32_t tag = kind == 0 ? TAG_PARITY : kind == 1 ? TAG_PERMK : TAG_KSEL;
                const U64x4 w = rng().draw(idx, aux, uint32_t(pass), tag);
                if (kind == 0) {
                    if ((w.w[0] >> 63) == 0) atomicOr(&sh.coin[lv >> 5], 1u << (lv & 31));   // u < 1/2
                } else if (kind == 1) {
                    sh.keys[lv] = w;
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) sh.lab[lv][4 * (kind - 2) + j] = uint8_t(below(w.w[j], uint32_t(lv)));
                }
            }
        }
        __syncthreads();
        // 4. roles (the "random choice" of Alg. 4.3): a permutation pi of the
        //    participants gives slot pi^-1(r) the rank r.  Only ranks from n0 on
        //    (leaves, then the thermalised set) are ever looked up, so only they
        //    are computed, with the inverse permutation: the ranks from the
        //    level-0 quota on by warps 1.. while warp 0 plans (warp 0 afterwards
        //    in a single-warp CTA), those the leaf rule borrows from level 0
        //    once the plan is known.  The plan is attempted once, and once more
        //    after the leaf rule has lowered the depth (one call site: the
        //    plan is long code, and one copy of it keeps the kernel small).
        Perm perm;
        perm.init(uint32_t(npart), sh.keyP0);
        const int nq0 = sh.Nq[0];
        for (int attempt = 0;; ++attempt) {
            if (warp == 0) plan_attempt();
            if (attempt == 0 && (warp > 0 || bs == 32)) {
                const int t0 = bs == 32 ? tid : tid - 32, st = bs == 32 ? bs : bs - 32;
                for (int r = nq0 + t0; r < npart; r += st) inv[r] = role_of(int(perm.inv(uint32_t(r))));
            }
            __syncthreads();
            if (attempt > 0 || sh.skip || !sh.cont) break;
            {
                // The first plan needs more leaves than the participants can give.
                // The rule then lowers the depth to just below one quota level
                // after another; those depths follow from the quotas alone, so up
                // to four warps test the next ones at once (feasibility only), and
                // warp 0 then plans the first feasible one in full.
                const int nsw = (bs >> 5) < 4 ? (bs >> 5) : 4;
                auto feasible_at = [&](int ct) -> bool {
                    int32_t *Dw = reinterpret_cast<int32_t *>(sh.red) + warp * 130, *rw = Dw + NLEV;
                    for (int j = lane; j < NLEV; j += 32) Dw[j] = 0;
                    __syncwarp();
                    int lv = ct;
                    while (lv >= 1 && sh.Nq[lv] + Dw[lv] == 0) --lv;
                    while (lv >= 1) {
                        int T = sh.Nq[lv] + Dw[lv];
                        if (T & 1) T += (sh.Nq[lv] >= 1 && ((sh.coin[lv >> 5] >> (lv & 31)) & 1u)) ? -1 : 1;
                        const int Cn = T >> 1;
                        if (lv == 1) {
                            if (lane == 0) Dw[0] += 2 * Cn;
                        } else if (Cn <= kPreLabels) {
                            if (lane < Cn) {
                                const int k = sh.lab[lv][lane];
                                atomicAdd(&Dw[k], 1);
                                atomicAdd(&Dw[lv - 1 - k], 1);
                            }
                        } else {
                            for (int k = lane; k < lv; k += 32) rw[k] = 0;
                            __syncwarp();
                            const int np = sh.npre[lv], cpre = Cn < np ? Cn : np;
                            for (int c = lane; c < cpre; c += 32) atomicAdd(&rw[sh.lab[lv][c]], 1);
                            for (int g = (np >> 2) + lane; g < (Cn + 3) >> 2; g += 32) {
                                const U64x4 w = rng().draw(uint64_t(g), uint64_t(lv), uint32_t(pass), TAG_KSEL);
    #pragma unroll
                                for (int j = 0; j < 4; ++j)
                                    if (4 * g + j < Cn) atomicAdd(&rw[below(w.w[j], uint32_t(lv))], 1);
                            }
                            __syncwarp();
                            for (int k = lane; k < lv; k += 32) Dw[k] += rw[k] + rw[lv - 1 - k];
                        }
                        __syncwarp();
                        --lv;
                        while (lv >= 1 && sh.Nq[lv] + Dw[lv] == 0) --lv;
                    }
                    const int n0q = sh.Nq[0], A = npart - n0q, d0 = Dw[0];
                    return d0 <= A || d0 - A <= n0q;
                };
                while (sh.cont) {
                    if (tid == 0) {
                        int c = sh.m_top;
                        for (int w = 0; w < nsw; ++w) sh.cand[w] = -1;
                        for (int w = 0; w < nsw; ++w) {
                            sh.cand[w] = c;
                            if (c == 0) break;                 // depth 0 needs no leaf: always feasible
                            int h = c;
                            while (h >= 1 && sh.Nq[h] == 0) --h;
                            c = (h >= 1 ? h : 1) - 1;
                        }
                        sh.cand_next = c;
                    }
                    __syncthreads();
                    if (warp < nsw) {
                        const int ct = sh.cand[warp];
                        const bool ok = ct >= 0 && feasible_at(ct);
                        if (lane == 0) sh.cand_ok[warp] = ok ? 1 : 0;
                    }
                    __syncthreads();
                    if (tid == 0) {
                        int chosen = -1;
                        for (int w = 0; w < nsw; ++w)
                            if (sh.cand[w] >= 0 && sh.cand_ok[w]) { chosen = sh.cand[w]; break; }
                        const int next = chosen >= 0 ? chosen : sh.cand_next;
                        sh.feas += sh.m_top - next;
                        sh.m_top = next;
                        sh.cont = chosen >= 0 ? 0 : 1;
                    }
                    __syncthreads();
                }
            }
        }
        if (sh.skip) break;
        const int m_eff = sh.m_eff, n0 = sh.n0, D0 = sh.D0, Dge1 = sh.Dge1;
        if (n0 < nq0) {
            for (int r = n0 + tid; r < nq0; r += bs) inv[r] = role_of(int(perm.inv(uint32_t(r))));
            __syncthreads();
        }
        // the stage's three components, from shared memory at each use (three
        // pointers held across the pass would cost registers)
        auto Vcx = [&]() { return sh.Vc; };
        auto Vcy = [&]() { return sh.Vc + sh.nVc; };
        auto Vcz = [&]() { return sh.Vc + 2 * sh.nVc; };
        if ((Mode == kWhole || sh.full) && pass == 0) {
            // which slots change: every rank from n0 on (leaves and thermalised)
            for (int r = n0 + tid; r < npart; r += bs) {
                const int i = inv[r];
                atomicOr(&sh.flags[i >> 5], 1u << (i & 31));
            }
        }
        if (Mode == kDual && !sh.full && pass == 0) {
            // stage the particles that change (every rank from n0 on: the
            // leaves, then the thermalised set) in rank order, Vc[r - n0]
            constexpr int U = 4;
            const int nv = sh.nVc;
            for (int j0 = tid; j0 < nv; j0 += U * bs) {
                Real x[U], y[U], z[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = j0 + u * bs;
                    if (j < nv) {
                        const int64_t g = base + inv[n0 + j];
                        x[u] = gx[g]; y[u] = gy[g]; z[u] = gz[g];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = j0 + u * bs;
                    if (j < nv) { Vcx()[j] = x[u]; Vcy()[j] = y[u]; Vcz()[j] = z[u]; }
                }
            }
            __syncthreads();
        }
        // position in Vc of the particle of rank r of this pass (r >= n0)
        const bool full = Mode == kWhole || sh.full;
        auto pos = [&](int r) -> int { return pass == 0 && !full ? r - n0 : inv[r]; };

        // 5. collision waves, level 1 first.  Levels of at most warp_level
        //    collisions (the deep ones) run in warp 0 alone, with warp-level
        //    synchronisation; a CTA barrier is needed only where a larger
        //    level follows them.
        Real *IBx = sh.IBuf, *IBy = sh.IBuf + (Dge1 + 1), *IBz = sh.IBuf + 2 * (Dge1 + 1);
        Real *OBx = sh.OBuf, *OBy = sh.OBuf + (D0 + 1), *OBz = sh.OBuf + 2 * (D0 + 1);
        const Real alpha = Real(sh.alpha), Sigma = Real(sh.Sigma);
        const double Sigma2 = double(Sigma) * double(Sigma);
        const int wb = TV == kWb ? prm.wb_length : 0;
        double *IL = sh.ILBuf, *OL = sh.OLBuf;
        auto level_setup = [&](int lv) {          // warp 0: label prefix and product key
            const int32_t *row = sh.Mt + tri(lv);
            int a0 = lane < lv ? row[lane] : 0, a1 = lane + 32 < lv ? row[lane + 32] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t0 = __shfl_up_sync(0xffffffffu, a0, o), t1 = __shfl_up_sync(0xffffffffu, a1, o);
                if (lane >= o) { a0 += t0; a1 += t1; }
            }
            a1 += __shfl_sync(0xffffffffu, a0, 31);
            if (lane < lv) sh.Pn[lane + 1] = a0;
            if (lane + 32 < lv) sh.Pn[lane + 33] = a1;
            if (lane == 0) sh.Pn[0] = 0;
        };
        auto collide_one = [&](int lv, int c, const Perm &pk) {
            // the draw and the product slots do not depend on the inputs:
            // issue them first so their latency overlaps the loads
            const U64x4 w = rng().draw(uint64_t(c), uint64_t(lv), uint32_t(pass), TAG_COLL);
            int t0, t1;
            pk.fwd2(uint32_t(2 * c), uint32_t(2 * c + 1), t0, t1);
            const int Dn = sh.D[lv], On = sh.O[lv], IBn = sh.IB[lv];
            const int32_t *row = sh.Mt + tri(lv), *srow = sh.St + tri(lv);
            // label of collision c: Pn[k] <= c < Pn[k+1]
            int lo_ = 0, hi_ = lv - 1;
            while (lo_ < hi_) {
                const int mid = (lo_ + hi_ + 1) >> 1;
                if (sh.Pn[mid] <= c) lo_ = mid; else hi_ = mid - 1;
            }
            const int k = lo_, j = lv - 1 - k, off = c - sh.Pn[k];
            const int s0 = srow[k] + off, s1 = srow[j] + row[j] + off;
            Real ax, ay, az, bx, by, bz;
            if (k == 0) { const int sl = pos(n0 + s0); ax = Vcx()[sl]; ay = Vcy()[sl]; az = Vcz()[sl]; }
            else { const int q = sh.IB[k] + s0; ax = IBx[q]; ay = IBy[q]; az = IBz[q]; }
            if (j == 0) { const int sl = pos(n0 + s1); bx = Vcx()[sl]; by = Vcy()[sl]; bz = Vcz()[sl]; }
            else { const int q = sh.IB[j] + s1; bx = IBx[q]; by = IBy[q]; bz = IBz[q]; }
            const Real dx = ax - bx, dy = ay - by, dz = az - bz;
            const Real g2 = dx * dx + dy * dy + dz * dz;
            Real g = Real(0);
            bool acc = true;
            if (sizeof(Real) == 8 && alpha == Real(1)) {
                // hard spheres in FP64: the bound and the acceptance on the squares
                if (lt_sqrt(double(Sigma), Sigma2, double(g2))) cnt[2] += 1;
                const double xs = double(Math<Real>::uni(w.w[0]) * Sigma);
                acc = lt_sqrt(xs, xs * xs, double(g2));
                if (acc) g = Math<Real>::sqrt_(g2);
            } else {
                g = Math<Real>::sqrt_(g2);
                if (alpha != Real(0)) {
                    const Real ga = (alpha == Real(1)) ? g : Math<Real>::pow_(g, alpha);
                    if (ga > Sigma) cnt[2] += 1;
                    const Real xi = Math<Real>::uni(w.w[0]);
                    acc = xi * Sigma < ga;
                }
            }
            Real oax = ax, oay = ay, oaz = az, obx = bx, oby = by, obz = bz;
            if (acc) {
                const Real ct = Real(2) * Math<Real>::uni(w.w[1]) - Real(1);
                const Real st = Math<Real>::sqrt_(fmax(Real(0), Real(1) - ct * ct));
                Real sp, cp;
                Math<Real>::angle(w.w[2], sp, cp);
                const Real sx = cp * st, sy = sp * st, sz = ct;
                const Real h = Real(0.5) * g;
                const Real cx = Real(0.5) * (ax + bx), cy = Real(0.5) * (ay + by), cz = Real(0.5) * (az + bz);
                oax = cx + h * sx; oay = cy + h * sy; oaz = cz + h * sz;
                obx = cx - h * sx; oby = cy - h * sy; obz = cz - h * sz;
                cnt[0] += 1;
            } else {
                cnt[1] += 1;
            }
            if (t0 < Dn) { const int q = IBn + t0; IBx[q] = oax; IBy[q] = oay; IBz[q] = oaz; }
            else { const int q = On + t0 - Dn; OBx[q] = oax; OBy[q] = oay; OBz[q] = oaz; }
            if (t1 < Dn) { const int q = IBn + t1; IBx[q] = obx; IBy[q] = oby; IBz[q] = obz; }
            else { const int q = On + t1 - Dn; OBx[q] = obx; OBy[q] = oby; OBz[q] = obz; }
            if (wb) {
                // length of this collision's tree (both products share it), from
                // its inputs' trees; an original particle has length 0
                double L;
                if (wb == TRMC_LEN_K) {
                    L = double(lv);
                } else {
                    const double La = k == 0 ? 0.0 : IL[sh.IB[k] + s0], Lb = j == 0 ? 0.0 : IL[sh.IB[j] + s1];
                    L = wb == TRMC_LEN_MIN ? 1.0 + (La < Lb ? La : Lb) : __dadd_rn(1.0, __dmul_rn(0.5, __dadd_rn(La, Lb)));
                }
                if (t0 < Dn) IL[IBn + t0] = L; else OL[On + t0 - Dn] = L;
                if (t1 < Dn) IL[IBn + t1] = L; else OL[On + t1 - Dn] = L;
            }
        };
        // 5a. The deep levels run one after the other in warp 0, mostly with a
        //     few collisions each, so their latency is the cell's critical
        //     path; the levels of up to a few collisions per thread are
        //     latency-bound too.  Everything of these levels' collisions that
        //     does not depend on the inputs -- label, input and output
        //     locations, the draw, the acceptance threshold and the scattering
        //     direction -- is computed first by the whole CTA; such a level
        //     then only loads its inputs, collides and stores.
        const int nWL = sh.nWL;
        if (nWL > 0) {
            const int nw = bs >> 5;
            for (int jl = warp; jl < nWL; jl += nw) {
                const int lv = sh.WL[jl];
                const int32_t *row = sh.Mt + tri(lv);
                int32_t *pr = sh.LP + tri(lv);
                const int r0 = lane < lv ? row[lane] : 0, r1 = lane + 32 < lv ? row[lane + 32] : 0;
                int a0 = r0, a1 = r1;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t0 = __shfl_up_sync(0xffffffffu, a0, o), t1 = __shfl_up_sync(0xffffffffu, a1, o);
                    if (lane >= o) { a0 += t0; a1 += t1; }
                }
                a1 += __shfl_sync(0xffffffffu, a0, 31);
                if (lane < lv) pr[lane] = a0 - r0;
                if (lane + 32 < lv) pr[lane + 32] = a1 - r1;
                // a level of at most 32 products: its dealing permutation as a
                // table, the rank of each product's key among the level's keys
                // (perm_rank2's own rule), in the level's label row, which the
                // plan no longer needs
                const int np = 2 * sh.C[lv];
                if (np <= 32) {
                    const uint32_t ky = lane < np ? rank_key(uint32_t(lane), sh.keys[lv].w[0]) : 0u;
                    uint32_t rk = 0;
                    for (int j = 0; j < np; ++j) rk += __shfl_sync(0xffffffffu, ky, j) < ky;
                    if (lane < np) sh.lab[lv][lane] = uint8_t(rk);
                }
            }
            __syncthreads();
            const int W = sh.WB[nWL];
            for (int i = tid; i < W; i += bs) {
                int lo_ = 0, hi_ = nWL - 1;
                while (lo_ < hi_) {
                    const int mid = (lo_ + hi_ + 1) >> 1;
                    if (sh.WB[mid] <= i) lo_ = mid; else hi_ = mid - 1;
                }
                const int lv = sh.WL[lo_], c = i - sh.WB[lo_];
                const int32_t *row = sh.Mt + tri(lv), *srow = sh.St + tri(lv), *pr = sh.LP + tri(lv);
                int ka = 0, kb = lv - 1;
                while (ka < kb) {
                    const int mid = (ka + kb + 1) >> 1;
                    if (pr[mid] <= c) ka = mid; else kb = mid - 1;
                }
                const int k = ka, j = lv - 1 - k, off = c - pr[k];
                const int s0 = srow[k] + off, s1 = srow[j] + row[j] + off;
                int2 sr, ds;
                sr.x = k == 0 ? ~pos(n0 + s0) : sh.IB[k] + s0;
                sr.y = j == 0 ? ~pos(n0 + s1) : sh.IB[j] + s1;
                int t0, t1;
                if (2 * sh.C[lv] <= 32) {
                    t0 = sh.lab[lv][2 * c];
                    t1 = sh.lab[lv][2 * c + 1];
                } else {
                    Perm pk;
                    pk.init(uint32_t(2 * sh.C[lv]), sh.keys[lv]);
                    pk.fwd2(uint32_t(2 * c), uint32_t(2 * c + 1), t0, t1);
                }
                const int Dn = sh.D[lv];
                ds.x = t0 < Dn ? sh.IB[lv] + t0 : ~(sh.O[lv] + t0 - Dn);
                ds.y = t1 < Dn ? sh.IB[lv] + t1 : ~(sh.O[lv] + t1 - Dn);
                const U64x4 w = rng().draw(uint64_t(c), uint64_t(lv), uint32_t(pass), TAG_COLL);
                const Real xs = alpha != Real(0) ? Math<Real>::uni(w.w[0]) * Sigma : Real(0);
                const Real ct = Real(2) * Math<Real>::uni(w.w[1]) - Real(1);
                const Real st = Math<Real>::sqrt_(fmax(Real(0), Real(1) - ct * ct));
                Real sp, cp;
                Math<Real>::angle(w.w[2], sp, cp);
                sh.psrc[i] = sr;
                sh.pdst[i] = ds;
                Real *rr = sh.prnd + 4 * size_t(i);
                rr[0] = xs; rr[1] = cp * st; rr[2] = sp * st; rr[3] = ct;
                if (sh.ntail > 0 && i >= sh.tail0) {
                    if (ds.x >= 0) sh.prodOf[ds.x - sh.tailbase] = i - sh.tail0;
                    if (ds.y >= 0) sh.prodOf[ds.y - sh.tailbase] = i - sh.tail0;
                    sh.done[i - sh.tail0] = 0;
                }
            }
            __syncthreads();
        }
        auto collide_pre = [&](int i, int lv) {
            const int2 sr = sh.psrc[i], ds = sh.pdst[i];
            const Real *rr = sh.prnd + 4 * size_t(i);
            const Real xs = rr[0], sx = rr[1], sy = rr[2], sz = rr[3];
            Real ax, ay, az, bx, by, bz;
            if (sr.x >= 0) { ax = IBx[sr.x]; ay = IBy[sr.x]; az = IBz[sr.x]; }
            else { const int sl = ~sr.x; ax = Vcx()[sl]; ay = Vcy()[sl]; az = Vcz()[sl]; }
            if (sr.y >= 0) { bx = IBx[sr.y]; by = IBy[sr.y]; bz = IBz[sr.y]; }
            else { const int sl = ~sr.y; bx = Vcx()[sl]; by = Vcy()[sl]; bz = Vcz()[sl]; }
            const Real dx = ax - bx, dy = ay - by, dz = az - bz;
            const Real g2 = dx * dx + dy * dy + dz * dz;
            Real g = Real(0);
            bool acc = true;
            if (sizeof(Real) == 8 && alpha == Real(1)) {
                if (lt_sqrt(double(Sigma), Sigma2, double(g2))) cnt[2] += 1;
                acc = lt_sqrt(double(xs), double(xs) * double(xs), double(g2));
                if (acc) g = Math<Real>::sqrt_(g2);
            } else {
                g = Math<Real>::sqrt_(g2);
                if (alpha != Real(0)) {
                    const Real ga = (alpha == Real(1)) ? g : Math<Real>::pow_(g, alpha);
                    if (ga > Sigma) cnt[2] += 1;
                    acc = xs < ga;
                }
            }
            Real oax = ax, oay = ay, oaz = az, obx = bx, oby = by, obz = bz;
            if (acc) {
                const Real h = Real(0.5) * g;
                const Real cx = Real(0.5) * (ax + bx), cy = Real(0.5) * (ay + by), cz = Real(0.5) * (az + bz);
                oax = cx + h * sx; oay = cy + h * sy; oaz = cz + h * sz;
                obx = cx - h * sx; oby = cy - h * sy; obz = cz - h * sz;
                cnt[0] += 1;
            } else {
                cnt[1] += 1;
            }
            if (ds.x >= 0) { IBx[ds.x] = oax; IBy[ds.x] = oay; IBz[ds.x] = oaz; }
            else { const int q = ~ds.x; OBx[q] = oax; OBy[q] = oay; OBz[q] = oaz; }
            if (ds.y >= 0) { IBx[ds.y] = obx; IBy[ds.y] = oby; IBz[ds.y] = obz; }
            else { const int q = ~ds.y; OBx[q] = obx; OBy[q] = oby; OBz[q] = obz; }
            if (wb) {
                double L;
                if (wb == TRMC_LEN_K) {
                    L = double(lv);
                } else {
                    const double La = sr.x >= 0 ? IL[sr.x] : 0.0, Lb = sr.y >= 0 ? IL[sr.y] : 0.0;
                    L = wb == TRMC_LEN_MIN ? 1.0 + (La < Lb ? La : Lb) : __dadd_rn(1.0, __dmul_rn(0.5, __dadd_rn(La, Lb)));
                }
                if (ds.x >= 0) IL[ds.x] = L; else OL[~ds.x] = L;
                if (ds.y >= 0) IL[ds.y] = L; else OL[~ds.y] = L;
            }
        };
        bool warp_only = false;      // the last level ran in warp 0 alone
        int jw = 0;                  // next recorded level in WL
        const int ntail = sh.ntail;
        const int lv_end = ntail > 0 ? sh.LB : m_eff;
        for (int lv = 1; lv <= lv_end; ++lv) {
            const int Cn = sh.C[lv];
            if (Cn == 0) continue;
            if (Cn <= a.warp_level) {
                warp_only = true;
                const int base = nWL > 0 ? sh.WB[jw++] : 0;
                if (warp != 0) continue;
                if (nWL > 0) {
                    for (int c = lane; c < Cn; c += 32) collide_pre(base + c, lv);
                    __syncwarp();
                    continue;
                }
                level_setup(lv);
                __syncwarp();
                Perm pk;
                pk.init(uint32_t(2 * Cn), sh.keys[lv]);
                for (int c = lane; c < Cn; c += 32) collide_one(lv, c, pk);
                __syncwarp();
            } else {
                if (warp_only) { __syncthreads(); warp_only = false; }
                if (Cn <= rec_max && nWL > 0) {
                    const int base = sh.WB[jw++];
                    for (int c = tid; c < Cn; c += bs) collide_pre(base + c, lv);
                    __syncthreads();
                    continue;
                }
                if (warp == 0) level_setup(lv);
                __syncthreads();
                Perm pk;
                pk.init(uint32_t(2 * Cn), sh.keys[lv]);
                for (int c = tid; c < Cn; c += bs) collide_one(lv, c, pk);
                __syncthreads();
            }
        }
        __syncthreads();
        if (ntail > 0) {
            // 5b. The tail in dependency order: every round, each record whose
            //     inputs were produced in earlier rounds (or come from leaves and
            //     lower levels) runs.  The number of rounds is the depth of the
            //     tail's collision graph, far below its number of levels (a
            //     level-n product depends on levels k and n-1-k, k uniform), and
            //     a round is at least the lowest pending level, so it ends.
            const int t0 = sh.tail0, base = sh.tailbase;
            int32_t *done = sh.done;
            const int32_t *prodOf = sh.prodOf;
            auto level_of = [&](int i) {
                int lo_ = 0, hi_ = nWL - 1;
                while (lo_ < hi_) {
                    const int mid = (lo_ + hi_ + 1) >> 1;
                    if (sh.WB[mid] <= i) lo_ = mid; else hi_ = mid - 1;
                }
                return sh.WL[lo_];
            };
            int round = 1;
            bool pending = true;
            for (;;) {
                if (!__syncthreads_or(pending)) break;
                if (round > NLEV) {          // impossible for a consistent plan; leave the cell unchanged
                    if (tid == 0) sh.skip = 2;
                    break;
                }
                pending = false;
                for (int r = tid; r < ntail; r += bs) {
                    if (done[r]) continue;
                    const int2 sr = sh.psrc[t0 + r];
                    bool ready = true;
                    if (sr.x >= base) { const int d = done[prodOf[sr.x - base]]; ready = d != 0 && d < round; }
                    if (ready && sr.y >= base) { const int d = done[prodOf[sr.y - base]]; ready = d != 0 && d < round; }
                    if (ready) {
                        collide_pre(t0 + r, wb == TRMC_LEN_K ? level_of(t0 + r) : 0);
                        done[r] = round;
                    } else {
                        pending = true;
                    }
                }
                ++round;
            }
            __syncthreads();
            if (sh.skip) break;
        }

        // 6. outputs replace the leaves.  What the collisions changed (sum of
        //    output - original over the leaves) and the thermalised set's own
        //    sums give the renormalisation target and the change of the
        //    adaptive indicator from the changed particles only, without
        //    cancelling two sums over the whole cell.
        {
            // cs[0..3]: change of momentum and energy over the leaves, cs[4..7]: the
            // thermalised set's momentum and energy, cs[8], cs[9]: the indicator's
            // change and the set's indicator (TRMC-RAD only)
            const bool rad = kRad;
            const Real Ux = Real(sh.U[0]);
            auto place = [&](Sum<Real> (&cs)[10], int jx) {
                const int sl = pos(n0 + jx);
                const Real ox = Vcx()[sl], oy = Vcy()[sl], oz = Vcz()[sl];
                const Real x = OBx[jx], y = OBy[jx], z = OBz[jx];
                Vcx()[sl] = x; Vcy()[sl] = y; Vcz()[sl] = z;
                if constexpr (sizeof(Real) == 8) {
                    cs[0].add(x - ox); cs[1].add(y - oy); cs[2].add(z - oz);
                    cs[3].add((x * x + y * y + z * z) - (ox * ox + oy * oy + oz * oz));
                    if (rad) cs[8].add(indicator(x, y, z, sh.U, kInd) - indicator(ox, oy, oz, sh.U, kInd));
                } else {
                    cs[0].add(x); cs[0].add(-ox); cs[1].add(y); cs[1].add(-oy); cs[2].add(z); cs[2].add(-oz);
                    cs[3].add_sq3(x, y, z); cs[3].sub_sq3(ox, oy, oz);
                    if (rad) cs[8].add(indicator_r(x, y, z, Ux, kInd) - indicator_r(ox, oy, oz, Ux, kInd));
                }
            };
            auto pool_add = [&](Sum<Real> (&cs)[10], int sl) {
                const Real x = Vcx()[sl], y = Vcy()[sl], z = Vcz()[sl];
                cs[4].add(x); cs[5].add(y); cs[6].add(z);
                cs[7].add_sq3(x, y, z);
                if (rad) {
                    if constexpr (sizeof(Real) == 8) cs[9].add(indicator(x, y, z, sh.U, kInd));
                    else cs[9].add(indicator_r(x, y, z, Ux, kInd));
                }
            };
            // TRMC-WB (Alg. 4.6): an output whose tree is longer than m_max is
            // not placed; its leaf joins the thermalised set, after the set's
            // own members, in output order.  A lone rejected output with no
            // thermalised set is kept: its only Maxwellian resample with the
            // same momentum and energy is itself.
            const bool wbm = TV == kWb;
            const double mmax = double(prm.m_fixed);
            const double *OL = sh.OLBuf;
            bool keep_all = false;
            if (wbm && sh.R == 0) {
                int tot = 0;
                for (int j0 = 0; j0 < D0; j0 += bs) tot += __syncthreads_count(j0 + tid < D0 && OL[j0 + tid] > mmax);
                keep_all = tot == 1;
            }
            // cs[0..3]: change of momentum and energy over the leaves, cs[4..7]: the
            // thermalised set's momentum and energy (rejected leaves with their
            // original velocities), cs[8], cs[9]: the indicator's change and the
            // set's indicator (TRMC-RAD only); canonical sums
            const int pool0 = n0 + D0, R = sh.R, nw = bs >> 5;
            for (int vw = warp; vw < kVW; vw += nw) {
                Sum<Real> cs[10];
                for (int jx = 32 * vw + lane; jx < D0; jx += 32 * kVW) {
                    if (wbm && !keep_all && OL[jx] > mmax) pool_add(cs, pos(n0 + jx));
                    else place(cs, jx);
                }
                for (int t = 32 * vw + lane; t < R; t += 32 * kVW) pool_add(cs, pos(pool0 + t));
                if (rad) vw_put<10>(cs, sh.red, vw);
                else vw_put<8>(cs, sh.red, vw);
            }
            int nrej = 0;
            if (wbm) {
                // the rejected leaves' slots, in output order
                for (int j0 = 0; j0 < D0; j0 += bs) {
                    const int jx = j0 + tid;
                    const bool rj = !keep_all && jx < D0 && OL[jx] > mmax;
                    int ex;
                    const int tot = block_flag_scan(rj, ex, sh.scan);
                    if (rj) sh.ext[nrej + ex] = pos(n0 + jx);
                    nrej += tot;
                }
            }
            const int Rx = R + nrej;
            double s[5], p[5];
            if (rad) {
                double t[10];
                vw_total<Real, 10>(sh.red, t);
                for (int j = 0; j < 4; ++j) { s[j] = t[j]; p[j] = t[4 + j]; }
                s[4] = t[8]; p[4] = t[9];
            } else {
                double t[8];
                vw_total<Real, 8>(sh.red, t);
                for (int j = 0; j < 4; ++j) { s[j] = t[j]; p[j] = t[4 + j]; }
                s[4] = 0.0; p[4] = 0.0;
            }
            if (tid == 0) {
                sh.dP[0] += s[0]; sh.dP[1] += s[1]; sh.dP[2] += s[2]; sh.dE += s[3]; sh.dS += s[4];
                sh.Pp[0] = p[0]; sh.Pp[1] = p[1]; sh.Pp[2] = p[2]; sh.Ep = p[3]; sh.Sp = p[4];
                sh.nrej = nrej;
                sh.R = Rx;
            }
        }
        // TRMC-RAD test (Sec. 4.3)
        if (tid == 0) {
            sh.cont = 0;
            if (kRad) {
                const int R = sh.R;
                double Sth = 0.0;
                if (R == 1) {
                    const int sl = pos(n0 + D0);
                    Sth = indicator(double(Vcx()[sl]), double(Vcy()[sl]), double(Vcz()[sl]), sh.U, kInd);
                } else if (R >= 2) {
                    const double Pt0 = sh.Pp[0] - sh.dP[0], Pt1 = sh.Pp[1] - sh.dP[1], Pt2 = sh.Pp[2] - sh.dP[2];
                    const double Et = sh.Ep - sh.dE;
                    double et = Et - (Pt0 * Pt0 + Pt1 * Pt1 + Pt2 * Pt2) / double(R);
                    if (et < 0.0) et = 0.0;
                    const double u0 = Pt0 / double(R), u1 = Pt1 / double(R), u2 = Pt2 / double(R);
                    if (kInd == TRMC_IND_M4) {
                        const double Tp = et / (3.0 * double(R));
                        const double uu = u0 * u0 + u1 * u1 + u2 * u2;
                        Sth = double(R) * (uu * uu + 10.0 * uu * Tp + 15.0 * Tp * Tp);
                    } else {
                        const double d = u0 - sh.U[0];
                        Sth = et / 3.0 + double(R) * d * d;
                    }
                }
                const double dS_total = sh.dS + (Sth - sh.Sp);
                const double E1 = (sh.S_pre != 0.0) ? fabs(dS_total) / fabs(double(sh.n) * sh.S_pre) : 0.0;
                const int m = sh.m;
                if (E1 > prm.delta2 && R > 0 && 2 * m <= prm.m_cap) {
                    if (pass == 0) {
                        // the continuation passes' position tables (at most R
                        // entries each), persistent: pass 0's buffers are done
                        sh.posA[0] = static_cast<int32_t *>(take(sh.smem_rest, sh.smem_rest_cap, sh.slab_rest,
                                                                 sh.slab_rest_cap, 4 * size_t(R)));
                        sh.posA[1] = static_cast<int32_t *>(take(sh.smem_rest, sh.smem_rest_cap, sh.slab_rest,
                                                                 sh.slab_rest_cap, 4 * size_t(R)));
                        if (!sh.posA[0] || !sh.posA[1]) sh.skip = 1;
                        if (sh.slab_rest > sh.slab_hi) sh.slab_hi = sh.slab_rest;
                    }
                    sh.cont = 1;
                    sh.n0_prev = n0; sh.D0_prev = D0;
                    sh.npart = R;
                    sh.lo = m + 1;
                    sh.m = 2 * m;
                    sh.pass = pass + 1;
                } else if (E1 < prm.delta1) {
                    sh.m_next = (m / 2 > prm.m_min) ? m / 2 : prm.m_min;
                } else {
                    sh.m_next = m;
                }
            } else {
                sh.m_next = sh.m;
            }
        }
        __syncthreads();
        if (!sh.cont) break;
    }
    if (sh.skip) {
        if (tid == 0) {
            raise_status(a.status, sh.skip == 2 ? TRMC_ERR_STATE : TRMC_ERR_CAPACITY, cell);
            if (a.stats) atomicAdd(&a.stats->capacity_skips, 1ull);
        }
        return Counts{{cnt[0], cnt[1], cnt[2]}};
    }

    // ---- 7. Maxwellian resampling of the thermalised set + renormalisation --
    const int pass = sh.pass, R = sh.R, R0 = sh.R - sh.nrej;
    const int32_t *posl = sh.posA[pass & 1];
    const int pool0 = sh.n0 + sh.D0, n0l = sh.n0;
    const int32_t *ext = sh.ext;
    auto Vcx = [&]() { return sh.Vc; };
    auto Vcy = [&]() { return sh.Vc + sh.nVc; };
    auto Vcz = [&]() { return sh.Vc + 2 * sh.nVc; };
    // position in Vc of thermalised member t (the set's own ranks, then the
    // leaves TRMC-WB sent to it)
    const bool full = Mode == kWhole || sh.full;
    auto pslot = [&](int t) {
        return t < R0 ? (pass == 0 ? (full ? sh.inv0[pool0 + t] : pool0 + t - n0l) : posl[pool0 + t]) : ext[t - R0];
    };
    const int warp = tid >> 5, nw = bs >> 5;
    const bool carry = a.cell_carry != nullptr;
    if (R >= 2) {
        // one pass for the samples and their first and second moments:
        // e = sum |z - zbar|^2 = sum |z|^2 - zbar . sum z (canonical sums)
        for (int vw = warp; vw < kVW; vw += nw) {
            Sum<Real> qs[4];
            for (int t = 32 * vw + lane; t < R; t += 32 * kVW) {
                Real z0, z1, z2;
                Math<Real>::normals(rng().draw(uint64_t(t), 0, 0, TAG_MAXW), z0, z1, z2);
                const int sl = pslot(t);
                Vcx()[sl] = z0; Vcy()[sl] = z1; Vcz()[sl] = z2;
                qs[0].add(z0); qs[1].add(z1); qs[2].add(z2);
                qs[3].add_sq3(z0, z1, z2);
            }
            vw_put<4>(qs, sh.red, vw);
        }
        double s[4], zq[4];
        vw_total<Real, 4>(sh.red, s, double(R), zq);       // zq[0..2]: the samples' mean
        const double zb0 = zq[0], zb1 = zq[1], zb2 = zq[2];
        const Real rz0 = Real(zb0), rz1 = Real(zb1), rz2 = Real(zb2);
        // target: what the set carried, minus the collisions' round-off change,
        // plus what earlier steps' rounding to the storage precision left over;
        // the energy scale and the mean are computed once, by four lanes
        if (tid < 4) {
            const double Pt0 = sh.Pp[0] - sh.dP[0] + sh.carry[0], Pt1 = sh.Pp[1] - sh.dP[1] + sh.carry[1],
                         Pt2 = sh.Pp[2] - sh.dP[2] + sh.carry[2];
            if (lane == 0) {
                const double Et = sh.Ep - sh.dE + sh.carry[3];
                sh.Pt[0] = Pt0; sh.Pt[1] = Pt1; sh.Pt[2] = Pt2; sh.Et = Et;
                double et = Et - (Pt0 * Pt0 + Pt1 * Pt1 + Pt2 * Pt2) / double(R);
                if (et < 0.0) et = 0.0;
                const double e = s[3] - (s[0] * zb0 + s[1] * zb1 + s[2] * zb2);
                sh.msc[0] = (e > 0.0) ? sqrt(et / e) : 0.0;
            } else {
                sh.msc[lane] = (lane == 1 ? Pt0 : lane == 2 ? Pt1 : Pt2) / double(R);
            }
        }
        __syncthreads();
        const double sc = sh.msc[0], u0 = sh.msc[1], u1 = sh.msc[2], u2 = sh.msc[3];
        // FP32-mixed: FP64 scale and targets, applied in float (the stored
        // result is a float either way); the stored set's canonical sums give
        // the carry
        const Real fs = Real(sc), f0 = Real(u0), f1 = Real(u1), f2 = Real(u2);
        for (int vw = warp; vw < kVW; vw += nw) {
            Sum<Real> rs[4];
            for (int t = 32 * vw + lane; t < R; t += 32 * kVW) {
                const int sl = pslot(t);
                Real x, y, z;
                if constexpr (sizeof(Real) == 8) {
                    x = u0 + sc * (Vcx()[sl] - zb0); y = u1 + sc * (Vcy()[sl] - zb1); z = u2 + sc * (Vcz()[sl] - zb2);
                } else {
                    x = f0 + fs * (Vcx()[sl] - rz0); y = f1 + fs * (Vcy()[sl] - rz1); z = f2 + fs * (Vcz()[sl] - rz2);
                }
                Vcx()[sl] = x; Vcy()[sl] = y; Vcz()[sl] = z;
                if (carry) { rs[0].add(x); rs[1].add(y); rs[2].add(z); rs[3].add_sq3(x, y, z); }
            }
            if (carry) vw_put<4>(rs, sh.red, vw);
        }
        if (carry) {
            // new carry: what the stored thermalised set misses of its target
            double r[4];
            vw_total<Real, 4>(sh.red, r);
            if (tid == 0) {
                sh.carry[0] = sh.Pt[0] - r[0]; sh.carry[1] = sh.Pt[1] - r[1]; sh.carry[2] = sh.Pt[2] - r[2];
                sh.carry[3] = sh.Et - r[3];
            }
        }
    }
    __syncthreads();
    if (a.cell_carry) {
        // with R <= 1 the carry takes the collisions' round-off change
        if (R < 2 && tid == 0) {
            sh.carry[0] -= sh.dP[0]; sh.carry[1] -= sh.dP[1]; sh.carry[2] -= sh.dP[2]; sh.carry[3] -= sh.dE;
        }
        if (tid == 0)
            for (int j = 0; j < 4; ++j) a.cell_carry[4 * int64_t(cell) + j] = sh.carry[j];
    }

    // ---- 8. write back the changed particles; cell max |v|^2 over the final
    //         velocities ------------------------------------------------------
    Real vm = 0;
    long long vmb = 0;
    auto vq = [&](Real x, Real y, Real z) {
        if constexpr (sizeof(Real) == 8)       // rounded exactly as the CPU reference rounds it
            vmb = max(vmb, __double_as_longlong(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z))));
        else
            vm = fmaxf(vm, __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z)));
    };
    const bool vmx = a.cell_vmax2 != nullptr;
    if (full) {
        // coalesced: every slot in order, the changed ones written
        for (int i = tid; i < n; i += bs) {
            const Real x = Vcx()[i], y = Vcy()[i], z = Vcz()[i];
            if ((sh.flags[i >> 5] >> (i & 31)) & 1u) { gx[base + i] = x; gy[base + i] = y; gz[base + i] = z; }
            if (vmx) vq(x, y, z);
        }
    } else {
        // scattered from the compact stage to the changed slots, then (for the
        // maximum) every particle from global memory, the changed ones as just
        // written (L2 holds the cell: it was read at the start of the step)
        const int n0f = sh.n0_first, nch = n - n0f;
        const int32_t *inv0 = sh.inv0;
        for (int j = tid; j < nch; j += bs) {
            const int64_t g = base + inv0[n0f + j];
            gx[g] = Vcx()[j]; gy[g] = Vcy()[j]; gz[g] = Vcz()[j];
        }
        if (vmx) {
            __syncthreads();
            constexpr int U = 2;
            for (int i0 = tid; i0 < n; i0 += U * bs) {
                Real x[U], y[U], z[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * bs;
                    if (i < n) { x[u] = gx[base + i]; y[u] = gy[base + i]; z[u] = gz[base + i]; }
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (i0 + u * bs < n) vq(x[u], y[u], z[u]);
            }
        }
    }
    if (vmx) {
        if constexpr (sizeof(Real) == 8) vm = __longlong_as_double(vmb);
        const double vmax = block_max_nonneg(double(vm), sh.red);
        if (tid == 0) a.cell_vmax2[cell] = vmax;
    }
    if (tid == 0) {
        if (kRad) a.m_max[cell] = sh.m_next;
        if (a.report) {
            int64_t *r = a.report + int64_t(cell) * TRMC_REPORT_LEN;
            r[0] = n; r[1] = sh.pass + 1; r[2] = sh.m_first; r[3] = sh.m; r[4] = sh.m_next; r[5] = R;
            r[7] = int64_t(n) - r[6] - int64_t(R - sh.nrej);
            r[11] = sh.feas; r[12] = sh.pdrop_tot; r[13] = sh.psurp_tot; r[15] = sh.nrej;
        }
    }
    return Counts{{cnt[0], cnt[1], cnt[2]}};
}

// Pre-pass of the large cells' moment sums: CTA (slot, vw) of one warp finds
// the slot's cell -- the first cell c = slot (mod kBigSlots) of at least
// kBigCell particles -- and sums virtual warp vw's lanes over it exactly as the
// collide kernel would (same loop, same vw_put), so the eight virtual warps of
// a large cell run on eight SMs.  GB300 issues FP64 at 2 lanes per clock and
// SM: alone, the one CTA of a cell of 1e5 FP64 particles spends about half its
// time here.
template <typename Real, bool M4>
__global__ void __launch_bounds__(32) bigsum_kernel(const Real *__restrict__ gx, const Real *__restrict__ gy,
                                                    const Real *__restrict__ gz, const int64_t *__restrict__ cell_start,
                                                    int n_cells, BigEntry *big, uint64_t stamp)
{
    // one warp per SM: many loads in flight per lane (same order of the sums)
    constexpr int K = M4 ? 5 : 4, U = 16;
    __shared__ double scr[kVW * 5];
    const int slot = blockIdx.x / kVW, vw = blockIdx.x % kVW, lane = threadIdx.x;
    int cell = -1;
    for (int c0 = slot; c0 < n_cells && cell < 0; c0 += 32 * kBigSlots) {
        const int c = c0 + lane * kBigSlots;
        const bool large = c < n_cells && cell_start[c + 1] - cell_start[c] >= kBigCell;
        const unsigned b = __ballot_sync(0xffffffffu, large);
        if (b) cell = c0 + (__ffs(b) - 1) * kBigSlots;
    }
    if (cell < 0) return;
    const int64_t base = cell_start[cell];
    const int n = int(cell_start[cell + 1] - base);
    Sum<Real> acc[5];
    for (int i0 = 32 * vw + lane; i0 < n; i0 += U * 32 * kVW) {
        Real x[U], y[U], z[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * 32 * kVW;
            if (i < n) { x[u] = gx[base + i]; y[u] = gy[base + i]; z[u] = gz[base + i]; }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * 32 * kVW;
            if (i < n) {
                acc[0].add(x[u]); acc[1].add(y[u]); acc[2].add(z[u]);
                acc[3].add_sq3(x[u], y[u], z[u]);
                if (M4) {
                    const Real e = x[u] * x[u] + y[u] * y[u] + z[u] * z[u];
                    acc[4].add(e * e);
                }
            }
        }
    }
    vw_put<K>(acc, scr, vw);
    __syncwarp();
    BigEntry *e = big + slot;
    if (lane < K) e->part[vw * K + lane] = scr[vw * K + lane];
    if (vw == 0 && lane == 0) { e->cell = cell; e->stamp = stamp; }
}

// Registers: the FP32 whole-mode kernel is built for three 256-thread CTAs
// per SM (at most 85 registers a thread; it then spills a few bytes), which
// runs the stationary shock's 2500-particle cells 4 % faster than two; the
// FP64 one, with more live FP64 state, for two; the dual-mode kernels for one
// CTA of up to 512 threads, the same 128 registers a thread as two of 256: a
// problem of one very large cell (the BKW cell of 1e5 particles) runs its
// parallel phases on twice the threads of one SM.
template <typename Real, int Mode, int TV>
__global__ void __launch_bounds__(Mode == kDual ? kThreadsDual : kThreads,
                                  Mode == kDual ? 1 : sizeof(Real) == 4 ? 3 : 2) collide_kernel(Args a)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ Sh<Real> sh;
    __shared__ int s_cell;
    char *slab = a.slabs + size_t(blockIdx.x) * a.slab_bytes;
    // the device step counter is read before any CTA can finish: it is
    // advanced only after every CTA of this launch has retired its last cell
    const uint64_t step = a.step_dev ? *a.step_dev : a.step;
    unsigned int n_max = 0;          // the largest cell this CTA met (thread 0)
    for (;;) {
        if (threadIdx.x == 0) s_cell = int(atomicAdd(&a.tickets[0], 1u));
        __syncthreads();
        const int ticket = s_cell;
        __syncthreads();
        if (ticket >= a.n_cells) break;
        const int cell = a.cell_order ? a.cell_order[ticket] : ticket;
        const long long t_start = clock64();
        const Counts k = process_cell<Real, Mode, TV>(a, step, sh, dsm, slab, cell);
        int cnt[3] = {k.c[0], k.c[1], k.c[2]};      // collisions, dummy, exceed
        if (threadIdx.x == 0 && unsigned(sh.n) > n_max) n_max = unsigned(sh.n);
        if (a.cell_cost && threadIdx.x == 0) {
            const unsigned long long dt = (unsigned long long)(clock64() - t_start) >> 4;
            a.cell_cost[cell] = dt > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(dt);
        }
        __syncthreads();
        // The slab is scratch that the next cell writes again before it reads
        // it: drop the lines this cell dirtied from L2 without writing them
        // back to DRAM (its 128-byte lines; the slab starts 256-byte aligned)
        for (char *p = slab + size_t(threadIdx.x) * 128; p < sh.slab_hi; p += size_t(blockDim.x) * 128)
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
        __syncthreads();
        if (a.report || a.stats) {
            block_sum_int<3>(cnt, sh.red);
            if (threadIdx.x == 0 && sh.n >= 2 && !sh.skip) {
                if (a.report) {
                    int64_t *r = a.report + int64_t(cell) * TRMC_REPORT_LEN;
                    r[8] = (long long)cnt[0]; r[9] = (long long)cnt[1]; r[10] = (long long)cnt[2];
                }
                if (a.stats) {
                    atomicAdd(&a.stats->collisions, (unsigned long long)cnt[0]);
                    atomicAdd(&a.stats->dummy, (unsigned long long)cnt[1]);
                    atomicAdd(&a.stats->exceed, (unsigned long long)cnt[2]);
                    atomicAdd(&a.stats->maxwell, (unsigned long long)(sh.R >= 2 ? sh.R : 0));
                    atomicAdd(&a.stats->passes, (unsigned long long)(sh.pass + 1));
                    atomicAdd(&a.stats->feas, (unsigned long long)sh.feas);
                    atomicAdd(&a.stats->cells, 1ull);
                    atomicAdd(&a.stats->changed, (unsigned long long)(sh.n - sh.n0_first));
                    atomicAdd(&a.stats->particles, (unsigned long long)sh.n);
                    if (sh.nrej) atomicAdd(&a.stats->wb_rejected, (unsigned long long)sh.nrej);
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        if (n_max) atomicMax(&a.tickets[2], n_max);
        __threadfence();
        const unsigned done = atomicAdd(&a.tickets[1], 1u);
        if (done == gridDim.x - 1) {
            // the last CTA: publish the launch's largest cell (the host picks the
            // next launch's mode from it) and reset the counters
            const unsigned biggest = atomicExch(&a.tickets[2], 0u);
            if (a.n_max_host) *a.n_max_host = biggest;
            a.tickets[0] = 0u;
            a.tickets[1] = 0u;
            if (a.step_dev) *a.step_dev = step + 1;
            __threadfence();
        }
    }
}

// Order of the next collide launch: longest cells first, by the times the
// previous launch measured (a counting sort over 64 buckets, two per octave;
// the order within a bucket is arbitrary, and results do not depend on it).
__device__ __forceinline__ int cost_bucket(uint32_t c)
{
    if (c == 0) return 0;
    const int l = 31 - __clz(c);
    const int half = l > 0 ? int((c >> (l - 1)) & 1u) : 0;
    const int b = 2 * l + half + 1;
    return b > 63 ? 63 : b;
}

__global__ void __launch_bounds__(1024) order_kernel(const uint32_t *cost, int n, int32_t *order)
{
    __shared__ int cnt[64];
    const int tid = threadIdx.x;
    if (tid < 64) cnt[tid] = 0;
    __syncthreads();
    for (int c = tid; c < n; c += blockDim.x) atomicAdd(&cnt[cost_bucket(cost[c])], 1);
    __syncthreads();
    if (tid == 0) {
        int s = 0;
        for (int b = 63; b >= 0; --b) { const int t = cnt[b]; cnt[b] = s; s += t; }
    }
    __syncthreads();
    for (int c = tid; c < n; c += blockDim.x) order[atomicAdd(&cnt[cost_bucket(cost[c])], 1)] = c;
}

// The kernel's dynamic shared-memory limit, set once per device to the most a
// CTA can have, so that every launch shape (and the allocation-free entry
// point) fits under it whatever order they come in.
template <typename Real, int Mode, int TV>
cudaError_t allow_max_smem(int device, int smem_optin)
{
    constexpr int kDev = 64;
    static bool done[kDev] = {};
    if (device >= 0 && device < kDev && done[device]) return cudaSuccess;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, collide_kernel<Real, Mode, TV>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(collide_kernel<Real, Mode, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_optin - int(fa.sharedSizeBytes));
    if (e == cudaSuccess && device >= 0 && device < kDev) done[device] = true;
    return e;
}

// The instantiation for a launch (staging mode, truncation), with its
// shared-memory limit raised.
using CollideFn = void (*)(Args);
template <typename Real, int Mode, int TV>
cudaError_t pick(int device, int smem_optin, CollideFn &fn)
{
    fn = collide_kernel<Real, Mode, TV>;
    return allow_max_smem<Real, Mode, TV>(device, smem_optin);
}

int variant_of(const trmc_collide_params *prm)
{
    if (prm->trunc == TRMC_TRUNC_RAD) return prm->indicator == TRMC_IND_M4 ? kRadM4 : kRadPxx;
    return prm->trunc == TRMC_TRUNC_WB ? kWb : kPlain;
}

template <typename Real>
cudaError_t collide_fn(int device, int smem_optin, bool dual, const trmc_collide_params *prm, CollideFn &fn)
{
    switch (variant_of(prm) + (dual ? 4 : 0)) {
    case kPlain: return pick<Real, kWhole, kPlain>(device, smem_optin, fn);
    case kRadPxx: return pick<Real, kWhole, kRadPxx>(device, smem_optin, fn);
    case kRadM4: return pick<Real, kWhole, kRadM4>(device, smem_optin, fn);
    case kWb: return pick<Real, kWhole, kWb>(device, smem_optin, fn);
    case 4 + kPlain: return pick<Real, kDual, kPlain>(device, smem_optin, fn);
    case 4 + kRadPxx: return pick<Real, kDual, kRadPxx>(device, smem_optin, fn);
    case 4 + kRadM4: return pick<Real, kDual, kRadM4>(device, smem_optin, fn);
    default: return pick<Real, kDual, kWb>(device, smem_optin, fn);
    }
}

// Does a cell of n particles fit in one CTA's shared memory staged whole
// (velocities, change bitmap, slot table)?  The same test as the kernel's.
template <typename Real>
size_t whole_bytes(uint64_t n)
{
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    return a16(3 * size_t(n) * sizeof(Real)) + a16(4 * size_t((n + 31) / 32)) + a16(4 * size_t(n));
}

template <typename Real>
bool fits_whole(uint64_t n, int smem) { return whole_bytes<Real>(n) <= size_t(smem); }

size_t static_cell_bytes(int64_t n, size_t real, bool wb);

// A launch whose largest cell needs at most 5/4 of a CTA's shared memory
// stays in the whole-staging mode when the cell fits its CTA's slab: the few
// cells that do not fit are staged whole in global memory, and every other
// cell keeps the faster kernel (more CTAs per SM).  Cells larger still are on
// the launch's critical path, and the dual kernel's compact staging serves
// them better.
template <typename Real>
bool near_whole(uint64_t n, int smem) { return whole_bytes<Real>(n) * 4 <= size_t(smem) * 5; }

// Dynamic shared memory of one CTA when per_sm CTAs share an SM: the SM's
// budget (226 KB where the device lets a CTA opt in to 200 KB or more, else
// the opt-in limit) split evenly, less the static part and 1 KB per CTA that
// the SM reserves; never more than one CTA may have.
template <typename Real>
int collide_smem(int smem_optin, int per_sm)
{
    const int budget = smem_optin >= 200 * 1024 ? 226 * 1024 : smem_optin;
    int smem = budget / per_sm - int(sizeof(Sh<Real>)) - 1024;
    if (smem > smem_optin - int(sizeof(Sh<Real>))) smem = smem_optin - int(sizeof(Sh<Real>));
    return smem > 0 ? smem : 0;
}

template <typename Real>
trmc_status launch_t(trmc_ctx *ctx, trmc_state *st, const trmc_collide_params *prm, uint64_t step,
                     int64_t *report, trmc_stats *stats, cudaStream_t s)
{
    // CTA size and CTAs per SM from the context (default 128 x 4): several
    // cells per SM overlap one cell's serial phases with the others' work;
    // the shared-memory budget of an SM is split evenly between them
    const int threads = ctx->collide_threads, per_sm_target = ctx->collide_ctas_per_sm;
    const int smem = collide_smem<Real>(int(ctx->smem_optin), per_sm_target);
    // the mode: staged whole, unless the previous launch met a cell too large
    // for shared memory and for the whole-mode rule above (the first launch
    // of a context does not know: dual)
    // (CTAs of more than kThreads threads run the dual kernel, the only one
    // built for them; it stages the cells that fit whole all the same)
    const uint64_t nmax = ctx->n_max_host ? *ctx->n_max_host : ~0ull;
    bool dual = threads > kThreads || !fits_whole<Real>(nmax, smem);
    const bool near = dual && threads <= kThreads && near_whole<Real>(nmax, smem);
    CollideFn fn = nullptr;
    cudaError_t e = collide_fn<Real>(ctx->device, int(ctx->smem_optin), dual && !near, prm, fn);
    if (e != cudaSuccess) return cuda_error(ctx, e, "cudaFuncSetAttribute(collide)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "occupancy(collide)");
    if (per_sm < 1) per_sm = 1;
    int grid = ctx->num_sms * per_sm;
    if (grid > st->n_cells) grid = st->n_cells;
    if (grid < 1) return TRMC_OK;
    if (near) {
        // whole mode if the largest cell, with room for its plan, fits a slab
        const size_t slab = (ctx->slabs_bytes / size_t(grid)) & ~size_t(255);
        dual = whole_bytes<Real>(nmax) + static_cell_bytes(int64_t(nmax), sizeof(Real), prm->trunc == TRMC_TRUNC_WB) >
               slab;
        if (dual) {
            e = collide_fn<Real>(ctx->device, int(ctx->smem_optin), true, prm, fn);
            if (e != cudaSuccess) return cuda_error(ctx, e, "cudaFuncSetAttribute(collide)");
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
            if (e != cudaSuccess) return cuda_error(ctx, e, "occupancy(collide)");
            if (per_sm < 1) per_sm = 1;
            grid = ctx->num_sms * per_sm;
            if (grid > st->n_cells) grid = st->n_cells;
        }
    }
    Args a;
    a.vx = st->vx; a.vy = st->vy; a.vz = st->vz;
    a.cell_start = st->cell_start;
    a.n_cells = st->n_cells;
    a.m_max = st->m_max;
    a.cell_param = st->cell_param;
    a.cell_key = st->cell_key;
    a.cell_vmax2 = st->cell_vmax2;
    a.cell_carry = st->cell_carry;
    a.step_dev = st->step_dev;
    a.cell_order = st->cell_order;
    a.cell_cost = st->cell_cost;
    a.problem_id = st->problem_id;
    a.seed = ctx->seed;
    a.step = step;
    a.prm = *prm;
    a.report = report;
    a.stats = stats;
    a.status = ctx->status;
    a.tickets = ctx->tickets;
    a.n_max_host = ctx->n_max_dev;
    a.big = nullptr;
    a.big_stamp = 0;
    if (dual && nmax >= uint64_t(kBigCell) && ctx->big) {
        // the large cells' moment sums over eight SMs each, first
        a.big = ctx->big;
        a.big_stamp = ++ctx->big_stamp;
        const bool m4 = prm->trunc == TRMC_TRUNC_RAD && prm->indicator == TRMC_IND_M4;
        const Real *vx = static_cast<const Real *>(st->vx), *vy = static_cast<const Real *>(st->vy),
                   *vz = static_cast<const Real *>(st->vz);
        if (m4) bigsum_kernel<Real, true><<<kBigSlots * kVW, 32, 0, s>>>(vx, vy, vz, st->cell_start, st->n_cells,
                                                                          ctx->big, a.big_stamp);
        else bigsum_kernel<Real, false><<<kBigSlots * kVW, 32, 0, s>>>(vx, vy, vz, st->cell_start, st->n_cells,
                                                                         ctx->big, a.big_stamp);
    }
    a.slabs = ctx->slabs;
    a.slab_bytes = (ctx->slabs_bytes / size_t(grid)) & ~size_t(255);
    a.smem_bytes = smem;
    a.warp_level = ctx->collide_warp_particles > 0 ? ctx->collide_warp_particles / 2
                   : sizeof(Real) == 8 ? kWarpLevel64 : kWarpLevel32;
    a.rec_per_thread = ctx->collide_records_per_thread > 0 ? ctx->collide_records_per_thread : kRecordPerThread;
    if (st->cell_cost && st->cell_order) order_kernel<<<1, 1024, 0, s>>>(st->cell_cost, st->n_cells, st->cell_order);
    fn<<<grid, threads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "collide launch");
    return TRMC_OK;
}

}  // namespace

trmc_status launch_collide(trmc_ctx *ctx, trmc_state *st, const trmc_collide_params *prm, uint64_t step,
                           int64_t *report, trmc_stats *stats, cudaStream_t s)
{
    if (ctx->precision == TRMC_FP64) return launch_t<double>(ctx, st, prm, step, report, stats, s);
    return launch_t<float>(ctx, st, prm, step, report, stats, s);
}

}  // namespace trmc

// ---- collision step without any allocation -----------------------------------
// Some callers cannot allocate device memory when they run the collision step:
// an application that advances the gas inside a section where cudaMalloc is
// not allowed (it may synchronise the whole device, or the host's memory
// manager owns every allocation), or a plug-in embedded in a program that
// hands it particle arrays but no allocator.  trmc_collide_static serves them:
// it needs no trmc_ctx, and its scratch (status word, work counter and the
// per-CTA overflow slabs for cells larger than shared memory) is one
// file-scope device array of TRMC_STATIC_SCRATCH_BYTES, which every GPU that
// loads the library keeps until the process exits.
namespace trmc {
namespace {

constexpr size_t kStaticControl = 4096;
static __device__ __align__(256) unsigned char g_static_scratch[TRMC_STATIC_SCRATCH_BYTES];

struct StaticDevice {
    bool ready = false;
    char *scratch = nullptr;   // device address of g_static_scratch on this device
    int num_sms = 0;
    int smem_optin = 0;
};
constexpr int kMaxDevices = 64;
StaticDevice g_static_dev[kMaxDevices];

// Working-set bound of one cell of n particles in the overflow slab: the
// slot table, the staged changed particles (at most n) and the continuation
// passes' position tables, the triangular plan tables at the deepest level,
// and product buffers for up to 4n consumers and n outputs (with TRMC-WB also
// their tree lengths and the rejected outputs' slots).
size_t static_cell_bytes(int64_t n, size_t real, bool wb)
{
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t N = size_t(n), T = size_t(TRMC_MCAP) * (TRMC_MCAP + 1) / 2 + 1;
    size_t b = a16(4 * N) + a16(3 * (N + 1) * real) + 2 * a16(4 * N) + 2 * a16(4 * T) +
               a16(3 * (3 * N + 1) * real) + a16(3 * (N + 1) * real) + 256;
    if (wb) b += a16(8 * (3 * N + 1)) + a16(8 * (N + 1)) + a16(4 * (N + 1));
    return b;
}

template <typename Real>
trmc_status launch_static(trmc_state *st, const trmc_collide_params *prm, uint64_t seed, uint64_t step,
                          int32_t max_cell, int *status_dev, cudaStream_t s)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TRMC_ERR_CUDA;
    StaticDevice &D = g_static_dev[dev];
    const int threads = 128, per_sm_target = 4;
    if (!D.ready) {
        // once per device, with that device current: the device address of the
        // scratch array (host code cannot use the array's name as a pointer)
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return TRMC_ERR_CUDA;
        if (cudaDeviceGetAttribute(&D.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TRMC_ERR_CUDA;
        if (cudaDeviceGetAttribute(&D.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return TRMC_ERR_CUDA;
        D.scratch = static_cast<char *>(p);
        D.ready = true;
    }
    const int smem = collide_smem<Real>(D.smem_optin, per_sm_target);
    CollideFn fn = nullptr;
    if (collide_fn<Real>(dev, D.smem_optin, true, prm, fn) != cudaSuccess) return TRMC_ERR_CUDA;
    const size_t avail = size_t(TRMC_STATIC_SCRATCH_BYTES) - kStaticControl;
    const size_t need = static_cell_bytes(max_cell, sizeof(Real), prm->trunc == TRMC_TRUNC_WB);
    int grid = int(std::min<size_t>(avail / need, size_t(D.num_sms) * per_sm_target));
    if (grid < 1) return TRMC_ERR_CAPACITY;       // a cell of max_cell particles cannot fit the scratch
    if (grid > st->n_cells) grid = st->n_cells;
    // the work counter must start at zero; the status word too
    if (cudaMemsetAsync(D.scratch, 0, kStaticControl, s) != cudaSuccess) return TRMC_ERR_CUDA;
    Args a;
    a.vx = st->vx; a.vy = st->vy; a.vz = st->vz;
    a.cell_start = st->cell_start;
    a.n_cells = st->n_cells;
    a.m_max = st->m_max;
    a.cell_param = st->cell_param;
    a.cell_key = st->cell_key;
    a.cell_vmax2 = st->cell_vmax2;
    a.cell_carry = st->cell_carry;
    a.step_dev = st->step_dev;
    a.cell_order = st->cell_order;
    a.cell_cost = nullptr;
    a.problem_id = st->problem_id;
    a.seed = seed;
    a.step = step;
    a.prm = *prm;
    a.report = nullptr;
    a.stats = nullptr;
    a.status = status_dev ? status_dev : reinterpret_cast<int *>(D.scratch);
    a.tickets = reinterpret_cast<unsigned int *>(D.scratch + 64);
    a.n_max_host = nullptr;
    a.big = nullptr;
    a.big_stamp = 0;
    a.slabs = D.scratch + kStaticControl;
    a.slab_bytes = (avail / size_t(grid)) & ~size_t(255);
    a.smem_bytes = smem;
    a.warp_level = sizeof(Real) == 8 ? kWarpLevel64 : kWarpLevel32;
    a.rec_per_thread = kRecordPerThread;
    fn<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? TRMC_OK : TRMC_ERR_CUDA;
}

}  // namespace
}  // namespace trmc

extern "C" trmc_status trmc_collide_static(trmc_state *state, const trmc_collide_params *p, int32_t precision,
                                           uint64_t seed, uint64_t step, int32_t max_cell_particles,
                                           int *status_dev, void *stream)
{
    using namespace trmc;
    if (precision != TRMC_FP64 && precision != TRMC_FP32_MIXED) return TRMC_ERR_ARG;
    if (check_collide_args(state, p)) return TRMC_ERR_ARG;          // the same checks as trmc_collide
    if (max_cell_particles < 0) return TRMC_ERR_ARG;
    if (state->n_cells == 0) return TRMC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == TRMC_FP64) return launch_static<double>(state, p, seed, step, max_cell_particles, status_dev, s);
    return launch_static<float>(state, p, seed, step, max_cell_particles, status_dev, s);
}


// ---- self-test of the FP64 angle and logarithm evaluations --------------------
namespace trmc {
namespace {
__global__ void fp64_selftest_kernel(const uint64_t *k, int n, double *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t w = k[i];
        double s, c, s_ref, c_ref;
        sincos_2pi(w >> 11, s, c);
        sincospi(2.0 * u01(w), &s_ref, &c_ref);
        double *o = out + 8 * size_t(i);
        o[0] = s; o[1] = c; o[2] = s_ref; o[3] = c_ref;
        o[4] = log_u53((w >> 11) + 1);
        o[5] = log(u01_open(w));
        const double x = __longlong_as_double(
            (long long)((w & ((1ull << 52) - 1ull)) | ((1ull + (w >> 53) % 2045ull) << 52)));
        o[6] = sqrt_pos(x);
        o[7] = sqrt(x);
    }
}
}  // namespace
}  // namespace trmc

extern "C" trmc_status trmc_fp64_selftest(const uint64_t *words_dev, int32_t n, double *out_dev, void *stream)
{
    if (n < 0 || (n > 0 && (!words_dev || !out_dev))) return TRMC_ERR_ARG;
    if (n == 0) return TRMC_OK;
    trmc::fp64_selftest_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0,
                                 static_cast<cudaStream_t>(stream)>>>(words_dev, n, out_dev);
    return cudaGetLastError() == cudaSuccess ? TRMC_OK : TRMC_ERR_CUDA;
}

// ---- self-test of the split's integer Iround ----------------------------------
namespace trmc {
namespace {
__global__ void split_selftest_kernel(const double *q, const int32_t *R, const uint64_t *K, int n, int32_t *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = iround_q(uint64_t(__double_as_longlong(q[i])), uint32_t(R[i]), K[i]);
}
}  // namespace
}  // namespace trmc

extern "C" trmc_status trmc_split_selftest(const double *q_dev, const int32_t *R_dev, const uint64_t *K_dev, int32_t n,
                                           int32_t *out_dev, void *stream)
{
    if (n < 0 || (n > 0 && (!q_dev || !R_dev || !K_dev || !out_dev))) return TRMC_ERR_ARG;
    if (n == 0) return TRMC_OK;
    trmc::split_selftest_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0,
                                  static_cast<cudaStream_t>(stream)>>>(q_dev, R_dev, K_dev, n, out_dev);
    return cudaGetLastError() == cudaSuccess ? TRMC_OK : TRMC_ERR_CUDA;
}
