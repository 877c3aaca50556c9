// trmc_device.cuh -- device primitives of libtrmc: counter-based random
// numbers, the pseudo-random permutation and block reductions.
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11).  The paper fixes no
// generator; a counter-based one lets every draw be addressed by
// (seed, problem | index, aux, cell, step/pass/tag), so a cell's result does
// not depend on launch shape or batch placement.
//
// Permutation of [0, n): it realises the "random choice" of particles in
// Alg. 4.3 without materialising shuffles, so every subset of it must be close
// to uniform.  For n <= 32 it is the order of n distinct hashed keys; above,
// an 8-round alternating Feistel network on the smallest 2^b >= n with cycle
// walking onto [0, n) (Black & Rogaway, CT-RSA 2002).
#pragma once
#include <cstdint>

namespace trmc {

enum Tag : uint32_t {
    TAG_INIT = 1, TAG_SPLIT = 2, TAG_PARITY = 3, TAG_KSEL = 4,
    TAG_PERM0 = 5, TAG_PERMK = 6, TAG_COLL = 7, TAG_MAXW = 8, TAG_RESERVOIR = 9
};

struct U64x4 { uint64_t w[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        const uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
        const uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
        const uint64_t n0 = hi1 ^ c1 ^ k0;
        const uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    U64x4 o;
    o.w[0] = c0; o.w[1] = c1; o.w[2] = c2; o.w[3] = c3;
    return o;
}

// Keyed stream of one cell: key = (seed, problem); the fourth counter word
// packs step, pass and purpose tag.  A draw is about 300 instructions and the
// collision kernel makes them in many places: one shared copy (not inlined)
// keeps the kernel's code small enough for the instruction caches.  The
// shared copy takes its words as arguments, which travel in registers; a
// member function would need its object's address, and so a copy of the
// object in local memory at every call (on GB300, with most of the SM's
// unified memory given to shared memory, local memory lives mostly in L2).
static __device__ __noinline__ U64x4 philox_draw(uint64_t index, uint64_t aux, uint64_t cell, uint64_t c3,
                                                 uint64_t seed, uint64_t problem)
{
    return philox4x64_10(index, aux, cell, c3, seed, problem);
}

struct CellRng {
    uint64_t seed, problem, cell, step;
    __device__ __forceinline__ U64x4 draw(uint64_t index, uint64_t aux, uint32_t pass, uint32_t tag) const
    {
        const uint64_t c3 = (step << 16) | (uint64_t(pass & 0xFFu) << 8) | uint64_t(tag & 0xFFu);
        return philox_draw(index, aux, cell, c3, seed, problem);
    }
};

// 53-bit uniforms on [0,1) and (0,1]; 24-bit float uniform; integer below n.
__device__ __forceinline__ double u01(uint64_t w) { return double(w >> 11) * 0x1.0p-53; }
__device__ __forceinline__ double u01_open(uint64_t w) { return double((w >> 11) + 1) * 0x1.0p-53; }
__device__ __forceinline__ float u01f(uint64_t w) { return float(uint32_t(w >> 40)) * 0x1.0p-24f; }
__device__ __forceinline__ float u01f_open(uint64_t w) { return float(uint32_t(w >> 40) + 1u) * 0x1.0p-24f; }
__device__ __forceinline__ uint32_t below(uint64_t w, uint32_t n)
{
    return uint32_t(((w >> 32) * uint64_t(n)) >> 32);
}

// ---- permutation of [0, n) ---------------------------------------------------
__device__ __forceinline__ uint32_t feistel_round(uint32_t r, uint64_t k)
{
    uint32_t z = (r ^ uint32_t(k)) * 0x9E3779B1u;
    z ^= z >> 15;
    z = (z + uint32_t(k >> 32)) * 0x85EBCA77u;
    z ^= z >> 13;
    return z;
}

// Round key r of the Feistel network: the draw's four words, then the same
// words with their 32-bit halves swapped.
__device__ __forceinline__ uint64_t swap32(uint64_t w) { return (w << 32) | (w >> 32); }

// One pass of the rounds (enc) and the rounds undone, last first (dec), on a
// b-bit word: A, the high ceil(b/2) bits, takes F of B in the even rounds; B,
// the low floor(b/2) bits, takes F of A in the odd ones.  Eight rounds for
// b <= 8, six for wider words (where six already pass the permutation pins at
// 10^5 keys).
__device__ __forceinline__ uint32_t feistel_enc(uint32_t x, uint32_t b, uint64_t k0, uint64_t k1, uint64_t k2,
                                                uint64_t k3)
{
    const uint32_t c = b >> 1, ma = (1u << (b - c)) - 1u, mb = (1u << c) - 1u;
    uint32_t A = x >> c, B = x & mb;
    A ^= feistel_round(B, k0) & ma; B ^= feistel_round(A, k1) & mb;
    A ^= feistel_round(B, k2) & ma; B ^= feistel_round(A, k3) & mb;
    A ^= feistel_round(B, swap32(k0)) & ma; B ^= feistel_round(A, swap32(k1)) & mb;
    if (b <= 8) { A ^= feistel_round(B, swap32(k2)) & ma; B ^= feistel_round(A, swap32(k3)) & mb; }
    return (A << c) | B;
}
__device__ __forceinline__ uint32_t feistel_dec(uint32_t y, uint32_t b, uint64_t k0, uint64_t k1, uint64_t k2,
                                                uint64_t k3)
{
    const uint32_t c = b >> 1, ma = (1u << (b - c)) - 1u, mb = (1u << c) - 1u;
    uint32_t A = y >> c, B = y & mb;
    if (b <= 8) { B ^= feistel_round(A, swap32(k3)) & mb; A ^= feistel_round(B, swap32(k2)) & ma; }
    B ^= feistel_round(A, swap32(k1)) & mb; A ^= feistel_round(B, swap32(k0)) & ma;
    B ^= feistel_round(A, k3) & mb; A ^= feistel_round(B, k2) & ma;
    B ^= feistel_round(A, k1) & mb; A ^= feistel_round(B, k0) & ma;
    return (A << c) | B;
}

// Key of item y for n <= 32: MurmurHash3's 32-bit finaliser (a bijection) of
// a bijection of y, so the keys of distinct items differ.
__device__ __forceinline__ uint32_t rank_key(uint32_t y, uint64_t k0)
{
    uint32_t h = (uint32_t(k0) ^ (y * 0x9E3779B9u)) + uint32_t(k0 >> 32);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// The evaluations below are noinline, each with one copy of the rounds: the
// collision kernel calls them from several phases, and on GB300 the size of
// its code (instruction fetch) costs more than the calls.
// n <= 32: pi(x0) | pi(x1) << 32, each the number of items with a smaller key
static __device__ __noinline__ uint64_t perm_rank2(uint32_t x0, uint32_t x1, uint32_t n, uint64_t k0)
{
    const uint32_t kx0 = rank_key(x0, k0), kx1 = rank_key(x1, k0);
    uint32_t y0 = 0, y1 = 0;
    for (uint32_t y = 0; y < n; ++y) {
        const uint32_t ky = rank_key(y, k0);
        y0 += ky < kx0;
        y1 += ky < kx1;
    }
    return uint64_t(y0) | (uint64_t(y1) << 32);
}
// n <= 32: pi^-1(y), the item whose key has y smaller ones
static __device__ __noinline__ uint32_t perm_rank_inv(uint32_t y, uint32_t n, uint64_t k0)
{
    for (uint32_t x = 0; x < n; ++x) {
        const uint32_t kx = rank_key(x, k0);
        uint32_t r = 0;
        for (uint32_t z = 0; z < n; ++z) r += rank_key(z, k0) < kx;
        if (r == y) return x;
    }
    return 0;     // not reached for y < n
}
// n > 32: encrypt x, and again while the word lies outside [0, n)
static __device__ __noinline__ uint32_t perm_walk(uint32_t x, uint32_t n, uint32_t b, uint64_t k0, uint64_t k1,
                                                  uint64_t k2, uint64_t k3)
{
    uint32_t y = x;
    do { y = feistel_enc(y, b, k0, k1, k2, k3); } while (y >= n);
    return y;
}
// n > 32: the cycle through y walked backwards
static __device__ __noinline__ uint32_t perm_walk_back(uint32_t y, uint32_t n, uint32_t b, uint64_t k0, uint64_t k1,
                                                       uint64_t k2, uint64_t k3)
{
    uint32_t x = y;
    do { x = feistel_dec(x, b, k0, k1, k2, k3); } while (x >= n);
    return x;
}

struct Perm {
    uint32_t n;
    uint32_t b;       // word width in bits: 2^(b-1) < n <= 2^b
    uint64_t k[4];

    __device__ __forceinline__ void init(uint32_t n_, const U64x4 &key)
    {
        n = n_;
        b = n_ <= 1 ? 0u : 32u - uint32_t(__clz(n_ - 1u));
        k[0] = key.w[0]; k[1] = key.w[1]; k[2] = key.w[2]; k[3] = key.w[3];
    }
    // pi(x0) and pi(x1) (a collision's two products), and pi^-1(y), for
    // arguments below n; the key words travel as arguments like philox_draw's
    __device__ __forceinline__ void fwd2(uint32_t x0, uint32_t x1, int &y0, int &y1) const
    {
        if (n <= 1) { y0 = y1 = 0; return; }
        if (n <= 32) {
            const uint64_t y = perm_rank2(x0, x1, n, k[0]);
            y0 = int(uint32_t(y));
            y1 = int(uint32_t(y >> 32));
            return;
        }
        y0 = int(perm_walk(x0, n, b, k[0], k[1], k[2], k[3]));
        y1 = int(perm_walk(x1, n, b, k[0], k[1], k[2], k[3]));
    }
    __device__ __forceinline__ uint32_t inv(uint32_t y) const
    {
        if (n <= 1) return 0;
        if (n <= 32) return perm_rank_inv(y, n, k[0]);
        return perm_walk_back(y, n, b, k[0], k[1], k[2], k[3]);
    }
};

// ---- warp / block reductions (fixed order, hence deterministic) --------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduction scratch: warp partials at [w*K + j] (w*K < 256: CTAs of up to 256
// threads for K = 16), block_sum totals at [256 + j], their quotients by a
// divisor at [264 + j] (K <= 8), the block_max total at [264].
constexpr int kRedScratch = 272;

// Sum K doubles over the block (K <= 16); every thread gets the totals and,
// with a divisor (K <= 8), the totals divided by it.
// scratch holds kRedScratch doubles.  Inside a warp the K values are
// reduce-scattered: at each of the first log2(P) shuffle steps (P = K rounded
// up to a power of two) a lane keeps half of its values and adds its
// partner's copies of them, so a warp spends P - 1 + log2(32/P) FP64 adds
// instead of 5K (GB300 issues FP64 at 2 lanes/clk/SM; a warp instruction costs
// 16 cycles whatever its active lanes).  Warp partials are then combined by
// warp 0 alone, lane j summing value j.  Fixed order, hence deterministic.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *scratch, double div = 0.0, double *quot = nullptr)
{
    static_assert(K >= 1 && K <= 16, "block_sum handles 1..16 values");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int P = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : 16, G = 32 / P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double t[P];
#pragma unroll
    for (int i = 0; i < P; ++i) t[i] = i < K ? v[i] : 0.0;
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
    if ((lane & (G - 1)) == 0 && idx < K) scratch[warp * K + idx] = t[0];
    __syncthreads();
    if (warp == 0 && lane < K) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += scratch[w * K + lane];
        scratch[256 + lane] = s;
        if (quot && K <= 8) scratch[264 + lane] = s / div;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = scratch[256 + j];
    if (quot && K <= 8) {
#pragma unroll
        for (int j = 0; j < K; ++j) quot[j] = scratch[264 + j];
    }
}

// a + b for unevaluated float pairs (hi, lo): TwoSum of the high parts, the
// low parts and the rounding error added, renormalised (about 48 bits)
__device__ __forceinline__ void ff_add(float &ah, float &al, float bh, float bl)
{
    const float s = ah + bh, bb = s - ah;
    float e = (ah - (s - bb)) + (bh - bb);
    e += al + bl;
    const float h = s + e;
    al = e - (h - s);
    ah = h;
}

// The same block sum for K compensated float partial sums (hi, lo), added as
// float pairs all the way, so no FP64 instruction is issued until warp 0
// converts the K totals.
template <int K>
__device__ __forceinline__ void block_sum_ff(const float (&vh)[K], const float (&vl)[K], double (&out)[K],
                                             double *scratch, double div = 0.0, double *quot = nullptr)
{
    static_assert(K >= 1 && K <= 16, "block_sum_ff handles 1..16 values");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int P = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : 16, G = 32 / P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    float th[P], tl[P];
#pragma unroll
    for (int i = 0; i < P; ++i) { th[i] = i < K ? vh[i] : 0.0f; tl[i] = i < K ? vl[i] : 0.0f; }
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
    float2 *sf = reinterpret_cast<float2 *>(scratch);
    if ((lane & (G - 1)) == 0 && idx < K) sf[warp * K + idx] = make_float2(th[0], tl[0]);
    __syncthreads();
    if (warp == 0 && lane < K) {
        float h = 0.0f, l = 0.0f;
        for (int w = 0; w < nw; ++w) { const float2 p = sf[w * K + lane]; ff_add(h, l, p.x, p.y); }
        const double s = double(h) + double(l);
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

// Sum K ints over the block; every thread gets the totals (K <= 8).
template <int K>
__device__ __forceinline__ void block_sum_int(int (&v)[K], double *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int *si = reinterpret_cast<int *>(scratch);
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = int(__reduce_add_sync(0xffffffffu, unsigned(v[j])));
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < K; ++j) si[warp * K + j] = v[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < K; ++j) {
        int s = 0;
        for (int w = 0; w < nw; ++w) s += si[w * K + j];
        v[j] = s;
    }
    __syncthreads();
}

// Maximum of a non-negative double over the block, on the bit patterns (they
// order like the values), so it costs no FP64 instruction.
__device__ __forceinline__ double block_max_nonneg(double v, double *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    long long *sl = reinterpret_cast<long long *>(scratch);
    if (lane == 0) sl[warp] = b;
    __syncthreads();
    long long m = sl[0];
    for (int w = 1; w < nw; ++w) m = max(m, sl[w]);
    __syncthreads();
    return __longlong_as_double(m);
}

__device__ __forceinline__ double block_max(double v, double *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = scratch[0];
        for (int w = 1; w < nw; ++w) m = fmax(m, scratch[w]);
        scratch[264] = m;
    }
    __syncthreads();
    return scratch[264];
}

}  // namespace trmc
