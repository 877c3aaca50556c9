/*
 * rng.c -- oracle random numbers.  TEST INFRASTRUCTURE ONLY (see trmc_oracle.h).
 *
 * The paper does not fix a generator.  The method's draws are keyed by
 * (step, cell, particle/collision, purpose) so that a cell's result does not
 * depend on which thread or launch computes it; a counter-based generator is
 * the natural fit.  We use Philox4x64-10 as defined by Salmon, Moraes, Dror and
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of
 *     (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
 * with the key bumped by the Weyl constants between rounds.
 *
 * The permutation of [0,n) realises Alg. 4.3's "random choice", so every
 * subset of it must be close to uniform.  Two constructions, by size:
 *  - n <= 32: the order of n keys.  Item y gets the 32-bit key
 *    fmix32((lo(w0) ^ y*0x9E3779B9) + hi(w0)) (fmix32: MurmurHash3's
 *    finaliser, a bijection, so the n keys are distinct), and pi(y) is the
 *    number of items with a smaller key.  Feistel networks are far from
 *    uniform on such small domains, whatever the number of rounds.
 *  - n > 32: an alternating Feistel network (Luby-Rackoff) on b-bit words,
 *    2^(b-1) < n <= 2^b: the high ceil(b/2) bits A and the low floor(b/2)
 *    bits B; eight rounds for b <= 8, six above, round r adding F(B, k_r) to A
 *    (r even) or F(A, k_r) to B (r odd) by exclusive or; round keys w0..w3 and
 *    then w0..w3 with their 32-bit halves swapped.  Restricted to [0,n) by
 *    cycle walking (Black & Rogaway, CT-RSA 2002), which takes fewer than two
 *    steps on average.
 * The four words w0..w3 are one Philox draw.
 */
#include "trmc_oracle.h"

#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

static void mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mul128(PHILOX_M0, c0, &hi0, &lo0);
        mul128(PHILOX_M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout: (index, aux, cell, step<<16 | pass<<8 | tag); key (seed, problem). */
void orc_draw(uint64_t seed, uint64_t problem, uint64_t index, uint64_t aux,
              uint64_t cell, uint64_t step, uint32_t pass, uint32_t tag, uint64_t out[4])
{
    uint64_t ctr[4] = { index, aux, cell,
                        (step << 16) | ((uint64_t)(pass & 0xFFu) << 8) | (uint64_t)(tag & 0xFFu) };
    uint64_t key[2] = { seed, problem };
    orc_philox4x64(ctr, key, out);
}

double orc_u01(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }
double orc_u01_open(uint64_t w) { return (double)((w >> 11) + 1) * 0x1.0p-53; }
uint32_t orc_below(uint64_t w, uint32_t n)
{
    return (uint32_t)(((w >> 32) * (uint64_t)n) >> 32);
}

/* --- permutation ---------------------------------------------------------- */
static uint32_t feistel_f(uint32_t r, uint64_t k)
{
    uint32_t z = (r ^ (uint32_t)k) * 0x9E3779B1u;
    z ^= z >> 15;
    z = (z + (uint32_t)(k >> 32)) * 0x85EBCA77u;
    z ^= z >> 13;
    return z;
}

static uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

void orc_prp_init(orc_prp *p, uint64_t n, const uint64_t key[4])
{
    p->n = n;
    int b = 1;
    while ((1ULL << b) < n) ++b;
    p->b = b;
    for (int i = 0; i < 4; ++i) p->key[i] = key[i];
}

/* the key of item y (n <= 32) */
static uint32_t rank_key(const orc_prp *p, uint64_t y)
{
    uint32_t lo = (uint32_t)p->key[0], hi = (uint32_t)(p->key[0] >> 32);
    return fmix32((lo ^ ((uint32_t)y * 0x9E3779B9u)) + hi);
}

/* rounds of the Feistel network: eight on words of up to 8 bits, six on
 * wider ones (where six already pass the permutation pins at 10^5 keys) */
static int feistel_rounds(const orc_prp *p)
{
    return p->b <= 8 ? 8 : 6;
}

/* round key r of the Feistel network */
static uint64_t round_key(const orc_prp *p, int r)
{
    uint64_t w = p->key[r & 3];
    return r < 4 ? w : (w << 32) | (w >> 32);
}

static uint64_t feistel_enc(const orc_prp *p, uint64_t x)
{
    int c = p->b / 2, a = p->b - c;
    uint64_t ma = (1ULL << a) - 1, mb = (1ULL << c) - 1;
    uint64_t A = x >> c, B = x & mb;
    for (int r = 0; r < feistel_rounds(p); ++r) {
        if (r % 2 == 0) A ^= (uint64_t)feistel_f((uint32_t)B, round_key(p, r)) & ma;
        else B ^= (uint64_t)feistel_f((uint32_t)A, round_key(p, r)) & mb;
    }
    return (A << c) | B;
}

static uint64_t feistel_dec(const orc_prp *p, uint64_t y)
{
    int c = p->b / 2, a = p->b - c;
    uint64_t ma = (1ULL << a) - 1, mb = (1ULL << c) - 1;
    uint64_t A = y >> c, B = y & mb;
    for (int r = feistel_rounds(p) - 1; r >= 0; --r) {
        if (r % 2 == 0) A ^= (uint64_t)feistel_f((uint32_t)B, round_key(p, r)) & ma;
        else B ^= (uint64_t)feistel_f((uint32_t)A, round_key(p, r)) & mb;
    }
    return (A << c) | B;
}

uint64_t orc_prp_fwd(const orc_prp *p, uint64_t x)
{
    if (p->n <= 1) return 0;
    if (p->n <= 32) {
        uint32_t kx = rank_key(p, x);
        uint64_t r = 0;
        for (uint64_t y = 0; y < p->n; ++y) r += rank_key(p, y) < kx;
        return r;
    }
    uint64_t y = feistel_enc(p, x);
    while (y >= p->n) y = feistel_enc(p, y);
    return y;
}

uint64_t orc_prp_inv(const orc_prp *p, uint64_t y)
{
    if (p->n <= 1) return 0;
    if (p->n <= 32) {
        for (uint64_t x = 0; x < p->n; ++x)
            if (orc_prp_fwd(p, x) == y) return x;
        return 0;     /* not reached for y < n */
    }
    uint64_t x = feistel_dec(p, y);
    while (x >= p->n) x = feistel_dec(p, x);
    return x;
}

/* forward tables of K permutations of [0,n) at once, for the statistical pins:
 * out[j][x] = pi_j(x), pi_j keyed by keys[j][0..3] */
void orc_prp_tables(uint64_t n, const uint64_t *keys, int64_t K, int32_t *out)
{
    for (int64_t j = 0; j < K; ++j) {
        orc_prp p;
        orc_prp_init(&p, n, keys + 4 * j);
        for (uint64_t x = 0; x < n; ++x) out[j * (int64_t)n + (int64_t)x] = (int32_t)orc_prp_fwd(&p, x);
    }
}
