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
 * The permutation is a 4-round balanced Feistel network on 2h-bit words
 * (Luby-Rackoff) restricted to [0,n) by cycle walking (Black & Rogaway 2002).
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

void orc_prp_init(orc_prp *p, uint64_t n, const uint64_t key[4])
{
    p->n = n;
    int h = 1;
    while ((1ULL << (2 * h)) < n) ++h;
    p->h = h;
    for (int i = 0; i < 4; ++i) p->key[i] = key[i];
}

static uint64_t feistel_enc(const orc_prp *p, uint64_t x)
{
    uint64_t mask = (1ULL << p->h) - 1;
    uint64_t L = x >> p->h, R = x & mask;
    for (int r = 0; r < 4; ++r) {
        uint64_t nl = R;
        uint64_t nr = L ^ ((uint64_t)feistel_f((uint32_t)R, p->key[r]) & mask);
        L = nl; R = nr;
    }
    return (L << p->h) | R;
}

static uint64_t feistel_dec(const orc_prp *p, uint64_t y)
{
    uint64_t mask = (1ULL << p->h) - 1;
    uint64_t L = y >> p->h, R = y & mask;
    for (int r = 3; r >= 0; --r) {
        uint64_t pr = L;
        uint64_t pl = R ^ ((uint64_t)feistel_f((uint32_t)L, p->key[r]) & mask);
        L = pl; R = pr;
    }
    return (L << p->h) | R;
}

uint64_t orc_prp_fwd(const orc_prp *p, uint64_t x)
{
    if (p->n <= 1) return 0;
    uint64_t y = feistel_enc(p, x);
    while (y >= p->n) y = feistel_enc(p, y);
    return y;
}

uint64_t orc_prp_inv(const orc_prp *p, uint64_t y)
{
    if (p->n <= 1) return 0;
    uint64_t x = feistel_dec(p, y);
    while (x >= p->n) x = feistel_dec(p, x);
    return x;
}
