/*
 * Counter-based generator for the oracle: Philox4x64 with 10 rounds, written
 * from its published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11): each round multiplies counter words 0
 * and 2 by two fixed odd constants, swaps the high/low halves across the
 * words and xors in the key, which is bumped by two Weyl constants.
 *
 * TEST INFRASTRUCTURE ONLY (see bs_oracle.h).
 */
#include "bs_oracle.h"

static const uint64_t PH_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PH_M1 = 0xCA5A826395121157ULL;
static const uint64_t PH_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PH_W1 = 0xBB67AE8584CAA73BULL;

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 prod = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(prod >> 64);
    *lo = (uint64_t)prod;
}

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(PH_M0, c0, &hi0, &lo0);
        mulhilo64(PH_M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PH_W0;
        k1 += PH_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Each 64-bit output word gives two uniforms: the top 24 bits of its high
 * and of its low 32-bit half, centred in their bins: (j + 1/2) 2^-24. */
void or_uniforms8(uint64_t seed, uint64_t chain_key, uint64_t c0, uint64_t c1,
                  uint64_t c2, double u[8])
{
    uint64_t ctr[4] = {c0, c1, c2, 0};
    uint64_t key[2] = {seed, chain_key};
    uint64_t w[4];
    or_philox4x64_10(ctr, key, w);
    const double scale = 1.0 / 16777216.0;
    for (int j = 0; j < 4; ++j) {
        uint64_t hi = w[j] >> 32, lo = w[j] & 0xFFFFFFFFULL;
        u[2 * j]     = ((double)(hi >> 8) + 0.5) * scale;
        u[2 * j + 1] = ((double)(lo >> 8) + 0.5) * scale;
    }
}
