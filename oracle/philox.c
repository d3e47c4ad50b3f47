/*
 * Philox4x32-10 counter-based generator, written from its published definition
 * (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11, section 4.2): ten rounds of a bijection on four
 * 32-bit words; each round multiplies words 0 and 2 by two fixed odd
 * multipliers, swaps the products' halves into new positions and XORs the round
 * key in; the two-word key is advanced by two Weyl increments between rounds.
 *
 * The paper (Szwed & Chmiel) only says that random particles and the random
 * scalars r2, r3 are drawn (section 3.1, section 3.3); which generator is left
 * open. Every random draw of the method is a pure function of
 * (seed, particle-in-swarm, swarm, iteration, tag, block) through this function.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"

static const uint32_t MUL0 = 0xD2511F53u;  /* multiplier applied to word 0 */
static const uint32_t MUL1 = 0xCD9E8D57u;  /* multiplier applied to word 2 */
static const uint32_t WEYL0 = 0x9E3779B9u; /* key increment, word 0 (golden ratio) */
static const uint32_t WEYL1 = 0xBB67AE85u; /* key increment, word 1 (sqrt(3) - 1) */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)MUL0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)MUL1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += WEYL0;
        k1 += WEYL1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag,
              uint32_t block, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, (tag << 24) | (block & 0xFFFFFFu)};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

double orc_u01(uint32_t u) {
    /* top 24 bits as a fraction: exact in fp32 and fp64, never 1.0 */
    return (double)(u >> 8) * (1.0 / 16777216.0);
}

uint32_t orc_below(uint32_t u, uint32_t k) {
    return (uint32_t)(((uint64_t)u * (uint64_t)k) >> 32);
}
