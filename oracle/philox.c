/*
 * Oracle (test infrastructure only): the counter-based generator.
 *
 * Philox4x32 with 10 rounds, written from its published definition
 * (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11): each round multiplies counter words
 * 0 and 2 by the two Philox multipliers, and the new counter is
 * (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key
 * is bumped by the two Weyl constants between rounds.
 *
 * The paper only asks for "a univariate R"; the generator, the counter
 * layout and the uniform conversion are this implementation's own reading
 * and are specified identically (not shared as code) on both sides:
 *   key     = (seed low 32 bits, seed high 32 bits)
 *   counter = (packet id low, packet id high, event index, draw block)
 *   uniform = ((r >> 8) | 1) * 2^-24   -- odd multiples of 2^-24, strictly
 *             inside (0,1), exact in FP32 and FP64, symmetric under u -> 1-u.
 */
#include "oracle.h"
#include <math.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void o_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double o_uniform(uint32_t r) {
  return ldexp((double)((r >> 8) | 1u), -24);
}

void o_philox_many(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n) {
  for (size_t i = 0; i < n; ++i) o_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}
