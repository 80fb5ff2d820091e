// isg_philox.cuh -- per-site Philox4x32-10 on the device.
//
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
//   (c0, c1, c2, c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key bumped by (W0, W1) between rounds.
//
// The counter of a site is (lo32(q), hi32(q), w2, w3) with q = j >> 2 the
// same-colour index over four, so within one launch only words 0 and 1 vary
// and only word 0 varies between the eight Philox calls of one 32-site word
// (q is a multiple of 8 there).  The first two rounds are therefore split:
//   round 0: the M1 product of w2 is launch-uniform (host-folded);
//   round 1: the M0 product of round-0's c0 = hi(M1 w2) ^ hi32(q) ^ k0 is
//            the same for the whole 32-site word (computed once per word).
// Each call then costs 18 wide multiplies and 19 three-input XORs instead
// of 20 and 20.  The round keys come from kernel parameters.
#pragma once

#include <cstdint>

#include "isg_internal.h"

namespace isg {

struct PhiloxWordPart {
    uint32_t r1_hi0;  // hi(M0 * c0') for round 1, c0' = r0_c0 ^ hi32(q)
    uint32_t r1_lo0;  // lo(M0 * c0'), the round-1 output word 3
};

__device__ __forceinline__ PhiloxWordPart philox_word_part(const PhiloxLaunch &pc, uint32_t q_hi)
{
    const uint64_t p = (uint64_t)kPhiloxM0 * (uint64_t)(pc.r0_c0 ^ q_hi);
    PhiloxWordPart w;
    w.r1_hi0 = (uint32_t)(p >> 32);
    w.r1_lo0 = (uint32_t)p;
    return w;
}

// Philox4x32-10 of counter (q_lo, q_hi, w2, w3) given the launch constants
// and the per-word part for q_hi; writes the four output words.
__device__ __forceinline__ void philox_site4(const PhiloxLaunch &pc, const PhiloxWordPart &wp,
                                             uint32_t q_lo, uint32_t &o0, uint32_t &o1,
                                             uint32_t &o2, uint32_t &o3)
{
    // round 0 (c0', c1' are per word / per launch and folded elsewhere)
    const uint64_t a = (uint64_t)kPhiloxM0 * (uint64_t)q_lo;
    const uint32_t c2 = (uint32_t)(a >> 32) ^ pc.r0_c2x;
    const uint32_t c3 = (uint32_t)a;
    // round 1
    const uint64_t b = (uint64_t)kPhiloxM1 * (uint64_t)c2;
    uint32_t x0 = (uint32_t)(b >> 32) ^ pc.r1_c0x;
    uint32_t x1 = (uint32_t)b;
    uint32_t x2 = wp.r1_hi0 ^ c3 ^ pc.rk1[1];
    uint32_t x3 = wp.r1_lo0;
    // rounds 2..9
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)x0;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)x2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ x1 ^ pc.rk0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ x3 ^ pc.rk1[r];
        x1 = (uint32_t)p1;
        x3 = (uint32_t)p0;
        x0 = n0;
        x2 = n2;
    }
    o0 = x0;
    o1 = x1;
    o2 = x2;
    o3 = x3;
}

}  // namespace isg
