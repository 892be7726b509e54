// philox.cuh -- the counter-based Gaussian draw of the sketch (Sec. 3.2.1).
#pragma once
#include <stdint.h>

namespace rutv {

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 64 x 64 -> 128-bit multiplies, key bumped by the Weyl constants.
__device__ __forceinline__ void philox4x64_10(uint64_t x[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0 = __umul64hi(M0, x[0]), lo0 = M0 * x[0];
        uint64_t hi1 = __umul64hi(M1, x[2]), lo1 = M1 * x[2];
        uint64_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
        x[0] = y0; x[1] = lo1; x[2] = y2; x[3] = lo0;
    }
}

// Four entries G(4k .. 4k+3, c) of the Gaussian matrix of block step `step`:
// counter (k, c, step, 0), key (seed, 0); each 64-bit word x gives
// u = (floor(x / 2^11) + 1) 2^-53 in (0, 1]; Box-Muller on the word pairs
// (0,1) -> rows 4k, 4k+1 and (2,3) -> rows 4k+2, 4k+3:
//   z_even = sqrt(-2 ln u_a) cos(2 pi u_b),  z_odd = sqrt(-2 ln u_a) sin(2 pi u_b).
__device__ __forceinline__ void gaussian4(uint64_t seed, int64_t step, int64_t k, int64_t c, double z[4]) {
    const double two_pi = 6.283185307179586476925286766559;
    const double inv53 = 1.0 / 9007199254740992.0;
    uint64_t x[4] = {(uint64_t)k, (uint64_t)c, (uint64_t)step, 0};
    philox4x64_10(x, seed, 0);
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
        double ua = ((double)(x[2 * pr] >> 11) + 1.0) * inv53;
        double ub = ((double)(x[2 * pr + 1] >> 11) + 1.0) * inv53;
        double rad = sqrt(-2.0 * log(ua));
        double s, co;
        sincos(two_pi * ub, &s, &co);
        z[2 * pr] = rad * co;
        z[2 * pr + 1] = rad * s;
    }
}

}  // namespace rutv
