// Exact reduction of an angle to a fraction of a turn, shared by the kernels
// that place points on a periodic grid (set_points, the Lagrange comparator).
//
// The doubled torus is 2 pi periodic in both angles, so a coordinate only
// matters as a fraction of a turn.  That fraction is computed exactly in
// integer arithmetic from the FP64 bit pattern: Y = floor(v / (2 pi) 2^64)
// mod 2^64 (Q0.64 turns), from the 53-bit significand times 1/(2 pi) held to
// 128 bits.  GB300 runs FP64 at a small fraction of its integer rate, and the
// fixed-point result is also more accurate (one unit in 2^-64 turns) than an
// FP64 product would be.
#pragma once

namespace {

// 1/(2 pi) as an unsigned Q0.128 number, floor(2^128 / (2 pi)) (Machin's formula).
#define DFS_INV_2PI_HI 0x28be60db9391054aULL
#define DFS_INV_2PI_LO 0x7f09d5f47d4d3770ULL

// Fraction of a turn of v in Q0.64.  False for inf/nan and for |v| >= 2^53,
// where FP64 no longer resolves a position within a turn.
__device__ __forceinline__ bool turns_q64(double v, unsigned long long &Y) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    int e = (int)((bits >> 52) & 0x7ff);
    if (e == 0x7ff) return false;
    unsigned long long m = bits & 0xfffffffffffffULL;
    if (e == 0) e = 1;                      // subnormal: m * 2^(1 - 1075)
    else m |= 1ULL << 52;                   // |v| = m * 2^(e - 1075)
    const int sh = 1139 - e;                // Y = floor(m * K * 2^-sh), K = 2^128 / (2 pi)
    if (sh < 64) return false;
    unsigned long long y = 0;
    if (sh < 192) {
        const unsigned long long hi0 = __umul64hi(m, DFS_INV_2PI_LO);
        const unsigned long long lo1 = m * DFS_INV_2PI_HI;
        const unsigned long long hi1 = __umul64hi(m, DFS_INV_2PI_HI);
        const unsigned long long p1 = hi0 + lo1;          // product bits 64..127
        const unsigned long long p2 = hi1 + (p1 < hi0);   // product bits 128..
        if (sh >= 128) {
            y = p2 >> (sh - 128);
        } else {
            const int s = sh - 64;
            y = s ? ((p1 >> s) | (p2 << (64 - s))) : p1;
        }
    }
    Y = (bits >> 63) ? 0ULL - y : y;
    return true;
}

}  // namespace
