// Integer arithmetic of the Ozaki schemes shared by the GEMM (gemm_oz.cu) and the O(r^5) products on the
// tensor cores (acse_zoz.cu): powers of two, the fixed-point value of an element, and the rounding of an
// exact integer back to FP64.  FP64 arithmetic is slow on this GPU, so all of them work on bit patterns.
#pragma once
#include <string.h>

// 2^n for -1022 <= n <= 1023, built from its bit pattern (exact)
__host__ __device__ __forceinline__ double oz_pow2(int n) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)(n + 1023) << 52);
#else
    const long long bits = (long long)(n + 1023) << 52;
    double d;
    memcpy(&d, &bits, sizeof(d));
    return d;
#endif
}

// Fixed-point value of one element: X = round(a 2^(nb - e)) from the bit pattern of a (ties away from
// zero), |X| <= 2^(nb-1) when |a| 2^-e < 1/2, nb <= 54 (integer arithmetic only: FP64 is slow on this GPU).
__device__ __forceinline__ long long oz_fixedb(unsigned long long bits, int nb, int e) {
    const int E = (int)((bits >> 52) & 0x7FF);
    const long long m = (long long)(bits & 0xFFFFFFFFFFFFFull) | (E ? (1ll << 52) : 0ll);
    const int sh = (E ? E : 1) - 1075 + nb - e;   // a = m 2^((E ? E : 1) - 1075)
    long long X;
    if (sh >= 0) X = m << sh;                      // < 2^(nb-1) by the choice of e
    else if (sh > -63) X = (m + (1ll << (-sh - 1))) >> -sh;
    else X = 0;
    return (bits >> 63) ? -X : X;
}

// The same for S six-bit slices: X = round(a 2^(6S - e)), |X| < 2^(6S-1).  The rounding drops bits below
// 2^-6S of the row scale, as the remainder x_{S+1} of the digit recursion does.
__device__ __forceinline__ long long oz_fixed(unsigned long long bits, int S, int e) { return oz_fixedb(bits, 6 * S, e); }

// acc 2^ex rounded to the nearest double (ties to even), with integer operations only (FP64 is slow on
// this GPU): the leading bit of |acc| fixes the exponent, the 53 bits below it the significand, the
// rest decides the rounding.  Results outside the normal range take the FP64 route.
__device__ __forceinline__ double oz_ll_scaled(long long acc, int ex) {
    if (acc == 0) return 0.0;
    const unsigned long long sign = acc < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned long long u = acc < 0 ? 0ull - (unsigned long long)acc : (unsigned long long)acc;
    int msb = 63 - __clzll((long long)u);
    unsigned long long mant;
    if (msb <= 52) {
        mant = u << (52 - msb);
    } else {
        const int sh = msb - 52;
        mant = u >> sh;
        const unsigned long long rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (mant & 1))) {
            if (++mant == (1ull << 53)) {
                mant >>= 1;
                ++msb;
            }
        }
    }
    const int E = msb + ex + 1023;
    if (E < 1 || E > 2046) return __ll2double_rn(acc) * oz_pow2(min(1023, max(-1022, ex)));
    return __longlong_as_double((long long)(sign | ((unsigned long long)E << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// (-1)^neg (hi 2^64 + lo) 2^ex rounded to the nearest double (ties to even) with integer operations: the
// leading 64 bits of the 128-bit magnitude are shifted down by one to fit a signed int64, every bit below
// them folded into the lowest bit (a sticky bit, below the rounding position), and that goes through the
// 64-bit rounding above.
__device__ __forceinline__ double oz_u128_scaled(unsigned long long hi, unsigned long long lo, bool neg, int ex) {
    unsigned long long top, rest;
    int e0;   // magnitude = top 2^e0 + (rest below it)
    if (hi != 0) {
        const int sh = __clzll((long long)hi);
        top = sh ? (hi << sh) | (lo >> (64 - sh)) : hi;
        rest = sh ? lo << sh : lo;
        e0 = 64 - sh;
    } else {
        if (lo == 0) return 0.0;
        const int sh = __clzll((long long)lo);
        top = lo << sh;
        rest = 0;
        e0 = -sh;
    }
    const long long v = (long long)((top >> 1) | (top & 1ull) | (rest != 0 ? 1ull : 0ull));
    return oz_ll_scaled(neg ? -v : v, ex + e0 + 1);
}
