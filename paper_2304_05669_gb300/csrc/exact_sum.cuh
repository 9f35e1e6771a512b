// In-order FP64 sums of float32 values, carried exactly in integers.
//
// A nonzero normal float is M * 2^(e - 150) with M < 2^24 and e its biased
// exponent (IEEE 754 binary32).  Take n values whose nonzero ones have
// exponents in [emin, emax]: each is an integer multiple of
// u = 2^(emin - 150) below 2^(emax - emin + 24) u, so every partial sum of
// them is an integer multiple of u below n * 2^(emax - emin + 24) u.  When
// emax - emin <= 29 - bitlen(n) that bound is at most 2^53 u, so every
// partial sum is exactly a double, every FP64 addition of the in-order sum
// (which starts at +0; zeros leave it unchanged) is exact, and the sum is
// acc * u with acc the int64 sum of the values in units of u -- which any
// order of integer additions reproduces.  GB300 issues FP64 at 1/64 of the
// float32 rate, so the integer route is the fast one; values outside it
// (a wider exponent range, subnormals, infinities, NaNs) are summed in
// FP64 in order by the caller.
#pragma once
#include <cstdint>

namespace fipt_exact {

constexpr int EMPTY_EMIN = 255;        // no nonzero value seen yet

// Largest exponent range for which n values sum exactly (negative: none).
__device__ __forceinline__ int spread_limit(int64_t n) {
    return 29 - (64 - __clzll((long long)n));
}

// Magnitude bits (sign cleared) of the smallest nonzero and the largest of
// a set of floats: for non-negative floats the bit patterns order as the
// values, so the two extremes give the exponent range and show whether any
// value is subnormal (a nonzero pattern below 2^23), infinite or NaN (at or
// above 0x7F800000).
struct Range {
    uint32_t lo = 0xFFFFFFFFu;     // smallest nonzero magnitude (all-ones: none)
    uint32_t hi = 0u;              // largest magnitude

    __device__ __forceinline__ void note(float v) {
        const uint32_t a = __float_as_uint(v) & 0x7FFFFFFFu;
        lo = min(lo, a != 0u ? a : 0xFFFFFFFFu);
        hi = max(hi, a);
    }
    // Outside the exact route whatever n is: a subnormal, an infinity or a NaN.
    __device__ __forceinline__ bool special() const {
        return hi >= 0x7F800000u || (hi != 0u && lo < 0x00800000u);
    }
    // Smallest exponent of the nonzero values (EMPTY_EMIN when all are zero).
    __device__ __forceinline__ int emin() const { return hi == 0u ? EMPTY_EMIN : (int)(lo >> 23); }
    // Whether n values spanning this range sum exactly (special() false).
    __device__ __forceinline__ bool exact_for(int64_t n) const {
        return hi == 0u || (int)(hi >> 23) - (int)(lo >> 23) <= spread_limit(n);
    }
};

// A normal (or zero) float in units of 2^(emin - 150); needs
// 0 <= exponent - emin <= 29.
__device__ __forceinline__ long long term(float v, int emin) {
    const uint32_t b = __float_as_uint(v);
    const bool nz = (b << 1) != 0u;
    const unsigned long long m = nz ? (unsigned long long)((b & 0x7FFFFFu) | 0x800000u) : 0ull;
    const int d = nz ? (int)((b >> 23) & 0xFFu) - emin : 0;
    const long long t = (long long)(m << d);
    return (b >> 31) ? -t : t;
}

// acc * 2^(emin - 150) as a double (|acc| < 2^53: exact), built from its
// bits; an exact cancellation gives +0 as FP64 addition does.
__device__ __forceinline__ double scaled_double(long long acc, int emin) {
    if (acc == 0) return 0.0;
    const unsigned long long a = acc < 0 ? (unsigned long long)(-acc) : (unsigned long long)acc;
    const int t = 63 - __clzll((long long)a);
    const unsigned long long bits = (acc < 0 ? (1ull << 63) : 0ull) |
                                    ((unsigned long long)(t + 1023 + emin - 150) << 52) |
                                    ((a << (52 - t)) & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

}  // namespace fipt_exact
