// Double <-> float conversion on the integer pipe.
//
// On GB300 a hardware FP64 -> FP32 conversion issues on the small FP64 unit
// (measured about 0.2 per clock per SM, ten times slower than an FP64 FMA),
// so kernels that convert every element become conversion-bound.  These
// versions take the IEEE-754 bit fields apart with integer instructions.
// d2f rounds to nearest, ties to even, exactly like the hardware conversion
// for every double of magnitude at least 2^-126 (the smallest normal float);
// a smaller magnitude gives a signed zero (the hardware would round to a
// subnormal float, or up to 2^-126), overflow gives a signed infinity, and a
// NaN gives a quiet NaN.  f2d is exact for every float, subnormals included
// (a NaN keeps its payload bits).
#pragma once

#include <stdint.h>

namespace omm {

__device__ __forceinline__ float sw_d2f(double d) {
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int de = (int)((b >> 52) & 0x7FF);                 // biased double exponent
    const int e = de - 1023 + 127;                           // biased float exponent
    const uint64_t m = b & 0xFFFFFFFFFFFFFull;               // 52-bit fraction
    if (de == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));  // inf / nan
    if (e <= 0) return __uint_as_float(sign);               // below 2^-126: signed zero
    if (e >= 255) return __uint_as_float(sign | 0x7F800000u);   // overflow: infinity
    uint32_t f = ((uint32_t)e << 23) | (uint32_t)(m >> 29);
    const uint32_t rem = (uint32_t)(m & 0x1FFFFFFFu);       // 29 dropped bits
    if (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) f += 1u;   // may carry into the exponent
    return __uint_as_float(sign | f);
}

__device__ __forceinline__ double sw_f2d(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    const uint32_t e = (u >> 23) & 0xFF;
    const uint64_t m = u & 0x7FFFFFu;
    if (e == 0) {
        if (m == 0) return __longlong_as_double((long long)sign);
        // subnormal float: normalise
        // m 2^-149 with the leading one at bit p = 23 - lz: 1.f x 2^(p - 149); shifting
        // by lz puts that one at bit 23, which the 23-bit mask then drops
        const int lz = __clz((int)m) - 8;                      // leading zeros inside the 24-bit field
        const uint64_t mm = (m << lz) & 0x7FFFFFull;
        const uint64_t ed = (uint64_t)(1023 - 126 - lz);
        return __longlong_as_double((long long)(sign | (ed << 52) | (mm << 29)));
    }
    if (e == 255) return __longlong_as_double((long long)(sign | (0x7FFull << 52) | (m << 29)));
    return __longlong_as_double((long long)(sign | ((uint64_t)(e - 127 + 1023) << 52) | (m << 29)));
}

// v * 2^e2 for a 64-bit integer v, rounded to nearest (ties to even); the
// caller keeps the result in the normal range (|v| 2^e2 between 2^-1000 and
// 2^1000).
__device__ __forceinline__ double sw_i64_scaled(int64_t v, int e2) {
    if (v == 0) return 0.0;
    const uint64_t sign = v < 0 ? (1ull << 63) : 0ull;
    const uint64_t a = v < 0 ? (0ull - (uint64_t)v) : (uint64_t)v;
    int p = 63 - __clzll((long long)a);                        // position of the leading one
    uint64_t q;
    if (p <= 52) {
        q = a << (52 - p);
    } else {
        const int sh = p - 52;
        q = a >> sh;
        const uint64_t rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (q & 1ull))) {
            q += 1ull;
            if (q >> 53) {
                q >>= 1;
                ++p;
            }
        }
    }
    return __longlong_as_double((long long)(sign | ((uint64_t)(1023 + p + e2) << 52) | (q & 0xFFFFFFFFFFFFFull)));
}

// x * 2^e by an exponent add when x and the result are normal; other cases
// (zero, subnormal, overflow, non-finite) go through ldexp.
__device__ __forceinline__ double sw_scale2(double x, int e) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int be = (int)((b >> 52) & 0x7FF);
    const int ne = be + e;
    if (be == 0 || be == 0x7FF || ne <= 0 || ne >= 0x7FF) return ldexp(x, e);
    return __longlong_as_double((long long)((b & ~(0x7FFull << 52)) | ((uint64_t)ne << 52)));
}

}  // namespace omm
