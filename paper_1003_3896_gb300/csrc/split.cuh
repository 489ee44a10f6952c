// split.cuh -- double-single split of a double (the paper's hi + lo
// coordinate format, Sect. 5.2) from its bits.
#pragma once

namespace nb {

// Double-single split of r: hi = RN_float(r), lo = RN_float(r - hi), taken
// from the bits of r with integer operations.  r = S 2^(E - 1075) with the
// 53-bit significand S; hi keeps the top 24 bits of S rounded to nearest
// even, and r - hi = d 2^(E - 1075) exactly, d = S - q 2^29 with |d| <= 2^28,
// whose float rounding is lo.  Equal bit for bit to the plain conversions
// for 2^-70 <= |r| < 2^101 (hi and lo normal floats); other r (zero, tiny,
// huge, non-finite) take the plain conversions.  The FP64 pipe, which runs at
// 1/77 of the FP32 rate here, otherwise carries three conversions and a
// subtraction per coordinate.
__device__ __forceinline__ void split_ds(double r, float &hi, float &lo)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(r);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E < 1023 - 70 || E > 1023 + 100) {
        hi = __double2float_rn(r);
        lo = __double2float_rn(r - (double)hi);
        return;
    }
    const unsigned long long S = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    unsigned int q = (unsigned int)(S >> 29);   // 24 bits, truncated
    const unsigned int rem = (unsigned int)(S & 0x1FFFFFFFu);
    const bool up = rem > 0x10000000u || (rem == 0x10000000u && (q & 1u));
    q += up ? 1u : 0u;
    const int d = (int)rem - (up ? 0x20000000 : 0);
    int ef = E - 1023 + 127;
    if (q == (1u << 24)) {   // rounding carried into the exponent
        q >>= 1;
        ++ef;
    }
    const unsigned int sign = (unsigned int)(b >> 63) << 31;
    hi = __int_as_float((int)(sign | ((unsigned int)ef << 23) | (q & 0x7FFFFFu)));
    const float scale = __int_as_float((E - 1075 + 127) << 23);   // 2^(E - 1075)
    lo = __fmul_rn(__int2float_rn(sign ? -d : d), scale);
}

// The double equal to float f, from its bits: the exponent rebiased, the
// fraction shifted into place (exact).  Zeros come from the sign bit alone;
// subnormal and non-finite f take the conversion instruction, which on this
// GPU runs on the FP64 pipe.
__device__ __forceinline__ double widen(float f)
{
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) {
        if ((u & 0x7FFFFFFFu) == 0u)
            return __longlong_as_double((long long)((unsigned long long)u << 32));
        return (double)f;
    }
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

}  // namespace nb
