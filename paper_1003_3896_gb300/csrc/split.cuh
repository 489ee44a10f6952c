// split.cuh -- double-single split of a double (the paper's hi + lo
// coordinate format, Sect. 5.2) from its bits, the widening of a float from
// its bits, and inverse square-root powers in double refined from a float
// estimate: arithmetic kept off the FP64 pipe, which on this GPU runs at 1/77
// of the FP32 rate.
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

// R^(-1/2) (POT) or R^(-3/2) in double for R >= 0, refined from the float
// estimate y0 = rsqrt.approx(R_f): R_f is R truncated to float and y0 is
// widened to double, both from their bits (the conversion instructions would
// run on the FP64 pipe, which bounds the FP64 pair kernel and the kick's
// field).  With R y0^2 = 1 - v, |v| < 2^-20 (the estimate's error and the
// truncation's),
//     R^(-1/2) = y0 (1 + v/2 + 3 v^2 / 8 + O(v^3)),
//     R^(-3/2) = y0^3 (1 + 3 v / 2 + 15 v^2 / 8 + O(v^3)),
// the dropped terms below 2^-58 relative; y0^2 is exact (y0 has 24 bits) and
// v is one fused multiply-add, so 5 or 6 FP64 operations replace the double
// rsqrt and the cube.  R outside the float range (the padding's 1e300, R = 0,
// non-finite R) takes the library rsqrt.
template <bool POT>
__device__ __forceinline__ double rsqrt_pow(double R)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(R);
    const int E = (int)(b >> 52);   // R >= 0: the sign bit is clear
    if (E < 1023 - 125 || E > 1023 + 126) {
        const double ri = rsqrt(R);
        return POT ? ri : ri * ri * ri;
    }
    const float rf = __int_as_float(((E - 1023 + 127) << 23) | (int)((b >> 29) & 0x7FFFFFu));
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(rf));
    const double y0 = widen(yf);
    const double q = __dmul_rn(y0, y0);
    const double v = __fma_rn(-R, q, 1.0);
    if (POT) return __fma_rn(y0, __dmul_rn(v, __fma_rn(v, 0.375, 0.5)), y0);
    const double y3 = __dmul_rn(q, y0);
    return __fma_rn(y3, __dmul_rn(v, __fma_rn(v, 1.875, 1.5)), y3);
}

}  // namespace nb
