// Double-binary32 ("double-word") arithmetic on the binary32 pipe: a value is
// an unevaluated pair (hi, lo) of binary32 words.  Products are exact by one
// FMA (p + e = a * b), sums by Knuth's TwoSum, and the low words are collected
// as in the double-word dot product of Ogita, Rump and Oishi (2005): about 48
// significant bits, binary64 class.  GB300 issues binary64 FMAs at ~1/60 of
// its binary32 rate, which makes this the fast binary64-class arithmetic.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace poro {

// ------------------------------------------------ error-free double-word ops
// Explicit round-to-nearest intrinsics keep the compiler from contracting or
// reassociating the transformations.
__device__ __forceinline__ void dw_mac(float& h, float& l, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float s = __fadd_rn(h, p);
    const float bb = __fsub_rn(s, h);
    const float er = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    h = s;
    l = __fadd_rn(l, __fadd_rn(er, e));
}

// acc += a * b with b a single binary32 word
__device__ __forceinline__ void dw_mac1(float& h, float& l, float ah, float al, float b) {
    const float p = __fmul_rn(ah, b);
    float e = __fmaf_rn(ah, b, -p);
    e = __fmaf_rn(al, b, e);
    const float s = __fadd_rn(h, p);
    const float bb = __fsub_rn(s, h);
    const float er = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    h = s;
    l = __fadd_rn(l, __fadd_rn(er, e));
}

// acc += a * (bh + bl) with a exact
__device__ __forceinline__ void dw_mac_x2(float& h, float& l, float a, float bh, float bl) {
    const float p = __fmul_rn(a, bh);
    float e = __fmaf_rn(a, bh, -p);
    e = __fmaf_rn(a, bl, e);
    const float s = __fadd_rn(h, p);
    const float bb = __fsub_rn(s, h);
    const float er = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    h = s;
    l = __fadd_rn(l, __fadd_rn(er, e));
}

// ------------------------------------- binary64 results on the integer pipe
// GB300 runs binary64 (conversions included) at ~1/60 of the binary32 rate,
// so the result is assembled from its binary32 words by bit manipulation.

// exact binary64 bit pattern of a binary32 value (binary32 subnormals,
// |x| < 1.2e-38, become signed zero; infinities and NaNs stay so)
__device__ __forceinline__ unsigned long long f2d_bits(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t ex = (b >> 23) & 0xFFu;
    const uint32_t dex = ex == 0xFFu ? 0x7FFu : ex + 896u;
    const uint32_t hi = ex ? ((b & 0x80000000u) | (dex << 20) | ((b >> 3) & 0xFFFFFu)) : (b & 0x80000000u);
    const uint32_t lo = ex ? (b << 29) : 0u;
    return ((unsigned long long)hi << 32) | lo;
}

// s + e as binary64 for a pair with |e| <= ulp(s) / 2 (TwoSum output): e is
// added to s's binary64 pattern in units of s's binary64 last place.  Exact
// when e's bits lie within 29 places below s's last bit (the sum then has at
// most 53 significant bits); otherwise e is truncated below that place.
__device__ __forceinline__ double pair_to_double(float s, float e) {
    unsigned long long d = f2d_bits(s);
    const uint32_t bs = __float_as_uint(s), be = __float_as_uint(e);
    const int exs = (int)((bs >> 23) & 0xFFu), exe = (int)((be >> 23) & 0xFFu);
    if (exs != 0 && exs != 0xFF && exe != 0) {
        const unsigned long long me = (unsigned long long)((be & 0x7FFFFFu) | 0x800000u);
        const bool opposite = ((bs ^ be) >> 31) != 0;
        // e in units of 2^(exp(s) - 52); one binade lower (half the unit) when s
        // is a power of two and e points towards zero
        int k = exe - exs + 29 + ((opposite && (bs & 0x7FFFFFu) == 0) ? 1 : 0);
        const unsigned long long delta = k >= 0 ? (me << k) : (k > -32 ? (me >> (-k)) : 0ull);
        d = opposite ? d - delta : d + delta;
    }
    return __longlong_as_double((long long)d);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float2 dw_split(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

// a + b for two double-word values
__device__ __forceinline__ float2 dw_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// ------------------------------------------------------- fixed-point words
// 2^k as binary32, k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// exact binary32 value of an integer v in [-2^22, 2^22]: v is added to the
// significand of 1.5 * 2^23 (unit last place 1; at v = 2^22 the pattern
// carries into the exponent of 2^24, still the right value), then that
// constant is subtracted (exact by Sterbenz's lemma)
__device__ __forceinline__ float small_int_to_float(int v) {
    return __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f);
}

// nearest integer to x * f for |x * f| < 2^22 and f a power of two: the
// exact product is rounded to the unit last place of 1.5 * 2^23 (a sum that
// rounds up to 2^24 gives the pattern of 2^24, i.e. v = 2^22)
__device__ __forceinline__ int round_to_int(float x, float f) {
    return __float_as_int(__fmaf_rn(x, f, 12582912.0f)) - 0x4B400000;
}

// exact double-word (h, l) of an integer |v| <= 2^44: v = a 2^22 + b with
// |a| <= 2^22 and b in [0, 2^22), both exact in binary32, joined by Fast2Sum
// (|a 2^22| > b unless a = 0)
__device__ __forceinline__ void int_to_dw(long long v, float& h, float& l) {
    const float fa = __fmul_rn(small_int_to_float((int)(v >> 22)), 4194304.0f);
    const float fb = small_int_to_float((int)(v & 0x3FFFFF));
    h = __fadd_rn(fa, fb);
    l = __fsub_rn(fb, __fsub_rn(h, fa));
}
__device__ __forceinline__ void int_to_dw(int v, float& h, float& l) {
    const float fa = __fmul_rn(small_int_to_float(v >> 22), 4194304.0f);
    const float fb = small_int_to_float(v & 0x3FFFFF);
    h = __fadd_rn(fa, fb);
    l = __fsub_rn(fb, __fsub_rn(h, fa));
}

}  // namespace poro
