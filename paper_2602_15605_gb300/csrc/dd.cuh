// dd.cuh -- double-float arithmetic (a value held as an unevaluated sum of
// two FP32 numbers) on the FP32 pipe, after Dekker (1971) and Knuth's
// two-sum.  The FP64 pipe of the target GPU is ~70x slower than its FP32
// pipe, so the mixed path keeps its per-element bookkeeping in this form.
// The error-free transformations rely on round-to-nearest FP32 and on the
// products being formed with explicit fmaf.
#pragma once
#include <cuda_runtime.h>

namespace cpl {

struct dfl {
    float h, l;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ dfl df_quick(float a, float b) {
    const float s = a + b;
    const float e = b - (s - a);
    return {s, e};
}

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_quick(p, e);
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    dfl s = df_two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return df_quick(s.h, s.l);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }

// exact double-float of an integer |v| < 2^31
__device__ __forceinline__ dfl df_from_int(int v) {
    const float h = __int2float_rn(v);
    const float l = __int2float_rn(v - __float2int_rn(h));
    return {h, l};
}

// exact double-float of the product of two integers |a|, |b| < 2^24 (the
// 32-bit conversions and the fma run on the FP32 pipe; 64-bit integer
// conversions would occupy the FP64 pipe)
__device__ __forceinline__ dfl df_int_prod(int a, int b) {
    const float fa = __int2float_rn(a), fb = __int2float_rn(b);
    const float p = __fmul_rn(fa, fb);
    return {p, fmaf(fa, fb, -p)};
}

// double-float of a 64-bit integer product (exact below 2^48)
__device__ __forceinline__ dfl df_from_ll(long long v) {
    const float h = __ll2float_rn(v);
    const float l = __ll2float_rn(v - __float2ll_rn(h));
    return {h, l};
}

// 1 / a (about 44 bits)
__device__ __forceinline__ dfl df_recip(dfl a) {
    const float q1 = 1.0f / a.h;
    // r = 1 - a q1, evaluated exactly to first order
    const float p = a.h * q1;
    float e = fmaf(a.h, q1, -p);
    e = fmaf(a.l, q1, e);
    const float r = (1.0f - p) - e;
    const float q2 = r / a.h;
    return df_quick(q1, q2);
}

// sqrt(a) for a > 0 (about 44 bits)
__device__ __forceinline__ dfl df_sqrt(dfl a) {
    const float s = sqrtf(a.h);
    const float p = s * s;
    float e = fmaf(s, s, -p);
    const float r = ((a.h - p) - e) + a.l;
    return df_quick(s, r / (2.0f * s));
}

// x * 2^k for an exponent that may leave the single-step range
__device__ __forceinline__ float scale2(float x, int k) {
    if (k < -252) return 0.0f;
    if (k > 254) k = 254;
    const int k1 = k / 2, k2 = k - k1;
    return x * __int_as_float((127 + k1) << 23) * __int_as_float((127 + k2) << 23);
}

// 2^k as a float for -126 <= k <= 127
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// floor(log2 |x|) for a normal nonzero float (exponent field only)
__device__ __forceinline__ int ilogbf_fast(float x) { return ((__float_as_int(x) >> 23) & 0xff) - 127; }

}  // namespace cpl

namespace cpl {

// Extended double-float: value (h + l) * 2^e with |h| in [1, 2) (or h = l = 0),
// so that products of widely scaled quantities never leave the FP32 range.
struct xdf {
    float h, l;
    int e;
};
static_assert(sizeof(xdf) == 12, "xdf tables are written by the host as three 32-bit words");

__device__ __forceinline__ xdf xdf_make(dfl m, int e) {
    if (m.h == 0.0f) return {0.0f, 0.0f, 0};
    const int k = ilogbf_fast(fabsf(m.h));
    return {scale2(m.h, -k), scale2(m.l, -k), e + k};
}

__device__ __forceinline__ xdf xdf_from_ll(long long v) { return xdf_make(df_from_ll(v), 0); }
__device__ __forceinline__ xdf xdf_from_int(int v) { return xdf_make(df_from_int(v), 0); }
// a b for |a|, |b| < 2^31 (relative error about 2^-48), on the FP32 pipe
__device__ __forceinline__ xdf xdf_int_mul(int a, int b) { return xdf_make(df_mul(df_from_int(a), df_from_int(b)), 0); }

__device__ __forceinline__ xdf xdf_mul(xdf a, xdf b) {
    if (a.h == 0.0f || b.h == 0.0f) return {0.0f, 0.0f, 0};
    return xdf_make(df_mul(dfl{a.h, a.l}, dfl{b.h, b.l}), a.e + b.e);
}

__device__ __forceinline__ xdf xdf_neg(xdf a) { return {-a.h, -a.l, a.e}; }

__device__ __forceinline__ xdf xdf_add(xdf a, xdf b) {
    if (a.h == 0.0f) return b;
    if (b.h == 0.0f) return a;
    if (a.e < b.e) {
        const xdf t = a;
        a = b;
        b = t;
    }
    const int d = b.e - a.e;          // <= 0
    if (d < -60) return a;
    const dfl s = df_add(dfl{a.h, a.l}, dfl{scale2(b.h, d), scale2(b.l, d)});
    return xdf_make(s, a.e);
}

__device__ __forceinline__ xdf xdf_recip(xdf a) {
    const dfl r = df_recip(dfl{a.h, a.l});
    return xdf_make(r, -a.e);
}

__device__ __forceinline__ xdf xdf_sqrt(xdf a) {
    if (a.h == 0.0f) return a;
    dfl m = {a.h, a.l};
    int e = a.e;
    if (e & 1) {
        m.h *= 2.0f;
        m.l *= 2.0f;
        e -= 1;
    }
    return xdf_make(df_sqrt(m), e / 2);
}

__device__ __forceinline__ xdf xdf_scale_int(xdf a, long long k) { return xdf_mul(a, xdf_from_ll(k)); }

// FP64 value of a (truncating below 2^-52 relative), built with integer
// operations only (the FP64 pipe is the scarce one).  Handles FP64
// subnormals and zero.
// (double) f from the bits for a normal f, 0 for a zero or subnormal f.
__device__ __forceinline__ double df_widen_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0x000fffffu);
    return __hiloint2double((int)hi, (int)(u << 29));
}
// FP64 of a double-float value: both parts widened from their bits and added
// once, i.e. the correctly rounded h + l (a low part below FP32's normal
// range, at most 2^-126 in absolute value, is dropped).
__device__ __forceinline__ double df_to_double(dfl a) { return df_widen_bits(a.h) + df_widen_bits(a.l); }

// (double) f * 2^k from the bits, for a normal f whose scaled exponent stays
// above FP64's normal range's bottom (else 0).
__device__ __forceinline__ double xdf_widen_bits(float f, int k) {
    const unsigned u = __float_as_uint(f);
    const int ef = (int)((u >> 23) & 0xffu);
    const int fd = ef + 896 + k;
    if (ef == 0 || fd < 1) return 0.0;
    const unsigned hi = (u & 0x80000000u) | ((unsigned)fd << 20) | ((u >> 3) & 0x000fffffu);
    return __hiloint2double((int)hi, (int)(u << 29));
}
// FP64 of (h + l) 2^e, h and l a normalised double-float pair: where h 2^e
// is a normal double at least 2^-960 in magnitude, both parts are widened
// from their bits and added once (the correctly rounded value; a low part
// that falls below FP64's normal range is far below its rounding); else the
// mantissa assembly of xdf_to_double_slow.
__device__ __forceinline__ double xdf_to_double_slow(xdf a);
__device__ __forceinline__ double xdf_to_double(xdf a) {
    const int eh = (int)((__float_as_uint(a.h) >> 23) & 0xffu);
    const int fh = eh + 896 + a.e;
    if (eh != 0 && eh != 255 && fh > 63 && fh < 2047) return xdf_widen_bits(a.h, a.e) + xdf_widen_bits(a.l, a.e);
    return xdf_to_double_slow(a);
}
__device__ __forceinline__ double xdf_to_double_slow(xdf a) {
    if (a.h == 0.0f) return 0.0;
    const unsigned long long sign = (a.h < 0.0f) ? (1ull << 63) : 0ull;
    const float ah = fabsf(a.h);
    const float al = (a.h < 0.0f) ? -a.l : a.l;
    long long M = (long long)((__float_as_uint(ah) & 0x7FFFFFu) | 0x800000u) << 29;   // ah * 2^52
    int e = a.e + ilogbf_fast(ah);                                                      // ah in [1, 2): 0
    if (al != 0.0f) {
        const float aal = fabsf(al);
        const int eal = ilogbf_fast(aal);
        const long long mal = (long long)((__float_as_uint(aal) & 0x7FFFFFu) | 0x800000u);
        const int sh = eal + 29 - ilogbf_fast(ah);
        long long add = 0;
        if (sh >= 0) add = mal << sh;
        else if (sh > -40) add = mal >> (-sh);
        M += (al < 0.0f) ? -add : add;
    }
    if (M >= (1ll << 53)) {
        M >>= 1;
        e += 1;
    } else if (M < (1ll << 52)) {
        M <<= 1;
        e -= 1;
    }
    const int biased = e + 1023;
    unsigned long long bits;
    if (biased >= 2047) {
        bits = sign | (0x7FFull << 52);
    } else if (biased >= 1) {
        bits = sign | ((unsigned long long)biased << 52) | ((unsigned long long)M & ((1ull << 52) - 1));
    } else {
        const int shift = 1 - biased;
        bits = (shift > 53) ? sign : (sign | ((unsigned long long)M >> shift));
    }
    return __longlong_as_double((long long)bits);
}

}  // namespace cpl
