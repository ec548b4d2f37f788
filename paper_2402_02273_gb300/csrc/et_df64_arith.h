// Double-float (DF64) pair arithmetic shared by the DF64 Taylor-term kernels
// (et_df64.cu, et_fused.cu).  A value is hi + lo in two FP32 numbers (48-bit
// significand).  Error-free transformations: TwoSum (Knuth) and the FMA-based
// TwoProduct; sums of products are compensated dot products in the manner of
// Ogita, Rump and Oishi (2005): high parts added with TwoSum, every rounding
// error and every hi*lo cross product collected in one FP32 correction, one
// renormalisation at the end; lo*lo products (relative size 2^-48) dropped.
// Intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn) keep the compiler from
// contracting or reassociating any step.
#pragma once

#include <cuda_runtime.h>

#include <cstring>

namespace et {
namespace df64 {

// Bit casts and the leading-bit count, on the device by intrinsics and on the
// host (where tests check from_double) by memcpy and the compiler builtin.
__host__ __device__ __forceinline__ unsigned long long bits_of(double v) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(v);
#else
    unsigned long long b;
    std::memcpy(&b, &v, sizeof(b));
    return b;
#endif
}
__host__ __device__ __forceinline__ float float_of(unsigned u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, sizeof(f));
    return f;
#endif
}
__host__ __device__ __forceinline__ int leading_bit(unsigned r) {  // r != 0
#ifdef __CUDA_ARCH__
    return 31 - __clz((int)r);
#else
    return 31 - __builtin_clz(r);
#endif
}

// A pair for an FP64 value, built from its bits with integer instructions
// only (GB300 runs FP64 conversions at its FP64 rate, 2 per clock per SM):
// hi = v rounded to 24 significant bits (half away from zero), lo = the signed
// remainder v - hi (at most 28 bits) cut to 24, so |v - (hi + lo)| <= 2^-48 |v|
// for 2^-70 <= |v| < 2^128.  A part below the FP32 normal range becomes a
// zero (absolute error under 2^-126); infinities, NaNs and values beyond the
// FP32 range give (+-inf or NaN, 0).
__host__ __device__ __forceinline__ float2 from_double(double v) {
    const unsigned long long bits = bits_of(v);
    const unsigned sign = (unsigned)(bits >> 32) & 0x80000000u;
    const unsigned long long mag = bits & 0x7fffffffffffffffull;
    const int e = (int)(mag >> 52);  // biased FP64 exponent
    const float zero = float_of(sign);
    if (e == 0x7ff) {
        const bool nan = (mag & 0xfffffffffffffull) != 0ull;
        return make_float2(float_of(sign | 0x7f800000u | (nan ? 0x400000u : 0u)), 0.f);
    }
    if (e - 896 <= 0) return make_float2(zero, zero);
    const unsigned long long rmag = mag + (1ull << 28);  // rounds at the 24th significant bit; may carry
    const int ef = (int)(rmag >> 52) - 896;              // biased FP32 exponent of hi
    if (ef >= 255) return make_float2(float_of(sign | 0x7f800000u), 0.f);
    const float hi = float_of(sign | ((unsigned)ef << 23) | ((unsigned)(rmag >> 29) & 0x7fffffu));
    const unsigned rem = (unsigned)mag & 0x1fffffffu;  // the 29 bits below hi's, of weight 2^(e - 1075)
    const bool up = (rem >> 28) != 0u;                 // hi was rounded up: the remainder is negative
    const unsigned r = up ? 0x20000000u - rem : rem;
    const unsigned lsign = up ? sign ^ 0x80000000u : sign;
    if (r == 0u) return make_float2(hi, zero);
    const int p = leading_bit(r);  // leading bit of r, 0..28
    const int el = e - 948 + p;    // biased FP32 exponent of lo
    if (el <= 0) return make_float2(hi, float_of(lsign));
    const unsigned mm = p >= 23 ? r >> (p - 23) : r << (23 - p);
    return make_float2(hi, float_of(lsign | ((unsigned)el << 23) | (mm & 0x7fffffu)));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Compensated accumulator of a sum of pair products.
struct DotAcc {
    float s, c;
};

__device__ __forceinline__ void dot_first(DotAcc& A, float2 a, float2 b) {
    A.s = __fmul_rn(a.x, b.x);
    float c = __fmaf_rn(a.x, b.x, -A.s);
    c = __fmaf_rn(a.x, b.y, c);
    A.c = __fmaf_rn(a.y, b.x, c);
}

__device__ __forceinline__ void dot_add(DotAcc& A, float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    const float ep = __fmaf_rn(a.x, b.x, -p);
    float s, es;
    two_sum(A.s, p, s, es);
    A.s = s;
    float c = __fmaf_rn(a.x, b.y, A.c);
    c = __fmaf_rn(a.y, b.x, c);
    A.c = __fadd_rn(c, __fadd_rn(ep, es));
}

__device__ __forceinline__ float2 dot_result(const DotAcc& A) {
    float s, e;
    two_sum(A.s, A.c, s, e);
    return make_float2(s, e);
}

__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    DotAcc A;
    dot_first(A, a, b);
    return dot_result(A);
}

// a * b + c as one compensated sum.
__device__ __forceinline__ float2 df_fma(float2 a, float2 b, float2 c) {
    DotAcc A;
    dot_first(A, a, b);
    float s, es;
    two_sum(A.s, c.x, s, es);
    A.s = s;
    A.c = __fadd_rn(__fadd_rn(A.c, c.y), es);
    return dot_result(A);
}

// a + b of two pairs (TwoSum of the high parts, low parts added to the error,
// one renormalisation).
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    float hi, lo;
    two_sum(s, e, hi, lo);
    return make_float2(hi, lo);
}

// Merges two compensated accumulators into A.
__device__ __forceinline__ void dot_merge(DotAcc& A, const DotAcc& B) {
    float s, e;
    two_sum(A.s, B.s, s, e);
    A.s = s;
    A.c = __fadd_rn(__fadd_rn(A.c, B.c), e);
}

// One Taylor term at a voxel: the 7-point stencil of the normalised operator
// on z (diagonal dt, weights towards +x, -x, +y, -y, +z, -z), optionally
// scaled by zscale, plus beta * b.  The eight products are summed in two
// independent compensated halves that are merged at the end, which halves the
// chain of dependent additions.
template <bool ZS>
__device__ __forceinline__ float2 stencil(float2 dt, float2 zc, float2 wxp, float2 zxp, float2 wxm, float2 zxm,
                                          float2 wyp, float2 zyp, float2 wym, float2 zym, float2 wzp, float2 zp,
                                          float2 wzm, float2 zm, float2 zscale, bool has_beta, float2 beta,
                                          float2 bval) {
    DotAcc A, B;
    dot_first(A, dt, zc);
    dot_first(B, wym, zym);
    dot_add(A, wxp, zxp);
    dot_add(B, wzp, zp);
    dot_add(A, wxm, zxm);
    dot_add(B, wzm, zm);
    dot_add(A, wyp, zyp);
    if (!ZS) {
        if (has_beta) dot_add(B, beta, bval);
        dot_merge(A, B);
        return dot_result(A);
    }
    dot_merge(A, B);
    const float2 acc = df_mul(zscale, dot_result(A));
    return has_beta ? df_fma(beta, bval, acc) : acc;
}

// The same term at a voxel whose six off-diagonal weights are all zero: the
// operations of stencil() with the products of zero weights left out.  Each
// left-out step adds an exact zero (a product 0 * z, an error term 0) to a
// sum, so the result is stencil()'s except possibly for the sign of a zero.
template <bool ZS>
__device__ __forceinline__ float2 stencil_diag(float2 dt, float2 zc, float2 zscale, bool has_beta, float2 beta,
                                               float2 bval) {
    DotAcc A;
    dot_first(A, dt, zc);
    if (!ZS) {
        if (has_beta) {
            DotAcc B;
            B.s = 0.f;
            B.c = 0.f;
            dot_add(B, beta, bval);
            dot_merge(A, B);
        }
        return dot_result(A);
    }
    const float2 acc = df_mul(zscale, dot_result(A));
    return has_beta ? df_fma(beta, bval, acc) : acc;
}

}  // namespace df64
}  // namespace et
