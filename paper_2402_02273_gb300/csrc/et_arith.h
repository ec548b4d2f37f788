// Per-voxel arithmetic of one Taylor term in the FP32 and DF64 value types,
// shared by the two-term kernels (et_fused.cu, et_quadpair.cu).  It is the
// arithmetic of the one-term kernels, operation for operation, so a voxel's
// result does not depend on which kernel computed it.
#pragma once

#include <cuda_runtime.h>

#include "et_df64_arith.h"

namespace et {

// Per-voxel arithmetic of one term, identical to the unfused kernels.  ZS: the
// stencil part is scaled by zscale (first term of an FP32 / DF64 chain).
template <typename T>
struct Arith;

template <>
struct Arith<float> {
    template <bool ZS>
    static __device__ __forceinline__ float stencil(float dt, float zc, float wxp, float zxp, float wxm, float zxm,
                                                    float wyp, float zyp, float wym, float zym, float wzp, float zp,
                                                    float wzm, float zm, float zscale, bool has_beta, float beta,
                                                    float bval) {
        float acc = dt * zc;
        acc = fmaf(wxp, zxp, acc);
        acc = fmaf(wxm, zxm, acc);
        acc = fmaf(wyp, zyp, acc);
        acc = fmaf(wym, zym, acc);
        acc = fmaf(wzp, zp, acc);
        acc = fmaf(wzm, zm, acc);
        if (ZS) acc *= zscale;
        if (has_beta) acc = fmaf(beta, bval, acc);
        return acc;
    }
    // The same term at a voxel whose six off-diagonal weights are zero: the
    // left-out multiply-adds each add an exact zero, so the result is
    // stencil()'s up to the sign of a zero.
    template <bool ZS>
    static __device__ __forceinline__ float diag(float dt, float zc, float zscale, bool has_beta, float beta,
                                                 float bval) {
        float acc = dt * zc;
        if (ZS) acc *= zscale;
        if (has_beta) acc = fmaf(beta, bval, acc);
        return acc;
    }
    // all six weights are zero (of either sign)
    static __device__ __forceinline__ bool zero6(float a, float b, float c, float d, float e, float f) {
        const unsigned o = __float_as_uint(a) | __float_as_uint(b) | __float_as_uint(c) | __float_as_uint(d) |
                           __float_as_uint(e) | __float_as_uint(f);
        return (o << 1) == 0u;
    }
    static __device__ __forceinline__ float axpy(float g, float x, float base) { return fmaf(g, x, base); }
    static __device__ __forceinline__ float scale(float g, float x) { return x * g; }
    static __device__ __forceinline__ double widen(float x) { return (double)x; }
    static __device__ __forceinline__ float zero() { return 0.f; }
};

template <>
struct Arith<float2> {
    template <bool ZS>
    static __device__ __forceinline__ float2 stencil(float2 dt, float2 zc, float2 wxp, float2 zxp, float2 wxm,
                                                     float2 zxm, float2 wyp, float2 zyp, float2 wym, float2 zym,
                                                     float2 wzp, float2 zp, float2 wzm, float2 zm, float2 zscale,
                                                     bool has_beta, float2 beta, float2 bval) {
        return df64::stencil<ZS>(dt, zc, wxp, zxp, wxm, zxm, wyp, zyp, wym, zym, wzp, zp, wzm, zm, zscale, has_beta,
                                 beta, bval);
    }
    template <bool ZS>
    static __device__ __forceinline__ float2 diag(float2 dt, float2 zc, float2 zscale, bool has_beta, float2 beta,
                                                  float2 bval) {
        return df64::stencil_diag<ZS>(dt, zc, zscale, has_beta, beta, bval);
    }
    static __device__ __forceinline__ bool zero6(float2 a, float2 b, float2 c, float2 d, float2 e, float2 f) {
        const unsigned o = __float_as_uint(a.x) | __float_as_uint(a.y) | __float_as_uint(b.x) | __float_as_uint(b.y) |
                           __float_as_uint(c.x) | __float_as_uint(c.y) | __float_as_uint(d.x) | __float_as_uint(d.y) |
                           __float_as_uint(e.x) | __float_as_uint(e.y) | __float_as_uint(f.x) | __float_as_uint(f.y);
        return (o << 1) == 0u;
    }
    static __device__ __forceinline__ float2 axpy(float2 g, float2 x, float2 base) { return df64::df_fma(g, x, base); }
    static __device__ __forceinline__ float2 scale(float2 g, float2 x) { return df64::df_mul(g, x); }
    static __device__ __forceinline__ double widen(float2 x) { return (double)x.x + (double)x.y; }
    static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
};

}  // namespace et
