// Residual of the FP32 and DF64 forms in pair arithmetic (et_df64_arith.h),
// shared by the single-grid kernel (et_df64.cu) and the batched one
// (et_kernels.cu).
//
// The residual of the step (Eq. 2 and the scheme of Section 3) is
// b = L u + rho u (1 - u) with the diagonal of the shifted Jacobian beside it.
// Here it is computed from the pair of each u (ush) and the 1/nu-scaled
// pair weights W (W.w[4] = -rowsum / nu): S = (L / nu) u by the stencil code
// of the Taylor terms, b = nu S + rho u (1 - u) and dt = W.w[4] + shift + k_u u
// (k_u = -2 rho / nu for the folded reaction, else 0).  About 2^-44 relative,
// on the FP32 pipes: the FP64 version of this kernel is bound by GB300's FP64
// rate.  FP32 outputs take the high part of the normalised pair (the nearest
// float).
#pragma once

#include <cuda_runtime.h>

#include "et_df64_arith.h"
#include "et_internal.h"

namespace et {

__device__ __forceinline__ void store_pair(float2* d, float2 v) { *d = v; }
__device__ __forceinline__ void store_pair(float* d, float2 v) { *d = v.x; }

// Returns |b| and |u| of the voxel (their high parts) in *babs, *uabs.
template <int OP, typename TO>
__device__ __forceinline__ void residual_pair_point(const Geom& G, const PairResidualArgs& R, int scheme,
                                                    TO* __restrict__ b, TO* __restrict__ dt, unsigned* flags, int i,
                                                    int j, int k, float* babs, float* uabs) {
    using namespace df64;
    const long long p = i + G.sy * j + G.sz * k;
    const float2* __restrict__ ush = R.ush;
    const Weights<float2>& W = R.W;
    const float2 zero = make_float2(0.f, 0.f);
    const float2 uc = ush[p];
    const float2 w4 = W.w[4][p];
    float2 S;
    if (zero_row_of(G, W.zrow, i, j, k)) {
        // a warp row without off-diagonal entries: the six products have zero
        // weights (the same sum up to the sign of a zero), their loads skipped
        S = stencil_diag<false>(w4, uc, zero, false, zero, zero);
    } else {
        const bool xm = i > 0, ym = j > 0, zmk = k > 0;
        const float2 wxm = xm ? (OP == ET_OP_CONSERVATIVE ? W.w[0][p - 1] : W.w[3][p]) : zero;
        const float2 wym = ym ? (OP == ET_OP_CONSERVATIVE ? W.w[1][p - G.sy] : W.w[3][p]) : zero;
        const float2 wzm = zmk ? (OP == ET_OP_CONSERVATIVE ? W.w[2][p - G.sz] : W.w[3][p]) : zero;
        S = stencil<false>(w4, uc, W.w[0][p], (i + 1 < G.nx) ? ush[p + 1] : zero, wxm, xm ? ush[p - 1] : zero,
                           W.w[1][p], (j + 1 < G.ny) ? ush[p + G.sy] : zero, wym, ym ? ush[p - G.sy] : zero,
                           W.w[2][p], (k + 1 < G.nz) ? ush[p + G.sz] : zero, wzm, zmk ? ush[p - G.sz] : zero, zero,
                           false, zero, zero);
    }
    const float2 one_minus_u = df_add(make_float2(1.f, 0.f), make_float2(-uc.x, -uc.y));
    const float2 bp = df_add(df_mul(R.nu, S), df_mul(R.rho, df_mul(uc, one_minus_u)));
    store_pair(&b[p], bp);
    store_pair(&dt[p], df_add(w4, df_fma(R.k_u, uc, R.shift)));
    *babs = fabsf(bp.x);
    *uabs = fabsf(uc.x);
    const float uh = uc.x;
    if (!isfinite(uh)) atomicOr(flags, ET_FLAG_NONFINITE);
    if (scheme == ET_SCHEME_ROSENBROCK && (uh < (float)-kRangeSlack || uh > (float)(1.0 + kRangeSlack)))
        atomicOr(flags, ET_FLAG_RANGE_IN);
}

}  // namespace et
