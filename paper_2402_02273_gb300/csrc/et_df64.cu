// Double-float (DF64) Taylor-term kernel for sm_103a.
//
// GB300 executes FP64 at 2 FMA per clock per SM against 128 FP32 FMA, so a
// stencil term carried out in pairs of FP32 numbers (value = hi + lo, a 48-bit
// significand, unit roundoff about 2^-48) runs on the FP32 pipes at a fraction
// of the FP64 issue time and leaves the kernel bound by memory traffic again.
// The pair arithmetic (et_df64_arith.h) uses TwoSum and FMA-based TwoProduct;
// the stencil sum is a compensated dot product.
//
// The recurrence is the normalised form used for FP32 (et_kernels.cu): the
// weights and the diagonal are divided by nu = ||A - mu I|| bound, so the
// vectors z stay O(|b| / nu) and the pairs never approach the FP32 range.
#include <cuda_runtime.h>

#include "et_df64_arith.h"
#include "et_internal.h"
#include "et_residual_pair.h"

namespace et {
namespace {

using namespace df64;

// Inputs of one voxel-plane of the term: everything except the centre value
// and the -z neighbour, which are carried from the previous plane.
struct PlaneDF {
    float2 dt, wxp, wxm, wyp, wym, zxp, zxm, zyp, zym, zp, wzp, bb, yy, w3;
    bool zero;  // the warp row has no off-diagonal entries: dt z + beta b only
};

// One (i, j) column of kTileZ planes of a term in pair arithmetic.  The z-march
// is software-pipelined: the loads of plane k+1 are issued before plane k is
// computed, so each thread keeps a whole plane of loads in flight while the
// FP32 pipes work.
template <int OP, int TZ>
__device__ __forceinline__ void term_column_df64(const Geom& G, const Weights<float2>& W,
                                                 const TermArgs<float2>& a, int i, int j, int tz) {
    // restrict-qualified locals: the stores of one plane do not alias the loads of
    // the next, so those loads may be issued before the stores
    const float2* __restrict__ z = a.zin;
    const float2* __restrict__ w0 = W.w[0];
    const float2* __restrict__ w1 = W.w[1];
    const float2* __restrict__ w2 = W.w[2];
    const float2* __restrict__ w3 = W.w[3];
    const float2* __restrict__ dtv = a.dt;
    const float2* __restrict__ bv = a.b;
    float2* __restrict__ zout = a.zout;
    float2* __restrict__ yacc = a.yacc;
    double* __restrict__ u = a.u;
    const float2 zero = make_float2(0.f, 0.f);
    const bool need_b = a.has_beta || (!a.horner && a.base_mode == 1);
    const bool need_y = !a.horner && a.base_mode == 0;
    const bool xp = i + 1 < G.nx, xm = i > 0, yp = j + 1 < G.ny, ym = j > 0;
    const int k0 = tz * TZ;
    const int k1 = min(k0 + TZ, G.nz);
    const long long tiles_x = (G.nx + 31) >> 5;
    auto load = [&](PlaneDF& L, long long q, int k) {
        L.zero = W.zrow && W.zrow[(i >> 5) + tiles_x * (j + (long long)G.ny * k)];
        L.dt = dtv[q];
        if (!L.zero) {
            L.wxp = w0[q];
            L.wyp = w1[q];
            L.wzp = w2[q];
            L.w3 = (OP == ET_OP_LITERAL) ? w3[q] : zero;
            L.wxm = (OP == ET_OP_CONSERVATIVE && xm) ? w0[q - 1] : zero;
            L.wym = (OP == ET_OP_CONSERVATIVE && ym) ? w1[q - G.sy] : zero;
            L.zxp = xp ? z[q + 1] : zero;
            L.zxm = xm ? z[q - 1] : zero;
            L.zyp = yp ? z[q + G.sy] : zero;
            L.zym = ym ? z[q - G.sy] : zero;
        } else {
            // every weight of the row is 0, its +z weight (the next plane's -z
            // weight) included
            L.wxp = L.wyp = L.wzp = L.w3 = L.wxm = L.wym = zero;
            L.zxp = L.zxm = L.zyp = L.zym = zero;
        }
        L.zp = (k + 1 < G.nz) ? z[q + G.sz] : zero;
        L.bb = need_b ? bv[q] : zero;
        L.yy = need_y ? yacc[q] : zero;
    };
    long long p = i + G.sy * j + G.sz * k0;
    float2 zm = (k0 > 0) ? z[p - G.sz] : zero;
    float2 wzm_c = (OP == ET_OP_CONSERVATIVE && k0 > 0) ? w2[p - G.sz] : zero;
    float2 zc = z[p];
    PlaneDF cur;
    load(cur, p, k0);
    for (int k = k0; k < k1; ++k, p += G.sz) {
        PlaneDF nxt;
        if (k + 1 < k1) load(nxt, p + G.sz, k + 1);
        // literal: the -e weight of every axis is w3[p] (0 on the near wall)
        const float2 wxm = (OP == ET_OP_CONSERVATIVE) ? cur.wxm : (xm ? cur.w3 : zero);
        const float2 wym = (OP == ET_OP_CONSERVATIVE) ? cur.wym : (ym ? cur.w3 : zero);
        const float2 wzm = (OP == ET_OP_CONSERVATIVE) ? wzm_c : ((k > 0) ? cur.w3 : zero);
        float2 acc;
        if (cur.zero)
            acc = a.has_zscale ? stencil_diag<true>(cur.dt, zc, a.zscale, a.has_beta != 0, a.beta, cur.bb)
                               : stencil_diag<false>(cur.dt, zc, a.zscale, a.has_beta != 0, a.beta, cur.bb);
        else
            acc = a.has_zscale
                      ? stencil<true>(cur.dt, zc, cur.wxp, cur.zxp, wxm, cur.zxm, cur.wyp, cur.zyp, wym, cur.zym,
                                      cur.wzp, cur.zp, wzm, zm, a.zscale, a.has_beta != 0, a.beta, cur.bb)
                      : stencil<false>(cur.dt, zc, cur.wxp, cur.zxp, wxm, cur.zxm, cur.wyp, cur.zyp, wym, cur.zym,
                                       cur.wzp, cur.zp, wzm, zm, a.zscale, a.has_beta != 0, a.beta, cur.bb);
        if (a.horner) {
            if (!a.last) {
                zout[p] = acc;
            } else {
                const float2 r = df_mul(a.gamma, acc);
                if (u) u[p] += (double)r.x + (double)r.y;
                else yacc[p] = r;
            }
        } else {
            float2 base;
            if (a.base_mode == 0) base = cur.yy;
            else if (a.base_mode == 1) base = df_mul(a.base_scale, cur.bb);
            else base = zc;
            float2 sum = df_fma(a.g, acc, base);
            if (!a.last) {
                zout[p] = acc;
                yacc[p] = sum;
            } else {
                sum = df_mul(a.gamma, sum);
                if (u) u[p] += (double)sum.x + (double)sum.y;
                else yacc[p] = sum;
            }
        }
        zm = zc;
        zc = cur.zp;
        wzm_c = cur.wzp;
        cur = nxt;
    }
}

// Same tiling and recurrence as term_kernel in et_kernels.cu, in pair arithmetic.
// The parameters are __grid_constant__: the column code takes them by
// reference, which otherwise makes a local copy (32-64 B of stack at 80
// registers).
template <int OP>
__global__ void __launch_bounds__(kThreads, 3)
term_kernel_df64(const __grid_constant__ Geom G, const __grid_constant__ Weights<float2> W,
                 const __grid_constant__ TermArgs<float2> a) {
    const int tiles_x = (G.nx + kBlockX - 1) / kBlockX;
    const int tiles_y = (G.ny + kBlockY - 1) / kBlockY;
    const int tiles_z = (G.nz + kTileZ - 1) / kTileZ;
    const int ntiles = tiles_x * tiles_y * tiles_z;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tx = t % tiles_x;
        const int rest = t / tiles_x;
        const int ty = rest % tiles_y;
        const int tz = rest / tiles_y;
        const int i = tx * kBlockX + threadIdx.x;
        const int j = ty * kBlockY + threadIdx.y;
        if (i >= G.nx || j >= G.ny) continue;
        term_column_df64<OP, kTileZ>(G, W, a, i, j, tz);
    }
}

// Batched form: blocks loop over the tiles of all grids of the launch.
template <int OP, int TZ>
__global__ void __launch_bounds__(kThreads, 2)
batch_term_df64_kernel(const BatchTerm<float2>* __restrict__ d, int count, long long tiles) {
    __shared__ BatchTerm<float2> sd;
    const int tid = threadIdx.x + kBlockX * threadIdx.y;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (d[mid].tile_begin <= tile) lo = mid;
            else hi = mid - 1;
        }
        __syncthreads();
        const int* src = reinterpret_cast<const int*>(d + lo);
        int* dst = reinterpret_cast<int*>(&sd);
        for (int w = tid; w < (int)(sizeof(BatchTerm<float2>) / 4); w += kThreads) dst[w] = src[w];
        __syncthreads();
        const long long lt = tile - sd.tile_begin;
        const int tiles_x = (sd.G.nx + kBlockX - 1) / kBlockX;
        const int tiles_y = (sd.G.ny + kBlockY - 1) / kBlockY;
        const int i = (int)(lt % tiles_x) * kBlockX + threadIdx.x;
        const long long rest = lt / tiles_x;
        const int j = (int)(rest % tiles_y) * kBlockY + threadIdx.y;
        const int tz = (int)(rest / tiles_y);
        if (i < sd.G.nx && j < sd.G.ny) term_column_df64<OP, TZ>(sd.G, sd.W, sd.a, i, j, tz);
    }
}

template <int OP, int TZ>
int batch_df64_blocks_per_sm() {
    static int cached = 0;
    if (!cached) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_term_df64_kernel<OP, TZ>, kThreads, 0) !=
                cudaSuccess ||
            b < 1)
            b = 1;
        cached = b;
    }
    return cached;
}

template <int OP, int TZ>
cudaError_t launch_batch_df64(const BatchTerm<float2>* d, int count, long long tiles, int sms, cudaStream_t stream) {
    const long long cap = (long long)(sms > 0 ? sms : 1) * batch_df64_blocks_per_sm<OP, TZ>();
    batch_term_df64_kernel<OP, TZ><<<(unsigned)(tiles < cap ? tiles : cap), dim3(kBlockX, kBlockY, 1), 0, stream>>>(
        d, count, tiles);
    return cudaGetLastError();
}

template <int OP>
int df64_blocks_per_sm() {
    static int cached = 0;
    if (!cached) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, term_kernel_df64<OP>, kThreads, 0) != cudaSuccess ||
            b < 1)
            b = 1;
        cached = b;
    }
    return cached;
}

template <int OP, typename TO>
__global__ void __launch_bounds__(kThreads)
residual_df64_kernel(const __grid_constant__ Geom G, const __grid_constant__ PairResidualArgs R, int scheme,
                     TO* __restrict__ b, TO* __restrict__ dt, unsigned* flags, unsigned long long* wnorm) {
    pdl_begin();  // launched by launch_pdl
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    float babs = 0.f, uabs = 0.f;
    if (i < G.nx && j < G.ny) residual_pair_point<OP, TO>(G, R, scheme, b, dt, flags, i, j, blockIdx.z, &babs, &uabs);
    // one warp per row of the 32 x 8 block
    if (wnorm)
        warp_norms(babs, uabs,
                   wnorm + 2 * ((blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z)) * kBlockY +
                                threadIdx.y));
}

}  // namespace

template <typename TO>
cudaError_t launch_residual_df64(const Geom& G, et_operator op, const PairResidualArgs& R, et_scheme scheme, TO* b,
                                 TO* dt, unsigned* flags, cudaStream_t stream, unsigned long long* wnorm) {
    const dim3 block(kBlockX, kBlockY, 1);
    const dim3 grid((G.nx + kBlockX - 1) / kBlockX, (G.ny + kBlockY - 1) / kBlockY, G.nz);
    if (op == ET_OP_CONSERVATIVE)
        return launch_pdl(residual_df64_kernel<ET_OP_CONSERVATIVE, TO>, grid, block, stream, G, R, (int)scheme, b,
                          dt, flags, wnorm);
    return launch_pdl(residual_df64_kernel<ET_OP_LITERAL, TO>, grid, block, stream, G, R, (int)scheme, b, dt,
                      flags, wnorm);
}

template cudaError_t launch_residual_df64<float2>(const Geom&, et_operator, const PairResidualArgs&, et_scheme,
                                                  float2*, float2*, unsigned*, cudaStream_t, unsigned long long*);
template cudaError_t launch_residual_df64<float>(const Geom&, et_operator, const PairResidualArgs&, et_scheme, float*,
                                                 float*, unsigned*, cudaStream_t, unsigned long long*);

cudaError_t prime_launch_limits_df64() {
    df64_blocks_per_sm<ET_OP_CONSERVATIVE>();
    df64_blocks_per_sm<ET_OP_LITERAL>();
    return cudaGetLastError();
}

cudaError_t launch_batch_term(et_operator op, int variant, const BatchTerm<float2>* d, int count, long long tiles,
                              int sms, cudaStream_t stream) {
    const BatchVariant v = batch_variant(ET_DF64, variant);
    if (op == ET_OP_CONSERVATIVE)
        return v.tile_z == 2 ? launch_batch_df64<ET_OP_CONSERVATIVE, 2>(d, count, tiles, sms, stream)
                             : launch_batch_df64<ET_OP_CONSERVATIVE, 4>(d, count, tiles, sms, stream);
    return v.tile_z == 2 ? launch_batch_df64<ET_OP_LITERAL, 2>(d, count, tiles, sms, stream)
                         : launch_batch_df64<ET_OP_LITERAL, 4>(d, count, tiles, sms, stream);
}

cudaError_t launch_term(const Geom& G, et_operator op, Weights<float2> W, const TermArgs<float2>& a,
                        cudaStream_t stream) {
    const dim3 block(kBlockX, kBlockY, 1);
    const long long tiles = (long long)((G.nx + kBlockX - 1) / kBlockX) * ((G.ny + kBlockY - 1) / kBlockY) *
                            ((G.nz + kTileZ - 1) / kTileZ);
    const int sms = G.sms > 0 ? G.sms : 1;
    if (op == ET_OP_CONSERVATIVE) {
        const long long cap = (long long)sms * df64_blocks_per_sm<ET_OP_CONSERVATIVE>();
        term_kernel_df64<ET_OP_CONSERVATIVE><<<(unsigned)(tiles < cap ? tiles : cap), block, 0, stream>>>(G, W, a);
    } else {
        const long long cap = (long long)sms * df64_blocks_per_sm<ET_OP_LITERAL>();
        term_kernel_df64<ET_OP_LITERAL><<<(unsigned)(tiles < cap ? tiles : cap), block, 0, stream>>>(G, W, a);
    }
    return cudaGetLastError();
}

}  // namespace et
