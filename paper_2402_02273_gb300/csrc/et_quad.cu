// FP32 Taylor term with four x-consecutive voxels ("a quad") per thread.
//
// At the grid sizes of one patient the FP32 chain stays in the 129 MB L2, and
// the one-voxel-per-thread term kernel is bound by instruction issue: about
// 110 instructions per voxel-term, most of them thirteen scalar loads with
// their address arithmetic and edge selects.  Here a thread moves 16-byte
// vectors: per plane one new z quad (the centre and -z quads are carried from
// the planes before), the +-y quads, and one quad of each weight, of the
// diagonal, of b and of the running sum.  The x neighbours at the two ends of
// a quad are the adjacent lanes' end values (warp shuffles; a scalar load at
// the ends of the warp).  The per-voxel arithmetic is that of the one-voxel
// kernel, operation for operation, so both give identical numbers.
//
// Layout: the quads of a plane are numbered row by row (a row holds nx / 4 of
// them; nx % 4 == 0 and 16-byte aligned fields are required); a block of 256
// threads takes 256 consecutive quads and marches over tz planes.
#include <cuda_runtime.h>

#include <cstdint>

#include "et_internal.h"

namespace et {
namespace {

constexpr int kQuadThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float at(const float4& v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set(float4& v, int e, float x) {
    if (e == 0) v.x = x;
    else if (e == 1) v.y = x;
    else if (e == 2) v.z = x;
    else v.w = x;
}

template <int OP>
__global__ void __launch_bounds__(kQuadThreads, 4)
term_quad_kernel(const __grid_constant__ Geom G, const __grid_constant__ Weights<float> W,
                 const __grid_constant__ TermArgs<float> a, int tz) {
    constexpr bool kCons = OP == ET_OP_CONSERVATIVE;
    // 32-bit index arithmetic throughout (n < 2^31 is required): 64-bit
    // division is a long software sequence
    const unsigned qx = (unsigned)G.nx >> 2;
    const unsigned nq = qx * (unsigned)G.ny;  // quads per plane
    const int k0 = (int)blockIdx.y * tz;
    const int k1 = min(k0 + tz, G.nz);
    const unsigned q = blockIdx.x * kQuadThreads + threadIdx.x;
    const bool active = q < nq;
    const unsigned qq = active ? q : nq - 1;  // idle lanes shadow the last quad: their loads stay in bounds
    const int j = (int)(qq / qx);
    const int i = 4 * (int)(qq - (unsigned)j * qx);
    const int sy = (int)G.sy, sz = (int)G.sz;
    const int lane = threadIdx.x & 31;
    const bool has_xm = i > 0, has_xp = i + 4 < G.nx;
    const bool has_ym = j > 0, has_yp = j + 1 < G.ny;

    const float* __restrict__ z = a.zin;
    const float* __restrict__ w0 = W.w[0];
    const float* __restrict__ w1 = W.w[1];
    const float* __restrict__ w2 = W.w[2];
    const float* __restrict__ w3 = W.w[3];
    const float* __restrict__ dtv = a.dt;
    const float* __restrict__ bv = a.b;
    float* __restrict__ zout = a.zout;
    float* __restrict__ yacc = a.yacc;
    double* __restrict__ u = a.u;
    const bool need_b = a.has_beta || (!a.horner && a.base_mode == 1);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    pdl_begin();  // launched as a programmatic dependent launch (launch_pdl)

    int p = i + sy * j + sz * k0;
    float4 zc = ld4(z + p);
    float4 zm = k0 > 0 ? ld4(z + p - sz) : zero4;
    float4 wzm = (kCons && k0 > 0) ? ld4(w2 + p - sz) : zero4;  // conservative: w2 of the plane below
    for (int k = k0; k < k1; ++k, p += sz) {
        const bool has_zp = k + 1 < G.nz;
        const float4 zp = has_zp ? ld4(z + p + sz) : zero4;
        const float4 zyp = has_yp ? ld4(z + p + sy) : zero4;
        const float4 zym = has_ym ? ld4(z + p - sy) : zero4;
        const float4 w0v = ld4(w0 + p);
        const float4 w1v = ld4(w1 + p);
        const float4 w2v = ld4(w2 + p);
        const float4 dv = ld4(dtv + p);
        const float4 bq = need_b ? ld4(bv + p) : zero4;
        float4 w3v = zero4, wym, wzmk;
        if (kCons) {
            wym = has_ym ? ld4(w1 + p - sy) : zero4;
            wzmk = wzm;
        } else {
            w3v = ld4(w3 + p);
            wym = has_ym ? w3v : zero4;
            wzmk = k > 0 ? w3v : zero4;
        }
        // x neighbours of the quad's end voxels
        float zl = __shfl_up_sync(kFull, zc.w, 1);
        float zr = __shfl_down_sync(kFull, zc.x, 1);
        float w0l = __shfl_up_sync(kFull, w0v.w, 1);
        if (lane == 0 && has_xm) {
            zl = z[p - 1];
            if (kCons) w0l = w0[p - 1];
        }
        if (lane == 31 && has_xp) zr = z[p + 4];
        if (!has_xm) {
            zl = 0.f;
            w0l = 0.f;
        }
        if (!has_xp) zr = 0.f;

        float4 r;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float zxp = e < 3 ? at(zc, e + 1) : zr;
            const float zxm = e > 0 ? at(zc, e - 1) : zl;
            const float wxm = kCons ? (e > 0 ? at(w0v, e - 1) : w0l) : ((e > 0 || has_xm) ? at(w3v, e) : 0.f);
            float acc = at(dv, e) * at(zc, e);
            acc = fmaf(at(w0v, e), zxp, acc);
            acc = fmaf(wxm, zxm, acc);
            acc = fmaf(at(w1v, e), at(zyp, e), acc);
            acc = fmaf(at(wym, e), at(zym, e), acc);
            acc = fmaf(at(w2v, e), at(zp, e), acc);
            acc = fmaf(at(wzmk, e), at(zm, e), acc);
            if (a.has_zscale) acc *= a.zscale;
            if (a.has_beta) acc = fmaf(a.beta, at(bq, e), acc);
            set(r, e, acc);
        }
        if (active) {
            if (a.horner) {
                if (!a.last) {
                    st4(zout + p, r);
                } else if (u) {
                    double2* up = reinterpret_cast<double2*>(u + p);
                    double2 u01 = up[0], u23 = up[1];
                    u01.x += (double)(r.x * a.gamma);
                    u01.y += (double)(r.y * a.gamma);
                    u23.x += (double)(r.z * a.gamma);
                    u23.y += (double)(r.w * a.gamma);
                    up[0] = u01;
                    up[1] = u23;
                } else {
                    st4(yacc + p, make_float4(r.x * a.gamma, r.y * a.gamma, r.z * a.gamma, r.w * a.gamma));
                }
            } else {
                float4 base;
                if (a.base_mode == 0) base = ld4(yacc + p);
                else if (a.base_mode == 1)
                    base = make_float4(a.base_scale * bq.x, a.base_scale * bq.y, a.base_scale * bq.z,
                                       a.base_scale * bq.w);
                else base = zc;
                const float4 sum = make_float4(fmaf(a.g, r.x, base.x), fmaf(a.g, r.y, base.y),
                                               fmaf(a.g, r.z, base.z), fmaf(a.g, r.w, base.w));
                if (!a.last) {
                    st4(zout + p, r);
                    st4(yacc + p, sum);
                } else if (u) {
                    double2* up = reinterpret_cast<double2*>(u + p);
                    double2 u01 = up[0], u23 = up[1];
                    u01.x += (double)(sum.x * a.gamma);
                    u01.y += (double)(sum.y * a.gamma);
                    u23.x += (double)(sum.z * a.gamma);
                    u23.y += (double)(sum.w * a.gamma);
                    up[0] = u01;
                    up[1] = u23;
                } else {
                    st4(yacc + p,
                        make_float4(sum.x * a.gamma, sum.y * a.gamma, sum.z * a.gamma, sum.w * a.gamma));
                }
            }
        }
        zm = zc;
        zc = zp;
        if (kCons) wzm = w2v;
    }
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

bool quad_eligible(const Geom& G, const Weights<float>& W, const TermArgs<float>& a) {
    if (G.nx % 4 != 0 || G.n >= (1ll << 31) || G.nz > 65535) return false;
    const void* ptrs[] = {W.w[0], W.w[1], W.w[2], W.w[3], a.zin, a.zout, a.b, a.dt, a.yacc, a.u};
    for (const void* p : ptrs)
        if (p && !aligned16(p)) return false;
    return true;
}

int quad_planes(const Geom& G) {
    // planes per thread: the longest z-march (up to 8 planes) that still gives
    // three blocks per SM, about one wave of the four resident ones.  Measured
    // at 128^3 (us per term): 1 plane 7.2, 2 planes 6.3, 4 planes 6.1 (the
    // choice), 8 planes 6.9, 16 planes 10.5.
    const long long nq = (long long)(G.nx / 4) * G.ny;
    const long long tiles_plane = (nq + kQuadThreads - 1) / kQuadThreads;
    const long long target = 3ll * (G.sms > 0 ? G.sms : 1);
    int tz = 1;
    while (tz < 8 && tiles_plane * ((G.nz + 2 * tz - 1) / (2 * tz)) >= target) tz *= 2;
    return tz;
}

cudaError_t launch_term_quad(const Geom& G, et_operator op, const Weights<float>& W, const TermArgs<float>& a,
                             cudaStream_t stream) {
    const int tz = quad_planes(G);
    const long long nq = (long long)(G.nx / 4) * G.ny;
    const dim3 grid((unsigned)((nq + kQuadThreads - 1) / kQuadThreads), (unsigned)((G.nz + tz - 1) / tz), 1);
    const dim3 block(kQuadThreads, 1, 1);
    if (op == ET_OP_CONSERVATIVE) return launch_pdl(term_quad_kernel<ET_OP_CONSERVATIVE>, grid, block, stream, G, W, a, tz);
    return launch_pdl(term_quad_kernel<ET_OP_LITERAL>, grid, block, stream, G, W, a, tz);
}

}  // namespace et
