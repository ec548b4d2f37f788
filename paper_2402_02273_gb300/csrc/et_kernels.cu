// CUDA kernels of the exponential-integrator step (arXiv 2402.02273, Sec. 2.1-2.2)
// for sm_103a.
//
// Four kernels make a step:
//   coeffs   (once per et_set_coeffs): face weights of L, minus its row sums,
//            and the bound max_p sum_{q != p} |L_pq|;
//   residual (once per step): b = L u^n + rho u^n (1 - u^n) (= A_n u^n + f(u^n),
//            eq. F / newF) and the diagonal of A_n - mu I;
//   term     (s*m - 1 per step): one term of the scaled Taylor recurrence of
//            exp(h (B - mu I)) applied to the augmented vector, see below;
//   stats    (once per step): min, max and sum of u^{n+1}.
//
// Scaled recurrence.  With h = tau / s, A~ = A - mu I and the augmented scalar
// a_k of sub-step k (a_0 = 1), the j-th Taylor term of exp(h(B - mu I)) [y; a]
// is g_j z^_j with g_j = h^j / j! and
//     z^_0 = y,   z^_{j+1} = A~ z^_j + a_k (-mu)^j b,
// so a term costs one stencil application plus two fused multiply-adds and
// needs no per-term rescaling.  The sub-step result is
//     y <- e^{mu h} (y + sum_{j=1..m} g_j z^_j),
// and on the last sub-step u^{n+1} = u^n + y is written directly.
//
// GB300 executes FP64 at 2 FMA per clock per SM (1/64 of FP32), so the FP64
// kernels are bound by FP64 instruction issue: every FP64 operation that is not
// part of the arithmetic above (comparisons, range checks, reductions of
// min/max) is done in integer or FP32 form instead.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "et_df64_arith.h"
#include "et_internal.h"
#include "et_residual_pair.h"

namespace et {
namespace {

__device__ __forceinline__ double harmonic_mean(double a, double b) {
    return (a > 0.0 && b > 0.0) ? 2.0 * a * b / (a + b) : 0.0;
}

// Monotone map of a double onto unsigned 64-bit integers (min/max by integer compare).
__device__ __forceinline__ unsigned long long order_key(double v) {
    const long long b = __double_as_longlong(v);
    return b < 0 ? ~(unsigned long long)b : ((unsigned long long)b | 0x8000000000000000ull);
}
__device__ __forceinline__ double order_key_inv(unsigned long long k) {
    return __longlong_as_double((k & 0x8000000000000000ull) ? (long long)(k & 0x7fffffffffffffffull)
                                                           : (long long)~k);
}
__device__ __forceinline__ bool nonfinite_bits(long long b) {
    return (b & 0x7ff0000000000000ll) == 0x7ff0000000000000ll;
}

dim3 voxel_grid(const Geom& G) {
    return dim3((G.nx + kBlockX - 1) / kBlockX, (G.ny + kBlockY - 1) / kBlockY, G.nz);
}

// ---------------------------------------------------------------------------
// coeffs: face weights, minus the row sums, and max_p sum_{q != p} |L_pq|.
template <int OP>
__global__ void __launch_bounds__(kThreads)
coeffs_kernel(Geom G, const double* __restrict__ D, double dscale, double inv_h2, double* __restrict__ w0,
              double* __restrict__ w1, double* __restrict__ w2, double* __restrict__ w3,
              double* __restrict__ w4, unsigned long long* rmax_bits, unsigned* flags) {
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int k = blockIdx.z;
    double absrow = 0.0;
    if (i < G.nx && j < G.ny) {
        const long long p = i + G.sy * j + G.sz * k;
        // the field is read as D * dscale (a product rounded once; exact for dscale = 1)
        const double Dp = D[p] * dscale;
        if (!(Dp >= 0.0) || !isfinite(Dp)) atomicOr(flags, ET_FLAG_D_INVALID);
        const int c[3] = {i, j, k};
        const int ext[3] = {G.nx, G.ny, G.nz};
        const long long st[3] = {1, G.sy, G.sz};
        double wp[3];
        double row = 0.0;
        for (int a = 0; a < 3; ++a) {
            const bool has_plus = c[a] + 1 < ext[a];
            const bool has_minus = c[a] > 0;
            const double Dq = has_plus ? D[p + st[a]] * dscale : 0.0;
            const double Dm = has_minus ? D[p - st[a]] * dscale : 0.0;
            double wplus, wminus;
            if (OP == ET_OP_CONSERVATIVE) {
                wplus = has_plus ? harmonic_mean(Dp, Dq) * inv_h2 : 0.0;
                wminus = has_minus ? harmonic_mean(Dm, Dp) * inv_h2 : 0.0;
            } else {
                wplus = has_plus ? (Dp + Dq) * inv_h2 : 0.0;
                wminus = has_minus ? 2.0 * Dp * inv_h2 : 0.0;
            }
            wp[a] = wplus;
            row += wplus + wminus;
            absrow += fabs(wplus) + fabs(wminus);
        }
        w0[p] = wp[0];
        w1[p] = wp[1];
        w2[p] = wp[2];
        w3[p] = (OP == ET_OP_LITERAL) ? 2.0 * Dp * inv_h2 : 0.0;
        w4[p] = -row;
    }
    // block maximum, then one atomic per block on the (monotone) bit pattern
    __shared__ double smax[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) absrow = fmax(absrow, __shfl_down_sync(0xffffffffu, absrow, off));
    const int tid = threadIdx.x + kBlockX * threadIdx.y;
    if ((tid & 31) == 0) smax[tid >> 5] = absrow;
    __syncthreads();
    if (tid == 0) {
        double m = smax[0];
        for (int w = 1; w < kThreads / 32; ++w) m = fmax(m, smax[w]);
        if (isfinite(m)) atomicMax(rmax_bits, (unsigned long long)__double_as_longlong(m));
    }
}

// Stores an FP64 value in the kernels' value types; FP64 -> (hi, lo) splits
// exactly up to the 48-bit significand of the pair.
__device__ __forceinline__ void store_value(double* d, double v) { *d = v; }
__device__ __forceinline__ void store_value(float* d, double v) { *d = (float)v; }
__device__ __forceinline__ void store_value(float2* d, double v) {
    const float hi = (float)v;
    *d = make_float2(hi, (float)(v - (double)hi));
}

template <typename T>
__global__ void convert_weights_kernel(long long n, const double* __restrict__ a0,
                                       const double* __restrict__ a1, const double* __restrict__ a2,
                                       const double* __restrict__ a3, double scale, T* __restrict__ f0,
                                       T* __restrict__ f1, T* __restrict__ f2, T* __restrict__ f3) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        store_value(&f0[p], a0[p] * scale);
        store_value(&f1[p], a1[p] * scale);
        store_value(&f2[p], a2[p] * scale);
        store_value(&f3[p], a3[p] * scale);
    }
}

// Weight towards -e at voxel p (0 on the near wall).
template <int OP, typename T>
__device__ __forceinline__ T minus_weight(const Weights<T>& W, int axis, long long p, long long stride,
                                          bool has_minus) {
    if (!has_minus) return T(0);
    return OP == ET_OP_CONSERVATIVE ? W.w[axis][p - stride] : W.w[3][p];
}

// ---------------------------------------------------------------------------
// Rows without off-diagonal entries, one flag per warp row (a ballot of the
// row's 32 x-consecutive voxels, the weights as the term kernels read them).
template <int OP>
__global__ void __launch_bounds__(kThreads)
zero_rows_kernel(Geom G, Weights<double> W, unsigned char* __restrict__ zrow, unsigned long long* count) {
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int k = blockIdx.z;
    const bool in = i < G.nx && j < G.ny;
    bool nonzero = false;
    if (in) {
        const long long p = i + G.sy * j + G.sz * k;
        nonzero = W.w[0][p] != 0.0 || minus_weight<OP, double>(W, 0, p, 1, i > 0) != 0.0 || W.w[1][p] != 0.0 ||
                  minus_weight<OP, double>(W, 1, p, G.sy, j > 0) != 0.0 || W.w[2][p] != 0.0 ||
                  minus_weight<OP, double>(W, 2, p, G.sz, k > 0) != 0.0;
    }
    const unsigned any = __ballot_sync(0xffffffffu, nonzero);
    const unsigned lanes = __ballot_sync(0xffffffffu, in);
    if (threadIdx.x == 0 && j < G.ny) {
        const bool zero = any == 0u;
        zrow[blockIdx.x + (long long)gridDim.x * (j + (long long)G.ny * k)] = zero ? 1 : 0;
        if (zero) atomicAdd(count, (unsigned long long)__popc(lanes));
    }
}

// ---------------------------------------------------------------------------
// residual: b = L u + rho u (1 - u), diag = rho(1 - 2u) - R - mu (or -R - mu).
// L u = sum_e w_e u_e - R u_p with R from the coefficient pass: 12 FP64
// operations per voxel; the range test on u runs on the integer bits.
// Returns |b| and |u| of the voxel in *babs, *uabs (the step's norms).
template <int OP, typename T>
__device__ __forceinline__ void residual_point(const Geom& G, const double* __restrict__ u, const Weights<double>& W,
                                               double rho, double dt_shift, double dt_scale, int scheme,
                                               T* __restrict__ b, T* __restrict__ dt, unsigned* flags, int i, int j,
                                               int k, double* babs, double* uabs) {
    const long long p = i + G.sy * j + G.sz * k;
    const double up = u[p];
    const double negR = W.w[4][p];
    double Lu = negR * up;
    // a warp row without off-diagonal entries (W.zrow, nullptr: none marked)
    // skips the six products with zero weights, their loads included
    const bool zero_row = W.zrow && W.zrow[(i >> 5) + (long long)((G.nx + 31) >> 5) * (j + (long long)G.ny * k)];
    if (!zero_row) {
        Lu = fma(W.w[0][p], (i + 1 < G.nx) ? u[p + 1] : 0.0, Lu);
        Lu = fma(minus_weight<OP, double>(W, 0, p, 1, i > 0), (i > 0) ? u[p - 1] : 0.0, Lu);
        Lu = fma(W.w[1][p], (j + 1 < G.ny) ? u[p + G.sy] : 0.0, Lu);
        Lu = fma(minus_weight<OP, double>(W, 1, p, G.sy, j > 0), (j > 0) ? u[p - G.sy] : 0.0, Lu);
        Lu = fma(W.w[2][p], (k + 1 < G.nz) ? u[p + G.sz] : 0.0, Lu);
        Lu = fma(minus_weight<OP, double>(W, 2, p, G.sz, k > 0), (k > 0) ? u[p - G.sz] : 0.0, Lu);
    }
    const double bp = fma(rho * up, 1.0 - up, Lu);
    double dp;
    if (scheme == ET_SCHEME_ROSENBROCK) dp = fma(-2.0 * rho, up, negR + dt_shift);
    else dp = negR + dt_shift;
    store_value(&b[p], bp);
    store_value(&dt[p], dp * dt_scale);
    *babs = fabs(bp);
    *uabs = fabs(up);
    const long long bits = __double_as_longlong(up);
    if (nonfinite_bits(bits)) atomicOr(flags, ET_FLAG_NONFINITE);
    if (scheme == ET_SCHEME_ROSENBROCK) {
        // u in [-slack, 1 + slack], compared on the bit patterns
        const long long hi = __double_as_longlong(1.0 + kRangeSlack);
        const long long lo = __double_as_longlong(kRangeSlack);
        const bool out = bits >= 0 ? bits > hi : (bits & 0x7fffffffffffffffll) > lo;
        if (out) atomicOr(flags, ET_FLAG_RANGE_IN);
    }
}

template <int OP, typename T>
__global__ void __launch_bounds__(kThreads)
residual_kernel(Geom G, const double* __restrict__ u, Weights<double> W, double rho, double dt_shift,
                double dt_scale, int scheme, T* __restrict__ b, T* __restrict__ dt, unsigned* flags,
                unsigned long long* wnorm) {
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int k = blockIdx.z;
    pdl_begin();  // launched by launch_pdl
    double babs = 0.0, uabs = 0.0;
    if (i < G.nx && j < G.ny)
        residual_point<OP, T>(G, u, W, rho, dt_shift, dt_scale, scheme, b, dt, flags, i, j, k, &babs, &uabs);
    // one warp per row of the 32 x 8 block
    if (wnorm)
        warp_norms(babs, uabs,
                   wnorm + 2 * ((blockIdx.x + gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z)) * kBlockY +
                                threadIdx.y));
}

// gamma * sum, rounded to the value type and widened, then added to u: the
// product is rounded on its own (never fused with the addition), so that u
// plus a recorded gamma * sum (the adjoint's segment states) is the same sum.
__device__ __forceinline__ double widened_product(double x, double g) { return __dmul_rn(x, g); }
__device__ __forceinline__ double widened_product(float x, float g) { return (double)(x * g); }

// One (i, j) column of TZ planes of a term, marching in z with the z-neighbours
// (and, for the conservative operator, the -z face weight) carried in registers.
template <int OP, typename T, int TZ>
__device__ __forceinline__ void term_column(const Geom& G, const Weights<T>& W, const TermArgs<T>& a, int i, int j,
                                            int tz) {
    // restrict-qualified locals: the stores of one plane do not alias the loads of
    // the next, so the compiler may issue those loads early
    const T* __restrict__ z = a.zin;
    const T* __restrict__ w0 = W.w[0];
    const T* __restrict__ w1 = W.w[1];
    const T* __restrict__ w2 = W.w[2];
    const T* __restrict__ w3 = W.w[3];
    const T* __restrict__ dtv = a.dt;
    const T* __restrict__ bv = a.b;
    T* __restrict__ zout = a.zout;
    T* __restrict__ yacc = a.yacc;
    double* __restrict__ u = a.u;
    const int k0 = tz * TZ;
    const int k1 = min(k0 + TZ, G.nz);
    long long p = i + G.sy * j + G.sz * k0;
    T zm = (k0 > 0) ? z[p - G.sz] : T(0);
    T wzm = (k0 > 0) ? (OP == ET_OP_CONSERVATIVE ? w2[p - G.sz] : w3[p]) : T(0);
    T zc = z[p];
#pragma unroll 2
    for (int k = k0; k < k1; ++k, p += G.sz) {
        const bool has_zp = k + 1 < G.nz;
        const T zp = has_zp ? z[p + G.sz] : T(0);
        const T wzp = w2[p];
        T acc = dtv[p] * zc;
        acc = fma(w0[p], (i + 1 < G.nx) ? z[p + 1] : T(0), acc);
        acc = fma((i > 0) ? (OP == ET_OP_CONSERVATIVE ? w0[p - 1] : w3[p]) : T(0), (i > 0) ? z[p - 1] : T(0), acc);
        acc = fma(w1[p], (j + 1 < G.ny) ? z[p + G.sy] : T(0), acc);
        acc = fma((j > 0) ? (OP == ET_OP_CONSERVATIVE ? w1[p - G.sy] : w3[p]) : T(0), (j > 0) ? z[p - G.sy] : T(0),
                  acc);
        acc = fma(wzp, zp, acc);
        acc = fma(wzm, zm, acc);
        if constexpr (!std::is_same<T, double>::value) {
            if (a.has_zscale) acc *= a.zscale;  // only the normalised (FP32) chain scales
        }
        if (a.has_beta) acc = fma(a.beta, bv[p], acc);
        if (a.horner) {
            if (!a.last) zout[p] = acc;
            else if (u) u[p] += widened_product(acc, a.gamma);
            else yacc[p] = acc * a.gamma;
        } else {
            T base;
            if (a.base_mode == 0) base = yacc[p];
            else if (a.base_mode == 1) base = a.base_scale * bv[p];
            else base = zc;
            T sum = fma(a.g, acc, base);
            if (!a.last) {
                zout[p] = acc;
                yacc[p] = sum;
            } else if (u) {
                u[p] += widened_product(sum, a.gamma);
            } else {
                yacc[p] = sum * a.gamma;
            }
        }
        zm = zc;
        zc = zp;
        wzm = (OP == ET_OP_CONSERVATIVE) ? wzp : (has_zp ? w3[p + G.sz] : T(0));
    }
}

// ---------------------------------------------------------------------------
// term: z^_{j+1} = A~ z^_j + beta b;  sum = base + g z^_{j+1};
// last term: sum *= gamma and either stored as the next y or added to u.
// Blocks loop over tiles so the grid matches the resident-block capacity.
template <int OP, typename T, int TZ>
__global__ void __launch_bounds__(kThreads)
term_kernel(Geom G, Weights<T> W, TermArgs<T> a) {
    const int tiles_x = (G.nx + kBlockX - 1) / kBlockX;
    const int tiles_y = (G.ny + kBlockY - 1) / kBlockY;
    const int tiles_z = (G.nz + TZ - 1) / TZ;
    const int ntiles = tiles_x * tiles_y * tiles_z;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tx = t % tiles_x;
        const int rest = t / tiles_x;
        const int ty = rest % tiles_y;
        const int tz = rest / tiles_y;
        const int i = tx * kBlockX + threadIdx.x;
        const int j = ty * kBlockY + threadIdx.y;
        if (i >= G.nx || j >= G.ny) continue;
        term_column<OP, T, TZ>(G, W, a, i, j, tz);
    }
}

// FP64 term, one voxel per thread over a (32 x 8 x nz)-block grid.  The FP64
// kernel is bound by the FP64 pipe, so it is kept lean for full occupancy
// (no plane loop, operands straight from the kernel parameters).
template <int OP>
__device__ __forceinline__ void term_point_f64(const Geom& G, const Weights<double>& W, const TermArgs<double>& a,
                                               int i, int j, int k, bool zero_row) {
    const long long p = i + G.sy * j + G.sz * k;
    const double* __restrict__ z = a.zin;
    const double zc = z[p];
    double acc = a.dt[p] * zc;
    // a zero row skips the six products with zero weights, their loads included
    if (!zero_row) {
        acc = fma(W.w[0][p], (i + 1 < G.nx) ? z[p + 1] : 0.0, acc);
        acc = fma(minus_weight<OP, double>(W, 0, p, 1, i > 0), (i > 0) ? z[p - 1] : 0.0, acc);
        acc = fma(W.w[1][p], (j + 1 < G.ny) ? z[p + G.sy] : 0.0, acc);
        acc = fma(minus_weight<OP, double>(W, 1, p, G.sy, j > 0), (j > 0) ? z[p - G.sy] : 0.0, acc);
        acc = fma(W.w[2][p], (k + 1 < G.nz) ? z[p + G.sz] : 0.0, acc);
        acc = fma(minus_weight<OP, double>(W, 2, p, G.sz, k > 0), (k > 0) ? z[p - G.sz] : 0.0, acc);
    }
    if (a.has_beta) acc = fma(a.beta, a.b[p], acc);
    if (a.horner) {
        // sub-step 0 by Horner's rule: no running sum to read or write
        if (!a.last) a.zout[p] = acc;
        else if (a.u) a.u[p] += widened_product(acc, a.gamma);
        else a.yacc[p] = acc * a.gamma;
        return;
    }
    double base;
    if (a.base_mode == 0) base = a.yacc[p];
    else if (a.base_mode == 1) base = a.base_scale * a.b[p];
    else base = zc;
    const double sum = fma(a.g, acc, base);
    if (!a.last) {
        a.zout[p] = acc;
        a.yacc[p] = sum;
    } else if (a.u) {
        a.u[p] += widened_product(sum, a.gamma);
    } else {
        a.yacc[p] = sum * a.gamma;
    }
}

template <int OP>
__global__ void __launch_bounds__(kThreads)
term_kernel_f64(Geom G, Weights<double> W, TermArgs<double> a) {
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int k = blockIdx.z;
    // the zero-row marks are written by et_set_coeffs, never by the chain: read
    // before the wait for the previous grid
    const bool zero_row = i < G.nx && j < G.ny && zero_row_of(G, W.zrow, i, j, k);
    pdl_begin();  // launched by launch_pdl
    if (i >= G.nx || j >= G.ny) return;
    term_point_f64<OP>(G, W, a, i, j, k, zero_row);
}

// ---------------------------------------------------------------------------
// stats: sum, min and max of u (min/max through integer order keys, one FP64
// add per voxel), the non-finite flag, then the step record; the F32 and DF64
// forms also take here the pair of each u, which their next residual reads.  A fixed grid of
// kStatsBlocks blocks fixes every summation order (bitwise reproducible).
// Block `blk` (of kStatsBlocks) of the reduction over u[0..n).
__device__ __forceinline__ void stats_body(long long n, const double* __restrict__ u, const StatsSink& s, int blk) {
    constexpr int kWarps = kStatsThreads / 32;
    __shared__ double ssum[kWarps];
    __shared__ unsigned long long smin[kWarps], smax[kWarps], snb[kWarps], snu[kWarps];
    __shared__ bool is_last;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    double sum = 0.0;
    unsigned long long kmin = ~0ull, kmax = 0ull;
    bool bad = false;
    // the residual's warp norm slots of this step (read first, so their
    // latency overlaps the pass over u)
    unsigned long long nb = 0ull, nu = 0ull;
    if (s.wnorm) {
        for (long long q = blk * (long long)kStatsThreads + tid; q < s.nwarps;
             q += (long long)kStatsBlocks * kStatsThreads) {
            const unsigned long long b0 = __ldcg(&s.wnorm[2 * q + 0]);
            const unsigned long long u0 = __ldcg(&s.wnorm[2 * q + 1]);
            nb = b0 > nb ? b0 : nb;
            nu = u0 > nu ? u0 : nu;
        }
    }
#pragma unroll 4
    for (long long p = blk * (long long)kStatsThreads + tid; p < n; p += (long long)kStatsBlocks * kStatsThreads) {
        const double v = u[p];
        if (s.ush) s.ush[p] = df64::from_double(v);
        sum += v;
        const unsigned long long key = order_key(v);
        kmin = key < kmin ? key : kmin;
        kmax = key > kmax ? key : kmax;
        bad |= nonfinite_bits(__double_as_longlong(v));
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(s.flags, ET_FLAG_NONFINITE);
    for (int off = 16; off > 0; off >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, off);
        const unsigned long long omin = __shfl_down_sync(0xffffffffu, kmin, off);
        const unsigned long long omax = __shfl_down_sync(0xffffffffu, kmax, off);
        const unsigned long long onb = __shfl_down_sync(0xffffffffu, nb, off);
        const unsigned long long onu = __shfl_down_sync(0xffffffffu, nu, off);
        kmin = omin < kmin ? omin : kmin;
        kmax = omax > kmax ? omax : kmax;
        nb = onb > nb ? onb : nb;
        nu = onu > nu ? onu : nu;
    }
    if (lane == 0) {
        ssum[warp] = sum;
        smin[warp] = kmin;
        smax[warp] = kmax;
        snb[warp] = nb;
        snu[warp] = nu;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kWarps; ++w) {
            sum += ssum[w];
            kmin = smin[w] < kmin ? smin[w] : kmin;
            kmax = smax[w] > kmax ? smax[w] : kmax;
            nb = snb[w] > nb ? snb[w] : nb;
            nu = snu[w] > nu ? snu[w] : nu;
        }
        s.partial[3 * blk + 0] = sum;
        s.partial[3 * blk + 1] = __longlong_as_double((long long)kmin);
        s.partial[3 * blk + 2] = __longlong_as_double((long long)kmax);
        if (s.wnorm) {
            s.npartial[2 * blk + 0] = __longlong_as_double((long long)nb);
            s.npartial[2 * blk + 1] = __longlong_as_double((long long)nu);
        }
        __threadfence();
        const unsigned ticket = atomicAdd(s.ticket, 1u);
        is_last = (ticket == kStatsBlocks - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    sum = 0.0;
    kmin = ~0ull;
    kmax = 0ull;
    for (int q = tid; q < kStatsBlocks; q += kStatsThreads) {
        sum += __ldcg(&s.partial[3 * q + 0]);
        const unsigned long long a = (unsigned long long)__double_as_longlong(__ldcg(&s.partial[3 * q + 1]));
        const unsigned long long b = (unsigned long long)__double_as_longlong(__ldcg(&s.partial[3 * q + 2]));
        kmin = a < kmin ? a : kmin;
        kmax = b > kmax ? b : kmax;
    }
    nb = 0ull;
    nu = 0ull;
    if (s.wnorm) {
        for (int q = tid; q < kStatsBlocks; q += kStatsThreads) {
            const unsigned long long b0 = (unsigned long long)__double_as_longlong(__ldcg(&s.npartial[2 * q + 0]));
            const unsigned long long u0 = (unsigned long long)__double_as_longlong(__ldcg(&s.npartial[2 * q + 1]));
            nb = b0 > nb ? b0 : nb;
            nu = u0 > nu ? u0 : nu;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, off);
        const unsigned long long omin = __shfl_down_sync(0xffffffffu, kmin, off);
        const unsigned long long omax = __shfl_down_sync(0xffffffffu, kmax, off);
        const unsigned long long onb = __shfl_down_sync(0xffffffffu, nb, off);
        const unsigned long long onu = __shfl_down_sync(0xffffffffu, nu, off);
        kmin = omin < kmin ? omin : kmin;
        kmax = omax > kmax ? omax : kmax;
        nb = onb > nb ? onb : nb;
        nu = onu > nu ? onu : nu;
    }
    __syncthreads();
    if (lane == 0) {
        ssum[warp] = sum;
        smin[warp] = kmin;
        smax[warp] = kmax;
        snb[warp] = nb;
        snu[warp] = nu;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kWarps; ++w) {
            sum += ssum[w];
            kmin = smin[w] < kmin ? smin[w] : kmin;
            kmax = smax[w] > kmax ? smax[w] : kmax;
            nb = snb[w] > nb ? snb[w] : nb;
            nu = snu[w] > nu ? snu[w] : nu;
        }
        const unsigned step = *s.step_counter;
        et_step_info rec;
        rec.umin = order_key_inv(kmin);
        rec.umax = order_key_inv(kmax);
        rec.mass = sum;
        rec.s = s.s;
        rec.m = s.m_dev ? *s.m_dev : s.m;
        if (s.wnorm) {
            // a-posteriori truncation estimate of the step: the remainder bound
            // of its (s, m) with the measured max |b| in place of its a-priori
            // bound, relative to max |u^n|
            const double bmax = __longlong_as_double((long long)nb), umax = __longlong_as_double((long long)nu);
            const double est = umax > 0.0 ? s.trunc_c * bmax / umax : (bmax > 0.0 ? INFINITY : 0.0);
            if (est > s.trunc_tol) atomicOr(s.flags, ET_FLAG_TRUNCATION);
            if (s.trunc_est) *s.trunc_est = est;
        }
        rec.flags = atomicOr(s.flags, 0u);
        rec.step = step;
        s.info[(size_t)step * (unsigned)s.info_stride] = rec;
        *s.last = rec;
        *s.step_counter = step + 1;
        *s.ticket = 0u;
        __threadfence();
    }
}

__global__ void __launch_bounds__(kStatsThreads) stats_kernel(long long n, const double* __restrict__ u,
                                                              StatsSink s) {
    pdl_begin();  // launched by launch_pdl
    stats_body(n, u, s, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Batched kernels: the descriptor of the block's grid is copied to shared
// memory once per tile, then the single-grid device functions run on it.

template <typename D>
__device__ __forceinline__ int find_desc(const D* __restrict__ d, int count, long long tile) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].tile_begin <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename D>
__device__ __forceinline__ void copy_desc(D& dst, const D* __restrict__ src) {
    static_assert(sizeof(D) % 4 == 0, "descriptor size");
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int* s = reinterpret_cast<const int*>(src);
    int* t = reinterpret_cast<int*>(&dst);
    for (int w = tid; w < (int)(sizeof(D) / 4); w += blockDim.x * blockDim.y) t[w] = s[w];
}

template <int OP, typename T>
__global__ void __launch_bounds__(kThreads)
batch_residual_kernel(const BatchResidual<T>* __restrict__ d, int count, int scheme, unsigned* flags) {
    __shared__ BatchResidual<T> sd;
    const long long tile = blockIdx.x;
    const int di = find_desc(d, count, tile);
    copy_desc(sd, d + di);
    __syncthreads();
    const long long lt = tile - sd.tile_begin;
    const int tiles_x = (sd.G.nx + kBlockX - 1) / kBlockX;
    const int tiles_y = (sd.G.ny + kBlockY - 1) / kBlockY;
    const int i = (int)(lt % tiles_x) * kBlockX + threadIdx.x;
    const long long rest = lt / tiles_x;
    const int j = (int)(rest % tiles_y) * kBlockY + threadIdx.y;
    const int k = (int)(rest / tiles_y);
    // |b| and |u| as doubles (FP64 form) or as the floats of their high parts
    using NormT = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
    NormT babs = 0, uabs = 0;
    if (i < sd.G.nx && j < sd.G.ny) {
        if constexpr (std::is_same<T, double>::value)
            residual_point<OP, T>(sd.G, sd.u, sd.W, sd.rho, sd.dt_shift, sd.dt_scale, scheme, sd.b, sd.dt, flags, i,
                                  j, k, &babs, &uabs);
        else
            residual_pair_point<OP, T>(sd.G, sd.P, scheme, sd.b, sd.dt, flags, i, j, k, &babs, &uabs);
    }
    if (sd.wnorm) warp_norms(babs, uabs, sd.wnorm + 2 * (tile * kBlockY + threadIdx.y));
}

// FP64, one tile (32 x 8 x 1) per block.  The descriptor's fields are read
// from the (read-only, cached) table itself: a block of zero rows does so
// little work that a copy to shared memory and its barrier would dominate
// (measured over the 64-grid batch: 1633 us per term with the copy, 1487
// without).  Held to 32 registers for 8 blocks per SM (with 40, 6 blocks per
// SM: 1734 us); the conservative instance keeps one 4-byte value on the
// stack, outside any loop.
template <int OP>
__global__ void __launch_bounds__(kThreads, 8)
batch_term_f64_kernel(const BatchTerm<double>* __restrict__ d, int count) {
    const unsigned tile = blockIdx.x;
    const BatchTerm<double>& sd = d[find_desc(d, count, (long long)tile)];
    // a grid's tiles number fewer than 2^31 (n < 2^31): 32-bit division
    const unsigned lt = tile - (unsigned)sd.tile_begin;
    const unsigned tiles_x = ((unsigned)sd.G.nx + kBlockX - 1) / kBlockX;
    const unsigned tiles_y = ((unsigned)sd.G.ny + kBlockY - 1) / kBlockY;
    const unsigned rest = lt / tiles_x;
    const int i = (int)(lt - rest * tiles_x) * kBlockX + threadIdx.x;
    const unsigned kk = rest / tiles_y;
    const int j = (int)(rest - kk * tiles_y) * kBlockY + threadIdx.y;
    const int k = (int)kk;
    if (i >= sd.G.nx || j >= sd.G.ny) return;
    term_point_f64<OP>(sd.G, sd.W, sd.a, i, j, k, zero_row_of(sd.G, sd.W.zrow, i, j, k));
}

// Blocks loop over tiles of TZ planes (grid = resident capacity).
template <int OP, typename T, int TZ>
__global__ void __launch_bounds__(kThreads)
batch_term_kernel(const BatchTerm<T>* __restrict__ d, int count, long long tiles) {
    __shared__ BatchTerm<T> sd;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int di = find_desc(d, count, tile);
        __syncthreads();
        copy_desc(sd, d + di);
        __syncthreads();
        const long long lt = tile - sd.tile_begin;
        const int tiles_x = (sd.G.nx + kBlockX - 1) / kBlockX;
        const int tiles_y = (sd.G.ny + kBlockY - 1) / kBlockY;
        const int i = (int)(lt % tiles_x) * kBlockX + threadIdx.x;
        const long long rest = lt / tiles_x;
        const int j = (int)(rest % tiles_y) * kBlockY + threadIdx.y;
        const int tz = (int)(rest / tiles_y);
        if (i < sd.G.nx && j < sd.G.ny) term_column<OP, T, TZ>(sd.G, sd.W, sd.a, i, j, tz);
    }
}

__global__ void __launch_bounds__(kStatsThreads) batch_stats_kernel(const BatchStats* __restrict__ d) {
    __shared__ BatchStats sd;
    const int di = blockIdx.x / kStatsBlocks;
    const int tid = threadIdx.x;
    const int* s = reinterpret_cast<const int*>(d + di);
    int* t = reinterpret_cast<int*>(&sd);
    for (int w = tid; w < (int)(sizeof(BatchStats) / 4); w += kStatsThreads) t[w] = s[w];
    __syncthreads();
    stats_body(sd.n, sd.u, sd.sink, blockIdx.x % kStatsBlocks);
}

template <int OP, typename T, int TZ>
int batch_blocks_per_sm() {
    static int cached = 0;
    if (!cached) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_term_kernel<OP, T, TZ>, kThreads, 0) !=
                cudaSuccess ||
            b < 1)
            b = 1;
        cached = b;
    }
    return cached;
}

// Resident blocks per SM of a term-kernel instantiation (looked up once).
// z-planes per thread: the FP64 kernel is bound by the FP64 pipe and runs best
// at full occupancy with one plane per thread (32 registers); the memory-bound
// FP32 kernel gains from marching over 4 planes.
template <typename T>
struct TermTile {
    static constexpr int kZ = std::is_same<T, double>::value ? 1 : kTileZ;
};

template <int OP, typename T>
int term_blocks_per_sm() {
    static int cached = 0;
    if (!cached) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, term_kernel<OP, T, TermTile<T>::kZ>, kThreads, 0) !=
                cudaSuccess ||
            b < 1)
            b = 1;
        cached = b;
    }
    return cached;
}

}  // namespace

cudaError_t launch_zero_rows(const Geom& G, et_operator op, const Weights<double>& W, unsigned char* zrow,
                             unsigned long long* count, cudaStream_t stream) {
    const dim3 block(kBlockX, kBlockY, 1);
    if (op == ET_OP_CONSERVATIVE)
        zero_rows_kernel<ET_OP_CONSERVATIVE><<<voxel_grid(G), block, 0, stream>>>(G, W, zrow, count);
    else
        zero_rows_kernel<ET_OP_LITERAL><<<voxel_grid(G), block, 0, stream>>>(G, W, zrow, count);
    return cudaGetLastError();
}

cudaError_t launch_coeffs(const Geom& G, const double* D, double inv_h2, et_operator op, double* const w[5],
                          unsigned long long* rmax_bits, unsigned* flags, cudaStream_t stream, double dscale) {
    const dim3 block(kBlockX, kBlockY, 1);
    if (op == ET_OP_CONSERVATIVE)
        coeffs_kernel<ET_OP_CONSERVATIVE><<<voxel_grid(G), block, 0, stream>>>(
            G, D, dscale, inv_h2, w[0], w[1], w[2], w[3], w[4], rmax_bits, flags);
    else
        coeffs_kernel<ET_OP_LITERAL><<<voxel_grid(G), block, 0, stream>>>(
            G, D, dscale, inv_h2, w[0], w[1], w[2], w[3], w[4], rmax_bits, flags);
    return cudaGetLastError();
}

template <typename T>
cudaError_t convert_weights_impl(const Geom& G, const double* const w[4], T* const wt[4], double scale,
                                 cudaStream_t stream) {
    const int threads = 256;
    long long blocks = (G.n + threads - 1) / threads;
    const long long cap = 16ll * (G.sms > 0 ? G.sms : 1);
    if (blocks > cap) blocks = cap;
    convert_weights_kernel<T><<<(unsigned)blocks, threads, 0, stream>>>(G.n, w[0], w[1], w[2], w[3], scale,
                                                                       wt[0], wt[1], wt[2], wt[3]);
    return cudaGetLastError();
}

cudaError_t launch_convert_weights(const Geom& G, const double* const w[4], float* const wf[4], double scale,
                                   cudaStream_t stream) {
    return convert_weights_impl<float>(G, w, wf, scale, stream);
}

cudaError_t launch_convert_weights(const Geom& G, const double* const w[4], float2* const wd[4], double scale,
                                   cudaStream_t stream) {
    return convert_weights_impl<float2>(G, w, wd, scale, stream);
}

template <typename T>
cudaError_t launch_residual(const Geom& G, et_operator op, const double* u, Weights<double> W, double rho,
                            double dt_shift, double dt_scale, et_scheme scheme, T* b, T* dt, unsigned* flags,
                            cudaStream_t stream, unsigned long long* wnorm) {
    const dim3 block(kBlockX, kBlockY, 1);
    if (op == ET_OP_CONSERVATIVE)
        return launch_pdl(residual_kernel<ET_OP_CONSERVATIVE, T>, voxel_grid(G), block, stream, G, u, W, rho, dt_shift,
                          dt_scale, (int)scheme, b, dt, flags, wnorm);
    return launch_pdl(residual_kernel<ET_OP_LITERAL, T>, voxel_grid(G), block, stream, G, u, W, rho, dt_shift,
                      dt_scale, (int)scheme, b, dt, flags, wnorm);
}

template <typename T>
cudaError_t launch_term(const Geom& G, et_operator op, Weights<T> W, const TermArgs<T>& a,
                        cudaStream_t stream) {
    const dim3 block(kBlockX, kBlockY, 1);
    if constexpr (std::is_same<T, double>::value) {
        if (op == ET_OP_CONSERVATIVE)
            return launch_pdl(term_kernel_f64<ET_OP_CONSERVATIVE>, voxel_grid(G), block, stream, G, W, a);
        return launch_pdl(term_kernel_f64<ET_OP_LITERAL>, voxel_grid(G), block, stream, G, W, a);
    }
    if constexpr (std::is_same<T, float>::value) {
        if (quad_eligible(G, W, a)) return launch_term_quad(G, op, W, a, stream);
    }
    constexpr int TZ = TermTile<T>::kZ;
    const long long tiles = (long long)((G.nx + kBlockX - 1) / kBlockX) * ((G.ny + kBlockY - 1) / kBlockY) *
                            ((G.nz + TZ - 1) / TZ);
    const int sms = G.sms > 0 ? G.sms : 1;
    if (op == ET_OP_CONSERVATIVE) {
        const long long cap = (long long)sms * term_blocks_per_sm<ET_OP_CONSERVATIVE, T>();
        term_kernel<ET_OP_CONSERVATIVE, T, TZ><<<(unsigned)(tiles < cap ? tiles : cap), block, 0, stream>>>(G, W, a);
    } else {
        const long long cap = (long long)sms * term_blocks_per_sm<ET_OP_LITERAL, T>();
        term_kernel<ET_OP_LITERAL, T, TZ><<<(unsigned)(tiles < cap ? tiles : cap), block, 0, stream>>>(G, W, a);
    }
    return cudaGetLastError();
}

cudaError_t prime_launch_limits() {
    term_blocks_per_sm<ET_OP_CONSERVATIVE, double>();
    term_blocks_per_sm<ET_OP_LITERAL, double>();
    term_blocks_per_sm<ET_OP_CONSERVATIVE, float>();
    term_blocks_per_sm<ET_OP_LITERAL, float>();
    prime_launch_limits_df64();
    prime_launch_limits_pair();
    prime_launch_limits_quad_pair();
    return cudaGetLastError();
}

int batch_variant_count(et_precision prec) { return prec == ET_F64 ? 3 : (prec == ET_F32 ? 4 : 2); }

BatchVariant batch_variant(et_precision prec, int v) {
    if (prec == ET_F64) {
        static const BatchVariant t[3] = {{1, 0}, {1, 1}, {2, 1}};
        return t[v];
    }
    if (prec == ET_F32) {
        static const BatchVariant t[4] = {{4, 1}, {2, 1}, {8, 1}, {1, 1}};
        return t[v];
    }
    static const BatchVariant t[2] = {{4, 1}, {2, 1}};
    return t[v];
}

template <int OP, typename T, int TZ>
cudaError_t launch_batch_persistent(const BatchTerm<T>* d, int count, long long tiles, int sms, cudaStream_t stream) {
    const long long cap = (long long)(sms > 0 ? sms : 1) * batch_blocks_per_sm<OP, T, TZ>();
    batch_term_kernel<OP, T, TZ><<<(unsigned)(tiles < cap ? tiles : cap), dim3(kBlockX, kBlockY, 1), 0, stream>>>(
        d, count, tiles);
    return cudaGetLastError();
}

template <int OP, typename T>
cudaError_t launch_batch_term_op(int variant, const BatchTerm<T>* d, int count, long long tiles, int sms,
                                 cudaStream_t stream) {
    const BatchVariant v = batch_variant(std::is_same<T, double>::value ? ET_F64 : ET_F32, variant);
    if (std::is_same<T, double>::value && !v.persistent) {
        if constexpr (std::is_same<T, double>::value)
            batch_term_f64_kernel<OP><<<(unsigned)tiles, dim3(kBlockX, kBlockY, 1), 0, stream>>>(d, count);
        return cudaGetLastError();
    }
    switch (v.tile_z) {
        case 1: return launch_batch_persistent<OP, T, 1>(d, count, tiles, sms, stream);
        case 2: return launch_batch_persistent<OP, T, 2>(d, count, tiles, sms, stream);
        case 4: return launch_batch_persistent<OP, T, 4>(d, count, tiles, sms, stream);
        default: return launch_batch_persistent<OP, T, 8>(d, count, tiles, sms, stream);
    }
}

template <typename T>
cudaError_t launch_batch_term(et_operator op, int variant, const BatchTerm<T>* d, int count, long long tiles, int sms,
                              cudaStream_t stream) {
    if (op == ET_OP_CONSERVATIVE) return launch_batch_term_op<ET_OP_CONSERVATIVE, T>(variant, d, count, tiles, sms, stream);
    return launch_batch_term_op<ET_OP_LITERAL, T>(variant, d, count, tiles, sms, stream);
}

template <typename T>
cudaError_t launch_batch_residual(et_operator op, int scheme, const BatchResidual<T>* d, int count, long long tiles,
                                  unsigned* flags, cudaStream_t stream) {
    if (op == ET_OP_CONSERVATIVE)
        batch_residual_kernel<ET_OP_CONSERVATIVE, T><<<(unsigned)tiles, dim3(kBlockX, kBlockY, 1), 0, stream>>>(
            d, count, scheme, flags);
    else
        batch_residual_kernel<ET_OP_LITERAL, T><<<(unsigned)tiles, dim3(kBlockX, kBlockY, 1), 0, stream>>>(
            d, count, scheme, flags);
    return cudaGetLastError();
}

cudaError_t launch_batch_stats(const BatchStats* d, int count, cudaStream_t stream) {
    batch_stats_kernel<<<(unsigned)(count * kStatsBlocks), kStatsThreads, 0, stream>>>(d);
    return cudaGetLastError();
}

template cudaError_t launch_batch_term<double>(et_operator, int, const BatchTerm<double>*, int, long long, int,
                                               cudaStream_t);
template cudaError_t launch_batch_term<float>(et_operator, int, const BatchTerm<float>*, int, long long, int,
                                              cudaStream_t);
template cudaError_t launch_batch_residual<double>(et_operator, int, const BatchResidual<double>*, int, long long,
                                                   unsigned*, cudaStream_t);
template cudaError_t launch_batch_residual<float>(et_operator, int, const BatchResidual<float>*, int, long long,
                                                  unsigned*, cudaStream_t);
template cudaError_t launch_batch_residual<float2>(et_operator, int, const BatchResidual<float2>*, int, long long,
                                                   unsigned*, cudaStream_t);

cudaError_t launch_stats(const Geom& G, const double* u, const StatsSink& sink, cudaStream_t stream) {
    return launch_pdl(stats_kernel, dim3(kStatsBlocks), dim3(kStatsThreads), stream, G.n, u, sink);
}

template cudaError_t launch_residual<double>(const Geom&, et_operator, const double*, Weights<double>,
                                             double, double, double, et_scheme, double*, double*, unsigned*,
                                             cudaStream_t, unsigned long long*);
template cudaError_t launch_term<double>(const Geom&, et_operator, Weights<double>,
                                         const TermArgs<double>&, cudaStream_t);
template cudaError_t launch_term<float>(const Geom&, et_operator, Weights<float>, const TermArgs<float>&,
                                        cudaStream_t);

}  // namespace et
