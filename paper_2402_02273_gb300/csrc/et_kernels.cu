// CUDA kernels of the exponential-integrator step (arXiv 2402.02273, Sec. 2.1-2.2)
// for sm_103a.
//
// Three kernels make a step:
//   coeffs   (once per et_set_coeffs): face weights of L and the row-sum bound;
//   residual (once per step): b = L u^n + rho u^n (1 - u^n) (= A_n u^n + f(u^n),
//            eq. F / newF) and the diagonal of A_n - mu I;
//   term     (s*m - 1 per step): one term of the scaled Taylor recurrence of
//            exp(h (B - mu I)) applied to the augmented vector, see below.
//
// Scaled recurrence.  With h = tau / s, A~ = A - mu I and the augmented scalar
// a_k of sub-step k (a_0 = 1), the j-th Taylor term of exp(h(B - mu I)) [y; a]
// is g_j z^_j with g_j = h^j / j! and
//     z^_0 = y,   z^_{j+1} = A~ z^_j + a_k (-mu)^j b,
// so a term costs one stencil application plus two fused multiply-adds and
// needs no per-term rescaling.  The sub-step result is
//     y <- e^{mu h} (y + sum_{j=1..m} g_j z^_j),
// and on the last sub-step u^{n+1} = u^n + y is written directly.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "et_internal.h"

namespace et {
namespace {

__device__ __forceinline__ double harmonic_mean(double a, double b) {
    return (a > 0.0 && b > 0.0) ? 2.0 * a * b / (a + b) : 0.0;
}

__device__ __forceinline__ unsigned linear_block() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// ---------------------------------------------------------------------------
// coeffs: face weights and max_p sum_{q != p} |L_pq|.
template <int OP>
__global__ void __launch_bounds__(kThreads)
coeffs_kernel(Geom G, const double* __restrict__ D, double inv_h2, double* __restrict__ w0,
              double* __restrict__ w1, double* __restrict__ w2, double* __restrict__ w3,
              unsigned long long* rmax_bits, unsigned* flags) {
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int k = blockIdx.z;
    double rowsum = 0.0;
    if (i < G.nx && j < G.ny) {
        const long long p = i + G.sy * j + G.sz * k;
        const double Dp = D[p];
        if (!(Dp >= 0.0) || !isfinite(Dp)) atomicOr(flags, ET_FLAG_D_INVALID);
        const int c[3] = {i, j, k};
        const int ext[3] = {G.nx, G.ny, G.nz};
        const long long st[3] = {1, G.sy, G.sz};
        double wp[3];
        for (int a = 0; a < 3; ++a) {
            const bool has_plus = c[a] + 1 < ext[a];
            const bool has_minus = c[a] > 0;
            const double Dq = has_plus ? D[p + st[a]] : 0.0;
            const double Dm = has_minus ? D[p - st[a]] : 0.0;
            double wplus, wminus;
            if (OP == ET_OP_CONSERVATIVE) {
                wplus = has_plus ? harmonic_mean(Dp, Dq) * inv_h2 : 0.0;
                wminus = has_minus ? harmonic_mean(Dm, Dp) * inv_h2 : 0.0;
            } else {
                wplus = has_plus ? (Dp + Dq) * inv_h2 : 0.0;
                wminus = has_minus ? 2.0 * Dp * inv_h2 : 0.0;
            }
            wp[a] = wplus;
            rowsum += fabs(wplus) + fabs(wminus);
        }
        w0[p] = wp[0];
        w1[p] = wp[1];
        w2[p] = wp[2];
        if (OP == ET_OP_LITERAL) w3[p] = 2.0 * Dp * inv_h2;
    }
    // block maximum, then one atomic per block on the (monotone) bit pattern
    __shared__ double smax[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) rowsum = fmax(rowsum, __shfl_down_sync(0xffffffffu, rowsum, off));
    const int tid = threadIdx.x + kBlockX * threadIdx.y;
    if ((tid & 31) == 0) smax[tid >> 5] = rowsum;
    __syncthreads();
    if (tid == 0) {
        double m = smax[0];
        for (int w = 1; w < kThreads / 32; ++w) m = fmax(m, smax[w]);
        if (isfinite(m)) atomicMax(rmax_bits, (unsigned long long)__double_as_longlong(m));
    }
}

__global__ void convert_weights_kernel(long long n, const double* __restrict__ a0,
                                       const double* __restrict__ a1, const double* __restrict__ a2,
                                       const double* __restrict__ a3, float* __restrict__ f0,
                                       float* __restrict__ f1, float* __restrict__ f2,
                                       float* __restrict__ f3) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        f0[p] = (float)a0[p];
        f1[p] = (float)a1[p];
        f2[p] = (float)a2[p];
        if (a3) f3[p] = (float)a3[p];
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
// residual: b = L u + rho u (1 - u), diag = c - R - mu (c = rho(1-2u) or 0).
template <int OP, typename T>
__global__ void __launch_bounds__(kThreads)
residual_kernel(Geom G, const double* __restrict__ u, Weights<double> W, double rho, double mu,
                int scheme, T* __restrict__ b, T* __restrict__ dt, unsigned* flags) {
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= G.nx || j >= G.ny) return;
    const long long p = i + G.sy * j + G.sz * k;
    const double up = u[p];
    const int c[3] = {i, j, k};
    const int ext[3] = {G.nx, G.ny, G.nz};
    const long long st[3] = {1, G.sy, G.sz};
    double Lu = 0.0, R = 0.0;
    for (int a = 0; a < 3; ++a) {
        const bool has_plus = c[a] + 1 < ext[a];
        const bool has_minus = c[a] > 0;
        const double wplus = W.w[a][p];
        const double wminus = minus_weight<OP, double>(W, a, p, st[a], has_minus);
        const double uplus = has_plus ? u[p + st[a]] : up;
        const double uminus = has_minus ? u[p - st[a]] : up;
        Lu += wplus * (uplus - up) + wminus * (uminus - up);
        R += wplus + wminus;
    }
    const double bp = Lu + rho * up * (1.0 - up);
    const double cp = (scheme == ET_SCHEME_ROSENBROCK) ? rho * (1.0 - 2.0 * up) : 0.0;
    b[p] = (T)bp;
    dt[p] = (T)(cp - R - mu);
    if (!isfinite(up)) atomicOr(flags, ET_FLAG_NONFINITE);
    if (scheme == ET_SCHEME_ROSENBROCK && (up < -kRangeSlack || up > 1.0 + kRangeSlack))
        atomicOr(flags, ET_FLAG_RANGE_IN);
}

// ---------------------------------------------------------------------------
// Block reduction of (min, max, sum) into per-block partials; the last block to
// finish reduces the partials in a fixed order (deterministic) and writes the
// step record.
__device__ void finish_stats(double vmin, double vmax, double vsum, const StatsSink& s) {
    __shared__ double sred[3][kThreads / 32];
    __shared__ bool is_last;
    const int tid = threadIdx.x + kBlockX * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5;
    for (int off = 16; off > 0; off >>= 1) {
        vmin = fmin(vmin, __shfl_down_sync(0xffffffffu, vmin, off));
        vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, off));
        vsum += __shfl_down_sync(0xffffffffu, vsum, off);
    }
    if (lane == 0) {
        sred[0][warp] = vmin;
        sred[1][warp] = vmax;
        sred[2][warp] = vsum;
    }
    __syncthreads();
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    if (tid == 0) {
        double a = sred[0][0], bmax = sred[1][0], c = sred[2][0];
        for (int w = 1; w < kThreads / 32; ++w) {
            a = fmin(a, sred[0][w]);
            bmax = fmax(bmax, sred[1][w]);
            c += sred[2][w];
        }
        const unsigned bid = linear_block();
        s.partial[3 * bid + 0] = a;
        s.partial[3 * bid + 1] = bmax;
        s.partial[3 * bid + 2] = c;
        __threadfence();
        const unsigned ticket = atomicAdd(s.ticket, 1u);
        is_last = (ticket == nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double lo = DBL_MAX, hi = -DBL_MAX, sum = 0.0;
    for (unsigned q = tid; q < nblocks; q += kThreads) {
        lo = fmin(lo, __ldcg(&s.partial[3 * q + 0]));
        hi = fmax(hi, __ldcg(&s.partial[3 * q + 1]));
        sum += __ldcg(&s.partial[3 * q + 2]);
    }
    for (int off = 16; off > 0; off >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, off));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, off));
        sum += __shfl_down_sync(0xffffffffu, sum, off);
    }
    __syncthreads();
    if (lane == 0) {
        sred[0][warp] = lo;
        sred[1][warp] = hi;
        sred[2][warp] = sum;
    }
    __syncthreads();
    if (tid == 0) {
        // thread 0 holds warp 0's result; add the other warps in order
        for (int w = 1; w < kThreads / 32; ++w) {
            lo = fmin(lo, sred[0][w]);
            hi = fmax(hi, sred[1][w]);
            sum += sred[2][w];
        }
        const unsigned step = *s.step_counter;
        et_step_info rec;
        rec.umin = lo;
        rec.umax = hi;
        rec.mass = sum;
        rec.s = s.s;
        rec.m = s.m;
        rec.flags = atomicOr(s.flags, 0u);
        rec.step = step;
        s.info[s.info_stride ? step : 0u] = rec;
        *s.last = rec;
        *s.step_counter = step + 1;
        *s.ticket = 0u;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// term: z^_{j+1} = A~ z^_j + beta b;  sum = base + g z^_{j+1};
// last term: sum *= gamma and either stored as the next y or added to u.
template <int OP, typename T, bool FINISH>
__global__ void __launch_bounds__(kThreads)
term_kernel(Geom G, Weights<T> W, TermArgs<T> a, StatsSink sink) {
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int k = blockIdx.z;
    double vmin = DBL_MAX, vmax = -DBL_MAX, vsum = 0.0;
    if (i < G.nx && j < G.ny) {
        const long long p = i + G.sy * j + G.sz * k;
        const T* __restrict__ z = a.zin;
        const T zc = z[p];
        T acc = a.dt[p] * zc;
        // +x / -x
        acc = fma(W.w[0][p], (i + 1 < G.nx) ? z[p + 1] : T(0), acc);
        acc = fma(minus_weight<OP, T>(W, 0, p, 1, i > 0), (i > 0) ? z[p - 1] : T(0), acc);
        // +y / -y
        acc = fma(W.w[1][p], (j + 1 < G.ny) ? z[p + G.sy] : T(0), acc);
        acc = fma(minus_weight<OP, T>(W, 1, p, G.sy, j > 0), (j > 0) ? z[p - G.sy] : T(0), acc);
        // +z / -z
        acc = fma(W.w[2][p], (k + 1 < G.nz) ? z[p + G.sz] : T(0), acc);
        acc = fma(minus_weight<OP, T>(W, 2, p, G.sz, k > 0), (k > 0) ? z[p - G.sz] : T(0), acc);
        if (a.beta != T(0)) acc = fma(a.beta, a.b[p], acc);
        T base;
        if (a.base_mode == 0) base = a.yacc[p];
        else if (a.base_mode == 1) base = a.base_scale * a.b[p];
        else base = zc;
        T sum = fma(a.g, acc, base);
        if (!a.last) {
            a.zout[p] = acc;
            a.yacc[p] = sum;
        } else {
            sum *= a.gamma;
            if (FINISH) {
                const double unew = a.u[p] + (double)sum;
                a.u[p] = unew;
                vmin = unew;
                vmax = unew;
                vsum = unew;
                if (!isfinite(unew)) atomicOr(sink.flags, ET_FLAG_NONFINITE);
            } else {
                a.yacc[p] = sum;
            }
        }
    }
    if (FINISH) finish_stats(vmin, vmax, vsum, sink);
}

dim3 stencil_grid(const Geom& G) {
    return dim3((G.nx + kBlockX - 1) / kBlockX, (G.ny + kBlockY - 1) / kBlockY, G.nz);
}

}  // namespace

cudaError_t launch_coeffs(const Geom& G, const double* D, double inv_h2, et_operator op, double* w0,
                          double* w1, double* w2, double* w3, unsigned long long* rmax_bits,
                          unsigned* flags, cudaStream_t stream) {
    const dim3 block(kBlockX, kBlockY, 1);
    if (op == ET_OP_CONSERVATIVE)
        coeffs_kernel<ET_OP_CONSERVATIVE><<<stencil_grid(G), block, 0, stream>>>(
            G, D, inv_h2, w0, w1, w2, w3, rmax_bits, flags);
    else
        coeffs_kernel<ET_OP_LITERAL><<<stencil_grid(G), block, 0, stream>>>(
            G, D, inv_h2, w0, w1, w2, w3, rmax_bits, flags);
    return cudaGetLastError();
}

cudaError_t launch_convert_weights(const Geom& G, const double* const w[4], float* const wf[4],
                                   cudaStream_t stream) {
    const int threads = 256;
    long long blocks = (G.n + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    convert_weights_kernel<<<(unsigned)blocks, threads, 0, stream>>>(G.n, w[0], w[1], w[2], w[3], wf[0],
                                                                    wf[1], wf[2], wf[3]);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const Geom& G, et_operator op, const double* u, Weights<double> W,
                            double rho, double mu, et_scheme scheme, T* b, T* dt, unsigned* flags,
                            cudaStream_t stream) {
    const dim3 block(kBlockX, kBlockY, 1);
    if (op == ET_OP_CONSERVATIVE)
        residual_kernel<ET_OP_CONSERVATIVE, T><<<stencil_grid(G), block, 0, stream>>>(
            G, u, W, rho, mu, (int)scheme, b, dt, flags);
    else
        residual_kernel<ET_OP_LITERAL, T><<<stencil_grid(G), block, 0, stream>>>(
            G, u, W, rho, mu, (int)scheme, b, dt, flags);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_term(const Geom& G, et_operator op, Weights<T> W, const TermArgs<T>& a,
                        const StatsSink& sink, cudaStream_t stream) {
    const dim3 block(kBlockX, kBlockY, 1);
    const dim3 grid = stencil_grid(G);
    const bool finish = a.last && a.u != nullptr;
    if (op == ET_OP_CONSERVATIVE) {
        if (finish)
            term_kernel<ET_OP_CONSERVATIVE, T, true><<<grid, block, 0, stream>>>(G, W, a, sink);
        else
            term_kernel<ET_OP_CONSERVATIVE, T, false><<<grid, block, 0, stream>>>(G, W, a, sink);
    } else {
        if (finish)
            term_kernel<ET_OP_LITERAL, T, true><<<grid, block, 0, stream>>>(G, W, a, sink);
        else
            term_kernel<ET_OP_LITERAL, T, false><<<grid, block, 0, stream>>>(G, W, a, sink);
    }
    return cudaGetLastError();
}

template cudaError_t launch_residual<double>(const Geom&, et_operator, const double*, Weights<double>,
                                             double, double, et_scheme, double*, double*, unsigned*,
                                             cudaStream_t);
template cudaError_t launch_residual<float>(const Geom&, et_operator, const double*, Weights<double>,
                                            double, double, et_scheme, float*, float*, unsigned*,
                                            cudaStream_t);
template cudaError_t launch_term<double>(const Geom&, et_operator, Weights<double>,
                                         const TermArgs<double>&, const StatsSink&, cudaStream_t);
template cudaError_t launch_term<float>(const Geom&, et_operator, Weights<float>,
                                        const TermArgs<float>&, const StatsSink&, cudaStream_t);

}  // namespace et
