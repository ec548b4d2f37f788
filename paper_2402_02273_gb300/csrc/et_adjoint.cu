// Adjoint (reverse-mode) kernels of the exponential-integrator step for sm_103a.
//
// Forward recurrence of one sub-step (et_kernels.cu, generic form with the
// normalisation nu = 1 for FP64):  with A^ = (A - mu I) / nu,
//     zeta_{j+1} = f_j A^ zeta_j + beta_j b,   S = base + sum_j g_j zeta_j,
//     y_{k+1} = gamma S,
// where f_j is 1 except on the first launched term of sub-step 0 (1/nu).  Its
// reverse, for a cotangent ybar_{k+1} and Sbar = gamma ybar_{k+1}, runs j
// downwards with w = zetabar_{j+1}:
//     zetabar_j = g_j Sbar + f_j A^T w,    bbar += beta_j w,
//     cbar_p   += f_j / nu * w_p x_p,      sbar_p += f_j / nu * (L^T w)_p x_p,
// x being the forward input of that term (zeta_j, y_k, or b).  cbar is the
// cotangent of the diagonal rho(1 - 2u^n) and sbar that of a uniform scale s
// of D (D -> s D), both per voxel; a step's sbar terms are summed in the value
// type and added to the FP64 total by the step kernel, reduced at the end.  Per step,
//     ubar^n = ubar^{n+1} + L^T bbar + rho (1 - 2u) bbar - 2 rho cbar,
//     rho-gradient += u(1-u) bbar + (1 - 2u) cbar,   s-gradient += bbar (L u),
// from b = L u + rho u (1-u) and c = rho (1 - 2u) (exponential Euler: no c).
//
// Transposes: the conservative operator is symmetric.  The literal one has
// row p with weight (D_p + D_{p+e}) towards +e and 2 D_p towards -e, so its
// transpose takes w_{p+e} with weight 2 D_{p+e} = w3[p+e] and w_{p-e} with
// weight D_{p-e} + D_p = w_e[p-e]; the diagonal is the same.
#include <cuda_runtime.h>

#include <cfloat>

#include "et_df64_arith.h"
#include "et_internal.h"

namespace et {
namespace {

// (A^T v)_p without the diagonal, from the (typed, 1/nu-scaled) weights.
template <int OP, typename T>
__device__ __forceinline__ T offdiag_transpose(const Weights<T>& W, const T* __restrict__ v, const Geom& G,
                                               int i, int j, int k, long long p) {
    T acc = T(0);
    const long long st[3] = {1, G.sy, G.sz};
    const int c[3] = {i, j, k};
    const int ext[3] = {G.nx, G.ny, G.nz};
    for (int a = 0; a < 3; ++a) {
        const bool has_plus = c[a] + 1 < ext[a];
        const bool has_minus = c[a] > 0;
        if (OP == ET_OP_CONSERVATIVE) {
            if (has_plus) acc = fma(W.w[a][p], v[p + st[a]], acc);
            if (has_minus) acc = fma(W.w[a][p - st[a]], v[p - st[a]], acc);
        } else {
            if (has_plus) acc = fma(W.w[3][p + st[a]], v[p + st[a]], acc);
            if (has_minus) acc = fma(W.w[a][p - st[a]], v[p - st[a]], acc);
        }
    }
    return acc;
}

template <int OP, typename T>
__global__ void __launch_bounds__(kThreads)
adj_term_kernel(Geom G, Weights<T> W, AdjTermArgs<T> a) {
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= G.nx || j >= G.ny) return;
    const long long p = i + G.sy * j + G.sz * k;
    // w = wscale * wsrc (wsrc = ybar_{k+1} on the first reverse term of a sub-step)
    const T wp = a.wscale * a.wsrc[p];
    // A conservative operator is symmetric: a row without off-diagonal entries
    // (W.zrow) is a column without them, and its transpose sum is the +0 that
    // offdiag_transpose forms from zero weights (the sum starts at +0 and every
    // product with a zero weight adds a zero to it).
    const bool skip = OP == ET_OP_CONSERVATIVE && zero_row_of(G, W.zrow, i, j, k);
    const T off = a.wscale * (skip ? T(0) : offdiag_transpose<OP, T>(W, a.wsrc, G, i, j, k, p));
    const T dtp = a.dt[p];
    const T atw = fma(dtp, wp, off);                     // A^T w
    const T sbar = a.gamma * a.ybar_next[p];             // Sbar
    const T out = fma(a.g, sbar, a.f * atw);             // g Sbar + f A^T w
    const T x = a.x[p];
    // L^T w / nu = off + (w4 / nu) w, with w4 = minus the row sum of L
    const T ltw = fma(a.negR[p], wp, off);
    // d A^/d c_p = e_p e_p^T / nu;  d A^/d s = L / nu (ltw already carries the 1/nu)
    a.cbar[p] = fma(a.f * a.inv_nu * wp, x, a.cbar[p]);
    a.sstep[p] = fma(a.f * ltw, x, a.sstep[p]);
    T bb = a.bbar[p];
    if (a.has_beta) bb = fma(a.beta, wp, bb);
    if (a.out_to_bbar) {
        bb += out;
    } else {
        a.zbar_out[p] = out;
    }
    a.bbar[p] = bb;
}

template <int OP, typename T>
__global__ void __launch_bounds__(kThreads)
adj_step_kernel(Geom G, Weights<double> W, const double* __restrict__ u, const T* __restrict__ bbar,
                const T* __restrict__ cbar, const T* __restrict__ sstep, const double* __restrict__ ubar_next,
                double rho, int scheme, double* __restrict__ ubar, double* __restrict__ sbar_acc,
                double* __restrict__ rbar_acc) {
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= G.nx || j >= G.ny) return;
    const long long p = i + G.sy * j + G.sz * k;
    const long long st[3] = {1, G.sy, G.sz};
    const int c[3] = {i, j, k};
    const int ext[3] = {G.nx, G.ny, G.nz};
    const double up = u[p];
    const double bp = (double)bbar[p];
    const double negR = W.w[4][p];
    // L^T bbar and L u
    double ltb = negR * bp, lu = negR * up;
    for (int a = 0; a < 3; ++a) {
        const bool has_plus = c[a] + 1 < ext[a];
        const bool has_minus = c[a] > 0;
        if (has_plus) {
            const double wt = (OP == ET_OP_CONSERVATIVE) ? W.w[a][p] : W.w[3][p + st[a]];
            ltb = fma(wt, (double)bbar[p + st[a]], ltb);
            lu = fma(W.w[a][p], u[p + st[a]], lu);
        }
        if (has_minus) {
            const double wt = W.w[a][p - st[a]];
            ltb = fma(wt, (double)bbar[p - st[a]], ltb);
            const double wm = (OP == ET_OP_CONSERVATIVE) ? W.w[a][p - st[a]] : W.w[3][p];
            lu = fma(wm, u[p - st[a]], lu);
        }
    }
    double ub = ubar_next[p] + ltb + rho * (1.0 - 2.0 * up) * bp;
    double rb = up * (1.0 - up) * bp;
    if (scheme == ET_SCHEME_ROSENBROCK) {
        const double cp = (double)cbar[p];
        ub -= 2.0 * rho * cp;
        rb += (1.0 - 2.0 * up) * cp;
    }
    ubar[p] = ub;
    rbar_acc[p] += rb;
    sbar_acc[p] += (double)sstep[p];
    sbar_acc[p] += bp * lu;
}

// Deterministic sum of a vector into *out (fixed grid, fixed order).
constexpr int kSumBlocks = 1024;
constexpr int kSumThreads = 256;

__global__ void __launch_bounds__(kSumThreads) sum_partials_kernel(long long n, const double* __restrict__ v,
                                                                   double* __restrict__ partial) {
    __shared__ double sh[kSumThreads / 32];
    double s = 0.0;
    for (long long p = blockIdx.x * (long long)kSumThreads + threadIdx.x; p < n;
         p += (long long)kSumBlocks * kSumThreads)
        s += v[p];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kSumThreads / 32; ++w) s += sh[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(32) sum_final_kernel(const double* __restrict__ partial, double* __restrict__ out) {
    double s = 0.0;
    for (int q = threadIdx.x; q < kSumBlocks; q += 32) s += partial[q];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) *out = s;
}

__global__ void cast_kernel(long long n, const double* __restrict__ src, double scale, float* __restrict__ dst) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        dst[p] = (float)(src[p] * scale);
}

__global__ void split_kernel(long long n, const double* __restrict__ src, double scale, float2* __restrict__ dst) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        dst[p] = df64::from_double(__dmul_rn(src[p], scale));
    }
}

template <typename T>
__global__ void add_widen_kernel(long long n, const double* __restrict__ u, const T* __restrict__ y,
                                 double* __restrict__ out) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        out[p] = u[p] + (double)y[p];
}

dim3 voxel_grid3(const Geom& G) {
    return dim3((G.nx + kBlockX - 1) / kBlockX, (G.ny + kBlockY - 1) / kBlockY, G.nz);
}

}  // namespace

size_t sum_partials_bytes() { return sizeof(double) * kSumBlocks; }

template <typename T>
cudaError_t launch_add_widen(long long n, const double* u, const T* y, double* out, cudaStream_t stream) {
    add_widen_kernel<T><<<1024, 256, 0, stream>>>(n, u, y, out);
    return cudaGetLastError();
}
template cudaError_t launch_add_widen<double>(long long, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_add_widen<float>(long long, const double*, const float*, double*, cudaStream_t);

cudaError_t launch_split(long long n, const double* src, double scale, float2* dst, cudaStream_t stream) {
    split_kernel<<<1024, 256, 0, stream>>>(n, src, scale, dst);
    return cudaGetLastError();
}

cudaError_t launch_cast(long long n, const double* src, double scale, float* dst, cudaStream_t stream) {
    cast_kernel<<<1024, 256, 0, stream>>>(n, src, scale, dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_term(const Geom& G, et_operator op, Weights<T> W, const AdjTermArgs<T>& a,
                            cudaStream_t stream) {
    const dim3 block(kBlockX, kBlockY, 1);
    if (op == ET_OP_CONSERVATIVE)
        adj_term_kernel<ET_OP_CONSERVATIVE, T><<<voxel_grid3(G), block, 0, stream>>>(G, W, a);
    else
        adj_term_kernel<ET_OP_LITERAL, T><<<voxel_grid3(G), block, 0, stream>>>(G, W, a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_step(const Geom& G, et_operator op, Weights<double> W, const double* u, const T* bbar,
                            const T* cbar, const T* sstep, const double* ubar_next, double rho, et_scheme scheme,
                            double* ubar, double* sbar_acc, double* rbar_acc, cudaStream_t stream) {
    const dim3 block(kBlockX, kBlockY, 1);
    if (op == ET_OP_CONSERVATIVE)
        adj_step_kernel<ET_OP_CONSERVATIVE, T><<<voxel_grid3(G), block, 0, stream>>>(
            G, W, u, bbar, cbar, sstep, ubar_next, rho, (int)scheme, ubar, sbar_acc, rbar_acc);
    else
        adj_step_kernel<ET_OP_LITERAL, T><<<voxel_grid3(G), block, 0, stream>>>(
            G, W, u, bbar, cbar, sstep, ubar_next, rho, (int)scheme, ubar, sbar_acc, rbar_acc);
    return cudaGetLastError();
}

cudaError_t launch_sum(long long n, const double* v, double* partial, double* out, cudaStream_t stream) {
    sum_partials_kernel<<<kSumBlocks, kSumThreads, 0, stream>>>(n, v, partial);
    sum_final_kernel<<<1, 32, 0, stream>>>(partial, out);
    return cudaGetLastError();
}

template cudaError_t launch_adj_term<double>(const Geom&, et_operator, Weights<double>, const AdjTermArgs<double>&,
                                             cudaStream_t);
template cudaError_t launch_adj_term<float>(const Geom&, et_operator, Weights<float>, const AdjTermArgs<float>&,
                                            cudaStream_t);
template cudaError_t launch_adj_step<double>(const Geom&, et_operator, Weights<double>, const double*,
                                             const double*, const double*, const double*, const double*, double,
                                             et_scheme, double*, double*, double*, cudaStream_t);
template cudaError_t launch_adj_step<float>(const Geom&, et_operator, Weights<double>, const double*, const float*,
                                            const float*, const float*, const double*, double, et_scheme, double*,
                                            double*, double*, cudaStream_t);

}  // namespace et
