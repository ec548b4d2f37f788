// Crank-Nicolson steps (Sec. 2.3, the paper's comparison method) by
// matrix-free conjugate gradients, FP64.
//
// The printed scheme drops u^t and flips the sign of the implicit term; it is
// read as the trapezoidal rule on the linearised system of the exponential
// step, (I - tau/2 A_n) u^{n+1} = (I + tau/2 A_n) u^n + tau f_n.  Started from
// u^n, the initial residual of that system is tau (A_n u^n + f_n) = tau b_n,
// so each step solves
//     M delta = tau b_n,   M = I - tau/2 A_n,   u^{n+1} = u^n + delta,
// with b_n and the diagonal of A_n from the exponential step's residual
// launch.  For the conservative operator M is symmetric positive definite
// (tau rho < 2), and conjugate gradients from delta = 0 converge in about
// sqrt(cond M) log(1/rtol) / 2 iterations.
//
// One iteration is three launches that keep every scalar on the device:
//   apply:  q = M p with the FP64 face weights (one voxel per thread, 32 x 8
//           tiles) and the partials of p.q; the last block forms alpha;
//   update: delta += alpha p, r -= alpha q and the partials of r.r (fixed grid);
//           the last block forms beta, counts the iteration and sets the done
//           flag once ||r|| <= rtol ||tau b_n||;
//   direction: p = r + beta p.
// Every launch returns at once when the done flag is set, so a run captured
// with a fixed iteration cap costs only empty launches past convergence.
// Reductions take fixed partials in a fixed order: the results do not depend
// on scheduling.
#include <cuda_runtime.h>

#include "et_cn.h"
#include "et_internal.h"

namespace et {
namespace {

constexpr int kCnThreads = 256;  // grid-stride kernels: kStatsBlocks blocks

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < nw; ++w) s += red[w];
    return s;  // valid on thread 0
}

// The last of nblocks blocks to arrive (one ticket per block) sums the
// partials in index order; returns true on that block's thread 0.
__device__ __forceinline__ bool last_block_sum(double mine, double* partial, unsigned nblocks, unsigned* ticket,
                                               double* total, double* red) {
    __shared__ bool is_last;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tid == 0) {
        partial[blk] = mine;
        __threadfence();
        is_last = atomicAdd(ticket, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double s = 0.0;
    const int nt = blockDim.x * blockDim.y;
    for (unsigned q = tid; q < nblocks; q += nt) s += __ldcg(&partial[q]);
    s = block_sum(s, red);
    if (tid == 0) {
        *total = s;
        *ticket = 0u;
    }
    return tid == 0;
}

__global__ void __launch_bounds__(kCnThreads) cn_init_kernel(long long n, double tau, double* __restrict__ r,
                                                             double* __restrict__ p, double* __restrict__ delta,
                                                             CnScalars* sc, double* partial, unsigned* ticket) {
    pdl_begin();
    __shared__ double red[32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)kCnThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kCnThreads) {
        const double v = tau * r[i];  // r holds b_n on entry
        r[i] = v;
        p[i] = v;
        delta[i] = 0.0;
        acc = fma(v, v, acc);
    }
    const double s = block_sum(acc, red);
    double total = 0.0;
    if (last_block_sum(s, partial, gridDim.x, ticket, &total, red)) {
        sc->rr = total;
        sc->rr0 = total;
        sc->iters = 0;
        sc->done = total > 0.0 ? 0 : 1;
    }
}

// q = M p = p - tau/2 (a_pp p + sum_e w_e p_e) with the conservative face
// weights (the -e weight is the neighbour's +e weight); partials of p.q.
__global__ void __launch_bounds__(kThreads) cn_apply_kernel(Geom G, const double* __restrict__ w0,
                                                            const double* __restrict__ w1,
                                                            const double* __restrict__ w2,
                                                            const double* __restrict__ diag, double half_tau,
                                                            const double* __restrict__ p, double* __restrict__ q,
                                                            CnScalars* sc, double* partial, unsigned* ticket) {
    pdl_begin();
    if (sc->done) return;
    __shared__ double red[32];
    const int i = blockIdx.x * kBlockX + threadIdx.x;
    const int j = blockIdx.y * kBlockY + threadIdx.y;
    const int k = blockIdx.z;
    double dot = 0.0;
    if (i < G.nx && j < G.ny) {
        const long long c = i + G.sy * j + G.sz * k;
        const double pc = p[c];
        double a = diag[c] * pc;
        if (i + 1 < G.nx) a = fma(w0[c], p[c + 1], a);
        if (i > 0) a = fma(w0[c - 1], p[c - 1], a);
        if (j + 1 < G.ny) a = fma(w1[c], p[c + G.sy], a);
        if (j > 0) a = fma(w1[c - G.sy], p[c - G.sy], a);
        if (k + 1 < G.nz) a = fma(w2[c], p[c + G.sz], a);
        if (k > 0) a = fma(w2[c - G.sz], p[c - G.sz], a);
        const double qv = fma(-half_tau, a, pc);
        q[c] = qv;
        dot = pc * qv;
    }
    const double s = block_sum(dot, red);
    double total = 0.0;
    if (last_block_sum(s, partial, gridDim.x * gridDim.y * gridDim.z, ticket, &total, red)) {
        sc->pq = total;
        sc->alpha = total > 0.0 ? sc->rr / total : 0.0;
    }
}

__global__ void __launch_bounds__(kCnThreads) cn_update_kernel(long long n, const double* __restrict__ p,
                                                               const double* __restrict__ q, double* __restrict__ r,
                                                               double* __restrict__ delta, double rtol2,
                                                               CnScalars* sc, double* partial, unsigned* ticket) {
    pdl_begin();
    if (sc->done) return;
    __shared__ double red[32];
    const double alpha = sc->alpha;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)kCnThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kCnThreads) {
        delta[i] = fma(alpha, p[i], delta[i]);
        const double rv = fma(-alpha, q[i], r[i]);
        r[i] = rv;
        acc = fma(rv, rv, acc);
    }
    const double s = block_sum(acc, red);
    double total = 0.0;
    if (last_block_sum(s, partial, gridDim.x, ticket, &total, red)) {
        sc->beta = sc->rr > 0.0 ? total / sc->rr : 0.0;
        sc->rr = total;
        sc->iters += 1;
        if (!(total > rtol2 * sc->rr0)) sc->done = 1;
    }
}

__global__ void __launch_bounds__(kCnThreads) cn_direction_kernel(long long n, const double* __restrict__ r,
                                                                  double* __restrict__ p, const CnScalars* sc) {
    pdl_begin();
    if (sc->done) return;
    const double beta = sc->beta;
    for (long long i = blockIdx.x * (long long)kCnThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kCnThreads)
        p[i] = fma(beta, p[i], r[i]);
}

// u += delta; a solve that stopped at the cap raises ET_FLAG_CG_CAP.
__global__ void __launch_bounds__(kCnThreads) cn_finish_kernel(long long n, const double* __restrict__ delta,
                                                               double* __restrict__ u, const CnScalars* sc,
                                                               unsigned* flags) {
    pdl_begin();
    for (long long i = blockIdx.x * (long long)kCnThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kCnThreads)
        u[i] += delta[i];
    if (blockIdx.x == 0 && threadIdx.x == 0 && !sc->done) atomicOr(flags, ET_FLAG_CG_CAP);
}

}  // namespace

cudaError_t launch_cn_init(long long n, double tau, double* r, double* p, double* delta, CnScalars* sc,
                           double* partial, unsigned* ticket, cudaStream_t st) {
    return launch_pdl(cn_init_kernel, dim3(kStatsBlocks), dim3(kCnThreads), st, n, tau, r, p, delta, sc, partial,
                      ticket);
}

cudaError_t launch_cn_iteration(const Geom& G, const double* const w[3], const double* diag, double tau,
                                double rtol, double* r, double* p, double* q, double* delta, CnScalars* sc,
                                double* bpartial, double* partial, unsigned* ticket, cudaStream_t st) {
    const dim3 grid((G.nx + kBlockX - 1) / kBlockX, (G.ny + kBlockY - 1) / kBlockY, G.nz);
    cudaError_t e = launch_pdl(cn_apply_kernel, grid, dim3(kBlockX, kBlockY, 1), st, G, w[0], w[1], w[2], diag,
                               0.5 * tau, (const double*)p, q, sc, bpartial, ticket);
    if (e != cudaSuccess) return e;
    e = launch_pdl(cn_update_kernel, dim3(kStatsBlocks), dim3(kCnThreads), st, G.n, (const double*)p,
                   (const double*)q, r, delta, rtol * rtol, sc, partial, ticket);
    if (e != cudaSuccess) return e;
    return launch_pdl(cn_direction_kernel, dim3(kStatsBlocks), dim3(kCnThreads), st, G.n, (const double*)r, p,
                      (const CnScalars*)sc);
}

cudaError_t launch_cn_finish(long long n, const double* delta, double* u, const CnScalars* sc, unsigned* flags,
                             cudaStream_t st) {
    return launch_pdl(cn_finish_kernel, dim3(kStatsBlocks), dim3(kCnThreads), st, n, delta, u, sc, flags);
}

}  // namespace et
