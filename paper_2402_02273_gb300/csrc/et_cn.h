// Crank-Nicolson steps by conjugate gradients on the device (et_cn.cu).  Not
// part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include "et_internal.h"

namespace et {

// Scalars of one conjugate-gradient solve, kept in device memory.
struct CnScalars {
    double rr, rr0, pq, alpha, beta;
    int iters, done;
};

// r = tau r (r holds b_n on entry), p = r, delta = 0, rr = rr0 = r.r.
cudaError_t launch_cn_init(long long n, double tau, double* r, double* p, double* delta, CnScalars* sc,
                           double* partial, unsigned* ticket, cudaStream_t st);
// One iteration (apply, update, direction).  w: the FP64 +x, +y, +z face
// weights; diag: the diagonal of A_n; bpartial: one double per 32 x 8 tile of
// the grid; partial: kStatsBlocks doubles.
cudaError_t launch_cn_iteration(const Geom& G, const double* const w[3], const double* diag, double tau,
                                double rtol, double* r, double* p, double* q, double* delta, CnScalars* sc,
                                double* bpartial, double* partial, unsigned* ticket, cudaStream_t st);
// u += delta, ET_FLAG_CG_CAP if the solve did not converge.
cudaError_t launch_cn_finish(long long n, const double* delta, double* u, const CnScalars* sc, unsigned* flags,
                             cudaStream_t st);

}  // namespace et
