// The launches of one step's Taylor chain on one grid's buffers (host side),
// shared by the single-grid driver (et_api.cu) and the batched form
// (et_batch_api.cu).
#pragma once

#include <cstddef>
#include <vector>

#include "et_internal.h"
#include "et_plan.h"

namespace et {

// One launch: a single Taylor term, or two consecutive terms of a sub-step
// for the pair kernel (et_fused.cu; a2 is used only then).
template <typename T>
struct ChainOp {
    bool pair;
    TermArgs<T> a1, a2;
};

// Buffers: b (also z_0 of sub-step 0), dt (diagonal), Y[2] (sub-step sums,
// ping-pong), Z[2] (terms, ping-pong); u receives the finished step.  With
// pairs, two consecutive terms of one sub-step share a launch; the first
// term's outputs are then not written and the term buffers alternate per
// launch.
template <typename T>
std::vector<ChainOp<T>> chain_ops(const ChainPlan& P, int s, const T* b, const T* dt, T* const Y[2], T* const Z[2],
                                  double* u, bool pairs) {
    std::vector<ChainOp<T>> ops;
    ops.reserve(P.terms.size());
    int zi = 0;  // next z buffer to write
    const T* zin = nullptr;
    auto args_of = [&](const PlannedTerm& t) {
        const int k = t.k, j = t.j;
        if (k == 0 && j == 1) zin = b;
        if (k > 0 && j == 0) zin = Y[k & 1];
        TermArgs<T> a;
        a.zin = zin;
        a.b = b;
        a.beta = Scalar<T>::make(t.beta);
        a.has_beta = t.beta != 0.0;
        a.zscale = Scalar<T>::make(t.zscale_val);
        a.has_zscale = t.zscale_on;
        a.dt = dt;
        a.g = Scalar<T>::make(t.gnext);
        a.gamma = Scalar<T>::make(t.last ? P.gamma * (t.horner ? t.gnext : 1.0) : 1.0);
        a.base_scale = Scalar<T>::make(t.base_scale);
        a.base_mode = t.base_mode;
        a.last = t.last;
        a.horner = t.horner;
        a.yacc = Y[(k + 1) & 1];
        a.u = (t.last && k == s - 1) ? u : nullptr;
        a.zout = t.last ? nullptr : Z[zi];
        return a;
    };
    for (size_t ti = 0; ti < P.terms.size(); ++ti) {
        const PlannedTerm& t = P.terms[ti];
        ChainOp<T> op;
        if (pairs && !t.last && ti + 1 < P.terms.size() && P.terms[ti + 1].k == t.k) {
            op.pair = true;
            op.a1 = args_of(t);  // its outputs stay on chip
            op.a1.zout = nullptr;
            op.a2 = args_of(P.terms[ti + 1]);
            ++ti;
            if (!op.a2.last) {
                zin = op.a2.zout;
                zi ^= 1;
            }
        } else {
            op.pair = false;
            op.a1 = args_of(t);
            op.a2 = op.a1;
            if (!t.last) {
                zin = op.a1.zout;
                zi ^= 1;
            }
        }
        ops.push_back(op);
    }
    return ops;
}

}  // namespace et
