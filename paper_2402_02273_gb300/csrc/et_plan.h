// Per-term scalars of one step's Taylor chain (shared by the single-grid and
// batched drivers and by the adjoint).  Not part of the public ABI.
#pragma once

#include <cmath>
#include <vector>

#include "et.h"

namespace et {

// One launched term of the chain, in forward order: it computes z_{j+1} of
// sub-step k from z_j (or from b / y_k on the first term of a sub-step).
struct PlannedTerm {
    int k, j;
    double beta;        // coefficient of b
    double gnext;       // weight of z_{j+1} in the sub-step sum
    double base_scale;  // base_mode 1: the first term's weight h on b
    int base_mode;      // 0: running sum; 1: h b; 2: y_k
    bool last;          // last term of its sub-step
    bool zscale_on;     // stencil part scaled by zscale_val (first term of sub-step 0)
    bool horner;        // a Horner step of sub-step 0
    double zscale_val;
};

struct ChainPlan {
    double gamma = 1.0;  // e^{mu h}
    double inv_nu = 1.0; // 1/nu (normalised forms) or 1
    std::vector<PlannedTerm> terms;
};

inline ChainPlan plan_chain(et_precision prec, double nu_form, int s, int m, double mu, double hstep) {
    ChainPlan P;
    const bool normalised = prec != ET_F64;
    const double nu = normalised ? nu_form : 1.0;
    const double hw = normalised ? hstep * nu : hstep;  // ratio of consecutive weights times (j+1)
    P.gamma = std::exp(mu * hstep);
    P.inv_nu = 1.0 / nu;
    double ak = 1.0;  // augmented scalar at the start of sub-step k
    for (int k = 0; k < s; ++k) {
        if (k == 0) {
            // Sub-step 0 starts from y_0 = 0, so its result is gamma P(A^) b with
            //   P(x) = sum_{j=1..m} g_j q_j(x),  q_1 = 1/nu,  q_{j+1}(x) = x q_j(x) + beta_j,
            // evaluated by Horner's rule: v = p_{m-1} b, v <- A^ v + p_i b (i = m-2..0).
            // FP64 uses the monic form (coefficients divided by p_{m-1}, folded into
            // the final factor); FP32 / DF64 keep p_{m-1} as a scale on the first
            // stencil so their vectors stay inside the FP32 range.
            std::vector<double> q(1, 1.0 / nu), pc(m, 0.0);
            double pw = 1.0;  // (-mu)^j
            double gj = 1.0;
            for (int j = 1; j <= m; ++j) {
                gj *= hw / j;
                for (size_t i = 0; i < q.size(); ++i) pc[i] += gj * q[i];
                if (j == m) break;
                pw *= -mu;
                const double beta = ak * pw / (normalised ? std::pow(nu, j + 1) : 1.0);
                q.insert(q.begin(), 0.0);  // x q_j
                q[0] += beta;
            }
            const double lead = pc[m - 1];
            for (int idx = 0; idx + 1 < m; ++idx) {
                const int i = m - 2 - idx;
                PlannedTerm t;
                t.k = 0;
                t.j = idx + 1;
                t.horner = true;
                t.beta = normalised ? pc[i] : pc[i] / lead;
                t.zscale_on = normalised && idx == 0;
                t.zscale_val = normalised ? lead : 1.0;
                t.last = (idx + 2 == m);
                t.gnext = t.last ? (normalised ? 1.0 : lead) : 0.0;  // final factor gamma * gnext
                t.base_scale = 0.0;
                t.base_mode = 0;
                P.terms.push_back(t);
            }
        } else {
            double pw = normalised ? 1.0 / nu : 1.0;  // (-mu)^j / nu^{j+1} (normalised) or (-mu)^j
            double gj = 1.0;                          // weight of term j
            for (int j = 0; j < m; ++j) {
                PlannedTerm t;
                t.k = k;
                t.j = j;
                t.horner = false;
                t.beta = ak * pw;
                t.gnext = gj * hw / (j + 1);
                t.base_scale = 0.0;
                t.base_mode = (j == 0) ? 2 : 0;  // y_k, read as the centre of z_0
                t.last = (j + 1 == m);
                t.zscale_on = false;
                t.zscale_val = 1.0;
                P.terms.push_back(t);
                pw *= -mu / nu;
                gj = t.gnext;
            }
        }
        // augmented scalar after the sub-step: e^{mu h} * sum_j a_k (-mu h)^j / j!
        double sum = 0.0, tt = 1.0;
        for (int j = 0; j <= m; ++j) {
            sum += tt;
            tt *= (-mu * hstep) / (j + 1);
        }
        ak = P.gamma * ak * sum;
    }
    return P;
}

}  // namespace et
