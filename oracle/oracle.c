/* Plain FP64 CPU oracle for the exponential-integrator step (arXiv 2402.02273).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the
 * benchmark's CPU baseline.  The product library neither links nor calls it.
 *
 * Everything below is written to be checked against the paper by eye:
 *   - the operator is the Sec. 2.1 finite-difference formula with ghost
 *     values equal to the centre value (zero normal derivative, eq. PDE);
 *   - the step is u^{n+1} = u^n + tau phi1(tau A)(A u^n + f(u^n)) (Sec. 2.2);
 *   - tau phi1(tau A) b is evaluated as the top block of exp(tau B) v_1 with
 *     the augmented matrix B = [[A, omega], [0, J]] (Sec. 2.2), written as
 *     the s-fold product of degree-m Taylor polynomials of tau B / s, applied
 *     factor by factor and term by term, P_j = (tau B / s)^j / j!.
 * No blocking, fusion or reordering beyond that; OpenMP only splits loops
 * over z-planes and every sum is taken plane by plane in a fixed order.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no -ffast-math).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static long nvox(const oracle_problem* P) { return (long)P->nx * P->ny * P->nz; }

/* Harmonic mean of two face-adjacent coefficients; 0 when either side is 0
 * (no flux into voxels with D = 0, "no tumor diffusion in the air", Sec. 2). */
static double harmonic_mean(double a, double b) {
    if (a <= 0.0 || b <= 0.0) return 0.0;
    return 2.0 * a * b / (a + b);
}

/* Diffusion part at voxel (i,j,k).  For each axis, with v+ / v- the values of
 * the forward / backward neighbours (the centre value when the neighbour lies
 * outside the box):
 *   literal (Sec. 2.1 formula):
 *     D_p (v+ - 2 v_p + v-) + D_{p+e} (v+ - v_p) - D_p (v_p - v-)
 *   conservative (div(D grad u) of eq. PDE with face coefficients):
 *     W_{p+e/2} (v+ - v_p) - W_{p-e/2} (v_p - v-),  W = harmonic mean of D
 * summed over x, y, z and divided by h^2. */
static double L_at(const oracle_problem* P, const double* v, int i, int j, int k) {
    const long sx = 1, sy = P->nx, sz = (long)P->nx * P->ny;
    const long p = i + sy * j + sz * k;
    const int coord[3] = {i, j, k};
    const int extent[3] = {P->nx, P->ny, P->nz};
    const long stride[3] = {sx, sy, sz};
    const double Dp = P->D[p];
    const double vp = v[p];
    double acc = 0.0;
    for (int a = 0; a < 3; ++a) {
        const int has_plus = coord[a] + 1 < extent[a];
        const int has_minus = coord[a] > 0;
        const double vplus = has_plus ? v[p + stride[a]] : vp;
        const double vminus = has_minus ? v[p - stride[a]] : vp;
        const double Dplus = has_plus ? P->D[p + stride[a]] : 0.0;
        const double Dminus = has_minus ? P->D[p - stride[a]] : 0.0;
        if (P->op == ORACLE_OP_LITERAL) {
            acc += Dp * (vplus - 2.0 * vp + vminus) + Dplus * (vplus - vp) - Dp * (vp - vminus);
        } else {
            acc += harmonic_mean(Dp, Dplus) * (vplus - vp) - harmonic_mean(Dminus, Dp) * (vp - vminus);
        }
    }
    return acc / (P->h * P->h);
}

/* Linear reaction coefficient folded into A (eq. F: rho (1 - 2 u^n) u). */
static double c_at(const oracle_problem* P, const double* un, long p) {
    if (P->scheme == ORACLE_SCHEME_EXPEULER) return 0.0;
    return P->rho * (1.0 - 2.0 * un[p]);
}

void oracle_apply_L(const oracle_problem* P, const double* v, double* out) {
    const long sy = P->nx, sz = (long)P->nx * P->ny;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) out[i + sy * j + sz * k] = L_at(P, v, i, j, k);
}

void oracle_apply_A(const oracle_problem* P, const double* un, const double* v, double* out) {
    const long sy = P->nx, sz = (long)P->nx * P->ny;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                const long p = i + sy * j + sz * k;
                out[p] = L_at(P, v, i, j, k) + c_at(P, un, p) * v[p];
            }
}

/* Row p of A, entries of eq. Amatrix divided by h^2 (literal) or the
 * harmonic-mean face weights (conservative); faces leaving the box are
 * dropped, and the diagonal is minus the sum of the kept off-diagonals plus
 * the reaction coefficient.  Order: centre, -x, +x, -y, +y, -z, +z. */
void oracle_row_A(const oracle_problem* P, const double* un, long p, double e[7]) {
    const long sy = P->nx, sz = (long)P->nx * P->ny;
    const int i = (int)(p % P->nx), j = (int)((p / sy) % P->ny), k = (int)(p / sz);
    const int coord[3] = {i, j, k};
    const int extent[3] = {P->nx, P->ny, P->nz};
    const long stride[3] = {1, sy, sz};
    const double h2 = P->h * P->h;
    const double Dp = P->D[p];
    double offsum = 0.0;
    for (int a = 0; a < 3; ++a) {
        double wminus = 0.0, wplus = 0.0;
        if (coord[a] > 0) {
            const double Dm = P->D[p - stride[a]];
            wminus = (P->op == ORACLE_OP_LITERAL) ? 2.0 * Dp / h2 : harmonic_mean(Dm, Dp) / h2;
        }
        if (coord[a] + 1 < extent[a]) {
            const double Dq = P->D[p + stride[a]];
            wplus = (P->op == ORACLE_OP_LITERAL) ? (Dp + Dq) / h2 : harmonic_mean(Dp, Dq) / h2;
        }
        e[1 + 2 * a] = wminus;
        e[2 + 2 * a] = wplus;
        offsum += wminus + wplus;
    }
    e[0] = -offsum + c_at(P, un, p);
}

void oracle_assemble_A(const oracle_problem* P, const double* un, double* entries) {
    const long n = nvox(P);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) oracle_row_A(P, un, p, entries + 7 * p);
}

double oracle_norm_inf_A(const oracle_problem* P, const double* un) {
    const long n = nvox(P);
    const long sz = (long)P->nx * P->ny;
    double* plane_max = (double*)calloc((size_t)P->nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < P->nz; ++k) {
        double m = 0.0;
        for (long p = k * sz; p < (k + 1) * sz; ++p) {
            double e[7];
            oracle_row_A(P, un, p, e);
            double r = fabs(e[0]);
            for (int q = 1; q < 7; ++q) r += fabs(e[q]);
            if (r > m) m = r;
        }
        plane_max[k] = m;
    }
    double m = 0.0;
    for (int k = 0; k < P->nz; ++k)
        if (plane_max[k] > m) m = plane_max[k];
    free(plane_max);
    (void)n;
    return m;
}

/* b = A u^n + f(u^n):  f = rho (u^n)^2 for the folded scheme (eq. newF with
 * u^t = u^{t-1}), f = rho u^n (1 - u^n) when A = L. */
void oracle_residual(const oracle_problem* P, const double* un, double* b) {
    const long n = nvox(P);
    oracle_apply_A(P, un, un, b);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) {
        const double f = (P->scheme == ORACLE_SCHEME_EXPEULER) ? P->rho * un[p] * (1.0 - un[p])
                                                               : P->rho * un[p] * un[p];
        b[p] += f;
    }
}

static double norm_inf(const double* v, long n, int nz) {
    const long plane = n / nz;
    double* pm = (double*)calloc((size_t)nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        double m = 0.0;
        for (long p = k * plane; p < (k + 1) * plane; ++p)
            if (fabs(v[p]) > m) m = fabs(v[p]);
        pm[k] = m;
    }
    double m = 0.0;
    for (int k = 0; k < nz; ++k)
        if (pm[k] > m) m = pm[k];
    free(pm);
    return m;
}

/* tau phi1(tau A) b as the top block of exp(tau B) v_1 (Sec. 2.2).
 *
 * Augmented vector w = [x; a; c] with B w = [A x + b a; c; 0] (omega = [b 0],
 * J = [[0 1],[0 0]]), v_1 = [0; 1; 0].  exp(tau B) = (exp(tau B / s))^s and
 * each factor is sum_{j=0}^{m} P_j, P_j = (tau B / s)^j / j!, applied to w
 * term by term: P_j w = (h / j) B (P_{j-1} w), h = tau / s.
 *
 * Choice of s and m (left open by the paper): s = ceil(beta / theta) with
 * beta = tau ||A||_inf, so theta_eff = h ||A||_inf <= theta.  For j >= 1 the
 * scalar parts of P_j w vanish, hence ||P_{j+1} w|| <= theta_eff/(j+1) ||P_j w||
 * and the remainder after term j is at most ||P_j w|| theta_eff/(j+1-theta_eff);
 * terms are added until that bound is below stop_tol * max(||x||, h ||b||)
 * (and at least 8 terms). */
int oracle_phi1_action(const oracle_problem* P, const double* un, const double* b, double tau,
                       const oracle_schedule* S, double* x, int* s_out, int* m_out) {
    const long n = nvox(P);
    const double theta = S ? S->theta : 0.5;
    const double stop_tol = S ? S->stop_tol : 1e-18;
    const int max_terms = S ? S->max_terms : 200;
    const double normA = oracle_norm_inf_A(P, un);
    const double beta = tau * normA;
    int s = (int)ceil(beta / theta);
    if (s < 1) s = 1;
    const double h = tau / s;
    const double theta_eff = h * normA;
    const double bnorm = norm_inf(b, n, P->nz);

    double* term = (double*)malloc((size_t)n * sizeof(double));
    double* next = (double*)malloc((size_t)n * sizeof(double));
    double* acc = (double*)malloc((size_t)n * sizeof(double));
    if (!term || !next || !acc) {
        free(term); free(next); free(acc);
        return -1;
    }
    /* w = v_1 */
    memset(x, 0, (size_t)n * sizeof(double));
    double a = 1.0, c = 0.0;
    int mmax = 0;
    int status = 0;

    for (int k = 1; k <= s && status == 0; ++k) {
        /* P_0 w = w */
        memcpy(term, x, (size_t)n * sizeof(double));
        double ta = a, tc = c;
        memcpy(acc, x, (size_t)n * sizeof(double));
        double acc_a = a, acc_c = c;
        int j = 1;
        for (;; ++j) {
            /* P_j w = (h / j) B (P_{j-1} w) */
            oracle_apply_A(P, un, term, next);
#pragma omp parallel for schedule(static)
            for (long p = 0; p < n; ++p) next[p] = (h / j) * (next[p] + b[p] * ta);
            const double na = (h / j) * tc;
            const double nc = 0.0;
#pragma omp parallel for schedule(static)
            for (long p = 0; p < n; ++p) acc[p] += next[p];
            acc_a += na;
            acc_c += nc;
            double* t = term; term = next; next = t;
            ta = na;
            tc = nc;
            if (j >= 8 && ta == 0.0 && tc == 0.0) {
                const double tn = norm_inf(term, n, P->nz);
                const double rem = tn * theta_eff / (j + 1 - theta_eff);
                const double xn = norm_inf(acc, n, P->nz);
                const double scale = xn > h * bnorm ? xn : h * bnorm;
                if (rem <= stop_tol * scale) break;
            }
            if (j >= max_terms) {
                status = -2;
                break;
            }
        }
        if (j > mmax) mmax = j;
        memcpy(x, acc, (size_t)n * sizeof(double));
        a = acc_a;
        c = acc_c;
    }
    free(term); free(next); free(acc);
    if (s_out) *s_out = s;
    if (m_out) *m_out = mmax;
    return status;
}

static void stats_of(const double* u, long n, int nz, oracle_stats* st) {
    const long plane = n / nz;
    double* ps = (double*)calloc((size_t)nz, sizeof(double));
    double* pmin = (double*)calloc((size_t)nz, sizeof(double));
    double* pmax = (double*)calloc((size_t)nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        double s = 0.0, lo = u[k * plane], hi = u[k * plane];
        for (long p = k * plane; p < (k + 1) * plane; ++p) {
            s += u[p];
            if (u[p] < lo) lo = u[p];
            if (u[p] > hi) hi = u[p];
        }
        ps[k] = s; pmin[k] = lo; pmax[k] = hi;
    }
    double s = 0.0, lo = pmin[0], hi = pmax[0];
    for (int k = 0; k < nz; ++k) {
        s += ps[k];
        if (pmin[k] < lo) lo = pmin[k];
        if (pmax[k] > hi) hi = pmax[k];
    }
    st->mass = s; st->umin = lo; st->umax = hi;
    free(ps); free(pmin); free(pmax);
}

/* One exponential-integrator step, u^{n+1} = u^n + tau phi1(tau A)(A u^n + f(u^n)). */
int oracle_step(const oracle_problem* P, double* u, double tau, const oracle_schedule* S,
                oracle_stats* st) {
    const long n = nvox(P);
    double* b = (double*)malloc((size_t)n * sizeof(double));
    double* x = (double*)malloc((size_t)n * sizeof(double));
    if (!b || !x) { free(b); free(x); return -1; }
    oracle_residual(P, u, b);
    int s = 0, m = 0;
    const int status = oracle_phi1_action(P, u, b, tau, S, x, &s, &m);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) u[p] += x[p];
    if (st) {
        stats_of(u, n, P->nz, st);
        st->s = s;
        st->m = m;
    }
    free(b); free(x);
    return status;
}

int oracle_run(const oracle_problem* P, double* u, double tau, int nsteps, const oracle_schedule* S,
               oracle_stats* stats) {
    for (int t = 0; t < nsteps; ++t) {
        const int status = oracle_step(P, u, tau, S, stats ? &stats[t] : NULL);
        if (status != 0) return status;
    }
    return 0;
}

/* (L^T v)_p: the transpose of the diffusion operator, from the row entries of
 * eq. Amatrix (entry (q, p) of row q for every neighbour q of p, and L_pp). */
static void apply_LT(const oracle_problem* P, const double* v, double* out) {
    const long sy = P->nx, sz = (long)P->nx * P->ny;
    const long n = nvox(P);
    double* zero_u = (double*)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < P->nz; ++k)
        for (int j = 0; j < P->ny; ++j)
            for (int i = 0; i < P->nx; ++i) {
                const long p = i + sy * j + sz * k;
                const int coord[3] = {i, j, k};
                const int extent[3] = {P->nx, P->ny, P->nz};
                const long stride[3] = {1, sy, sz};
                double e[7];
                oracle_row_A(P, zero_u, p, e);
                /* L_pp is minus the sum of the kept off-diagonal entries */
                double acc = -(e[1] + e[2] + e[3] + e[4] + e[5] + e[6]) * v[p];
                for (int a = 0; a < 3; ++a) {
                    double eq[7];
                    if (coord[a] > 0) { /* row q = p - e has entry towards +e equal to L_{q,p} */
                        oracle_row_A(P, zero_u, p - stride[a], eq);
                        acc += eq[2 + 2 * a] * v[p - stride[a]];
                    }
                    if (coord[a] + 1 < extent[a]) { /* row q = p + e, entry towards -e */
                        oracle_row_A(P, zero_u, p + stride[a], eq);
                        acc += eq[1 + 2 * a] * v[p + stride[a]];
                    }
                }
                out[p] = acc;
            }
    free(zero_u);
}

/* Reverse of oracle_step.  Forward, per sub-step k (x_0 = 0, augmented scalar
 * a = 1 throughout):  t_1 = h (A x_{k-1} + b),  t_j = (h/j) A t_{j-1},
 * x_k = x_{k-1} + t_1 + ... + t_J;  then u^{n+1} = u^n + x_s, with
 * A = L + diag(c), c = rho (1 - 2u^n) (folded scheme) or 0, b = L u^n + rho u^n (1 - u^n).
 * Reverse, from xbar = ubar_next:
 *   tbar_J = xbar;  tbar_j = xbar + (h/(j+1)) A^T tbar_{j+1};
 *   xbar_{k-1} = xbar + h A^T tbar_1;   bbar += h tbar_1;
 *   cbar_p += h tbar_1,p x_{k-1},p + sum_{j>=2} (h/j) tbar_j,p t_{j-1},p;
 *   d/ds (L -> sL) += h <tbar_1, L x_{k-1}> + sum_{j>=2} (h/j) <tbar_j, L t_{j-1}>;
 * then ubar = ubar_next + L^T bbar + rho (1 - 2u) bbar - 2 rho cbar,
 * d/drho += <u(1-u), bbar> + <1 - 2u, cbar>,  d/ds += <bbar, L u>. */
int oracle_step_adjoint(const oracle_problem* P, const double* un, double tau, const oracle_schedule* S,
                        const double* ubar_next, double* ubar, double* grad_rho, double* grad_dscale) {
    const long n = nvox(P);
    const double theta = S ? S->theta : 0.5;
    const double stop_tol = S ? S->stop_tol : 1e-18;
    const int max_terms = S ? S->max_terms : 200;
    const int folded = P->scheme != ORACLE_SCHEME_EXPEULER;
    const double normA = oracle_norm_inf_A(P, un);
    int s = (int)ceil(tau * normA / theta);
    if (s < 1) s = 1;
    const double h = tau / s;
    const double theta_eff = h * normA;

    double* b = (double*)malloc((size_t)n * sizeof(double));
    double* xs = (double*)malloc((size_t)(s + 1) * n * sizeof(double)); /* x_0 .. x_s */
    int* nterms = (int*)calloc((size_t)s, sizeof(int));
    double* work = (double*)malloc((size_t)n * sizeof(double));
    double* work2 = (double*)malloc((size_t)n * sizeof(double));
    double* bbar = (double*)calloc((size_t)n, sizeof(double));
    double* cbar = (double*)calloc((size_t)n, sizeof(double));
    double* xbar = (double*)malloc((size_t)n * sizeof(double));
    double* tbar = (double*)malloc((size_t)n * sizeof(double));
    double* tbar_prev = (double*)malloc((size_t)n * sizeof(double));
    double* tstore = NULL;
    if (!b || !xs || !nterms || !work || !work2 || !bbar || !cbar || !xbar || !tbar || !tbar_prev) return -1;

    /* b = L u + rho u (1 - u) (equal to A u + f for both schemes, eq. F) */
    oracle_apply_L(P, un, b);
    for (long p = 0; p < n; ++p) b[p] += P->rho * un[p] * (1.0 - un[p]);
    const double bnorm = norm_inf(b, n, P->nz);

    /* forward sub-steps, recording x_k and the number of terms */
    memset(xs, 0, (size_t)n * sizeof(double));
    for (int k = 1; k <= s; ++k) {
        double* xprev = xs + (size_t)(k - 1) * n;
        double* xk = xs + (size_t)k * n;
        memcpy(xk, xprev, (size_t)n * sizeof(double));
        memcpy(work, xprev, (size_t)n * sizeof(double)); /* term */
        double ta = 1.0;
        int j = 1;
        for (;; ++j) {
            oracle_apply_A(P, un, work, work2);
            for (long p = 0; p < n; ++p) work2[p] = (h / j) * (work2[p] + b[p] * ta);
            ta = 0.0;
            for (long p = 0; p < n; ++p) xk[p] += work2[p];
            double* t = work; work = work2; work2 = t;
            if (j >= 8) {
                const double tn = norm_inf(work, n, P->nz);
                const double xn = norm_inf(xk, n, P->nz);
                const double scale = xn > h * bnorm ? xn : h * bnorm;
                if (tn * theta_eff / (j + 1 - theta_eff) <= stop_tol * scale) break;
            }
            if (j >= max_terms) break;
        }
        nterms[k - 1] = j;
    }

    /* reverse sub-steps */
    memcpy(xbar, ubar_next, (size_t)n * sizeof(double));
    double gscale = 0.0;
    for (int k = s; k >= 1; --k) {
        const int J = nterms[k - 1];
        const double* xprev = xs + (size_t)(k - 1) * n;
        /* recompute t_1 .. t_J of this sub-step */
        tstore = (double*)realloc(tstore, (size_t)(J + 1) * n * sizeof(double));
        oracle_apply_A(P, un, xprev, work);
        for (long p = 0; p < n; ++p) tstore[n + p] = h * (work[p] + b[p]);
        for (int j = 2; j <= J; ++j) {
            oracle_apply_A(P, un, tstore + (size_t)(j - 1) * n, work);
            for (long p = 0; p < n; ++p) tstore[(size_t)j * n + p] = (h / j) * work[p];
        }
        /* tbar_J = xbar, then down to tbar_1 */
        memcpy(tbar, xbar, (size_t)n * sizeof(double));
        for (int j = J; j >= 2; --j) {
            /* t_j = (h/j) A t_{j-1}: contributions of tbar_j */
            const double* tprev = tstore + (size_t)(j - 1) * n;
            oracle_apply_L(P, tprev, work);
            for (long p = 0; p < n; ++p) {
                cbar[p] += (h / j) * tbar[p] * tprev[p];
                gscale += (h / j) * tbar[p] * work[p];
            }
            /* tbar_{j-1} = xbar + (h/j) A^T tbar_j */
            apply_LT(P, tbar, work);
            for (long p = 0; p < n; ++p) {
                const double cp = folded ? P->rho * (1.0 - 2.0 * un[p]) : 0.0;
                tbar_prev[p] = xbar[p] + (h / j) * (work[p] + cp * tbar[p]);
            }
            double* t = tbar; tbar = tbar_prev; tbar_prev = t;
        }
        /* t_1 = h (A x_{k-1} + b) */
        oracle_apply_L(P, xprev, work);
        for (long p = 0; p < n; ++p) {
            cbar[p] += h * tbar[p] * xprev[p];
            gscale += h * tbar[p] * work[p];
            bbar[p] += h * tbar[p];
        }
        apply_LT(P, tbar, work);
        for (long p = 0; p < n; ++p) {
            const double cp = folded ? P->rho * (1.0 - 2.0 * un[p]) : 0.0;
            xbar[p] = xbar[p] + h * (work[p] + cp * tbar[p]);
        }
    }
    /* x_0 = 0 does not depend on anything: xbar_0 is dropped.
     * u^{n+1} = u^n + x_s; b and c depend on u^n, rho and the D scale. */
    apply_LT(P, bbar, work);
    oracle_apply_L(P, un, work2);
    double grho = 0.0;
    for (long p = 0; p < n; ++p) {
        double up = un[p];
        ubar[p] = ubar_next[p] + work[p] + P->rho * (1.0 - 2.0 * up) * bbar[p];
        grho += up * (1.0 - up) * bbar[p];
        gscale += bbar[p] * work2[p];
        if (folded) {
            ubar[p] += -2.0 * P->rho * cbar[p];
            grho += (1.0 - 2.0 * up) * cbar[p];
        }
    }
    if (grad_rho) *grad_rho += grho;
    if (grad_dscale) *grad_dscale += gscale;
    free(b); free(xs); free(nterms); free(work); free(work2); free(bbar); free(cbar);
    free(xbar); free(tbar); free(tbar_prev); free(tstore);
    return 0;
}
