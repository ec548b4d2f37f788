/* Plain FP64 CPU oracle for the exponential-integrator step of the
 * Fisher-Kolmogorov tumour model (Pabisz, Munoz-Matute, Paszynski,
 * arXiv 2402.02273).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and oracle.c are used by the test
 * suite, by the smoke check and by the benchmark's CPU baseline; the product
 * library never includes, links or calls them, and shares no code with them.
 *
 * Grid: nx * ny * nz cell-centred voxels of width h, voxel (i, j, k) stored at
 * p = i + nx * (j + ny * k) (x fastest), zero-flux walls (Sec. 2, eq. PDE).
 * All arrays are FP64 of length nx * ny * nz.
 */
#ifndef ET_ORACLE_H
#define ET_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Operator readings of Sec. 2.1 (see oracle.c for both). */
#define ORACLE_OP_CONSERVATIVE 0 /* div(D grad u), harmonic-mean faces     */
#define ORACLE_OP_LITERAL      1 /* the printed FD formula / eq. Amatrix   */

/* Linearisation of the reaction (eq. F / newF of Sec. 2.1). */
#define ORACLE_SCHEME_ROSENBROCK 0 /* A = L + diag(rho(1-2u^n)), f = rho (u^n)^2 */
#define ORACLE_SCHEME_EXPEULER   1 /* A = L,                     f = rho u(1-u) */

typedef struct {
    int nx, ny, nz;
    double h;
    const double* D;  /* per-voxel diffusion coefficient, >= 0 */
    int op;           /* ORACLE_OP_*     */
    int scheme;       /* ORACLE_SCHEME_* */
    double rho;       /* proliferation rate */
} oracle_problem;

/* Sub-stepping control of the phi1 action (Sec. 2.2): s = ceil(beta / theta),
 * terms added until the remainder bound drops below stop_tol relative. */
typedef struct {
    double theta;     /* default 0.5   */
    double stop_tol;  /* default 1e-18 */
    int max_terms;    /* default 200   */
} oracle_schedule;

typedef struct {
    double mass, umin, umax; /* of u^{n+1} */
    int s, m;                /* sub-steps and the largest number of terms used */
} oracle_stats;

void oracle_set_threads(int nthreads);
int oracle_get_threads(void);

/* out = A v, A from u^n per the problem's operator and scheme (eq. Amatrix). */
void oracle_apply_A(const oracle_problem* P, const double* un, const double* v, double* out);
/* out = L v (diffusion part only). */
void oracle_apply_L(const oracle_problem* P, const double* v, double* out);
/* Dense row p of A: 7 entries (centre, -x, +x, -y, +y, -z, +z); 0 where absent. */
void oracle_row_A(const oracle_problem* P, const double* un, long p, double entries[7]);
/* ||A||_inf from the row entries (Gershgorin row sums). */
double oracle_norm_inf_A(const oracle_problem* P, const double* un);
/* The rows of A_n for every voxel p, as oracle_row_A writes them, at
 * entries[7 p .. 7 p + 6] (for assembling a sparse matrix). */
void oracle_assemble_A(const oracle_problem* P, const double* un, double* entries);
/* b = A u^n + f(u^n). */
void oracle_residual(const oracle_problem* P, const double* un, double* b);
/* x = tau * phi1(tau A) b through exp(tau B) v_1 (augmented matrix, s sub-steps). */
int oracle_phi1_action(const oracle_problem* P, const double* un, const double* b, double tau,
                       const oracle_schedule* S, double* x, int* s_out, int* m_out);
/* u <- u + tau phi1(tau A)(A u + f(u)), in place; returns 0 on success. */
int oracle_step(const oracle_problem* P, double* u, double tau, const oracle_schedule* S,
                oracle_stats* st);
/* nsteps steps in place; stats[nsteps] may be NULL. */
int oracle_run(const oracle_problem* P, double* u, double tau, int nsteps, const oracle_schedule* S,
               oracle_stats* stats);

/* Discrete adjoint of oracle_step (reverse mode through the same loops, with
 * the schedule s and the number of Taylor terms of every sub-step frozen at
 * the values the forward step takes from u^n).  Given ubar_next = dJ/du^{n+1},
 * writes ubar = dJ/du^n and adds dJ/drho to *grad_rho and d/ds J(s D)|_{s=1}
 * to *grad_dscale. */
int oracle_step_adjoint(const oracle_problem* P, const double* un, double tau, const oracle_schedule* S,
                        const double* ubar_next, double* ubar, double* grad_rho, double* grad_dscale);

#ifdef __cplusplus
}
#endif
#endif
