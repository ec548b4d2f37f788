// Host side of the C ABI declared in include/et.h: argument checks, workspace
// layout, the (s, m) selector, the per-step launch sequence and its CUDA-graph
// replay.  No PyTorch dependency: the caller passes raw device pointers and a
// cudaStream_t.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <type_traits>
#include <vector>

#include "et.h"
#include "et_chain.h"
#include "et_cn.h"
#include "et_internal.h"
#include "et_plan.h"

using namespace et;

namespace {

thread_local char g_create_error[512] = "";

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Bytes of one value of the term kernels' type.
size_t value_bytes(et_precision prec) { return prec == ET_F32 ? 4 : 8; }

struct Layout {
    size_t w[5];      // FP64 coefficient fields (all forms; the residual reads them)
    size_t wt[5];     // typed, 1/nu-scaled copies of w[0..4] (F32, DF64)
    size_t wpair[5];  // F32: the same scaled weights as pairs, read by the residual
    size_t vec[6];    // b, dt, Y0, Y1, Z0, Z1 in the kernels' value type
    size_t stage;     // n doubles for host transfers
    size_t ushadow;   // F32, DF64: the pair of each u, read by the pair-arithmetic residual
    size_t partial;   // 3 * kStatsBlocks doubles
    size_t wnorm;     // 2 * kBlockY * nblocks: the residual warps' max |b|, max |u^n|
    size_t npartial;  // 2 * kStatsBlocks doubles: the stats blocks' maxima of those
    size_t zrow;      // one byte per warp row: rows without off-diagonal entries
    size_t misc;      // counters, flags, info slots
    size_t total;
    unsigned nblocks;
};

constexpr size_t kMiscBytes = 2048;  // counters, flags, info slot; truncation estimate at 1024, CN scalars at 1536,
                                     // zero-row count at 1600

bool make_layout(int nx, int ny, int nz, et_precision prec, Layout* L) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return false;
    const long long n = (long long)nx * ny * nz;
    if (n >= (1ll << 31)) return false;
    if (nz > 65535) return false;
    const unsigned gx = (unsigned)((nx + kBlockX - 1) / kBlockX);
    const unsigned gy = (unsigned)((ny + kBlockY - 1) / kBlockY);
    const unsigned long long nb = (unsigned long long)gx * gy * (unsigned)nz;
    if (nb >= (1ull << 31)) return false;
    L->nblocks = (unsigned)nb;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    const size_t vb = value_bytes(prec);
    for (int a = 0; a < 5; ++a) L->w[a] = take(8ull * n);
    for (int a = 0; a < 5; ++a) L->wt[a] = (prec != ET_F64) ? take(vb * n) : SIZE_MAX;
    for (int a = 0; a < 5; ++a) L->wpair[a] = (prec == ET_F32) ? take(8ull * n) : SIZE_MAX;
    for (int v = 0; v < 6; ++v) L->vec[v] = take(vb * n);
    L->stage = take(8ull * n);
    L->ushadow = prec != ET_F64 ? take(8ull * n) : SIZE_MAX;
    L->partial = take(3ull * 8ull * kStatsBlocks);
    L->wnorm = take(2ull * 8ull * kBlockY * nb);
    L->npartial = take(2ull * 8ull * kStatsBlocks);
    {
        Geom G;
        G.nx = nx;
        G.ny = ny;
        G.nz = nz;
        L->zrow = take((size_t)zero_row_bytes(G));
    }
    L->misc = take(kMiscBytes);
    L->total = off;
    return true;
}

// The scalars of the coefficient setup that a captured run bakes into its
// kernel arguments (the weights themselves are read from device memory when
// the graph runs, so a new D with the same scalars reuses the graph).
struct CoeffKey {
    double nu = 0.0, rmax = 0.0, rho = 0.0;
    int op = -1, scheme = -1;
    bool opt_set = false;
    et_options opt{};
};

bool same_coeffs(const CoeffKey& a, const CoeffKey& b) {
    // bit patterns, so that a NaN never matches and -0 differs from +0
    auto eq = [](double x, double y) { return std::memcmp(&x, &y, sizeof(double)) == 0; };
    if (!eq(a.nu, b.nu) || !eq(a.rmax, b.rmax) || !eq(a.rho, b.rho) || a.op != b.op || a.scheme != b.scheme ||
        a.opt_set != b.opt_set)
        return false;
    if (!a.opt_set) return true;
    const et_options &x = a.opt, &y = b.opt;
    return eq(x.tol, y.tol) && eq(x.theta_max, y.theta_max) && x.shift == y.shift && x.force_s == y.force_s &&
           x.force_m == y.force_m && x.use_graph == y.use_graph && x.single_terms == y.single_terms &&
           x.timeout_probe_us == y.timeout_probe_us && x.every_row == y.every_row;
}

struct GraphEntry {
    CoeffKey coeffs;
    double* u = nullptr;
    et_step_info* info = nullptr;
    double tau = 0.0;
    int nsteps = 0;
    bool timing = false;
    cudaGraphExec_t exec = nullptr;
    unsigned long long stamp = 0;
    long long term_launches = 0, other_launches = 0;
};

struct Schedule {
    int s = 0, m = 0;
    double mu = 0.0, theta = 0.0;
};

struct ResolvedOptions {
    double tol, theta_max;
    int shift, force_s, force_m, use_graph;
    int single_terms;  // 1: one term per launch; -1: two where possible; 0: per form
    unsigned long long probe_ns;  // test hook of the two-term kernel's bounded waits (0: off)
    bool skip_zero_rows;          // one-term kernels skip rows without off-diagonal entries
};

ResolvedOptions resolve(const et_options* o, et_precision prec) {
    ResolvedOptions r;
    r.tol = (o && o->tol > 0) ? o->tol : (prec == ET_F32 ? 1e-7 : 1e-13);
    r.shift = (o && o->shift == 0) ? 0 : 1;
    if (o && o->shift < 0) r.shift = 1;
    // Unshifted, the Taylor partial sums of a sub-step grow like e^theta before
    // cancelling, so theta is capped for rounding; shifted, the e^{mu h} factor
    // of each sub-step cancels that growth and theta is capped only to keep the
    // sums far inside the FP32 range.
    const double cap_default = r.shift ? 32.0 : (prec == ET_F32 ? 1.5 : 7.0);
    r.theta_max = (o && o->theta_max > 0) ? o->theta_max : cap_default;
    r.force_s = (o && o->force_s > 0) ? o->force_s : 0;
    r.force_m = (o && o->force_m > 0) ? o->force_m : 0;
    r.use_graph = (o && o->use_graph < 0) ? 0 : 1;
    r.single_terms = !o ? 0 : (o->single_terms > 0 ? 1 : (o->single_terms < 0 ? -1 : 0));
    r.probe_ns = (o && o->timeout_probe_us > 0) ? 1000ull * (unsigned long long)o->timeout_probe_us : 0;
    r.skip_zero_rows = !(o && o->every_row != 0);
    return r;
}

}  // namespace

struct et_grid {
    int nx, ny, nz;
    long long n;
    double h;
    et_precision prec;
    int device;
    char* ws;
    size_t ws_bytes;
    Layout L;
    Geom G;
    cudaStream_t stream;
    cudaStream_t capture;  // private stream used only for graph capture
    // device views
    double* w[5];
    void* wt[5];
    void* vec[6];
    double* stage;
    double* partial;
    PairPlan* pair;  // tensor maps of the two-term kernel (F32 / DF64), or nullptr
    float2* wres[5];  // F32, DF64: the 1/nu-scaled pair weights the residual reads
    float2* ush;      // F32, DF64: the pair copy of u (nullptr for F64)
    unsigned long long* rmax_bits;
    unsigned* flags;
    unsigned* ticket;
    unsigned* step_counter;
    et_step_info* info_slot;
    unsigned long long* wnorm;  // residual warps' norm slots of the truncation estimate
    double* npartial;           // the stats blocks' maxima of those
    double* trunc_est;          // the latest step's estimate
    unsigned char* zrow;        // rows without off-diagonal entries (Weights::zrow)
    unsigned long long* zrow_count;  // voxels in those rows
    // Crank-Nicolson: device scalars of the solve and the captured step
    CnScalars* cn_sc;
    cudaGraphExec_t cn_exec;
    CoeffKey cn_key;
    double* cn_u;
    et_step_info* cn_info;
    double cn_tau, cn_rtol;
    int cn_cap;
    // model state
    bool coeffs_set;
    et_operator op;
    et_scheme scheme;
    double rho;
    double rmax;
    double nu;  // ||A - mu I||_inf bound: the FP32 / DF64 recurrences are scaled by 1/nu
    et_options opt;
    bool opt_set;
    // graph cache and timing
    std::vector<GraphEntry> graphs;
    unsigned long long stamp;
    bool timing;
    std::vector<cudaEvent_t> ev;  // 2 per step of the last timed run
    int timed_steps;
    long long last_term_launches, last_other_launches;
    char err[512];
};

namespace {

et_status fail(et_grid* g, et_status st, const char* fmt, ...) {
    char* dst = g ? g->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return st;
}

#define ET_CUDA(g, call)                                                                      \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((g), ET_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

// Keeps the caller's current device across a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

CoeffKey coeff_key(const et_grid* g) {
    CoeffKey k;
    k.nu = g->nu;
    k.rmax = g->rmax;
    k.rho = g->rho;
    k.op = (int)g->op;
    k.scheme = (int)g->scheme;
    k.opt_set = g->opt_set;
    if (g->opt_set) k.opt = g->opt;
    return k;
}

void clear_graphs(et_grid* g) {
    for (auto& e : g->graphs)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    g->graphs.clear();
}

void clear_events(et_grid* g) {
    for (auto e : g->ev) cudaEventDestroy(e);
    g->ev.clear();
    g->timed_steps = 0;
}

et_status schedule_for(const et_grid* g, double tau, Schedule* S) {
    return et_select_schedule(tau, g->rmax, g->rho, g->scheme, g->prec, g->opt_set ? &g->opt : nullptr,
                              &S->s, &S->m, &S->mu, &S->theta);
}

template <typename T>
struct Buffers {
    Weights<T> W;  // w[4] unused by the term kernels
    const T* b;
    T* dt;
    T* Y[2];
    T* Z[2];
};

template <typename T>
Buffers<T> typed_buffers(et_grid* g) {
    Buffers<T> B;
    for (int a = 0; a < 4; ++a) B.W.w[a] = g->prec == ET_F64 ? (const T*)g->w[a] : (const T*)g->wt[a];
    B.W.w[4] = nullptr;
    // the one-term kernels skip the rows without off-diagonal entries
    B.W.zrow = resolve(g->opt_set ? &g->opt : nullptr, g->prec).skip_zero_rows ? g->zrow : nullptr;
    B.b = (const T*)g->vec[0];
    B.dt = (T*)g->vec[1];
    B.Y[0] = (T*)g->vec[2];
    B.Y[1] = (T*)g->vec[3];
    B.Z[0] = (T*)g->vec[4];
    B.Z[1] = (T*)g->vec[5];
    return B;
}

// Enqueues the s*m - 1 Taylor-term launches of one step (Sec. 2.2); counts
// them in *launches.
//
// FP64 runs the scaled recurrence of et_kernels.cu, z^_{j+1} = A~ z^_j +
// a_k (-mu)^j b with weights g_j = h^j / j!.  FP32 and DF64 run it normalised
// by nu (weights and diagonal already divided by nu): zeta_j = z^_j / nu^j,
//     zeta_{j+1} = (A~/nu) zeta_j + a_k (-mu)^j / nu^{j+1} b,
// with weights theta^j / j!, theta = h nu, so the vectors stay O(|b| / nu).
// On sub-step 0, zeta_1 = b / nu is read as b with the stencil part scaled by
// 1 / nu (zscale).
// Two consecutive terms of a sub-step per launch (et_fused.cu)?  Only F32 and
// DF64 grids whose rows the two-term kernel can address.  By default DF64
// always; F32 only when the fields of its chain (about 32 B per voxel) exceed
// about 1.4 times the 129 MB L2: while they (largely) fit, the four-voxel
// one-term kernel is the faster, beyond, the pair's halved HBM traffic wins.
// Measured, us per term (one-term / half a pair): 128^3 6.1 / 10.4, 160^3
// 16.5 / 19.5, 192^3 35.5 / 31.1.
bool use_pairs(const et_grid* g) {
    if (g->prec == ET_F64 || !g->pair || !pair_preferred(g->op, g->prec)) return false;
    const int t = resolve(g->opt_set ? &g->opt : nullptr, g->prec).single_terms;
    if (t != 0) return t < 0;
    // FP32: one term per launch (four-voxel kernel) while the Horner chain's
    // seven fields (28 B a voxel) stay well inside the L2, two per launch
    // beyond (us per term, one / two per launch: 128^3 5.8 / 8.2, 160^3
    // 17.4 / 14.2, 192^3 35.0 / 23.5)
    constexpr double kL2Bytes = 129.0e6;
    return g->prec == ET_DF64 || 28.0 * (double)g->n > 0.75 * kL2Bytes;
}

// Test hook of the two-term kernel's bounded waits (et_options.timeout_probe_us).
unsigned long long probe_ns(const et_grid* g) { return g->opt_set ? resolve(&g->opt, g->prec).probe_ns : 0; }

ChainPlan plan_chain(const et_grid* g, const Schedule& S, double hstep) {
    return et::plan_chain(g->prec, g->nu, S.s, S.m, S.mu, hstep);
}

// Storage of a recorded forward step for the adjoint: z_j of sub-step k at
// zstore + (k m + j) n and y_k at ystore + k n (values of type T).
template <typename T>
struct ChainRecord {
    T* zstore = nullptr;
    T* ystore = nullptr;
    long long n = 0;
    int m = 0;
    T* z(int k, int j) const { return zstore + ((long long)k * m + j) * n; }
    T* y(int k) const { return ystore + (long long)k * n; }
};

// Enqueues the s*m - 1 Taylor-term launches of one step (Sec. 2.2); counts
// them in *launches.
//
// FP64 runs the scaled recurrence of et_kernels.cu, z^_{j+1} = A~ z^_j +
// a_k (-mu)^j b with weights g_j = h^j / j!.  FP32 and DF64 run it normalised
// by nu (weights and diagonal already divided by nu): zeta_j = z^_j / nu^j,
//     zeta_{j+1} = (A~/nu) zeta_j + a_k (-mu)^j / nu^{j+1} b,
// with weights theta^j / j!, theta = h nu, so the vectors stay O(|b| / nu).
// On sub-step 0, zeta_1 = b / nu is read as b with the stencil part scaled by
// 1 / nu (zscale).  With `rec`, every z_j and y_k goes to the record instead
// of the ping-pong buffers and u is left unchanged.
template <typename T>
cudaError_t enqueue_chain(et_grid* g, const Buffers<T>& B, double* u, const Schedule& S, double hstep,
                          cudaStream_t st, long long* launches, const ChainRecord<T>* rec = nullptr) {
    const ChainPlan P = plan_chain(g, S, hstep);
    const int s = S.s;
    if (!rec) {
        // consecutive terms of a sub-step in pairs where chosen (use_pairs)
        const bool pairs = !std::is_same<T, double>::value && use_pairs(g);
        T* const Y[2] = {B.Y[0], B.Y[1]};
        T* const Z[2] = {B.Z[0], B.Z[1]};
        for (const ChainOp<T>& op : chain_ops<T>(P, s, B.b, B.dt, Y, Z, u, pairs)) {
            cudaError_t e;
            if constexpr (std::is_same<T, double>::value) {
                e = launch_term(g->G, g->op, B.W, op.a1, st);
            } else {
                // FP32 Horner pairs on the vector two-term kernel where it
                // applies, other pairs on the TMA-fed one
                bool vec = false;
                if constexpr (std::is_same<T, float>::value) {
                    vec = op.pair && vec_pair_eligible<T>(g->G, g->op, B.W, op.a1, op.a2);
                    if (vec) e = launch_term_vec_pair<T>(g->G, g->op, B.W, op.a1, op.a2, st);
                }
                if (!vec)
                    e = op.pair ? launch_term_pair(g->pair, g->G, g->op, op.a1, op.a2, g->flags, st, probe_ns(g))
                                : launch_term(g->G, g->op, B.W, op.a1, st);
            }
            if (e != cudaSuccess) return e;
            ++*launches;
        }
        return cudaSuccess;
    }
    // recorded chain (adjoint): every term to its own buffer; where pairs are
    // chosen (use_pairs) the pair kernel stores both terms
    const bool pairs = !std::is_same<T, double>::value && use_pairs(g);
    const T* zin = nullptr;
    auto rec_args = [&](const PlannedTerm& t) {
        const int k = t.k, j = t.j;
        if (k == 0 && j == 1) zin = B.b;
        if (k > 0 && j == 0) zin = rec->y(k);
        TermArgs<T> a;
        a.zin = zin;
        a.b = B.b;
        a.beta = Scalar<T>::make(t.beta);
        a.has_beta = t.beta != 0.0;
        a.zscale = Scalar<T>::make(t.zscale_val);
        a.has_zscale = t.zscale_on;
        a.dt = B.dt;
        a.g = Scalar<T>::make(t.gnext);
        a.gamma = Scalar<T>::make(t.last ? P.gamma * (t.horner ? t.gnext : 1.0) : 1.0);
        a.base_scale = Scalar<T>::make(t.base_scale);
        a.base_mode = t.base_mode;
        a.last = t.last;
        a.horner = t.horner;
        a.yacc = rec->y(k + 1);
        a.u = nullptr;
        a.zout = t.last ? nullptr : rec->z(k, j + 1);
        return a;
    };
    if constexpr (!std::is_same<T, double>::value) {
        if (pairs) {
            for (size_t ti = 0; ti < P.terms.size(); ++ti) {
                const PlannedTerm& t = P.terms[ti];
                cudaError_t e;
                if (!t.last && ti + 1 < P.terms.size() && P.terms[ti + 1].k == t.k) {
                    const TermArgs<T> a1 = rec_args(t);
                    zin = a1.zout;
                    const TermArgs<T> a2 = rec_args(P.terms[ti + 1]);
                    ++ti;
                    PairMaps M;
                    if (!pair_maps_for(g->pair, g->G, g->prec, a1.zin, B.b, B.dt, &M)) return cudaErrorInvalidValue;
                    e = launch_term_pair_maps(M, g->G, g->op, a1, a2, g->flags, st, probe_ns(g));
                    if (!a2.last) zin = a2.zout;
                } else {
                    const TermArgs<T> a = rec_args(t);
                    e = launch_term(g->G, g->op, B.W, a, st);
                    if (!t.last) zin = a.zout;
                }
                if (e != cudaSuccess) return e;
                ++*launches;
            }
            return cudaSuccess;
        }
    }
    for (const PlannedTerm& t : P.terms) {
        const TermArgs<T> a = rec_args(t);
        const cudaError_t e = launch_term(g->G, g->op, B.W, a, st);
        if (e != cudaSuccess) return e;
        ++*launches;
        if (!t.last) zin = a.zout;
    }
    return cudaSuccess;
}

// b and the shifted diagonal of the F32 / DF64 forms from the pair copy ush of u.
template <typename T>
cudaError_t enqueue_pair_residual(et_grid* g, const float2* ush, const Buffers<T>& B, double dt_shift,
                                  cudaStream_t st, unsigned long long* wnorm = nullptr) {
    PairResidualArgs R = pair_residual_args(ush, g->wres, g->nu, g->rho, dt_shift, g->scheme);
    R.W.zrow = B.W.zrow;  // the term chain's zero rows, skipped by the residual too
    return launch_residual_df64<T>(g->G, g->op, R, g->scheme, const_cast<T*>(B.b), B.dt, g->flags, st, wnorm);
}

template <typename T>
et_status enqueue_form(et_grid* g, double* u, const Schedule& S, double hstep, double dt_shift,
                       cudaStream_t st, cudaEvent_t ev_begin, unsigned evflags, long long* term_launches,
                       long long* other_launches) {
    Buffers<T> B = typed_buffers<T>(g);
    cudaError_t e;
    if constexpr (!std::is_same<T, double>::value) {
        // F32, DF64: the residual in pair arithmetic from the pair copy of u, on
        // the FP32 pipes (the FP64 residual is bound by GB300's FP64 rate)
        e = enqueue_pair_residual<T>(g, g->ush, B, dt_shift, st, g->wnorm);
    } else {
        Weights<double> W64;
        for (int a = 0; a < 5; ++a) W64.w[a] = g->w[a];
        W64.zrow = B.W.zrow;  // the term chain's zero rows, skipped by the residual too
        e = launch_residual<T>(g->G, g->op, u, W64, g->rho, dt_shift, 1.0, g->scheme, const_cast<T*>(B.b), B.dt,
                               g->flags, st, g->wnorm);
    }
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "residual launch: %s", cudaGetErrorString(e));
    ++*other_launches;
    if (ev_begin) ET_CUDA(g, cudaEventRecordWithFlags(ev_begin, st, evflags));
    e = enqueue_chain<T>(g, B, u, S, hstep, st, term_launches);
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "term launch: %s", cudaGetErrorString(e));
    return ET_OK;
}

// Residual plus the term chain of one step on stream st.
et_status enqueue_step(et_grid* g, double* u, double tau, const Schedule& S, et_step_info* info,
                       int info_stride, cudaStream_t st, cudaEvent_t ev_begin, cudaEvent_t ev_end,
                       bool external_events, long long* term_launches, long long* other_launches) {
    StatsSink sink;
    sink.partial = g->partial;
    sink.ticket = g->ticket;
    sink.step_counter = g->step_counter;
    sink.flags = g->flags;
    sink.info = info;
    sink.info_stride = info_stride;
    sink.last = g->info_slot;
    sink.s = S.s;
    sink.m = S.m;
    sink.ush = g->ush;
    sink.wnorm = g->wnorm;
    sink.nwarps = (long long)g->G.nblocks * kBlockY;
    sink.npartial = g->npartial;
    sink.trunc_c = truncation_factor(tau, g->rmax, g->rho, g->scheme, g->prec, g->opt_set ? &g->opt : nullptr, S.s,
                                     S.m);
    sink.trunc_tol = resolve(g->opt_set ? &g->opt : nullptr, g->prec).tol;
    sink.trunc_est = g->trunc_est;
    const double hstep = tau / S.s;
    const double dt_shift = (g->scheme == ET_SCHEME_ROSENBROCK ? g->rho : 0.0) - S.mu;
    const unsigned evflags = external_events ? cudaEventRecordExternal : cudaEventRecordDefault;
    et_status rc;
    if (g->prec == ET_F64)
        rc = enqueue_form<double>(g, u, S, hstep, dt_shift, st, ev_begin, evflags, term_launches, other_launches);
    else if (g->prec == ET_F32)
        rc = enqueue_form<float>(g, u, S, hstep, dt_shift, st, ev_begin, evflags, term_launches, other_launches);
    else
        rc = enqueue_form<float2>(g, u, S, hstep, dt_shift, st, ev_begin, evflags, term_launches, other_launches);
    if (rc != ET_OK) return rc;
    cudaError_t e;
    if (ev_end) ET_CUDA(g, cudaEventRecordWithFlags(ev_end, st, evflags));
    e = launch_stats(g->G, u, sink, st);
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "stats launch: %s", cudaGetErrorString(e));
    ++*other_launches;
    return ET_OK;
}

et_status ensure_events(et_grid* g, int nsteps) {
    if (!g->timing) return ET_OK;
    if ((int)g->ev.size() >= 2 * nsteps) return ET_OK;
    clear_graphs(g);  // graphs hold references to the old events
    clear_events(g);
    g->ev.resize(2 * (size_t)nsteps, nullptr);
    for (auto& e : g->ev) ET_CUDA(g, cudaEventCreate(&e));
    return ET_OK;
}

// The pair copy of u that the F32 / DF64 residual reads, taken at the start of
// a run; the stats launch that ends every step writes it for the next one.
et_status start_pair_copy(et_grid* g, const double* u, cudaStream_t st) {
    const cudaError_t e = launch_split(g->n, u, 1.0, g->ush, st);
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "split launch: %s", cudaGetErrorString(e));
    return ET_OK;
}

// Enqueues a whole run (counter reset + nsteps steps) on stream st.
et_status enqueue_run(et_grid* g, double* u, double tau, int nsteps, et_step_info* info, cudaStream_t st,
                      bool external_events) {
    Schedule S;
    et_status rc = schedule_for(g, tau, &S);
    if (rc != ET_OK) return fail(g, rc, "no (s, m) meets the tolerance for tau = %g", tau);
    ET_CUDA(g, cudaMemsetAsync(g->step_counter, 0, sizeof(unsigned), st));
    et_step_info* dst = info ? info : g->info_slot;
    const int stride = info ? 1 : 0;
    long long tl = 0, ol = 0;
    if (g->ush) {
        rc = start_pair_copy(g, u, st);
        if (rc != ET_OK) return rc;
        ++ol;
    }
    for (int t = 0; t < nsteps; ++t) {
        cudaEvent_t e0 = g->timing ? g->ev[2 * t] : nullptr;
        cudaEvent_t e1 = g->timing ? g->ev[2 * t + 1] : nullptr;
        rc = enqueue_step(g, u, tau, S, dst, stride, st, e0, e1, external_events, &tl, &ol);
        if (rc != ET_OK) return rc;
    }
    g->last_term_launches = tl;
    g->last_other_launches = ol;
    g->timed_steps = g->timing ? nsteps : 0;
    return ET_OK;
}

et_status run_impl(et_grid* g, double* u, double tau, int nsteps, et_step_info* info) {
    if (!g->coeffs_set) return fail(g, ET_ERR_STATE, "et_set_coeffs has not been called");
    if (!u || !aligned8(u)) return fail(g, ET_ERR_ARG, "u must be a non-NULL 8-byte aligned device pointer");
    if (info && !aligned8(info)) return fail(g, ET_ERR_ARG, "info must be 8-byte aligned");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(g, ET_ERR_ARG, "tau must be finite and > 0");
    if (nsteps < 1) return fail(g, ET_ERR_ARG, "nsteps must be >= 1");
    Schedule S;
    if (schedule_for(g, tau, &S) != ET_OK)
        return fail(g, ET_ERR_ARG, "no (s, m) meets the tolerance for tau = %g", tau);
    et_status rc = ensure_events(g, nsteps);
    if (rc != ET_OK) return rc;
    const ResolvedOptions ro = resolve(g->opt_set ? &g->opt : nullptr, g->prec);
    if (!ro.use_graph) return enqueue_run(g, u, tau, nsteps, info, g->stream, false);

    const CoeffKey key = coeff_key(g);
    for (auto& e : g->graphs) {
        if (e.u == u && e.info == info && e.tau == tau && e.nsteps == nsteps && e.timing == g->timing &&
            same_coeffs(e.coeffs, key)) {
            e.stamp = ++g->stamp;
            ET_CUDA(g, cudaGraphLaunch(e.exec, g->stream));
            g->last_term_launches = e.term_launches;
            g->last_other_launches = e.other_launches;
            g->timed_steps = e.timing ? nsteps : 0;
            return ET_OK;
        }
    }
    // capture on the private stream, then launch on the caller's stream
    ET_CUDA(g, cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_run(g, u, tau, nsteps, info, g->capture, true);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(g->capture, &graph);
    if (rc != ET_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess) return fail(g, ET_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(g, ET_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    if (g->graphs.size() >= 8) {
        size_t oldest = 0;
        for (size_t i = 1; i < g->graphs.size(); ++i)
            if (g->graphs[i].stamp < g->graphs[oldest].stamp) oldest = i;
        cudaGraphExecDestroy(g->graphs[oldest].exec);
        g->graphs.erase(g->graphs.begin() + oldest);
    }
    GraphEntry ent;
    ent.coeffs = key;
    ent.u = u;
    ent.info = info;
    ent.tau = tau;
    ent.nsteps = nsteps;
    ent.timing = g->timing;
    ent.exec = exec;
    ent.stamp = ++g->stamp;
    ent.term_launches = g->last_term_launches;
    ent.other_launches = g->last_other_launches;
    g->graphs.push_back(ent);
    ET_CUDA(g, cudaGraphLaunch(exec, g->stream));
    return ET_OK;
}

et_status set_coeffs_impl(et_grid* g, const double* D, double rho, et_operator op, et_scheme scheme,
                          const et_options* opt, double dscale = 1.0) {
    if (!(dscale >= 0.0) || !std::isfinite(dscale)) return fail(g, ET_ERR_ARG, "dscale must be finite and >= 0");
    if (!(rho >= 0.0) || !std::isfinite(rho)) return fail(g, ET_ERR_ARG, "rho must be finite and >= 0");
    if (op != ET_OP_CONSERVATIVE && op != ET_OP_LITERAL) return fail(g, ET_ERR_ARG, "unknown operator %d", (int)op);
    if (scheme != ET_SCHEME_ROSENBROCK && scheme != ET_SCHEME_EXPEULER)
        return fail(g, ET_ERR_ARG, "unknown scheme %d", (int)scheme);
    if (opt) {
        if (opt->tol < 0 || !std::isfinite(opt->tol)) return fail(g, ET_ERR_ARG, "options.tol must be >= 0");
        if (opt->theta_max < 0 || !std::isfinite(opt->theta_max))
            return fail(g, ET_ERR_ARG, "options.theta_max must be >= 0");
        if (opt->force_m == 1) return fail(g, ET_ERR_ARG, "options.force_m must be 0 or >= 2");
        if (opt->force_s < 0 || opt->force_m < 0) return fail(g, ET_ERR_ARG, "forced s, m must be >= 0");
        if (opt->timeout_probe_us < 0 || opt->timeout_probe_us > 1000000)
            return fail(g, ET_ERR_ARG, "options.timeout_probe_us must be in [0, 1000000]");
        if (opt->every_row != 0 && opt->every_row != 1) return fail(g, ET_ERR_ARG, "options.every_row must be 0 or 1");
    }
    // cached graphs stay: a run reuses one only if its coefficient scalars match
    g->coeffs_set = false;
    ET_CUDA(g, cudaMemsetAsync(g->rmax_bits, 0, sizeof(unsigned long long), g->stream));
    ET_CUDA(g, cudaMemsetAsync(g->flags, 0, sizeof(unsigned), g->stream));
    ET_CUDA(g, cudaMemsetAsync(g->ticket, 0, sizeof(unsigned), g->stream));
    const double inv_h2 = 1.0 / (g->h * g->h);
    cudaError_t e = launch_coeffs(g->G, D, inv_h2, op, g->w, g->rmax_bits, g->flags, g->stream, dscale);
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "coeffs launch: %s", cudaGetErrorString(e));
    {
        Weights<double> W64;
        for (int a = 0; a < 5; ++a) W64.w[a] = g->w[a];
        ET_CUDA(g, cudaMemsetAsync(g->zrow_count, 0, sizeof(unsigned long long), g->stream));
        e = launch_zero_rows(g->G, op, W64, g->zrow, g->zrow_count, g->stream);
        if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "zero-row launch: %s", cudaGetErrorString(e));
    }
    unsigned long long bits = 0;
    unsigned flags = 0;
    ET_CUDA(g, cudaMemcpyAsync(&bits, g->rmax_bits, sizeof(bits), cudaMemcpyDeviceToHost, g->stream));
    ET_CUDA(g, cudaMemcpyAsync(&flags, g->flags, sizeof(flags), cudaMemcpyDeviceToHost, g->stream));
    ET_CUDA(g, cudaStreamSynchronize(g->stream));
    ET_CUDA(g, cudaMemsetAsync(g->flags, 0, sizeof(unsigned), g->stream));
    if (flags & ET_FLAG_D_INVALID) return fail(g, ET_ERR_NUMERIC, "D has negative or non-finite values");
    double rmax;
    std::memcpy(&rmax, &bits, sizeof(rmax));
    g->rmax = rmax;
    {
        const ResolvedOptions ro = resolve(opt, g->prec);
        const double rho_c = (scheme == ET_SCHEME_ROSENBROCK) ? rho * (1.0 + 2.0 * kRangeSlack) : 0.0;
        const double nu = ro.shift ? rmax + rho_c : 2.0 * rmax + rho_c;
        g->nu = nu > 0.0 ? nu : 1.0;
        // the two-term kernel skips voxels without off-diagonal entries too
        pair_plan_set_skip(g->pair, ro.skip_zero_rows);
    }
    if (g->prec != ET_F64) {
        const double* src[4] = {g->w[0], g->w[1], g->w[2], g->w[3]};
        if (g->prec == ET_F32) {
            float* dst[4] = {(float*)g->wt[0], (float*)g->wt[1], (float*)g->wt[2], (float*)g->wt[3]};
            e = launch_convert_weights(g->G, src, dst, 1.0 / g->nu, g->stream);
            if (e == cudaSuccess) e = launch_cast(g->n, g->w[4], 1.0 / g->nu, (float*)g->wt[4], g->stream);
            float2* pdst[4] = {g->wres[0], g->wres[1], g->wres[2], g->wres[3]};
            if (e == cudaSuccess) e = launch_convert_weights(g->G, src, pdst, 1.0 / g->nu, g->stream);
            if (e == cudaSuccess) e = launch_split(g->n, g->w[4], 1.0 / g->nu, g->wres[4], g->stream);
        } else {
            float2* dst[4] = {(float2*)g->wt[0], (float2*)g->wt[1], (float2*)g->wt[2], (float2*)g->wt[3]};
            e = launch_convert_weights(g->G, src, dst, 1.0 / g->nu, g->stream);
            if (e == cudaSuccess) e = launch_split(g->n, g->w[4], 1.0 / g->nu, (float2*)g->wt[4], g->stream);
        }
        if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "weight conversion: %s", cudaGetErrorString(e));
    }
    g->rho = rho;
    g->op = op;
    g->scheme = scheme;
    g->opt_set = opt != nullptr;
    if (opt) g->opt = *opt;
    g->coeffs_set = true;
    return ET_OK;
}

// ---------------------------------------------------------------------------
// Adjoint (vector-Jacobian product) of nsteps steps, checkpointed.

// Adjoint workspace: checkpoints, the states of one segment, and the recorded
// forward steps of that segment (per step: b, the diagonal, every z_j and y_k).
struct AdjLayout {
    size_t zstore, ystore, bstore, dtstore, ckpt, seg, ubar[2], bbar, cbar, sstep, zbar[2], ybar[2], sacc, racc,
        partial,
        slots;
    size_t total;
    size_t zstep, ystep;  // bytes of one step's z and y records
    int nck, ck;
};

bool adj_layout(const et_grid* g, const Schedule& S, int nsteps, int ck, AdjLayout* A) {
    const size_t n = (size_t)g->n;
    const size_t vb = value_bytes(g->prec);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    A->nck = (nsteps + ck - 1) / ck;
    A->ck = ck;
    A->zstep = (size_t)S.s * S.m * vb * n;
    A->ystep = (size_t)(S.s + 1) * vb * n;
    A->zstore = take((size_t)ck * A->zstep);
    A->ystore = take((size_t)ck * A->ystep);
    A->bstore = take((size_t)ck * vb * n);
    A->dtstore = take((size_t)ck * vb * n);
    A->ckpt = take((size_t)A->nck * 8 * n);
    A->seg = take((size_t)ck * 8 * n);
    for (int i = 0; i < 2; ++i) A->ubar[i] = take(8 * n);
    A->bbar = take(vb * n);
    A->cbar = take(vb * n);
    A->sstep = take(vb * n);
    for (int i = 0; i < 2; ++i) A->zbar[i] = take(vb * n);
    for (int i = 0; i < 2; ++i) A->ybar[i] = take(vb * n);
    A->sacc = take(8 * n);
    A->racc = take(8 * n);
    A->partial = take(sum_partials_bytes());
    A->slots = take(64);
    A->total = off;
    return true;
}

// Buffers and record of step `slot` of the current segment.
template <typename T>
Buffers<T> slot_buffers(et_grid* g, char* ws, const AdjLayout& A, int slot, ChainRecord<T>* rec) {
    Buffers<T> B = typed_buffers<T>(g);
    const size_t vb = sizeof(T) * (size_t)g->n;
    B.b = (const T*)(ws + A.bstore + (size_t)slot * vb);
    B.dt = (T*)(ws + A.dtstore + (size_t)slot * vb);
    rec->zstore = (T*)(ws + A.zstore + (size_t)slot * A.zstep);
    rec->ystore = (T*)(ws + A.ystore + (size_t)slot * A.ystep);
    rec->n = g->n;
    return B;
}

// Forward step from u^n into the record of `slot`: its b, diagonal, every
// z_j and y_k (y_s + u^n is u^{n+1}).
template <typename T>
et_status record_step(et_grid* g, const Schedule& S, double hstep, const double* un, char* ws, const AdjLayout& A,
                      int slot, cudaStream_t st) {
    ChainRecord<T> rec;
    rec.m = S.m;
    Buffers<T> B = slot_buffers<T>(g, ws, A, slot, &rec);
    Weights<double> W64;
    for (int a = 0; a < 5; ++a) W64.w[a] = g->w[a];
    const double dt_shift = (g->scheme == ET_SCHEME_ROSENBROCK ? g->rho : 0.0) - S.mu;
    cudaError_t e;
    if constexpr (std::is_same<T, double>::value) {
        e = launch_residual<T>(g->G, g->op, un, W64, g->rho, dt_shift, 1.0, g->scheme, const_cast<T*>(B.b), B.dt,
                               g->flags, st);
    } else {
        // the residual of the forward step, from the pair of u^n
        e = launch_split(g->n, un, 1.0, g->ush, st);
        if (e == cudaSuccess) e = enqueue_pair_residual<T>(g, g->ush, B, dt_shift, st);
    }
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "residual launch: %s", cudaGetErrorString(e));
    long long launches = 0;
    e = enqueue_chain<T>(g, B, nullptr, S, hstep, st, &launches, &rec);
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "recording launch: %s", cudaGetErrorString(e));
    return ET_OK;
}

// Reverse of one recorded step: given ubar_next = dJ/du^{n+1}, writes ubar =
// dJ/du^n and accumulates the per-voxel rho and D-scale cotangents.
template <typename T>
et_status enqueue_step_adjoint(et_grid* g, const Schedule& S, double hstep, const double* un,
                               const double* ubar_next, double* ubar, char* ws, const AdjLayout& A, int slot,
                               cudaStream_t st) {
    const long long n = g->n;
    Weights<double> W64;
    for (int a = 0; a < 5; ++a) W64.w[a] = g->w[a];
    ChainRecord<T> rec;
    rec.m = S.m;
    Buffers<T> B = slot_buffers<T>(g, ws, A, slot, &rec);
    cudaError_t e;
    // 2. reverse the chain
    T* bbar = (T*)(ws + A.bbar);
    T* cbar = (T*)(ws + A.cbar);
    T* zbar[2] = {(T*)(ws + A.zbar[0]), (T*)(ws + A.zbar[1])};
    T* ybar[2] = {(T*)(ws + A.ybar[0]), (T*)(ws + A.ybar[1])};
    double* sacc = (double*)(ws + A.sacc);
    double* racc = (double*)(ws + A.racc);
    ET_CUDA(g, cudaMemsetAsync(bbar, 0, sizeof(T) * n, st));
    ET_CUDA(g, cudaMemsetAsync(cbar, 0, sizeof(T) * n, st));
    T* sstep = (T*)(ws + A.sstep);
    ET_CUDA(g, cudaMemsetAsync(sstep, 0, sizeof(T) * n, st));
    const T* ynext;  // cotangent of y_{k+1}
    int yi = 0;
    if constexpr (std::is_same<T, double>::value) {
        ynext = ubar_next;
    } else {
        e = launch_cast(n, ubar_next, 1.0, ybar[0], st);
        if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "cast launch: %s", cudaGetErrorString(e));
        ynext = ybar[0];
        yi = 1;
    }
    const ChainPlan P = plan_chain(g, S, hstep);
    Weights<T> WT = B.W;
    WT.w[4] = g->prec == ET_F64 ? (const T*)g->w[4] : (const T*)g->wt[4];
    int zi = 0;
    const T* wprev = nullptr;  // zbar_{j+1} from the previous reverse term
    for (int idx = (int)P.terms.size() - 1; idx >= 0; --idx) {
        const PlannedTerm& t = P.terms[idx];
        const int k = t.k, j = t.j;
        const bool first_reverse = t.last;            // j = m - 1: w = g_m Sbar
        const bool into_b = (k == 0 && j == 1);        // forward input is b
        const bool into_y = (k > 0 && j == 0);         // forward input is y_k
        AdjTermArgs<T> a;
        if (first_reverse) {
            a.wsrc = ynext;
            a.wscale = Scalar<T>::make(t.gnext * P.gamma);
        } else {
            a.wsrc = wprev;
            a.wscale = Scalar<T>::make(1.0);
        }
        a.dt = B.dt;
        a.negR = WT.w[4];
        a.ybar_next = ynext;
        a.gamma = Scalar<T>::make(P.gamma);
        // coefficient of the forward input in the sub-step sum
        // (Horner steps: the input enters the result only through the polynomial)
        double gin;
        if (t.horner) gin = 0.0;
        else if (into_y) gin = 1.0;
        else gin = P.terms[idx - 1].gnext;
        a.g = Scalar<T>::make(gin);
        a.f = Scalar<T>::make(t.zscale_on ? t.zscale_val : 1.0);
        a.inv_nu = Scalar<T>::make(P.inv_nu);
        a.x = into_b ? B.b : (into_y ? rec.y(k) : rec.z(k, j));
        a.has_beta = t.beta != 0.0;
        a.beta = Scalar<T>::make(t.beta);
        a.bbar = bbar;
        a.cbar = cbar;
        a.sstep = sstep;
        a.out_to_bbar = into_b;
        if (into_y) {
            a.zbar_out = ybar[yi];
        } else {
            a.zbar_out = zbar[zi];
        }
        e = launch_adj_term<T>(g->G, g->op, WT, a, st);
        if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "adjoint term launch: %s", cudaGetErrorString(e));
        if (into_y) {
            // ybar_k is the cotangent of the previous sub-step's result
            ynext = ybar[yi];
            yi ^= 1;
        } else if (!into_b) {
            wprev = zbar[zi];
            zi ^= 1;
        }
    }
    // 3. through b = L u + rho u (1 - u) and c = rho (1 - 2u) to u^n, rho, D scale
    e = launch_adj_step<T>(g->G, g->op, W64, un, bbar, cbar, sstep, ubar_next, g->rho, g->scheme, ubar, sacc, racc,
                           st);
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "adjoint step launch: %s", cudaGetErrorString(e));
    return ET_OK;
}

// Forward pass from u (in place) keeping u^0, u^ck, u^2ck, ... as checkpoints;
// all nsteps steps when `full`, else the nsteps - 1 the adjoint needs.
et_status forward_checkpoints(et_grid* g, double* u, double tau, int nsteps, const Schedule& S, char* ws,
                              const AdjLayout& A, bool full) {
    cudaStream_t st = g->stream;
    const long long n = g->n;
    const size_t nb = 8ull * n;
    double* ckpt = (double*)(ws + A.ckpt);
    long long tl = 0, ol = 0;
    ET_CUDA(g, cudaMemcpyAsync(ckpt, u, nb, cudaMemcpyDeviceToDevice, st));
    if (g->ush) {
        const et_status rc = start_pair_copy(g, u, st);
        if (rc != ET_OK) return rc;
    }
    const int last = full ? nsteps : nsteps - 1;
    for (int t = 0; t < last; ++t) {
        et_status rc = enqueue_step(g, u, tau, S, g->info_slot, 0, st, nullptr, nullptr, false, &tl, &ol);
        if (rc != ET_OK) return rc;
        if ((t + 1) % A.ck == 0 && t + 1 < nsteps)
            ET_CUDA(g, cudaMemcpyAsync(ckpt + (size_t)((t + 1) / A.ck) * n, u, nb, cudaMemcpyDeviceToDevice, st));
    }
    return ET_OK;
}

// Reverse pass from the checkpoints: each segment is run forward once with
// every step recorded, then its steps are reversed.
template <typename T>
et_status reverse_from_checkpoints(et_grid* g, double tau, int nsteps, const double* ubar_final, double* ubar0,
                                   double* grad_rho, double* grad_dscale, char* ws, const AdjLayout& A,
                                   const Schedule& S) {
    cudaStream_t st = g->stream;
    const long long n = g->n;
    const size_t nb = 8ull * n;
    const double hstep = tau / S.s;
    const int ck = A.ck;
    double* ckpt = (double*)(ws + A.ckpt);
    double* seg = (double*)(ws + A.seg);
    double* ub[2] = {(double*)(ws + A.ubar[0]), (double*)(ws + A.ubar[1])};
    ET_CUDA(g, cudaMemcpyAsync(ub[0], ubar_final, nb, cudaMemcpyDeviceToDevice, st));
    ET_CUDA(g, cudaMemsetAsync(ws + A.sacc, 0, nb, st));
    ET_CUDA(g, cudaMemsetAsync(ws + A.racc, 0, nb, st));
    int cur = 0;
    for (int sgi = A.nck - 1; sgi >= 0; --sgi) {
        const int n0 = sgi * ck;
        const int n1 = std::min(n0 + ck, nsteps);
        // record the segment's steps; u^{t+1} = u^t + y_s of step t
        ET_CUDA(g, cudaMemcpyAsync(seg, ckpt + (size_t)sgi * n, nb, cudaMemcpyDeviceToDevice, st));
        for (int t = n0; t < n1; ++t) {
            const int slot = t - n0;
            double* ut = seg + (size_t)slot * n;
            et_status rc = record_step<T>(g, S, hstep, ut, ws, A, slot, st);
            if (rc != ET_OK) return rc;
            if (t + 1 < n1) {
                const T* ys = (const T*)(ws + A.ystore + (size_t)slot * A.ystep) + (size_t)S.s * n;
                const cudaError_t e = launch_add_widen<T>(n, ut, ys, ut + n, st);
                if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "state update: %s", cudaGetErrorString(e));
            }
        }
        for (int t = n1 - 1; t >= n0; --t) {
            et_status rc = enqueue_step_adjoint<T>(g, S, hstep, seg + (size_t)(t - n0) * n, ub[cur], ub[cur ^ 1],
                                                   ws, A, t - n0, st);
            if (rc != ET_OK) return rc;
            cur ^= 1;
        }
    }
    ET_CUDA(g, cudaMemcpyAsync(ubar0, ub[cur], nb, cudaMemcpyDeviceToDevice, st));
    double* partial = (double*)(ws + A.partial);
    double* slots = (double*)(ws + A.slots);
    cudaError_t e = launch_sum(n, (double*)(ws + A.racc), partial, slots + 0, st);
    if (e == cudaSuccess) e = launch_sum(n, (double*)(ws + A.sacc), partial, slots + 1, st);
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "reduction launch: %s", cudaGetErrorString(e));
    double host[2] = {0.0, 0.0};
    ET_CUDA(g, cudaMemcpyAsync(host, slots, sizeof(host), cudaMemcpyDeviceToHost, st));
    ET_CUDA(g, cudaStreamSynchronize(st));
    if (grad_rho) *grad_rho = host[0];
    if (grad_dscale) *grad_dscale = host[1];
    return ET_OK;
}

// Common checks of the adjoint entry points; fills the schedule and layout.
et_status adjoint_setup(et_grid* g, double tau, int nsteps, int checkpoint_every, void* workspace,
                        size_t workspace_bytes, Schedule* S, AdjLayout* A) {
    if (!g->coeffs_set) return fail(g, ET_ERR_STATE, "et_set_coeffs has not been called");
    if (g->prec == ET_DF64) return fail(g, ET_ERR_UNSUPPORTED, "the adjoint is provided for ET_F64 and ET_F32");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(g, ET_ERR_ARG, "tau must be finite and > 0");
    if (nsteps < 1 || checkpoint_every < 1) return fail(g, ET_ERR_ARG, "nsteps and checkpoint_every must be >= 1");
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0)
        return fail(g, ET_ERR_ARG, "workspace must be a 256-byte aligned device pointer");
    if (schedule_for(g, tau, S) != ET_OK) return fail(g, ET_ERR_ARG, "no (s, m) for tau = %g", tau);
    adj_layout(g, *S, nsteps, std::min(checkpoint_every, nsteps), A);
    if (workspace_bytes < A->total)
        return fail(g, ET_ERR_ARG, "adjoint workspace has %zu bytes, %zu needed", workspace_bytes, A->total);
    clear_graphs(g);  // the forward steps below run without graphs
    return ET_OK;
}

}  // namespace

namespace et {

// The factor C of the a-posteriori truncation estimate C max|b| / max|u^n| of
// a step with s sub-steps of degree m: the remainder bound that
// et_select_schedule holds below tol, tau e^{2 tau rho'} theta^m / m!
// (1 + tau nu / (m + 1)) / (1 - theta / (m + 1)), without the a-priori bound
// (2 rmax + rho') max|u| on max|b| (which the device measures instead).
// Infinite where theta >= m + 1 (the bound does not converge).
double truncation_factor(double tau, double rmax, double rho, et_scheme scheme, et_precision precision,
                         const et_options* options, int s, int m) {
    const ResolvedOptions o = resolve(options, precision);
    const double rho_c = (scheme == ET_SCHEME_ROSENBROCK) ? rho * (1.0 + 2.0 * kRangeSlack) : 0.0;
    const double nu = o.shift ? rmax + rho_c : 2.0 * rmax + rho_c;
    const double beta = tau * nu;
    const double theta = beta / s;
    if (theta == 0.0) return 0.0;
    if (theta >= m + 1) return INFINITY;
    const double logc = std::log(tau) + 2.0 * tau * rho_c + m * std::log(theta) - std::lgamma(m + 1.0) +
                        std::log1p(beta / (m + 1)) - std::log1p(-theta / (m + 1));
    return std::exp(logc);
}

double resolved_tol(const et_options* options, et_precision precision) { return resolve(options, precision).tol; }

}  // namespace et

namespace {

// Conjugate-gradient iterations that reach a relative residual rtol for
// M = I - tau/2 A_n: with Gershgorin, the eigenvalues of A_n lie in
// [-(2 rmax + rho'), rho'], so those of M in [1 - tau rho'/2, 1 + tau (rmax + rho'/2)];
// the classical bound ||r_k|| <= 2 sqrt(kappa) ((sqrt(kappa) - 1) / (sqrt(kappa) + 1))^k ||r_0||
// then gives the cap (two iterations of margin for rounding).
int cn_cap_of(const et_grid* g, double tau, double rtol) {
    const double rho_c = (g->scheme == ET_SCHEME_ROSENBROCK) ? g->rho * (1.0 + 2.0 * kRangeSlack) : 0.0;
    const double lo = 1.0 - 0.5 * tau * rho_c;
    const double hi = 1.0 + tau * (g->rmax + 0.5 * rho_c);
    const double sk = std::sqrt(hi / lo);
    if (sk <= 1.0 + 1e-12) return 2;
    const double k = std::log(2.0 * sk / rtol) / std::log((sk + 1.0) / (sk - 1.0));
    return (int)std::ceil(k) + 2;
}

// One Crank-Nicolson step on stream st: residual (b_n and the diagonal of
// A_n), the solve of M delta = tau b_n, u += delta, the step record.
et_status enqueue_cn_step(et_grid* g, double* u, double tau, double rtol, int cap, et_step_info* info,
                          int info_stride, cudaStream_t st) {
    double* r = (double*)g->vec[0];
    double* diag = (double*)g->vec[1];
    double* p = (double*)g->vec[2];
    double* q = (double*)g->vec[3];
    double* delta = (double*)g->vec[4];
    Weights<double> W64;
    for (int a = 0; a < 5; ++a) W64.w[a] = g->w[a];
    const double dt_shift = g->scheme == ET_SCHEME_ROSENBROCK ? g->rho : 0.0;  // the diagonal of A_n itself
    cudaError_t e = launch_residual<double>(g->G, g->op, u, W64, g->rho, dt_shift, 1.0, g->scheme, r, diag,
                                            g->flags, st);
    if (e == cudaSuccess) e = launch_cn_init(g->n, tau, r, p, delta, g->cn_sc, g->partial, g->ticket, st);
    const double* w[3] = {g->w[0], g->w[1], g->w[2]};
    for (int it = 0; it < cap && e == cudaSuccess; ++it)
        e = launch_cn_iteration(g->G, w, diag, tau, rtol, r, p, q, delta, g->cn_sc, (double*)g->wnorm, g->partial,
                                g->ticket, st);
    if (e == cudaSuccess) e = launch_cn_finish(g->n, delta, u, g->cn_sc, g->flags, st);
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "Crank-Nicolson launch: %s", cudaGetErrorString(e));
    StatsSink sink;
    sink.partial = g->partial;
    sink.ticket = g->ticket;
    sink.step_counter = g->step_counter;
    sink.flags = g->flags;
    sink.info = info;
    sink.info_stride = info_stride;
    sink.last = g->info_slot;
    sink.s = 0;  // a Crank-Nicolson step: m is its conjugate-gradient iterations
    sink.m = 0;
    sink.m_dev = &g->cn_sc->iters;
    sink.ush = nullptr;
    e = launch_stats(g->G, u, sink, st);
    if (e != cudaSuccess) return fail(g, ET_ERR_CUDA, "stats launch: %s", cudaGetErrorString(e));
    return ET_OK;
}

}  // namespace

extern "C" {

int et_version(void) { return ET_VERSION; }

const char* et_status_string(et_status s) {
    switch (s) {
        case ET_OK: return "ok";
        case ET_ERR_ARG: return "invalid argument";
        case ET_ERR_STATE: return "invalid call order";
        case ET_ERR_CUDA: return "CUDA error";
        case ET_ERR_NUMERIC: return "numeric error";
        case ET_ERR_TIMEOUT: return "device wait timed out";
        case ET_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* et_last_error(const et_grid* g) { return g ? g->err : g_create_error; }

size_t et_workspace_bytes(int nx, int ny, int nz, et_precision precision) {
    if (precision != ET_F64 && precision != ET_F32 && precision != ET_DF64) return 0;
    Layout L;
    if (!make_layout(nx, ny, nz, precision, &L)) return 0;
    return L.total;
}

et_status et_select_schedule(double tau, double rmax, double rho, et_scheme scheme, et_precision precision,
                             const et_options* options, int* s_out, int* m_out, double* mu_out,
                             double* theta_out) {
    if (!(tau > 0.0) || !std::isfinite(tau) || !(rmax >= 0.0) || !std::isfinite(rmax) || !(rho >= 0.0) ||
        !std::isfinite(rho))
        return ET_ERR_ARG;
    const ResolvedOptions o = resolve(options, precision);
    const double rho_c = (scheme == ET_SCHEME_ROSENBROCK) ? rho * (1.0 + 2.0 * kRangeSlack) : 0.0;
    const double mu = o.shift ? -rmax : 0.0;
    const double nu = o.shift ? rmax + rho_c : 2.0 * rmax + rho_c;
    const double beta = tau * nu;
    const double kappa = tau * (2.0 * rmax + rho_c) * std::exp(2.0 * tau * rho_c);
    const int s_lo = o.force_s ? o.force_s : 1, s_hi = o.force_s ? o.force_s : 4096;
    const int m_lo = o.force_m ? o.force_m : 2, m_hi = o.force_m ? o.force_m : 96;
    long long best = std::numeric_limits<long long>::max();
    int bs = 0, bm = 0;
    for (int s = s_lo; s <= s_hi; ++s) {
        if (2ll * s - 1 > best) break;
        const double theta = beta / s;
        if (!o.force_s && theta > o.theta_max) continue;
        for (int m = m_lo; m <= m_hi; ++m) {
            bool ok;
            if (o.force_m) {
                ok = true;
            } else if (kappa == 0.0 || theta == 0.0) {
                ok = true;
            } else if (theta >= m + 1) {
                ok = false;
            } else {
                const double logE = std::log(kappa) + m * std::log(theta) - std::lgamma(m + 1.0) +
                                    std::log1p(beta / (m + 1)) - std::log1p(-theta / (m + 1));
                ok = logE <= std::log(o.tol);
            }
            if (ok) {
                const long long cost = (long long)s * m - 1;
                if (cost < best) {
                    best = cost;
                    bs = s;
                    bm = m;
                }
                break;
            }
        }
    }
    if (!bs) return ET_ERR_ARG;
    if (s_out) *s_out = bs;
    if (m_out) *m_out = bm;
    if (mu_out) *mu_out = mu;
    if (theta_out) *theta_out = beta / bs;
    return ET_OK;
}

et_status et_create_grid(int nx, int ny, int nz, double h, et_precision precision, void* workspace,
                         size_t workspace_bytes, void* cuda_stream, et_grid** out) {
    if (!out) return fail(nullptr, ET_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    if (precision != ET_F64 && precision != ET_F32 && precision != ET_DF64)
        return fail(nullptr, ET_ERR_ARG, "unknown precision");
    Layout L;
    if (!make_layout(nx, ny, nz, precision, &L))
        return fail(nullptr, ET_ERR_ARG, "grid %d x %d x %d is empty or too large", nx, ny, nz);
    if (!(h > 0.0) || !std::isfinite(h)) return fail(nullptr, ET_ERR_ARG, "h must be finite and > 0");
    if (!workspace) return fail(nullptr, ET_ERR_ARG, "workspace must not be NULL");
    if (((uintptr_t)workspace % kAlign) != 0) return fail(nullptr, ET_ERR_ARG, "workspace must be 256-byte aligned");
    if (workspace_bytes < L.total)
        return fail(nullptr, ET_ERR_ARG, "workspace has %zu bytes, %zu needed", workspace_bytes, L.total);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, ET_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    et_grid* g = new (std::nothrow) et_grid();
    if (!g) return fail(nullptr, ET_ERR_ARG, "out of host memory");
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->n = (long long)nx * ny * nz;
    g->h = h;
    g->prec = precision;
    g->device = dev;
    g->ws = (char*)workspace;
    g->ws_bytes = workspace_bytes;
    g->L = L;
    g->G.nx = nx;
    g->G.ny = ny;
    g->G.nz = nz;
    g->G.n = g->n;
    g->G.sy = nx;
    g->G.sz = (long long)nx * ny;
    g->G.nblocks = L.nblocks;
    g->G.sms = 0;
    e = cudaDeviceGetAttribute(&g->G.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = prime_launch_limits();
    if (e != cudaSuccess) {
        delete g;
        return fail(nullptr, ET_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    }
    g->stream = (cudaStream_t)cuda_stream;
    for (int a = 0; a < 5; ++a) g->w[a] = (double*)(g->ws + L.w[a]);
    for (int a = 0; a < 5; ++a) g->wt[a] = precision != ET_F64 ? (void*)(g->ws + L.wt[a]) : nullptr;
    for (int v = 0; v < 6; ++v) g->vec[v] = (void*)(g->ws + L.vec[v]);
    g->stage = (double*)(g->ws + L.stage);
    g->ush = precision != ET_F64 ? (float2*)(g->ws + L.ushadow) : nullptr;
    for (int a = 0; a < 5; ++a)
        g->wres[a] = precision == ET_F32    ? (float2*)(g->ws + L.wpair[a])
                     : precision == ET_DF64 ? (float2*)g->wt[a]
                                            : nullptr;
    g->partial = (double*)(g->ws + L.partial);
    g->pair = nullptr;
    if (precision != ET_F64) {
        const void* wt4[4] = {g->wt[0], g->wt[1], g->wt[2], g->wt[3]};
        const void* yz[4] = {g->vec[2], g->vec[3], g->vec[4], g->vec[5]};
        g->pair = pair_plan_create(g->G, precision, wt4, g->vec[0], g->vec[1], yz);  // nullptr: one term per launch
    }
    char* misc = g->ws + L.misc;
    g->rmax_bits = (unsigned long long*)(misc + 0);
    g->flags = (unsigned*)(misc + 8);
    g->ticket = (unsigned*)(misc + 12);
    g->step_counter = (unsigned*)(misc + 16);
    g->info_slot = (et_step_info*)(misc + 64);
    g->wnorm = (unsigned long long*)(g->ws + L.wnorm);
    g->npartial = (double*)(g->ws + L.npartial);
    g->trunc_est = (double*)(misc + 1024);
    g->cn_sc = (CnScalars*)(misc + 1536);
    g->zrow = (unsigned char*)(g->ws + L.zrow);
    g->zrow_count = (unsigned long long*)(misc + 1600);
    g->cn_exec = nullptr;
    g->cn_u = nullptr;
    g->cn_info = nullptr;
    g->cn_tau = g->cn_rtol = 0.0;
    g->cn_cap = 0;
    g->coeffs_set = false;
    g->rmax = 0.0;
    g->nu = 1.0;
    g->rho = 0.0;
    g->opt_set = false;
    std::memset(&g->opt, 0, sizeof(g->opt));
    g->stamp = 0;
    g->timing = false;
    g->timed_steps = 0;
    g->last_term_launches = g->last_other_launches = 0;
    g->err[0] = 0;
    e = cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        pair_plan_destroy(g->pair);
        delete g;
        return fail(nullptr, ET_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(misc, 0, kMiscBytes, g->stream);
    if (e != cudaSuccess) {
        cudaStreamDestroy(g->capture);
        pair_plan_destroy(g->pair);
        delete g;
        return fail(nullptr, ET_ERR_CUDA, "workspace clear: %s", cudaGetErrorString(e));
    }
    *out = g;
    return ET_OK;
}

et_status et_set_coeffs(et_grid* g, const double* D, double rho, et_operator op, et_scheme scheme,
                        const et_options* options) {
    NvtxRange nvtx_range("et_set_coeffs");
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    if (!D || !aligned8(D)) return fail(g, ET_ERR_ARG, "D must be a non-NULL 8-byte aligned device pointer");
    DeviceGuard dg(g->device);
    return set_coeffs_impl(g, D, rho, op, scheme, options);
}

et_status et_set_coeffs_scaled(et_grid* g, const double* D, double dscale, double rho, et_operator op,
                               et_scheme scheme, const et_options* options) {
    NvtxRange nvtx_range("et_set_coeffs_scaled");
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    if (!D || !aligned8(D)) return fail(g, ET_ERR_ARG, "D must be a non-NULL 8-byte aligned device pointer");
    DeviceGuard dg(g->device);
    return set_coeffs_impl(g, D, rho, op, scheme, options, dscale);
}
et_status et_set_coeffs_host(et_grid* g, const double* D_host, double rho, et_operator op, et_scheme scheme,
                             const et_options* options) {
    NvtxRange nvtx_range("et_set_coeffs_host");
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    if (!D_host) return fail(g, ET_ERR_ARG, "D_host must not be NULL");
    DeviceGuard dg(g->device);
    ET_CUDA(g, cudaMemcpyAsync(g->stage, D_host, 8ull * g->n, cudaMemcpyHostToDevice, g->stream));
    return set_coeffs_impl(g, g->stage, rho, op, scheme, options);
}

et_status et_step(et_grid* g, double* u, double tau, et_step_info* info) {
    NvtxRange nvtx_range("et_step");
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    DeviceGuard dg(g->device);
    return run_impl(g, u, tau, 1, info);
}

et_status et_run(et_grid* g, double* u, double tau, int nsteps, et_step_info* info) {
    NvtxRange nvtx_range("et_run");
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    DeviceGuard dg(g->device);
    return run_impl(g, u, tau, nsteps, info);
}

et_status et_run_host(et_grid* g, double* u_host, double tau, int nsteps, et_step_info* info_host) {
    NvtxRange nvtx_range("et_run_host");
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    if (!u_host) return fail(g, ET_ERR_ARG, "u_host must not be NULL");
    if (nsteps < 1) return fail(g, ET_ERR_ARG, "nsteps must be >= 1");
    DeviceGuard dg(g->device);
    if (!g->coeffs_set) return fail(g, ET_ERR_STATE, "et_set_coeffs has not been called");
    ET_CUDA(g, cudaMemcpyAsync(g->stage, u_host, 8ull * g->n, cudaMemcpyHostToDevice, g->stream));
    // records go to the internal slot (last step); per-step records need a device array
    et_status rc = run_impl(g, g->stage, tau, nsteps, nullptr);
    if (rc != ET_OK) return rc;
    ET_CUDA(g, cudaMemcpyAsync(u_host, g->stage, 8ull * g->n, cudaMemcpyDeviceToHost, g->stream));
    return et_sync_info(g, info_host);
}

et_status et_sync_info(et_grid* g, et_step_info* host_out) {
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    DeviceGuard dg(g->device);
    et_step_info rec;
    unsigned flags = 0;
    ET_CUDA(g, cudaMemcpyAsync(&rec, g->info_slot, sizeof(rec), cudaMemcpyDeviceToHost, g->stream));
    ET_CUDA(g, cudaMemcpyAsync(&flags, g->flags, sizeof(flags), cudaMemcpyDeviceToHost, g->stream));
    ET_CUDA(g, cudaStreamSynchronize(g->stream));
    ET_CUDA(g, cudaMemsetAsync(g->flags, 0, sizeof(unsigned), g->stream));
    if (host_out) *host_out = rec;
    if (flags & ET_FLAG_TIMEOUT) return fail(g, ET_ERR_TIMEOUT, "a device-side wait ran out; the run is not valid");
    if (flags & ET_FLAG_NONFINITE) return fail(g, ET_ERR_NUMERIC, "non-finite density met");
    if (flags & ET_FLAG_CG_CAP)
        return fail(g, ET_ERR_NUMERIC, "a Crank-Nicolson solve reached its iteration cap before its tolerance");
    if (flags & ET_FLAG_RANGE_IN)
        return fail(g, ET_ERR_NUMERIC, "density outside [0, 1] (+-1e-3): the step bound does not hold");
    return ET_OK;
}

et_status et_cn_run(et_grid* g, double* u, double tau, int nsteps, double rtol, int max_iter, et_step_info* info) {
    NvtxRange nvtx_range("et_cn_run");
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    if (!g->coeffs_set) return fail(g, ET_ERR_STATE, "et_set_coeffs has not been called");
    if (g->prec != ET_F64) return fail(g, ET_ERR_UNSUPPORTED, "Crank-Nicolson steps run on ET_F64 grids");
    if (g->op != ET_OP_CONSERVATIVE)
        return fail(g, ET_ERR_UNSUPPORTED, "Crank-Nicolson steps need the conservative (symmetric) operator");
    if (!u || !aligned8(u)) return fail(g, ET_ERR_ARG, "u must be a non-NULL 8-byte aligned device pointer");
    if (info && !aligned8(info)) return fail(g, ET_ERR_ARG, "info must be 8-byte aligned");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(g, ET_ERR_ARG, "tau must be finite and > 0");
    if (g->scheme == ET_SCHEME_ROSENBROCK && !(0.5 * tau * g->rho * (1.0 + 2.0 * kRangeSlack) < 1.0))
        return fail(g, ET_ERR_ARG, "tau rho must be below 2 (I - tau/2 A is then positive definite)");
    if (nsteps < 1) return fail(g, ET_ERR_ARG, "nsteps must be >= 1");
    if (!(rtol > 0.0 && rtol < 1.0)) return fail(g, ET_ERR_ARG, "rtol must be in (0, 1)");
    if (max_iter < 0 || max_iter > 100000) return fail(g, ET_ERR_ARG, "max_iter must be in [0, 100000]");
    DeviceGuard dg(g->device);
    const int cap = max_iter > 0 ? max_iter : cn_cap_of(g, tau, rtol);
    et_step_info* dst = info ? info : g->info_slot;
    const int stride = info ? 1 : 0;
    ET_CUDA(g, cudaMemsetAsync(g->step_counter, 0, sizeof(unsigned), g->stream));
    ET_CUDA(g, prime_launch_limits());
    const ResolvedOptions ro = resolve(g->opt_set ? &g->opt : nullptr, g->prec);
    if (!ro.use_graph) {
        for (int t = 0; t < nsteps; ++t) {
            const et_status rc = enqueue_cn_step(g, u, tau, rtol, cap, dst, stride, g->stream);
            if (rc != ET_OK) return rc;
        }
        return ET_OK;
    }
    // one step captured once and replayed: the step index comes from the device
    const CoeffKey key = coeff_key(g);
    const bool same = g->cn_exec && g->cn_u == u && g->cn_info == dst && g->cn_tau == tau && g->cn_rtol == rtol &&
                      g->cn_cap == cap && same_coeffs(g->cn_key, key);
    if (!same) {
        if (g->cn_exec) cudaGraphExecDestroy(g->cn_exec);
        g->cn_exec = nullptr;
        ET_CUDA(g, cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal));
        const et_status rc = enqueue_cn_step(g, u, tau, rtol, cap, dst, stride, g->capture);
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(g->capture, &graph);
        if (rc != ET_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ce != cudaSuccess) return fail(g, ET_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&g->cn_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            g->cn_exec = nullptr;
            return fail(g, ET_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        }
        g->cn_u = u;
        g->cn_info = dst;
        g->cn_tau = tau;
        g->cn_rtol = rtol;
        g->cn_cap = cap;
        g->cn_key = key;
    }
    for (int t = 0; t < nsteps; ++t) ET_CUDA(g, cudaGraphLaunch(g->cn_exec, g->stream));
    return ET_OK;
}

int et_cn_iteration_cap(const et_grid* g, double tau, double rtol) {
    if (!g || !g->coeffs_set || !(tau > 0.0) || !(rtol > 0.0 && rtol < 1.0)) return 0;
    return cn_cap_of(g, tau, rtol);
}

et_status et_get_zero_rows(et_grid* g, long long* voxels) {
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    if (!voxels) return fail(g, ET_ERR_ARG, "voxels must not be NULL");
    if (!g->coeffs_set) return fail(g, ET_ERR_STATE, "et_set_coeffs has not been called");
    DeviceGuard dg(g->device);
    unsigned long long c = 0;
    ET_CUDA(g, cudaMemcpyAsync(&c, g->zrow_count, sizeof(c), cudaMemcpyDeviceToHost, g->stream));
    ET_CUDA(g, cudaStreamSynchronize(g->stream));
    *voxels = (long long)c;
    return ET_OK;
}

et_status et_get_truncation(et_grid* g, double* estimate) {
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    if (!estimate) return fail(g, ET_ERR_ARG, "estimate must not be NULL");
    DeviceGuard dg(g->device);
    double est = 0.0;
    ET_CUDA(g, cudaMemcpyAsync(&est, g->trunc_est, sizeof(est), cudaMemcpyDeviceToHost, g->stream));
    ET_CUDA(g, cudaStreamSynchronize(g->stream));
    *estimate = est;
    return ET_OK;
}

et_status et_get_schedule(const et_grid* g, double tau, int* s, int* m, double* mu, double* theta) {
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    if (!g->coeffs_set) return fail(const_cast<et_grid*>(g), ET_ERR_STATE, "et_set_coeffs has not been called");
    Schedule S;
    et_status rc = schedule_for(g, tau, &S);
    if (rc != ET_OK) return fail(const_cast<et_grid*>(g), rc, "no (s, m) for tau = %g", tau);
    if (s) *s = S.s;
    if (m) *m = S.m;
    if (mu) *mu = S.mu;
    if (theta) *theta = S.theta;
    return ET_OK;
}

et_status et_set_stream(et_grid* g, void* cuda_stream) {
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    g->stream = (cudaStream_t)cuda_stream;
    return ET_OK;
}

et_status et_enable_timing(et_grid* g, int enable) {
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    DeviceGuard dg(g->device);
    if ((bool)enable != g->timing) {
        clear_graphs(g);
        if (!enable) clear_events(g);
        g->timing = enable != 0;
    }
    return ET_OK;
}

et_status et_get_timing(et_grid* g, double* term_ms, long long* term_launches, long long* other_launches) {
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    DeviceGuard dg(g->device);
    double total = 0.0;
    if (g->timing && g->timed_steps > 0) {
        ET_CUDA(g, cudaStreamSynchronize(g->stream));
        for (int t = 0; t < g->timed_steps; ++t) {
            float ms = 0.f;
            ET_CUDA(g, cudaEventElapsedTime(&ms, g->ev[2 * t], g->ev[2 * t + 1]));
            total += ms;
        }
    }
    if (term_ms) *term_ms = total;
    if (term_launches) *term_launches = g->last_term_launches;
    if (other_launches) *other_launches = g->last_other_launches;
    return ET_OK;
}

et_status et_get_info(const et_grid* g, long long* nvoxels, size_t* ws_used, double* rmax) {
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    if (nvoxels) *nvoxels = g->n;
    if (ws_used) *ws_used = g->L.total;
    if (rmax) *rmax = g->coeffs_set ? g->rmax : 0.0;
    return ET_OK;
}

size_t et_vjp_workspace_bytes(const et_grid* g, double tau, int nsteps, int checkpoint_every) {
    if (!g || !g->coeffs_set || nsteps < 1 || checkpoint_every < 1) return 0;
    Schedule S;
    if (schedule_for(g, tau, &S) != ET_OK) return 0;
    AdjLayout A;
    adj_layout(g, S, nsteps, std::min(checkpoint_every, nsteps), &A);
    return A.total;
}

et_status et_vjp(et_grid* g, const double* u0, double tau, int nsteps, int checkpoint_every,
                 const double* ubar_final, double* ubar0, double* grad_rho, double* grad_dscale,
                 void* workspace, size_t workspace_bytes) {
    NvtxRange nvtx_range("et_vjp");
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    DeviceGuard dg(g->device);
    if (!u0 || !ubar_final || !ubar0 || !aligned8(u0) || !aligned8(ubar_final) || !aligned8(ubar0))
        return fail(g, ET_ERR_ARG, "u0, ubar_final and ubar0 must be 8-byte aligned device pointers");
    Schedule S;
    AdjLayout A;
    et_status rc = adjoint_setup(g, tau, nsteps, checkpoint_every, workspace, workspace_bytes, &S, &A);
    if (rc != ET_OK) return rc;
    char* ws = (char*)workspace;
    // the checkpoint pass runs on the first segment-state slot
    double* u = (double*)(ws + A.seg);
    ET_CUDA(g, cudaMemcpyAsync(u, u0, 8ull * g->n, cudaMemcpyDeviceToDevice, g->stream));
    rc = forward_checkpoints(g, u, tau, nsteps, S, ws, A, false);
    if (rc != ET_OK) return rc;
    if (g->prec == ET_F64)
        return reverse_from_checkpoints<double>(g, tau, nsteps, ubar_final, ubar0, grad_rho, grad_dscale, ws, A, S);
    return reverse_from_checkpoints<float>(g, tau, nsteps, ubar_final, ubar0, grad_rho, grad_dscale, ws, A, S);
}

et_status et_run_checkpointed(et_grid* g, double* u, double tau, int nsteps, int checkpoint_every, void* workspace,
                              size_t workspace_bytes) {
    NvtxRange nvtx_range("et_run_checkpointed");
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    DeviceGuard dg(g->device);
    if (!u || !aligned8(u)) return fail(g, ET_ERR_ARG, "u must be an 8-byte aligned device pointer");
    Schedule S;
    AdjLayout A;
    et_status rc = adjoint_setup(g, tau, nsteps, checkpoint_every, workspace, workspace_bytes, &S, &A);
    if (rc != ET_OK) return rc;
    return forward_checkpoints(g, u, tau, nsteps, S, (char*)workspace, A, true);
}

et_status et_vjp_checkpointed(et_grid* g, double tau, int nsteps, int checkpoint_every, const double* ubar_final,
                              double* ubar0, double* grad_rho, double* grad_dscale, void* workspace,
                              size_t workspace_bytes) {
    NvtxRange nvtx_range("et_vjp_checkpointed");
    if (!g) return fail(nullptr, ET_ERR_ARG, "grid is NULL");
    DeviceGuard dg(g->device);
    if (!ubar_final || !ubar0 || !aligned8(ubar_final) || !aligned8(ubar0))
        return fail(g, ET_ERR_ARG, "ubar_final and ubar0 must be 8-byte aligned device pointers");
    Schedule S;
    AdjLayout A;
    et_status rc = adjoint_setup(g, tau, nsteps, checkpoint_every, workspace, workspace_bytes, &S, &A);
    if (rc != ET_OK) return rc;
    char* ws = (char*)workspace;
    if (g->prec == ET_F64)
        return reverse_from_checkpoints<double>(g, tau, nsteps, ubar_final, ubar0, grad_rho, grad_dscale, ws, A, S);
    return reverse_from_checkpoints<float>(g, tau, nsteps, ubar_final, ubar0, grad_rho, grad_dscale, ws, A, S);
}

void et_destroy(et_grid* g) {
    if (!g) return;
    {
        DeviceGuard dg(g->device);
        clear_graphs(g);
        clear_events(g);
        if (g->cn_exec) cudaGraphExecDestroy(g->cn_exec);
        if (g->capture) cudaStreamDestroy(g->capture);
    }
    pair_plan_destroy(g->pair);
    delete g;
}

}  // extern "C"
