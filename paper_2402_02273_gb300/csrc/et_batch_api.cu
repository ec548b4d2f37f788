// Batched form of the C ABI (include/et.h, et_batch_*): many grids of
// different sizes, each with its own diffusion field, proliferation rate and
// (s, m) schedule, advanced together.  Every step is one batched residual
// launch, one batched launch per Taylor-term index (covering every grid that
// has that term) and one batched stats launch; the whole run is captured as
// one CUDA graph.  The kernel variant of the term launches (planes per tile,
// looping blocks or one tile per block) is chosen by timing the candidates on
// the batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "et.h"
#include "et_chain.h"
#include "et_internal.h"
#include "et_plan.h"

using namespace et;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxBatch = 1024;
constexpr int kMaxTermLaunches = 1024;  // per step
thread_local char g_batch_error[512] = "";

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
size_t value_bytes(et_precision prec) { return prec == ET_F32 ? 4 : 8; }
// flags, per-grid rmax bits, tickets and step counters, per-grid step records,
// then per grid the truncation estimate
size_t misc_head_bytes(int count) { return 128ull * count + 1024; }
size_t misc_bytes(int count) { return misc_head_bytes(count) + 64ull * count; }

size_t term_desc_bytes(et_precision prec) {
    return prec == ET_F64 ? sizeof(BatchTerm<double>)
                          : (prec == ET_F32 ? sizeof(BatchTerm<float>) : sizeof(BatchTerm<float2>));
}
size_t pair_desc_bytes(et_precision prec) {
    return prec == ET_F64 ? 0 : (prec == ET_F32 ? sizeof(BatchPair<float>) : sizeof(BatchPair<float2>));
}
// F32 Horner pairs on the four-voxel two-term kernel
size_t qpair_desc_bytes(et_precision prec) { return prec == ET_F32 ? sizeof(VecPairGrid<float>) : 0; }
// Per grid: up to kMaxTermLaunches single terms, or half as many pairs, plus
// its residual and stats descriptors.
size_t desc_bytes_per_instance(et_precision prec) {
    const size_t res = prec == ET_F64 ? sizeof(BatchResidual<double>)
                                      : (prec == ET_F32 ? sizeof(BatchResidual<float>) : sizeof(BatchResidual<float2>));
    return (size_t)kMaxTermLaunches * term_desc_bytes(prec) +
           (size_t)(kMaxTermLaunches / 2) * (pair_desc_bytes(prec) + qpair_desc_bytes(prec)) + res +
           sizeof(BatchStats) + 128;
}

struct BatchLayout {
    // wpair: F32 pair weights of the residual; ush: F32 / DF64 pair copy of u
    // wnorm: the residual warps' norm slots (2 per warp, 8 warps per residual
    // tile of every grid); npartial: per grid the stats blocks' maxima of them
    // zrow: per grid one byte per warp row without off-diagonal entries
    // (Weights::zrow), zcount: per grid the voxels of those rows
    size_t w[5], wt[5], wpair[5], vec[6], stage, ush, partial, wnorm, npartial, desc, tune_desc, misc, zrow, zcount;
    size_t total;
    long long ntot;
    long long res_tiles;  // 32 x 8 residual tiles of all grids
};

bool batch_layout(int count, const int* dims, et_precision prec, BatchLayout* L, std::vector<long long>* offs,
                  std::vector<long long>* zoffs = nullptr) {
    if (count < 1 || count > kMaxBatch || !dims) return false;
    long long ntot = 0, res_tiles = 0, zbytes = 0;
    offs->assign(count + 1, 0);
    if (zoffs) zoffs->assign(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        const int nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
        if (nx <= 0 || ny <= 0 || nz <= 0) return false;
        const long long n = (long long)nx * ny * nz;
        (*offs)[i] = ntot;
        ntot += n;
        res_tiles += (long long)((nx + kBlockX - 1) / kBlockX) * ((ny + kBlockY - 1) / kBlockY) * nz;
        if (zoffs) (*zoffs)[i] = zbytes;
        zbytes += (long long)((nx + kBlockX - 1) / kBlockX) * ny * nz;
    }
    if (zoffs) (*zoffs)[count] = zbytes;
    L->res_tiles = res_tiles;
    (*offs)[count] = ntot;
    if (ntot >= (1ll << 40)) return false;
    L->ntot = ntot;
    const size_t vb = value_bytes(prec);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    for (int a = 0; a < 5; ++a) L->w[a] = take(8ull * ntot);
    for (int a = 0; a < 5; ++a) L->wt[a] = (prec != ET_F64) ? take(vb * ntot) : SIZE_MAX;
    for (int a = 0; a < 5; ++a) L->wpair[a] = (prec == ET_F32) ? take(8ull * ntot) : SIZE_MAX;
    for (int v = 0; v < 6; ++v) L->vec[v] = take(vb * ntot);
    L->stage = take(8ull * ntot);
    L->ush = (prec != ET_F64) ? take(8ull * ntot) : SIZE_MAX;
    L->partial = take(3ull * 8ull * kStatsBlocks * count);
    L->wnorm = take(2ull * 8ull * kBlockY * (unsigned long long)L->res_tiles);
    L->npartial = take(2ull * 8ull * kStatsBlocks * count);
    L->desc = take(desc_bytes_per_instance(prec) * count);
    L->tune_desc = take((term_desc_bytes(prec) + pair_desc_bytes(prec) + qpair_desc_bytes(prec)) * count + 256);
    L->misc = take(misc_bytes(count));
    L->zrow = take((size_t)zbytes);
    L->zcount = take(8ull * count);
    L->total = off;
    return true;
}

struct Sched {
    int s = 0, m = 0;
    double mu = 0.0, theta = 0.0;
};

}  // namespace

struct et_batch {
    int count;
    std::vector<int> dims;
    std::vector<long long> offs;
    std::vector<long long> zoffs;  // per grid: byte offset of its zero-row flags
    long long ntot;
    double h;
    et_precision prec;
    int device, sms;
    char* ws;
    size_t ws_bytes;
    BatchLayout L;
    cudaStream_t stream, capture;
    // model
    bool coeffs_set;
    et_operator op;
    et_scheme scheme;
    std::vector<double> rho, rmax, nu;
    et_options opt;
    bool opt_set;
    // tables and graph
    double table_tau;
    int table_variant;
    int nlaunch;                         // term launches per step
    // per launch index of a step: single-term descriptors (count, tiles, first)
    // and two-term descriptors (count, tiles, first)
    std::vector<int> single_count, pair_count, qpair_count;
    std::vector<long long> single_tiles, pair_tiles, single_first, pair_first, qpair_tiles, qpair_first;
    size_t pair_table_offset;              // byte offset of the two-term descriptors
    size_t qpair_table_offset;             // byte offset of the four-voxel two-term descriptors (F32)
    std::vector<PairPlan*> pair_plans;     // per grid (F32 / DF64), nullptr: one term per launch
    long long res_tiles;
    double graph_tau;
    int graph_steps;
    double* graph_u;
    et_step_info* graph_info;
    int graph_variant;
    cudaGraphExec_t exec;
    int variant;  // autotuned kernel variant (-1: not tuned yet)
    char err[512];
};

namespace {

et_status bfail(et_batch* b, et_status st, const char* fmt, ...) {
    char* dst = b ? b->err : g_batch_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return st;
}

#define BT_CUDA(b, call)                                                                        \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return bfail((b), ET_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

struct BDeviceGuard {
    int prev = -1;
    explicit BDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~BDeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

Geom geom_of(const et_batch* b, int i) {
    Geom G;
    G.nx = b->dims[3 * i];
    G.ny = b->dims[3 * i + 1];
    G.nz = b->dims[3 * i + 2];
    G.n = (long long)G.nx * G.ny * G.nz;
    G.sy = G.nx;
    G.sz = (long long)G.nx * G.ny;
    G.nblocks = (unsigned)(((G.nx + kBlockX - 1) / kBlockX) * ((G.ny + kBlockY - 1) / kBlockY) * G.nz);
    G.sms = b->sms;
    return G;
}

long long tiles_of(const Geom& G, int tz) {
    return (long long)((G.nx + kBlockX - 1) / kBlockX) * ((G.ny + kBlockY - 1) / kBlockY) * ((G.nz + tz - 1) / tz);
}

char* misc(et_batch* b) { return b->ws + b->L.misc; }
unsigned* flags_of(et_batch* b) { return (unsigned*)(misc(b) + 0); }
unsigned long long* rmax_bits_of(et_batch* b, int i) { return (unsigned long long*)(misc(b) + 64 + 8ull * i); }
double* trunc_est_of(et_batch* b, int i) { return (double*)(misc(b) + misc_head_bytes(b->count) + 64ull * i); }
unsigned* ticket_of(et_batch* b, int i) { return (unsigned*)(misc(b) + 64 + 8ull * b->count + 8ull * i); }
unsigned* counter_of(et_batch* b, int i) { return ticket_of(b, i) + 1; }
et_step_info* slot_of(et_batch* b, int i) {
    return (et_step_info*)(misc(b) + align_up(64 + 16ull * b->count) + 64ull * i);
}

template <typename T>
T* field(et_batch* b, size_t region, int i) {
    return (T*)(b->ws + region) + b->offs[i];
}

// Pair weight a of grid i read by the F32 / DF64 residual.
float2* pair_weight(et_batch* b, int a, int i) {
    return field<float2>(b, b->prec == ET_F32 ? b->L.wpair[a] : b->L.wt[a], i);
}

et_status sched_of(const et_batch* b, int i, double tau, Sched* S) {
    const et_status rc = et_select_schedule(tau, b->rmax[i], b->rho[i], b->scheme, b->prec,
                                            b->opt_set ? &b->opt : nullptr, &S->s, &S->m, &S->mu, &S->theta);
    return rc;
}

template <typename T>
Weights<T> typed_weights(et_batch* b, int i) {
    Weights<T> W;
    for (int a = 0; a < 5; ++a)
        W.w[a] = b->prec == ET_F64 ? (const T*)field<double>(b, b->L.w[a], i) : field<T>(b, b->L.wt[a], i);
    // the one-term kernels skip the warp rows without off-diagonal entries
    // (their products all have zero weights) unless every row is asked for
    const bool every_row = b->opt_set && b->opt.every_row != 0;
    W.zrow = every_row ? nullptr : (const unsigned char*)(b->ws + b->L.zrow) + b->zoffs[i];
    return W;
}

// Kernel variants: the single-term variants of batch_variant (planes per tile,
// looping blocks) and, for F32 / DF64, each of them again with two-term
// launches (the first half of the index range).
int total_variants(et_precision prec) {
    return prec == ET_F64 ? batch_variant_count(prec) : 2 * batch_variant_count(prec);
}
bool variant_pairs(et_precision prec, int v) { return prec != ET_F64 && v < batch_variant_count(prec); }
int single_variant(et_precision prec, int v) { return v % batch_variant_count(prec); }

size_t align64(size_t x) { return (x + 63) / 64 * 64; }

// Host-side tables of one step: the residual and stats descriptors of every
// grid, then for every launch index l the single-term and the two-term
// descriptors of the grids whose chain has an l-th launch.  tuning: the step
// result goes to the staging field instead of u.
template <typename T>
et_status build_tables(et_batch* b, double* u, double tau, int variant, std::vector<char>& bytes, bool tuning) {
    const int C = b->count;
    const int tz = batch_variant(b->prec, single_variant(b->prec, variant)).tile_z;
    const bool want_pairs = variant_pairs(b->prec, variant) && !(b->opt_set && b->opt.single_terms > 0);
    std::vector<Sched> S(C);
    std::vector<ChainPlan> plans(C);
    for (int i = 0; i < C; ++i) {
        if (sched_of(b, i, tau, &S[i]) != ET_OK)
            return bfail(b, ET_ERR_ARG, "no (s, m) meets the tolerance for grid %d at tau = %g", i, tau);
        plans[i] = plan_chain(b->prec, b->nu[i], S[i].s, S[i].m, S[i].mu, tau / S[i].s);
        if ((int)plans[i].terms.size() > kMaxTermLaunches)
            return bfail(b, ET_ERR_UNSUPPORTED, "more than %d terms per step", kMaxTermLaunches);
    }
    // residual descriptors
    std::vector<BatchResidual<T>> res(C);
    long long rt = 0;
    for (int i = 0; i < C; ++i) {
        BatchResidual<T>& r = res[i];
        r.G = geom_of(b, i);
        r.u = u + b->offs[i];
        for (int a = 0; a < 5; ++a) r.W.w[a] = field<double>(b, b->L.w[a], i);
        // the FP64 residual skips the products of zero rows as the term chain does
        r.W.zrow = b->prec == ET_F64 ? typed_weights<T>(b, i).zrow : nullptr;
        r.rho = b->rho[i];
        r.dt_shift = (b->scheme == ET_SCHEME_ROSENBROCK ? b->rho[i] : 0.0) - S[i].mu;
        r.dt_scale = b->prec == ET_F64 ? 1.0 : 1.0 / b->nu[i];
        std::memset(&r.P, 0, sizeof(r.P));
        if (b->prec != ET_F64) {
            float2* wres[5];
            for (int a = 0; a < 5; ++a) wres[a] = pair_weight(b, a, i);
            r.P = pair_residual_args(field<float2>(b, b->L.ush, i), wres, b->nu[i], b->rho[i], r.dt_shift, b->scheme);
            r.P.W.zrow = typed_weights<T>(b, i).zrow;  // zero rows skipped as in the term chain
        }
        r.b = field<T>(b, b->L.vec[0], i);
        r.dt = field<T>(b, b->L.vec[1], i);
        r.wnorm = tuning ? nullptr : (unsigned long long*)(b->ws + b->L.wnorm);
        r.tile_begin = rt;
        rt += tiles_of(r.G, 1);
    }
    b->res_tiles = rt;
    // every grid runs its own chain, launch by launch
    std::vector<std::vector<ChainOp<T>>> ops(C);
    int nl = 0;
    for (int i = 0; i < C; ++i) {
        T* const Y[2] = {field<T>(b, b->L.vec[2], i), field<T>(b, b->L.vec[3], i)};
        T* const Z[2] = {field<T>(b, b->L.vec[4], i), field<T>(b, b->L.vec[5], i)};
        double* ui = tuning ? field<double>(b, b->L.stage, i) : u + b->offs[i];
        const bool pairs = want_pairs && b->pair_plans[i] != nullptr;
        ops[i] = chain_ops<T>(plans[i], S[i].s, field<T>(b, b->L.vec[0], i), field<T>(b, b->L.vec[1], i), Y, Z, ui,
                              pairs);
        nl = std::max(nl, (int)ops[i].size());
    }
    b->nlaunch = nl;
    b->single_count.assign(nl, 0);
    b->pair_count.assign(nl, 0);
    b->single_tiles.assign(nl, 0);
    b->pair_tiles.assign(nl, 0);
    b->single_first.assign(nl, 0);
    b->pair_first.assign(nl, 0);
    b->qpair_count.assign(nl, 0);
    b->qpair_tiles.assign(nl, 0);
    b->qpair_first.assign(nl, 0);
    std::vector<BatchTerm<T>> singles;
    std::vector<BatchPair<T>> pairs;
    std::vector<VecPairGrid<T>> qpairs;
    for (int l = 0; l < nl; ++l) {
        b->single_first[l] = (long long)singles.size();
        b->pair_first[l] = (long long)pairs.size();
        b->qpair_first[l] = (long long)qpairs.size();
        long long st = 0, pt = 0, qt = 0;
        for (int i = 0; i < C; ++i) {
            if (l >= (int)ops[i].size()) continue;
            const ChainOp<T>& op = ops[i][l];
            bool quad = false;
            if constexpr (std::is_same<T, float>::value) {
                // FP32 Horner pairs: the vector two-term kernel where it applies
                const Geom G = geom_of(b, i);
                const Weights<T> W = typed_weights<T>(b, i);
                if (op.pair && vec_pair_eligible<T>(G, b->op, W, op.a1, op.a2)) {
                    const int tz = G.nz < 32 ? G.nz : 32;
                    qpairs.push_back(vec_pair_grid<T>(G, W, op.a1, op.a2, tz, qt));
                    qt += vec_pair_tiles<T>(G, tz);
                    quad = true;
                }
            }
            if (quad) continue;
            if (op.pair) {
                BatchPair<T> d;
                std::memset(&d, 0, sizeof(d));
                if (!pair_maps(b->pair_plans[i], op.a1.zin, &d.M))
                    return bfail(b, ET_ERR_UNSUPPORTED, "grid %d: no tensor map for a two-term launch", i);
                d.G = geom_of(b, i);
                d.a1 = op.a1;
                d.a2 = op.a2;
                d.tz = batch_pair_tz(d.G);
                d.tile_begin = pt;
                pt += tiles_of(d.G, d.tz);
                pairs.push_back(d);
            } else {
                BatchTerm<T> d;
                std::memset(&d, 0, sizeof(d));
                d.G = geom_of(b, i);
                d.W = typed_weights<T>(b, i);
                d.a = op.a1;
                d.tile_begin = st;
                st += tiles_of(d.G, tz);
                singles.push_back(d);
            }
        }
        b->single_count[l] = (int)((long long)singles.size() - b->single_first[l]);
        b->pair_count[l] = (int)((long long)pairs.size() - b->pair_first[l]);
        b->single_tiles[l] = st;
        b->pair_tiles[l] = pt;
        b->qpair_count[l] = (int)((long long)qpairs.size() - b->qpair_first[l]);
        b->qpair_tiles[l] = qt;
    }
    // stats descriptors
    std::vector<BatchStats> stv(C);
    for (int i = 0; i < C; ++i) {
        stv[i].n = geom_of(b, i).n;
        stv[i].u = u + b->offs[i];
        StatsSink& sk = stv[i].sink;
        sk.partial = (double*)(b->ws + b->L.partial) + 3ull * kStatsBlocks * i;
        sk.ticket = ticket_of(b, i);
        sk.step_counter = counter_of(b, i);
        sk.flags = flags_of(b);
        sk.info = nullptr;  // set per run
        sk.info_stride = 0;
        sk.last = slot_of(b, i);
        sk.s = S[i].s;
        sk.m = S[i].m;
        sk.ush = b->prec != ET_F64 ? field<float2>(b, b->L.ush, i) : nullptr;
        sk.wnorm = tuning ? nullptr : (unsigned long long*)(b->ws + b->L.wnorm) + 2ll * kBlockY * res[i].tile_begin;
        sk.nwarps = (long long)kBlockY * tiles_of(res[i].G, 1);
        sk.npartial = (double*)(b->ws + b->L.npartial) + 2ull * kStatsBlocks * i;
        sk.trunc_c = truncation_factor(tau, b->rmax[i], b->rho[i], b->scheme, b->prec, b->opt_set ? &b->opt : nullptr,
                                       S[i].s, S[i].m);
        sk.trunc_tol = resolved_tol(b->opt_set ? &b->opt : nullptr, b->prec);
        sk.trunc_est = trunc_est_of(b, i);
    }
    // [residual x C][stats x C][single terms][pad to 64 bytes][two-term]
    // [pad][four-voxel two-term]
    const size_t head = sizeof(BatchResidual<T>) * C + sizeof(BatchStats) * C;
    b->pair_table_offset = align64(head + sizeof(BatchTerm<T>) * singles.size());
    b->qpair_table_offset = align64(b->pair_table_offset + sizeof(BatchPair<T>) * pairs.size());
    bytes.assign(b->qpair_table_offset + sizeof(VecPairGrid<T>) * qpairs.size(), 0);
    char* p = bytes.data();
    std::memcpy(p, res.data(), sizeof(BatchResidual<T>) * C);
    std::memcpy(p + sizeof(BatchResidual<T>) * C, stv.data(), sizeof(BatchStats) * C);
    if (!singles.empty()) std::memcpy(p + head, singles.data(), sizeof(BatchTerm<T>) * singles.size());
    if (!pairs.empty()) std::memcpy(p + b->pair_table_offset, pairs.data(), sizeof(BatchPair<T>) * pairs.size());
    if (!qpairs.empty())
        std::memcpy(p + b->qpair_table_offset, qpairs.data(), sizeof(VecPairGrid<T>) * qpairs.size());
    return ET_OK;
}

// The launches of launch index l from a table at dtab (single terms at
// dtab + head, two-term descriptors at dtab + pair_table_offset).
template <typename T>
cudaError_t launch_index(et_batch* b, const char* dsingles, const char* dpairs, const char* dqpairs, int l,
                         int variant, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (b->single_count[l] > 0)
        e = launch_batch_term(b->op, single_variant(b->prec, variant),
                              reinterpret_cast<const BatchTerm<T>*>(dsingles) + b->single_first[l], b->single_count[l],
                              b->single_tiles[l], b->sms, st);
    if constexpr (!std::is_same<T, double>::value) {
        if (e == cudaSuccess && b->pair_count[l] > 0)
            e = launch_batch_term_pair<T>(b->op, reinterpret_cast<const BatchPair<T>*>(dpairs) + b->pair_first[l],
                                          b->pair_count[l], b->pair_tiles[l], b->sms, flags_of(b), st,
                                          b->opt_set && b->opt.timeout_probe_us > 0
                                              ? 1000ull * (unsigned long long)b->opt.timeout_probe_us
                                              : 0ull);
        if constexpr (std::is_same<T, float>::value) {
            if (e == cudaSuccess && b->qpair_count[l] > 0)
                e = launch_batch_term_vec_pair<T>(b->op,
                                                  reinterpret_cast<const VecPairGrid<T>*>(dqpairs) + b->qpair_first[l],
                                                  b->qpair_count[l], b->qpair_tiles[l], b->sms, st);
        }
    }
    return e;
}

template <typename T>
et_status enqueue_batch_step(et_batch* b, char* dtab, cudaStream_t st) {
    const int C = b->count;
    const BatchResidual<T>* res = (const BatchResidual<T>*)dtab;
    const BatchStats* sts = (const BatchStats*)(dtab + sizeof(BatchResidual<T>) * C);
    const char* dsingles = dtab + sizeof(BatchResidual<T>) * C + sizeof(BatchStats) * C;
    const char* dpairs = dtab + b->pair_table_offset;
    const char* dqpairs = dtab + b->qpair_table_offset;
    cudaError_t e = launch_batch_residual<T>(b->op, (int)b->scheme, res, C, b->res_tiles, flags_of(b), st);
    if (e != cudaSuccess) return bfail(b, ET_ERR_CUDA, "batched residual: %s", cudaGetErrorString(e));
    for (int l = 0; l < b->nlaunch; ++l) {
        e = launch_index<T>(b, dsingles, dpairs, dqpairs, l, b->table_variant, st);
        if (e != cudaSuccess) return bfail(b, ET_ERR_CUDA, "batched term: %s", cudaGetErrorString(e));
    }
    e = launch_batch_stats(sts, C, st);
    if (e != cudaSuccess) return bfail(b, ET_ERR_CUDA, "batched stats: %s", cudaGetErrorString(e));
    return ET_OK;
}

template <typename T>
et_status upload_tables(et_batch* b, double* u, double tau, int variant, et_step_info* info, bool tuning) {
    std::vector<char> bytes;
    et_status rc = build_tables<T>(b, u, tau, variant, bytes, tuning);
    if (rc != ET_OK) return rc;
    // the per-run info destination goes into the stats descriptors
    BatchStats* st = (BatchStats*)(bytes.data() + sizeof(BatchResidual<T>) * b->count);
    for (int i = 0; i < b->count; ++i) {
        st[i].sink.info = info ? info + i : slot_of(b, i);
        st[i].sink.info_stride = info ? b->count : 0;
    }
    char* dst = b->ws + b->L.desc;
    BT_CUDA(b, cudaMemcpyAsync(dst, bytes.data(), bytes.size(), cudaMemcpyHostToDevice, b->stream));
    BT_CUDA(b, cudaStreamSynchronize(b->stream));  // bytes is a pageable host vector
    b->table_tau = tau;
    b->table_variant = variant;
    return ET_OK;
}

// Times the first launch index (every grid's first single or two-term launch)
// for every kernel variant and scores it per Taylor term advanced; keeps the
// fastest one-term variant, with two-term launches if those are faster still.
// us_out[v]: microseconds per term of the batch.
template <typename T>
et_status autotune(et_batch* b, double tau, double* us_out) {
    const int nv = total_variants(b->prec);
    cudaEvent_t e0, e1;
    BT_CUDA(b, cudaEventCreate(&e0));
    BT_CUDA(b, cudaEventCreate(&e1));
    double best = 1e300;
    int best_v = 0;
    std::vector<double> times(nv, 1e300);
    const int C = b->count;
    const size_t head = sizeof(BatchResidual<T>) * C + sizeof(BatchStats) * C;
    for (int v = 0; v < nv; ++v) {
        // tables with the step result redirected to the staging field
        std::vector<char> bytes;
        et_status rc = build_tables<T>(b, field<double>(b, b->L.stage, 0), tau, v, bytes, true);
        if (rc != ET_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rc;
        }
        // the descriptors of launch index 0 only
        const size_t ns = sizeof(BatchTerm<T>) * b->single_count[0];
        const size_t np = pair_desc_bytes(b->prec) * b->pair_count[0];
        const size_t nq = qpair_desc_bytes(b->prec) * b->qpair_count[0];
        char* dst = b->ws + b->L.tune_desc;
        const size_t poff = align64(ns);
        const size_t qoff = align64(poff + np);
        cudaError_t ce = cudaSuccess;
        if (ns) ce = cudaMemcpyAsync(dst, bytes.data() + head + sizeof(BatchTerm<T>) * b->single_first[0], ns,
                                     cudaMemcpyHostToDevice, b->stream);
        if (ce == cudaSuccess && np)
            ce = cudaMemcpyAsync(dst + poff, bytes.data() + b->pair_table_offset, np, cudaMemcpyHostToDevice,
                                 b->stream);
        if (ce == cudaSuccess && nq)
            ce = cudaMemcpyAsync(dst + qoff, bytes.data() + b->qpair_table_offset, nq, cudaMemcpyHostToDevice,
                                 b->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
        // voxel-terms advanced by launch index 0
        double vterms = 0.0, voxels = 0.0;
        for (int i = 0; i < C; ++i) voxels += (double)geom_of(b, i).n;
        {
            const BatchTerm<T>* sd = reinterpret_cast<const BatchTerm<T>*>(bytes.data() + head);
            for (int q = 0; q < b->single_count[0]; ++q) vterms += (double)sd[q].G.n;
            if constexpr (!std::is_same<T, double>::value) {
                const BatchPair<T>* pd = reinterpret_cast<const BatchPair<T>*>(bytes.data() + b->pair_table_offset);
                for (int q = 0; q < b->pair_count[0]; ++q) vterms += 2.0 * (double)pd[q].G.n;
                const VecPairGrid<T>* qd = reinterpret_cast<const VecPairGrid<T>*>(bytes.data() + b->qpair_table_offset);
                for (int q = 0; q < b->qpair_count[0]; ++q) vterms += 2.0 * (double)qd[q].G.n;
            }
        }
        // launch_index reads single_first / pair_first: point them at the copies
        b->single_first[0] = 0;
        b->pair_first[0] = 0;
        b->qpair_first[0] = 0;
        float ms = 0.f;
        for (int r = 0; r < 4 && ce == cudaSuccess; ++r) {  // one warm-up launch, then three timed
            if (r == 1) ce = cudaEventRecord(e0, b->stream);
            if (ce == cudaSuccess) ce = launch_index<T>(b, dst, dst + poff, dst + qoff, 0, v, b->stream);
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, b->stream);
        if (ce != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return bfail(b, ET_ERR_CUDA, "autotune timing failed: %s", cudaGetErrorString(cudaGetLastError()));
        }
        const double us = ms * 1e3 / 3.0 * (vterms > 0.0 ? voxels / vterms : 1.0);
        times[v] = us;
        if (us_out) us_out[v] = us;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // The fastest one-term variant also runs the leftover single terms of the
    // two-term variants, so it is chosen on its own; two-term launches are then
    // kept if their best time per term beats it.
    const int nsv = batch_variant_count(b->prec);
    int best_single = nv - nsv;
    for (int v = nv - nsv; v < nv; ++v)
        if (times[v] < times[best_single]) best_single = v;
    best_v = best_single;
    if (nv > nsv) {
        double best_pair = times[0];
        for (int v = 1; v < nsv; ++v) best_pair = std::min(best_pair, times[v]);
        if (best_pair < times[best_single]) best_v = best_single - nsv;  // the same single variant, with pairs
    }
    (void)best;
    b->variant = best_v;
    b->table_tau = -1.0;  // tables must be rebuilt for the chosen variant
    return ET_OK;
}

void clear_graph(et_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

template <typename T>
et_status run_impl(et_batch* b, double* u, double tau, int nsteps, et_step_info* info) {
    if (b->variant < 0) {
        et_status rc = autotune<T>(b, tau, nullptr);
        if (rc != ET_OK) return rc;
    }
    const bool same = b->exec && b->graph_tau == tau && b->graph_steps == nsteps && b->graph_u == u &&
                      b->graph_info == info && b->graph_variant == b->variant;
    if (same) {
        BT_CUDA(b, cudaGraphLaunch(b->exec, b->stream));
        return ET_OK;
    }
    clear_graph(b);
    et_status rc = upload_tables<T>(b, u, tau, b->variant, info, false);
    if (rc != ET_OK) return rc;
    BT_CUDA(b, cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    rc = ET_OK;
    for (int i = 0; i < b->count && rc == ET_OK; ++i)
        if (cudaMemsetAsync(counter_of(b, i), 0, sizeof(unsigned), b->capture) != cudaSuccess) rc = ET_ERR_CUDA;
    // the pair copy of u for the first residual (F32 / DF64); each step's
    // stats launch writes it for the next
    if (rc == ET_OK && b->prec != ET_F64 &&
        launch_split(b->ntot, u, 1.0, field<float2>(b, b->L.ush, 0), b->capture) != cudaSuccess)
        rc = ET_ERR_CUDA;
    for (int t = 0; t < nsteps && rc == ET_OK; ++t) rc = enqueue_batch_step<T>(b, b->ws + b->L.desc, b->capture);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->capture, &graph);
    if (rc != ET_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc == ET_ERR_CUDA ? bfail(b, rc, "capture failed") : rc;
    }
    if (ce != cudaSuccess) return bfail(b, ET_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return bfail(b, ET_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    b->graph_tau = tau;
    b->graph_steps = nsteps;
    b->graph_u = u;
    b->graph_info = info;
    b->graph_variant = b->variant;
    BT_CUDA(b, cudaGraphLaunch(b->exec, b->stream));
    return ET_OK;
}

}  // namespace

extern "C" {

size_t et_batch_workspace_bytes(int count, const int* dims, et_precision precision) {
    if (precision != ET_F64 && precision != ET_F32 && precision != ET_DF64) return 0;
    BatchLayout L;
    std::vector<long long> offs;
    if (!batch_layout(count, dims, precision, &L, &offs)) return 0;
    return L.total;
}

et_status et_batch_create(int count, const int* dims, double h, et_precision precision, void* workspace,
                          size_t workspace_bytes, void* cuda_stream, et_batch** out) {
    if (!out) return bfail(nullptr, ET_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    if (precision != ET_F64 && precision != ET_F32 && precision != ET_DF64)
        return bfail(nullptr, ET_ERR_ARG, "unknown precision");
    BatchLayout L;
    std::vector<long long> offs, zoffs;
    if (!batch_layout(count, dims, precision, &L, &offs, &zoffs))
        return bfail(nullptr, ET_ERR_ARG, "batch of %d grids is empty, too large or has an empty grid", count);
    for (int i = 0; i < count; ++i)
        if (dims[3 * i + 2] > 65535 || (long long)dims[3 * i] * dims[3 * i + 1] * dims[3 * i + 2] >= (1ll << 31))
            return bfail(nullptr, ET_ERR_ARG, "grid %d is too large", i);
    if (!(h > 0.0) || !std::isfinite(h)) return bfail(nullptr, ET_ERR_ARG, "h must be finite and > 0");
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0)
        return bfail(nullptr, ET_ERR_ARG, "workspace must be a 256-byte aligned device pointer");
    if (workspace_bytes < L.total)
        return bfail(nullptr, ET_ERR_ARG, "workspace has %zu bytes, %zu needed", workspace_bytes, L.total);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bfail(nullptr, ET_ERR_CUDA, "device query failed");
    et_batch* b = new (std::nothrow) et_batch();
    if (!b) return bfail(nullptr, ET_ERR_ARG, "out of host memory");
    b->count = count;
    b->dims.assign(dims, dims + 3 * count);
    b->offs = offs;
    b->zoffs = zoffs;
    b->ntot = L.ntot;
    b->h = h;
    b->prec = precision;
    b->device = dev;
    b->sms = sms;
    b->ws = (char*)workspace;
    b->ws_bytes = workspace_bytes;
    b->L = L;
    b->stream = (cudaStream_t)cuda_stream;
    b->coeffs_set = false;
    b->opt_set = false;
    std::memset(&b->opt, 0, sizeof(b->opt));
    b->rho.assign(count, 0.0);
    b->rmax.assign(count, 0.0);
    b->nu.assign(count, 1.0);
    b->table_tau = -1.0;
    b->table_variant = -1;
    b->nlaunch = 0;
    b->res_tiles = 0;
    b->graph_tau = -1.0;
    b->graph_steps = 0;
    b->graph_u = nullptr;
    b->graph_info = nullptr;
    b->graph_variant = -1;
    b->exec = nullptr;
    b->variant = -1;
    b->err[0] = 0;
    b->pair_table_offset = 0;
    b->qpair_table_offset = 0;
    b->pair_plans.assign(count, nullptr);
    if (precision != ET_F64) {
        // tensor maps of every grid's fields for the two-term kernel (nullptr:
        // its rows are not a 16-byte multiple, or its fields are not 16-byte
        // aligned in the concatenated layout; that grid runs one term per launch)
        const size_t es = value_bytes(precision);
        for (int i = 0; i < count; ++i) {
            auto at = [&](size_t region) { return (const void*)(b->ws + region + es * (size_t)offs[i]); };
            const void* wt4[4] = {at(L.wt[0]), at(L.wt[1]), at(L.wt[2]), at(L.wt[3])};
            const void* yz[4] = {at(L.vec[2]), at(L.vec[3]), at(L.vec[4]), at(L.vec[5])};
            b->pair_plans[i] = pair_plan_create(geom_of(b, i), precision, wt4, at(L.vec[0]), at(L.vec[1]), yz);
        }
    }
    if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess ||
        prime_launch_limits() != cudaSuccess ||
        cudaMemsetAsync(b->ws + L.misc, 0, misc_bytes(count), b->stream) != cudaSuccess) {
        for (PairPlan* P : b->pair_plans) pair_plan_destroy(P);
        delete b;
        return bfail(nullptr, ET_ERR_CUDA, "batch set-up failed");
    }
    *out = b;
    return ET_OK;
}

et_status et_batch_set_coeffs(et_batch* b, const double* D, const double* rho, et_operator op, et_scheme scheme,
                              const et_options* options) {
    NvtxRange nvtx_range("et_batch_set_coeffs");
    if (!b) return bfail(nullptr, ET_ERR_ARG, "batch is NULL");
    if (!D || ((uintptr_t)D & 7u) || !rho) return bfail(b, ET_ERR_ARG, "D (device) and rho (host) must be given");
    if (op != ET_OP_CONSERVATIVE && op != ET_OP_LITERAL) return bfail(b, ET_ERR_ARG, "unknown operator");
    if (scheme != ET_SCHEME_ROSENBROCK && scheme != ET_SCHEME_EXPEULER) return bfail(b, ET_ERR_ARG, "unknown scheme");
    for (int i = 0; i < b->count; ++i)
        if (!(rho[i] >= 0.0) || !std::isfinite(rho[i])) return bfail(b, ET_ERR_ARG, "rho[%d] must be finite and >= 0", i);
    if (options) {
        if (options->tol < 0 || !std::isfinite(options->tol)) return bfail(b, ET_ERR_ARG, "options.tol must be >= 0");
        if (options->theta_max < 0 || !std::isfinite(options->theta_max))
            return bfail(b, ET_ERR_ARG, "options.theta_max must be >= 0");
        if (options->force_m == 1) return bfail(b, ET_ERR_ARG, "options.force_m must be 0 or >= 2");
        if (options->force_s < 0 || options->force_m < 0) return bfail(b, ET_ERR_ARG, "forced s, m must be >= 0");
        if (options->timeout_probe_us < 0 || options->timeout_probe_us > 1000000)
            return bfail(b, ET_ERR_ARG, "options.timeout_probe_us must be in [0, 1000000]");
        if (options->every_row != 0 && options->every_row != 1)
            return bfail(b, ET_ERR_ARG, "options.every_row must be 0 or 1");
    }
    BDeviceGuard dg(b->device);
    clear_graph(b);
    b->coeffs_set = false;
    b->table_tau = -1.0;
    const double inv_h2 = 1.0 / (b->h * b->h);
    BT_CUDA(b, cudaMemsetAsync(misc(b), 0, misc_bytes(b->count), b->stream));
    BT_CUDA(b, cudaMemsetAsync(b->ws + b->L.zcount, 0, 8ull * b->count, b->stream));
    for (int i = 0; i < b->count; ++i) {
        double* w[5];
        for (int a = 0; a < 5; ++a) w[a] = field<double>(b, b->L.w[a], i);
        cudaError_t e =
            launch_coeffs(geom_of(b, i), D + b->offs[i], inv_h2, op, w, rmax_bits_of(b, i), flags_of(b), b->stream);
        if (e != cudaSuccess) return bfail(b, ET_ERR_CUDA, "coeffs launch: %s", cudaGetErrorString(e));
        // the warp rows without off-diagonal entries of this grid's operator
        Weights<double> W64;
        for (int a = 0; a < 5; ++a) W64.w[a] = w[a];
        e = launch_zero_rows(geom_of(b, i), op, W64, (unsigned char*)(b->ws + b->L.zrow) + b->zoffs[i],
                             (unsigned long long*)(b->ws + b->L.zcount) + i, b->stream);
        if (e != cudaSuccess) return bfail(b, ET_ERR_CUDA, "zero-row launch: %s", cudaGetErrorString(e));
    }
    std::vector<unsigned long long> bits(b->count);
    unsigned flags = 0;
    BT_CUDA(b, cudaMemcpyAsync(bits.data(), rmax_bits_of(b, 0), 8ull * b->count, cudaMemcpyDeviceToHost, b->stream));
    BT_CUDA(b, cudaMemcpyAsync(&flags, flags_of(b), sizeof(flags), cudaMemcpyDeviceToHost, b->stream));
    BT_CUDA(b, cudaStreamSynchronize(b->stream));
    BT_CUDA(b, cudaMemsetAsync(flags_of(b), 0, sizeof(unsigned), b->stream));
    if (flags & ET_FLAG_D_INVALID) return bfail(b, ET_ERR_NUMERIC, "D has negative or non-finite values");
    b->op = op;
    b->scheme = scheme;
    b->opt_set = options != nullptr;
    if (options) b->opt = *options;
    const bool shift = !(options && options->shift == 0);
    for (PairPlan* P : b->pair_plans) pair_plan_set_skip(P, !(options && options->every_row != 0));
    for (int i = 0; i < b->count; ++i) {
        std::memcpy(&b->rmax[i], &bits[i], sizeof(double));
        b->rho[i] = rho[i];
        const double rho_c = scheme == ET_SCHEME_ROSENBROCK ? rho[i] * (1.0 + 2.0 * kRangeSlack) : 0.0;
        const double nu = shift ? b->rmax[i] + rho_c : 2.0 * b->rmax[i] + rho_c;
        b->nu[i] = nu > 0.0 ? nu : 1.0;
        if (b->prec != ET_F64) {
            const Geom G = geom_of(b, i);
            const double* src[4];
            for (int a = 0; a < 4; ++a) src[a] = field<double>(b, b->L.w[a], i);
            cudaError_t e;
            if (b->prec == ET_F32) {
                float* dst[4];
                for (int a = 0; a < 4; ++a) dst[a] = field<float>(b, b->L.wt[a], i);
                e = launch_convert_weights(G, src, dst, 1.0 / b->nu[i], b->stream);
                if (e == cudaSuccess)
                    e = launch_cast(G.n, field<double>(b, b->L.w[4], i), 1.0 / b->nu[i], field<float>(b, b->L.wt[4], i),
                                    b->stream);
            } else {
                float2* dst[4];
                for (int a = 0; a < 4; ++a) dst[a] = field<float2>(b, b->L.wt[a], i);
                e = launch_convert_weights(G, src, dst, 1.0 / b->nu[i], b->stream);
            }
            // the pair weights of the residual (DF64: the term weights themselves)
            float2* pw[4];
            for (int a = 0; a < 4; ++a) pw[a] = pair_weight(b, a, i);
            if (e == cudaSuccess && b->prec == ET_F32) e = launch_convert_weights(G, src, pw, 1.0 / b->nu[i], b->stream);
            if (e == cudaSuccess)
                e = launch_split(G.n, field<double>(b, b->L.w[4], i), 1.0 / b->nu[i], pair_weight(b, 4, i), b->stream);
            if (e != cudaSuccess) return bfail(b, ET_ERR_CUDA, "weight conversion: %s", cudaGetErrorString(e));
        }
    }
    b->coeffs_set = true;
    b->variant = -1;
    return ET_OK;
}

et_status et_batch_run(et_batch* b, double* u, double tau, int nsteps, et_step_info* info) {
    NvtxRange nvtx_range("et_batch_run");
    if (!b) return bfail(nullptr, ET_ERR_ARG, "batch is NULL");
    if (!b->coeffs_set) return bfail(b, ET_ERR_STATE, "et_batch_set_coeffs has not been called");
    if (!u || ((uintptr_t)u & 7u)) return bfail(b, ET_ERR_ARG, "u must be an 8-byte aligned device pointer");
    if (info && ((uintptr_t)info & 7u)) return bfail(b, ET_ERR_ARG, "info must be 8-byte aligned");
    if (!(tau > 0.0) || !std::isfinite(tau)) return bfail(b, ET_ERR_ARG, "tau must be finite and > 0");
    if (nsteps < 1) return bfail(b, ET_ERR_ARG, "nsteps must be >= 1");
    BDeviceGuard dg(b->device);
    if (b->prec == ET_F64) return run_impl<double>(b, u, tau, nsteps, info);
    if (b->prec == ET_F32) return run_impl<float>(b, u, tau, nsteps, info);
    return run_impl<float2>(b, u, tau, nsteps, info);
}

et_status et_batch_autotune(et_batch* b, double tau, int* variant, double* us_per_variant) {
    NvtxRange nvtx_range("et_batch_autotune");
    if (!b) return bfail(nullptr, ET_ERR_ARG, "batch is NULL");
    if (!b->coeffs_set) return bfail(b, ET_ERR_STATE, "et_batch_set_coeffs has not been called");
    if (!(tau > 0.0) || !std::isfinite(tau)) return bfail(b, ET_ERR_ARG, "tau must be finite and > 0");
    BDeviceGuard dg(b->device);
    clear_graph(b);
    et_status rc;
    if (b->prec == ET_F64) rc = autotune<double>(b, tau, us_per_variant);
    else if (b->prec == ET_F32) rc = autotune<float>(b, tau, us_per_variant);
    else rc = autotune<float2>(b, tau, us_per_variant);
    if (rc == ET_OK && variant) *variant = b->variant;
    return rc;
}

et_status et_batch_set_variant(et_batch* b, int variant) {
    if (!b) return bfail(nullptr, ET_ERR_ARG, "batch is NULL");
    if (variant < 0 || variant >= total_variants(b->prec)) return bfail(b, ET_ERR_ARG, "no variant %d", variant);
    BDeviceGuard dg(b->device);
    clear_graph(b);
    b->variant = variant;
    b->table_tau = -1.0;
    return ET_OK;
}

int et_batch_variant_count(et_precision precision) {
    if (precision != ET_F64 && precision != ET_F32 && precision != ET_DF64) return 0;
    return total_variants(precision);
}

et_status et_batch_sync_info(et_batch* b, et_step_info* host_out) {
    if (!b) return bfail(nullptr, ET_ERR_ARG, "batch is NULL");
    BDeviceGuard dg(b->device);
    std::vector<et_step_info> rec(b->count);
    unsigned flags = 0;
    for (int i = 0; i < b->count; ++i)
        BT_CUDA(b, cudaMemcpyAsync(&rec[i], slot_of(b, i), sizeof(et_step_info), cudaMemcpyDeviceToHost, b->stream));
    BT_CUDA(b, cudaMemcpyAsync(&flags, flags_of(b), sizeof(flags), cudaMemcpyDeviceToHost, b->stream));
    BT_CUDA(b, cudaStreamSynchronize(b->stream));
    BT_CUDA(b, cudaMemsetAsync(flags_of(b), 0, sizeof(unsigned), b->stream));
    if (host_out) std::memcpy(host_out, rec.data(), sizeof(et_step_info) * b->count);
    if (flags & ET_FLAG_TIMEOUT) return bfail(b, ET_ERR_TIMEOUT, "a device-side wait ran out; the run is not valid");
    if (flags & ET_FLAG_NONFINITE) return bfail(b, ET_ERR_NUMERIC, "non-finite density met");
    if (flags & ET_FLAG_RANGE_IN) return bfail(b, ET_ERR_NUMERIC, "density outside [0, 1] (+-1e-3)");
    return ET_OK;
}

et_status et_batch_get_schedule(const et_batch* b, double tau, int* s, int* m) {
    if (!b) return bfail(nullptr, ET_ERR_ARG, "batch is NULL");
    if (!b->coeffs_set) return bfail(const_cast<et_batch*>(b), ET_ERR_STATE, "et_batch_set_coeffs has not been called");
    for (int i = 0; i < b->count; ++i) {
        Sched S;
        if (sched_of(b, i, tau, &S) != ET_OK) return bfail(const_cast<et_batch*>(b), ET_ERR_ARG, "no (s, m) for grid %d", i);
        if (s) s[i] = S.s;
        if (m) m[i] = S.m;
    }
    return ET_OK;
}

et_status et_batch_get_zero_rows(et_batch* b, long long* voxels, long long* total) {
    if (!b) return bfail(nullptr, ET_ERR_ARG, "batch is NULL");
    if (!b->coeffs_set) return bfail(b, ET_ERR_STATE, "et_batch_set_coeffs has not been called");
    BDeviceGuard dg(b->device);
    std::vector<unsigned long long> c(b->count);
    BT_CUDA(b, cudaMemcpyAsync(c.data(), b->ws + b->L.zcount, 8ull * b->count, cudaMemcpyDeviceToHost, b->stream));
    BT_CUDA(b, cudaStreamSynchronize(b->stream));
    long long sum = 0;
    for (int i = 0; i < b->count; ++i) {
        if (voxels) voxels[i] = (long long)c[i];
        sum += (long long)c[i];
    }
    if (total) *total = sum;
    return ET_OK;
}

et_status et_batch_set_stream(et_batch* b, void* cuda_stream) {
    if (!b) return bfail(nullptr, ET_ERR_ARG, "batch is NULL");
    b->stream = (cudaStream_t)cuda_stream;
    return ET_OK;
}

const char* et_batch_last_error(const et_batch* b) { return b ? b->err : g_batch_error; }

void et_batch_destroy(et_batch* b) {
    if (!b) return;
    {
        BDeviceGuard dg(b->device);
        clear_graph(b);
        if (b->capture) cudaStreamDestroy(b->capture);
    }
    for (PairPlan* P : b->pair_plans) pair_plan_destroy(P);
    delete b;
}

}  // extern "C"
