// et_step_static: one exponential-integrator step that allocates nothing.
//
// Some callers cannot call cudaMalloc or any allocating routine: code running
// inside a host framework that owns all device memory through its own pool
// and forbids side allocations, code called while a memory budget is locked,
// or plug-ins that must not grow the process footprint at call time.  For
// them this entry point keeps its scratch (face weights, residual, diagonal,
// Taylor-term vectors, reduction partials and counters) in one file-scope
// static __device__ array of fixed size instead of a caller-provided
// workspace.  The caller still passes the inputs (D) and the in/out density u.
//
// Limits and behaviour:
//  - at most kStaticMaxVoxels = 64^3 = 262144 voxels and at most 65536 thread
//    blocks of the 32 x 8 stencil tile; larger grids are rejected with
//    ET_ERR_ARG, and so are grids with nz > 65535 (the z extent of a launch).
//    The array is 11 FP64 fields of 64^3 voxels plus 3 x 8 x kStatsBlocks
//    bytes of reduction partials (about 14 KiB) and 256 bytes of counters:
//    22 MiB held on every GPU that loads it until exit.
//  - the first call in a CUDA context of a device (the primary context, or a
//    new one after cudaDeviceReset) looks up the array's device address with
//    cudaGetSymbolAddress while that device is current, and caches it keyed by
//    the context's unique id; make that first call before any stream capture.
//  - every call shares the array: two calls whose work overlaps on the GPU
//    (different streams, or different host threads) race and corrupt each
//    other.  Counters are cleared at the start of each call; every other
//    region is fully written before it is read.
//  - the call synchronises the stream twice (after the coefficient pass, to
//    read the operator bound that fixes s and m, and at the end, to report
//    device flags).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "et.h"
#include "et_internal.h"

namespace {

using namespace et;

constexpr long long kStaticMaxVoxels = 64ll * 64 * 64;
constexpr unsigned kStaticMaxBlocks = 65536;
constexpr size_t kFieldBytes = 8ull * kStaticMaxVoxels;          // one FP64 field
constexpr int kFields = 11;                                      // 5 weights, b, dt, Y0, Y1, Z0, Z1
constexpr size_t kPartialBytes = 3ull * 8ull * kStatsBlocks;
constexpr size_t kCounterBytes = 256;
constexpr size_t kStaticScratchBytes = kFields * kFieldBytes + kPartialBytes + kCounterBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // id of the context the address belongs to

// Unique id of the current CUDA context (0 if the driver cannot say).  Ids are
// never reused, unlike context handles, so an address cached for a context
// that was destroyed (cudaDeviceReset) is never taken for its successor.
unsigned long long current_context_id() {
    typedef int (*ctx_current_fn)(void**);
    typedef int (*ctx_id_fn)(void*, unsigned long long*);
    static ctx_current_fn get_current = nullptr;
    static ctx_id_fn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<ctx_current_fn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<ctx_id_fn>(p);
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

et_status report(char* msg, size_t msg_len, et_status st, const char* fmt, ...) {
    if (msg && msg_len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(msg, msg_len, fmt, ap);
        va_end(ap);
    }
    return st;
}

// Device address of the static array in the current context of device `dev`:
// looked up once per context and cached; looked up on every call if the
// driver gives no context id.
cudaError_t scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = (unsigned char*)p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" ET_API et_status et_step_static(int nx, int ny, int nz, double h, const double* D, double rho,
                                           et_operator op, et_scheme scheme, double* u, double tau,
                                           void* cuda_stream, char* msg, size_t msg_len) {
    if (msg && msg_len) msg[0] = 0;
    if (nx <= 0 || ny <= 0 || nz <= 0)
        return report(msg, msg_len, ET_ERR_ARG, "grid %d x %d x %d is empty", nx, ny, nz);
    const long long n = (long long)nx * ny * nz;
    if (n > kStaticMaxVoxels)
        return report(msg, msg_len, ET_ERR_ARG,
                      "grid %d x %d x %d has %lld voxels; the static scratch holds at most %lld (64^3)",
                      nx, ny, nz, n, kStaticMaxVoxels);
    if (nz > 65535)
        return report(msg, msg_len, ET_ERR_ARG, "grid %d x %d x %d: nz = %d exceeds 65535, the z extent of a launch",
                      nx, ny, nz, nz);
    const unsigned long long nblocks = (unsigned long long)((nx + kBlockX - 1) / kBlockX) *
                                       ((ny + kBlockY - 1) / kBlockY) * (unsigned long long)nz;
    if (nblocks > kStaticMaxBlocks)
        return report(msg, msg_len, ET_ERR_ARG,
                      "grid %d x %d x %d needs %llu thread blocks of the 32 x 8 tile; at most %u "
                      "are supported", nx, ny, nz, nblocks, kStaticMaxBlocks);
    if (!(h > 0.0) || !std::isfinite(h)) return report(msg, msg_len, ET_ERR_ARG, "h must be finite and > 0");
    if (!(tau > 0.0) || !std::isfinite(tau)) return report(msg, msg_len, ET_ERR_ARG, "tau must be finite and > 0");
    if (!(rho >= 0.0) || !std::isfinite(rho)) return report(msg, msg_len, ET_ERR_ARG, "rho must be finite and >= 0");
    if (op != ET_OP_CONSERVATIVE && op != ET_OP_LITERAL) return report(msg, msg_len, ET_ERR_ARG, "unknown operator");
    if (scheme != ET_SCHEME_ROSENBROCK && scheme != ET_SCHEME_EXPEULER)
        return report(msg, msg_len, ET_ERR_ARG, "unknown scheme");
    if (!D || !u || ((uintptr_t)D & 7u) || ((uintptr_t)u & 7u))
        return report(msg, msg_len, ET_ERR_ARG, "D and u must be non-NULL 8-byte aligned device pointers");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report(msg, msg_len, ET_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return report(msg, msg_len, ET_ERR_UNSUPPORTED, "device index %d", dev);
    unsigned char* base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess)
        return report(msg, msg_len, ET_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)cuda_stream;

    double* field[kFields];
    for (int f = 0; f < kFields; ++f) field[f] = (double*)(base + f * kFieldBytes);
    double* partial = (double*)(base + kFields * kFieldBytes);
    unsigned char* counters = base + kFields * kFieldBytes + kPartialBytes;
    unsigned long long* rmax_bits = (unsigned long long*)(counters + 0);
    unsigned* flags = (unsigned*)(counters + 8);
    unsigned* ticket = (unsigned*)(counters + 12);
    unsigned* step_counter = (unsigned*)(counters + 16);
    et_step_info* record = (et_step_info*)(counters + 64);

    Geom G;
    G.nx = nx;
    G.ny = ny;
    G.nz = nz;
    G.n = n;
    G.sy = nx;
    G.sz = (long long)nx * ny;
    G.nblocks = (unsigned)nblocks;
    G.sms = 0;

#define STATIC_CUDA(call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return report(msg, msg_len, ET_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

    STATIC_CUDA(cudaDeviceGetAttribute(&G.sms, cudaDevAttrMultiProcessorCount, dev));
    STATIC_CUDA(prime_launch_limits());
    // counters start at zero on every call; the array keeps the previous call's contents
    STATIC_CUDA(cudaMemsetAsync(counters, 0, kCounterBytes, st));
    STATIC_CUDA(launch_coeffs(G, D, 1.0 / (h * h), op, field, rmax_bits, flags, st));
    unsigned long long bits = 0;
    unsigned dflags = 0;
    STATIC_CUDA(cudaMemcpyAsync(&bits, rmax_bits, sizeof(bits), cudaMemcpyDeviceToHost, st));
    STATIC_CUDA(cudaMemcpyAsync(&dflags, flags, sizeof(dflags), cudaMemcpyDeviceToHost, st));
    STATIC_CUDA(cudaStreamSynchronize(st));
    if (dflags & ET_FLAG_D_INVALID) return report(msg, msg_len, ET_ERR_NUMERIC, "D has negative or non-finite values");
    double rmax;
    std::memcpy(&rmax, &bits, sizeof(rmax));

    int s = 0, m = 0;
    double mu = 0.0, theta = 0.0;
    if (et_select_schedule(tau, rmax, rho, scheme, ET_F64, nullptr, &s, &m, &mu, &theta) != ET_OK)
        return report(msg, msg_len, ET_ERR_ARG, "no (s, m) meets the tolerance for tau = %g", tau);

    Weights<double> W;
    for (int a = 0; a < 5; ++a) W.w[a] = field[a];
    double* b = field[5];
    double* dt = field[6];
    double* Y[2] = {field[7], field[8]};
    double* Z[2] = {field[9], field[10]};
    const double dt_shift = (scheme == ET_SCHEME_ROSENBROCK ? rho : 0.0) - mu;
    STATIC_CUDA(launch_residual<double>(G, op, u, W, rho, dt_shift, 1.0, scheme, b, dt, flags, st));

    StatsSink sink;
    sink.partial = partial;
    sink.ticket = ticket;
    sink.step_counter = step_counter;
    sink.flags = flags;
    sink.info = record;
    sink.info_stride = 0;
    sink.last = record;
    sink.s = s;
    sink.m = m;
    sink.ush = nullptr;

    // the scaled Taylor recurrence of exp(h (B - mu I)) on [y; a], sub-step by sub-step
    const double hs = tau / s;
    const double gamma = std::exp(mu * hs);
    double ak = 1.0;
    int zi = 0;
    for (int k = 0; k < s; ++k) {
        double* yacc = Y[(k + 1) & 1];
        const double* zin = (k == 0) ? b : Y[k & 1];
        double pw = (k == 0) ? -mu : 1.0;  // (-mu)^j at the first launched term
        double gj = (k == 0) ? hs : 1.0;   // g_j = h^j / j!
        for (int j = (k == 0) ? 1 : 0; j < m; ++j) {
            TermArgs<double> a;
            a.zin = zin;
            a.b = b;
            a.beta = ak * pw;
            a.has_beta = (ak * pw) != 0.0;
            a.zscale = 1.0;
            a.has_zscale = 0;
            a.horner = 0;
            a.dt = dt;
            const double gnext = gj * hs / (j + 1);
            a.g = gnext;
            a.gamma = 1.0;
            a.base_scale = 0.0;
            a.base_mode = (k == 0 && j == 1) ? 1 : ((k > 0 && j == 0) ? 2 : 0);
            if (a.base_mode == 1) a.base_scale = hs;
            a.last = (j + 1 == m);
            a.yacc = yacc;
            a.u = nullptr;
            a.zout = a.last ? nullptr : Z[zi];
            if (a.last) {
                a.gamma = gamma;
                if (k == s - 1) a.u = u;
            }
            STATIC_CUDA(launch_term<double>(G, op, W, a, st));
            if (!a.last) {
                zin = Z[zi];
                zi ^= 1;
            }
            pw *= -mu;
            gj = gnext;
        }
        double sum = 0.0, t = 1.0;
        for (int j = 0; j <= m; ++j) {
            sum += t;
            t *= (-mu * hs) / (j + 1);
        }
        ak = gamma * ak * sum;
    }
    STATIC_CUDA(launch_stats(G, u, sink, st));
    STATIC_CUDA(cudaMemcpyAsync(&dflags, flags, sizeof(dflags), cudaMemcpyDeviceToHost, st));
    STATIC_CUDA(cudaStreamSynchronize(st));
#undef STATIC_CUDA
    if (dflags & ET_FLAG_NONFINITE) return report(msg, msg_len, ET_ERR_NUMERIC, "non-finite density met");
    if (dflags & ET_FLAG_RANGE_IN)
        return report(msg, msg_len, ET_ERR_NUMERIC, "density outside [0, 1] (+-1e-3): the step bound does not hold");
    return ET_OK;
}
