// Internal declarations shared by the host driver (et_api.cu) and the kernels
// (et_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <utility>

#include "et.h"
#include <nvtx3/nvToolsExt.h>

namespace et {

// NVTX range over one call of the C ABI (header-only NVTX: a no-op unless a
// tool such as ncu --nvtx is attached).  Kernels a call enqueues, and graphs
// it launches, carry the range's name in the tool's view.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Density range accepted by the a-priori bound |1 - 2u| <= 1 + 2 * kRangeSlack
// of the folded scheme (ET_FLAG_RANGE_IN outside it).
constexpr double kRangeSlack = 1e-3;

// Thread-block shape of the stencil kernels: 32 voxels along x (one warp per
// row, coalesced) by 8 rows along y; one z-plane per block.
// Programmatic dependent launch.  A kernel launched by launch_pdl calls
// pdl_begin() before its first memory access: it lets the next grid in the
// stream be scheduled as soon as all of its own blocks run, and waits until
// the previous grid has finished and its stores are visible (after a plain
// launch the wait returns at once).  Short kernels then overlap their launch
// and block set-up with the previous kernel's tail.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.launch_dependents;");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t stream, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int kBlockX = 32;
constexpr int kBlockY = 8;
constexpr int kThreads = kBlockX * kBlockY;

// Coefficient fields of L (Sec. 2.1), one value per voxel:
//   w[0..2]: weight towards +x, +y, +z (0 on the far wall);
//   conservative: weight towards -e is w[e][p - e] (0 on the near wall);
//   literal:      weight towards -e is w[3][p] = 2 D_p / h^2 (0 on the near wall);
//   w[4]: minus the sum of the kept off-diagonal weights of row p (the
//         diagonal of L); FP64 only, read by the residual kernel.
template <typename T>
struct Weights {
    const T* w[5];
    // Rows without off-diagonal entries: one byte per warp row (32
    // x-consecutive voxels of one grid row, index (i >> 5) + ceil(nx / 32) (j +
    // ny k)), 1 where every off-diagonal weight of its voxels is zero (voxels
    // in and next to D = 0 tissue); a term there is dt z + beta b.  nullptr:
    // no rows are skipped.
    const unsigned char* zrow = nullptr;
};

// Tile of the stencil kernels: a 32 x 8 block of threads, each thread marching
// over kTileZ consecutive z-planes; blocks loop over tiles (grid-stride).
constexpr int kTileZ = 4;

// Per-launch geometry.
struct Geom {
    int nx, ny, nz;
    long long n;
    long long sy, sz;  // strides of y and z
    unsigned nblocks;  // blocks of a one-voxel-per-thread stencil launch (coeffs, residual)
    int sms;           // multiprocessors of the device
};
// Whether voxel (i, j, k)'s warp row (32 x-consecutive voxels) has no
// off-diagonal entries of the operator (the same for all its lanes; zrow
// nullptr: none marked).
__device__ __forceinline__ bool zero_row_of(const Geom& G, const unsigned char* zrow, int i, int j, int k) {
    return zrow && zrow[(i >> 5) + (long long)((G.nx + 31) >> 5) * (j + (long long)G.ny * k)];
}

// Marks the warp rows without off-diagonal entries of the operator (zrow, as
// in Weights) and adds their voxels to *count.
cudaError_t launch_zero_rows(const Geom& G, et_operator op, const Weights<double>& W, unsigned char* zrow,
                             unsigned long long* count, cudaStream_t stream);
inline long long zero_row_bytes(const Geom& G) { return (long long)((G.nx + 31) / 32) * G.ny * G.nz; }

// Device-side accumulation of per-step observables: block partials, a ticket
// counter for the last-block reduction, the step index and the flag word.
constexpr int kStatsBlocks = 608;  // 4 per SM; fixed, so the summation order is fixed
constexpr int kStatsThreads = 256;
// Norms of a step for its a-posteriori truncation estimate: every warp of the
// residual launch writes max |b| and max |u^n| of its voxels (bit patterns of
// non-negative doubles) to its own slot; the stats launch that ends the step
// reduces the slots with its pass over u (two more partials a block).
struct StatsSink {
    double* partial;        // 3 * kStatsBlocks: sum, min key, max key
    unsigned* ticket;       // last-block counter, returns to 0 after each step
    unsigned* step_counter; // step index within the current run
    unsigned* flags;        // ET_FLAG_* word
    et_step_info* info;     // destination base
    int info_stride;        // records step t at info[t * info_stride] (0: always info[0])
    et_step_info* last;     // internal copy of the latest record (read by et_sync_info)
    int s, m;               // recorded in the info
    const int* m_dev = nullptr;  // non-null: m is read from here (iterations of a Crank-Nicolson solve)
    float2* ush;            // F32 / DF64: receives the pair of each u (nullptr: none)
    // truncation estimate (nullptr wnorm: none): est = trunc_c max|b| / max|u^n|,
    // ET_FLAG_TRUNCATION when est > trunc_tol; est is stored to *trunc_est
    const unsigned long long* wnorm = nullptr;  // [nwarps][2]: max |b|, max |u^n| of each residual warp
    long long nwarps = 0;
    double* npartial = nullptr;                 // 2 * kStatsBlocks: the blocks' maxima of the slots
    double trunc_c = 0.0, trunc_tol = 0.0;
    double* trunc_est = nullptr;
};

// Writes the maxima of |b| and |u| over the calling warp's lanes to the warp's
// slot (lanes without a voxel pass 0).  Every lane of the warp must call it.
// (the FP32 / DF64 residual passes the high parts as floats: their maxima are
// taken on the float bits and widened once, off GB300's slow FP64 pipe)
__device__ __forceinline__ void warp_norms(float babs, float uabs, unsigned long long* slot) {
    unsigned kb = __float_as_uint(babs), ku = __float_as_uint(uabs);
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned ob = __shfl_down_sync(0xffffffffu, kb, off);
        const unsigned ou = __shfl_down_sync(0xffffffffu, ku, off);
        kb = ob > kb ? ob : kb;
        ku = ou > ku ? ou : ku;
    }
    if ((threadIdx.x & 31) == 0) {
        slot[0] = (unsigned long long)__double_as_longlong((double)__uint_as_float(kb));
        slot[1] = (unsigned long long)__double_as_longlong((double)__uint_as_float(ku));
    }
}
__device__ __forceinline__ void warp_norms(double babs, double uabs, unsigned long long* slot) {
    unsigned long long kb = (unsigned long long)__double_as_longlong(babs);
    unsigned long long ku = (unsigned long long)__double_as_longlong(uabs);
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ob = __shfl_down_sync(0xffffffffu, kb, off);
        const unsigned long long ou = __shfl_down_sync(0xffffffffu, ku, off);
        kb = ob > kb ? ob : kb;
        ku = ou > ku ? ou : ku;
    }
    if ((threadIdx.x & 31) == 0) {
        slot[0] = kb;
        slot[1] = ku;
    }
}

// Scalars of the kernels' value types: double (FP64), float (FP32) and
// float2 = (hi, lo) double-float pairs (DF64, value hi + lo).
template <typename T>
struct Scalar;
template <>
struct Scalar<double> {
    static double make(double v) { return v; }
};
template <>
struct Scalar<float> {
    static float make(double v) { return (float)v; }
};
template <>
struct Scalar<float2> {
    static float2 make(double v) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    }
};

// Arguments of one Taylor-term launch (scaled recurrence, see et_kernels.cu).
template <typename T>
struct TermArgs {
    const T* zin;    // z_j, read with a one-voxel halo
    T* zout;         // z_{j+1}; nullptr on the last term of a sub-step
    const T* b;      // residual, added with coefficient beta when has_beta
    T beta;
    int has_beta;
    T zscale;        // factor on the stencil part (first term of the FP32 / DF64 chain)
    int has_zscale;
    const T* dt;     // diagonal of A - mu I
    int base_mode;   // 0: yacc[p]; 1: base_scale * b[p]; 2: zin[p]
    T base_scale;
    T g;             // weight of z_{j+1} in the sub-step sum
    T gamma;         // e^{mu h}, applied on the last term (1 otherwise)
    int last;        // last term of the sub-step
    int horner;      // Horner step of sub-step 0: output acc itself (no running sum)
    T* yacc;         // sub-step sum (read when base_mode == 0, written unless finishing)
    double* u;       // non-null on the last term of the step: u += gamma * sum
};

// Arguments of one reverse Taylor-term launch (et_adjoint.cu).
template <typename T>
struct AdjTermArgs {
    const T* wsrc;       // w / wscale, read with a one-voxel halo
    T wscale;
    const T* dt;         // diagonal of A^ (as in the forward pass)
    const T* negR;       // minus the row sums of L, times 1/nu
    const T* ybar_next;  // cotangent of the sub-step result; Sbar = gamma * ybar_next
    T gamma;
    T g;                 // coefficient of Sbar in the output
    T f;                 // factor of the forward term on A^ (1, or 1/nu on the first term)
    T inv_nu;
    const T* x;          // forward input of this term
    int has_beta;
    T beta;
    T* bbar;             // cotangent of b (accumulated)
    T* cbar;             // cotangent of the diagonal rho(1 - 2u) (accumulated)
    T* sstep;            // per-voxel cotangent of the D scale, this step's terms
    int out_to_bbar;     // the output adds to bbar instead of zbar_out
    T* zbar_out;
};

// Batched form: one launch covers many grids.  Each grid's part of a launch is
// a descriptor in device memory (fields already offset to the grid's slice of
// the concatenated workspace) with the index of its first tile; blocks find
// their grid by binary search over tile_begin.
template <typename T>
struct BatchTerm {
    Geom G;
    Weights<T> W;
    TermArgs<T> a;
    long long tile_begin;
};

// Inputs of the pair-arithmetic residual of the F32 and DF64 forms: the pair
// of each u (df64::from_double), the 1/nu-scaled pair weights (w[4] = -rowsum / nu), nu,
// rho, the diagonal shift / nu and the coefficient of u in the diagonal.
struct PairResidualArgs {
    const float2* ush;
    Weights<float2> W;
    float2 nu, rho, shift, k_u;
};

// One grid of the batched residual: FP64 from u (F64 form) or in pair
// arithmetic from P (F32, DF64).
template <typename T>
struct BatchResidual {
    Geom G;
    const double* u;
    Weights<double> W;
    double rho, dt_shift, dt_scale;
    PairResidualArgs P;
    T* b;
    T* dt;
    unsigned long long* wnorm;  // the batch's warp norm slots, indexed by tile (nullptr: none)
    long long tile_begin;
};

struct BatchStats {
    long long n;
    const double* u;
    StatsSink sink;
};

// Kernel variants of the batched term launch, chosen by the autotuner:
// planes per tile and whether blocks loop over tiles.
struct BatchVariant {
    int tile_z;
    int persistent;
};
int batch_variant_count(et_precision prec);
BatchVariant batch_variant(et_precision prec, int v);

template <typename T>
cudaError_t launch_batch_term(et_operator op, int variant, const BatchTerm<T>* d, int count, long long tiles,
                              int sms, cudaStream_t stream);
cudaError_t launch_batch_term(et_operator op, int variant, const BatchTerm<float2>* d, int count, long long tiles,
                              int sms, cudaStream_t stream);
template <typename T>
cudaError_t launch_batch_residual(et_operator op, int scheme, const BatchResidual<T>* d, int count, long long tiles,
                                  unsigned* flags, cudaStream_t stream);
cudaError_t launch_batch_stats(const BatchStats* d, int count, cudaStream_t stream);

// Kernel launchers (et_kernels.cu).  All enqueue on `stream` and return the
// launch error.  launch_coeffs reads the diffusion field as D * dscale.
cudaError_t launch_coeffs(const Geom& G, const double* D, double inv_h2, et_operator op,
                          double* const w[5], unsigned long long* rmax_bits, unsigned* flags,
                          cudaStream_t stream, double dscale = 1.0);
// Typed copies of w[0..3] scaled by `scale` (1 / nu for the FP32 and DF64 forms).
cudaError_t launch_convert_weights(const Geom& G, const double* const w[4], float* const wf[4],
                                   double scale, cudaStream_t stream);
cudaError_t launch_convert_weights(const Geom& G, const double* const w[4], float2* const wd[4],
                                   double scale, cudaStream_t stream);
// The FP64 residual of the F64 form (instantiated for double): dt_shift is
// rho - mu (folded scheme) or -mu (exponential Euler); the diagonal is stored
// times dt_scale.
template <typename T>
cudaError_t launch_residual(const Geom& G, et_operator op, const double* u, Weights<double> W,
                            double rho, double dt_shift, double dt_scale, et_scheme scheme, T* b,
                            T* dt, unsigned* flags, cudaStream_t stream, unsigned long long* wnorm = nullptr);
// FP32 term with four voxels per thread (et_quad.cu), the same arithmetic as
// the one-voxel kernel; needs nx % 4 == 0 and 16-byte aligned fields.
bool quad_eligible(const Geom& G, const Weights<float>& W, const TermArgs<float>& a);
cudaError_t launch_term_quad(const Geom& G, et_operator op, const Weights<float>& W, const TermArgs<float>& a,
                             cudaStream_t stream);
template <typename T>
cudaError_t launch_term(const Geom& G, et_operator op, Weights<T> W, const TermArgs<T>& a,
                        cudaStream_t stream);
// double-float form (et_df64.cu)
cudaError_t launch_term(const Geom& G, et_operator op, Weights<float2> W, const TermArgs<float2>& a,
                        cudaStream_t stream);
// Tensor maps of the two-term kernel for one grid and launch (et_fused.cu):
// z_j with a two-voxel halo, the weights, the diagonal and b.
struct PairMaps {
    CUtensorMap zj, w0, w1, w2, dt, b, w3;
    // voxels whose six off-diagonal weights are zero take dt z + beta b only
    int skip_zero;
};

// One grid of a batched two-term launch.
template <typename T>
struct BatchPair {
    PairMaps M;
    Geom G;
    TermArgs<T> a1, a2;
    long long tile_begin;
    int tz;  // planes per column segment
};

// Two consecutive terms of one sub-step (a1 not last) in one TMA-fed launch
// (et_fused.cu): a1's outputs are not written, a2's are.  probe_ns > 0 (a test
// hook, et_options.timeout_probe_us) makes each block first wait that long on
// a barrier nothing completes, so the launch reports ET_FLAG_TIMEOUT.  The plan holds the
// tensor maps of one grid's fields: typed weights wt[0..3], b, the diagonal
// dt and the vectors Y0, Y1, Z0, Z1 (a1.zin must be b or one of these).
// pair_plan_create returns nullptr where TMA cannot address the rows.
struct PairPlan;
PairPlan* pair_plan_create(const Geom& G, et_precision prec, const void* const wt[4], const void* b, const void* dt,
                           const void* const yz[4]);
void pair_plan_destroy(PairPlan* P);
// Whether the plan's launches skip the products of voxels without
// off-diagonal entries (set by et_set_coeffs from options.every_row).
void pair_plan_set_skip(PairPlan* P, bool skip);
template <typename T>
cudaError_t launch_term_pair(const PairPlan* P, const Geom& G, et_operator op, const TermArgs<T>& a1,
                             const TermArgs<T>& a2, unsigned* flags, cudaStream_t stream,
                             unsigned long long probe_ns = 0);
// Fills the tensor maps of a pair launch (a1.zin selects the z_j map); false
// if a1.zin is none of the plan's vectors.
bool pair_maps(const PairPlan* P, const void* zin, PairMaps* out);
// Tensor maps for a pair launch on other buffers than the plan's (z_j, b and
// the diagonal encoded now; the weights from the plan).
bool pair_maps_for(const PairPlan* P, const Geom& G, et_precision prec, const void* zin, const void* b,
                   const void* dt, PairMaps* out);
// A pair launch with explicit tensor maps; a1.zout non-null also stores the
// first term (a recorded chain).
template <typename T>
cudaError_t launch_term_pair_maps(const PairMaps& M, const Geom& G, et_operator op, const TermArgs<T>& a1,
                                  const TermArgs<T>& a2, unsigned* flags, cudaStream_t stream,
                                  unsigned long long probe_ns = 0);
// Whether two terms per launch beat two one-term launches for this operator
// and form (resident blocks per SM of the pair kernel: at least 2).
bool pair_preferred(et_operator op, et_precision prec);
// Planes per column segment of a grid in a batched launch.
int batch_pair_tz(const Geom& G);
// Batched two-term launch over count grids (device table d, tiles in all).
template <typename T>
cudaError_t launch_batch_term_pair(et_operator op, const BatchPair<T>* d, int count, long long tiles, int sms,
                                   unsigned* flags, cudaStream_t stream, unsigned long long probe_ns = 0);
// Two consecutive Horner terms of sub-step 0 in one launch, one 16-byte vector
// of each field per thread (four FP32 voxels), on full-width tiles of th rows
// and tz planes, fed by asynchronous copies (et_quadpair.cu); the per-voxel
// arithmetic of the one-term kernels.  Eligible: FP32 (instantiated for
// float; DF64 keeps the TMA-fed kernel), nx % 4 == 0, nx <= 256, 16-byte
// aligned fields, n < 2^31, a1 and a2 Horner terms (a1 not last, a2 not
// scaled) on the same b and diagonal.
template <typename T>
struct VecPairGrid {
    Geom G;
    Weights<T> W;
    TermArgs<T> a1, a2;
    long long tile_begin;  // first tile of this grid in a batched launch
    int th, tz;            // rows and planes of a tile
};
template <typename T>
bool vec_pair_eligible(const Geom& G, et_operator op, const Weights<T>& W, const TermArgs<T>& a1,
                       const TermArgs<T>& a2);
template <typename T>
int vec_pair_rows(const Geom& G);
template <typename T>
long long vec_pair_tiles(const Geom& G, int tz);
template <typename T>
VecPairGrid<T> vec_pair_grid(const Geom& G, const Weights<T>& W, const TermArgs<T>& a1, const TermArgs<T>& a2,
                             int tz, long long tile_begin);
template <typename T>
cudaError_t launch_term_vec_pair(const Geom& G, et_operator op, const Weights<T>& W, const TermArgs<T>& a1,
                                 const TermArgs<T>& a2, cudaStream_t stream);
// Batched launch over count grids (device table d, tiles in all).
template <typename T>
cudaError_t launch_batch_term_vec_pair(et_operator op, const VecPairGrid<T>* d, int count, long long tiles, int sms,
                                       cudaStream_t stream);
cudaError_t prime_launch_limits_quad_pair();
// min, max and sum of u and the non-finite flag into the step record.
cudaError_t launch_stats(const Geom& G, const double* u, const StatsSink& sink, cudaStream_t stream);
// Adjoint launchers (et_adjoint.cu).
template <typename T>
cudaError_t launch_adj_term(const Geom& G, et_operator op, Weights<T> W, const AdjTermArgs<T>& a,
                            cudaStream_t stream);
template <typename T>
cudaError_t launch_adj_step(const Geom& G, et_operator op, Weights<double> W, const double* u, const T* bbar,
                            const T* cbar, const T* sstep, const double* ubar_next, double rho, et_scheme scheme,
                            double* ubar, double* sbar_acc, double* rbar_acc, cudaStream_t stream);
// Deterministic sum of v[0..n) into *out; partial holds sum_partials_bytes().
size_t sum_partials_bytes();
cudaError_t launch_sum(long long n, const double* v, double* partial, double* out, cudaStream_t stream);
// out[p] = u[p] + y[p] in FP64 (y widened as the last term of a step adds it)
template <typename T>
cudaError_t launch_add_widen(long long n, const double* u, const T* y, double* out, cudaStream_t stream);
// dst[p] = src[p] * scale as a pair (df64::from_double of the FP64 product)
cudaError_t launch_split(long long n, const double* src, double scale, float2* dst, cudaStream_t stream);
// The residual of the FP32 and DF64 forms in pair arithmetic from the pair
// copy of u: b = nu (L~ u) + rho u (1 - u) and the diagonal w4~ + shift + k u,
// stored in the form's value type.
// PairResidualArgs of a grid with scaling nu, rate rho and the diagonal shift
// (rho for the folded reaction, minus the series shift mu).
inline PairResidualArgs pair_residual_args(const float2* ush, float2* const w[5], double nu, double rho,
                                           double dt_shift, et_scheme scheme) {
    PairResidualArgs R;
    R.ush = ush;
    for (int a = 0; a < 5; ++a) R.W.w[a] = w[a];
    R.nu = Scalar<float2>::make(nu);
    R.rho = Scalar<float2>::make(rho);
    R.shift = Scalar<float2>::make(dt_shift / nu);
    R.k_u = Scalar<float2>::make(scheme == ET_SCHEME_ROSENBROCK ? -2.0 * rho / nu : 0.0);
    return R;
}
template <typename TO>
cudaError_t launch_residual_df64(const Geom& G, et_operator op, const PairResidualArgs& R, et_scheme scheme, TO* b,
                                 TO* dt, unsigned* flags, cudaStream_t stream, unsigned long long* wnorm = nullptr);
// dst[p] = (float)(src[p] * scale)
cudaError_t launch_cast(long long n, const double* src, double scale, float* dst, cudaStream_t stream);

// Factor C of the a-posteriori truncation estimate C max|b| / max|u^n| of one
// step with s sub-steps of degree m (et_api.cu).
double truncation_factor(double tau, double rmax, double rho, et_scheme scheme, et_precision precision,
                         const et_options* options, int s, int m);
// The truncation tolerance the options resolve to (options.tol or the form's default).
double resolved_tol(const et_options* options, et_precision precision);
// Looks up launch limits (resident blocks per SM) before any stream capture.
cudaError_t prime_launch_limits();
cudaError_t prime_launch_limits_df64();
cudaError_t prime_launch_limits_pair();

}  // namespace et
