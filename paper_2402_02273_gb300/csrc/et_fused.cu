// Two consecutive Taylor terms in one launch (temporal blocking) for the FP32
// and DF64 forms on sm_103a, fed by TMA.
//
// Terms j and j+1 of one sub-step are
//     z_a = A~ z_j + beta_1 b,          z_b = A~ z_a + beta_2 b,
// (with the running sums  S_a = base + g_1 z_a,  S_b = S_a + g_2 z_b  outside
// the Horner sub-step).  A block owns a 32 x 8 column of the grid and marches
// through a segment of its z-range.  For every plane q one thread issues TMA
// tile loads (cp.async.bulk.tensor) of z_j with a two-voxel halo (box 36 x 12
// for DF64, 40 x 12 for FP32, whose x origin is moved to a 16-byte boundary)
// and of the weights, the diagonal and b with a one-voxel halo into a ring of
// shared-memory stages completed by an mbarrier; loads run one plane ahead of
// the arithmetic.  The TMA unit fills voxels outside the grid with zeros, so
// the zero-flux walls need no branches: every weight of an outside voxel and
// every outside value reads as 0, exactly the terms the unfused kernels skip.
// The first term is evaluated on the one-voxel halo of the plane (34 x 10, one
// voxel per thread of an 11-warp block) into a four-plane shared ring, the
// second on the interior (8 warps) two planes behind, so the two need only the
// one barrier per plane; the plane-below values of the first term are carried
// in registers.  z_a never reaches memory: a pair of terms moves about
// the bytes of one unfused term.  The per-voxel arithmetic (order of the
// multiply-adds, pair arithmetic for DF64) is that of the unfused kernels, so
// both give identical numbers.
//
// Eligible grids: rows of a 16-byte multiple (nx even for DF64, a multiple of
// 4 for FP32), as TMA requires of the global strides; other grids run one
// term per launch.  The same body serves one grid (kernel parameters), a
// table of grids (the batched form) and recorded chains of the adjoint (the
// first term is then stored too, to the record).
//
// Every mbarrier wait is bounded; a wait that runs out sets ET_FLAG_TIMEOUT,
// waits (bounded) for the block's copies still in flight and ends the block.
// A test hook (probe_ns > 0) makes every block's first wait also wait, for at
// most probe_ns, on a barrier that nothing completes, so that this path runs
// without stalling the device.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>
#include <new>
#include <type_traits>

#include "et_arith.h"
#include "et_df64_arith.h"
#include "et_internal.h"

namespace et {

struct PairPlan {
    CUtensorMap zj[5];       // 12-row boxes of b, Y0, Y1, Z0, Z1
    const void* zj_ptr[5];
    CUtensorMap w0, w1, w2, dt, b, w3;  // w1: 11 rows; the others 10
    int skip_zero = 1;
};

namespace {

constexpr int kPairThreads = 352;       // 11 warps: one per voxel of the 34 x 10 halo plane
constexpr int kHaloX = kBlockX + 2;     // 34
constexpr int kHaloY = kBlockY + 2;     // 10
constexpr int kHalo = kHaloX * kHaloY;  // 340
constexpr int kRing = 4;                // z_a planes kept: the second term's three and the one being written
constexpr int kWaitTries = 1 << 24;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

template <typename T>
struct Shape {
    static constexpr int ES = sizeof(T);
    static constexpr int BX = ES == 8 ? 36 : 40;  // box width (x origin x0 - XO, 16-byte aligned)
    static constexpr int XO = ES == 8 ? 2 : 4;
    __host__ __device__ static constexpr int box(int rows) { return rows * BX * ES; }
    __host__ __device__ static constexpr int pad(int b) { return (b + 127) / 128 * 128; }
    static constexpr int kZj = 0;                        // 12 rows from y0 - 2
    static constexpr int kW1 = pad(box(12));             // 11 rows from y0 - 2
    static constexpr int kW0 = kW1 + pad(box(11));       // 10 rows from y0 - 1 (also w2, dt, b, w3)
    static constexpr int kW2 = kW0 + pad(box(10));
    static constexpr int kDt = kW2 + pad(box(10));
    static constexpr int kB = kDt + pad(box(10));
    static constexpr int kW3 = kB + pad(box(10));
    __host__ __device__ static constexpr int stage_bytes(bool literal) { return kW3 + (literal ? pad(box(10)) : 0); }
    __host__ __device__ static constexpr unsigned tx_bytes(bool literal) {
        return box(12) + box(11) + 4 * box(10) + (literal ? box(10) : 0);
    }
    // stages loaded ahead of the one consumed: two where three blocks per SM
    // still fit (FP32, conservative: 68 KB a block), else one
    __host__ __device__ static constexpr int prefetch(bool literal) { return (ES == 4 && !literal) ? 2 : 1; }
    // + planes L - 3 (second term), L - 1, L (first term), L - 2
    __host__ __device__ static constexpr int stages(bool literal) { return prefetch(literal) + 4; }
    __host__ __device__ static constexpr int smem_bytes(bool literal) {
        // + one mbarrier per stage and the probe barrier
        return 128 + stages(literal) * stage_bytes(literal) + kRing * kHalo * ES + (stages(literal) + 1) * 8;
    }
};

// Kernel variants: Horner pair (sub-step 0) or running-sum pair; the first
// term scaled by zscale; the sum's base read from z_j itself (first term of a
// later sub-step) instead of the running sum.
// kModeTable: the term shapes are read per grid (batched launches).
enum : int { kModeHorner = 1, kModeZscale = 2, kModeBaseZ = 4, kModeTable = 8 };

// ---- mbarrier and TMA (inline PTX) -----------------------------------------

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity to complete, for at most about
// limit_ns of the global timer (and kWaitTries polls).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long limit_ns = kWaitNs) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (int i = 0; i < kWaitTries; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// ---- the kernel --------------------------------------------------------------

// Where the tiles of a launch come from: one grid (kernel parameters) or a
// table of grids (the batched form), tiles numbered grid after grid.
template <typename T>
struct OneGrid {
    const PairMaps* M;
    const Geom* G;
    const TermArgs<T>* a1;
    const TermArgs<T>* a2;
    int tz;
    long long total;
    __device__ __forceinline__ int find(long long) const { return 0; }
    __device__ __forceinline__ const PairMaps* maps(int) const { return M; }
    __device__ __forceinline__ const Geom& geom(int) const { return *G; }
    __device__ __forceinline__ const TermArgs<T>& first(int) const { return *a1; }
    __device__ __forceinline__ const TermArgs<T>& second(int) const { return *a2; }
    __device__ __forceinline__ int planes(int) const { return tz; }
    __device__ __forceinline__ long long begin(int) const { return 0; }
};

template <typename T>
struct GridTable {
    const BatchPair<T>* d;
    int count;
    long long total;
    __device__ __forceinline__ int find(long long tile) const {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (d[mid].tile_begin <= tile) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    }
    __device__ __forceinline__ const PairMaps* maps(int i) const { return &d[i].M; }
    __device__ __forceinline__ const Geom& geom(int i) const { return d[i].G; }
    __device__ __forceinline__ const TermArgs<T>& first(int i) const { return d[i].a1; }
    __device__ __forceinline__ const TermArgs<T>& second(int i) const { return d[i].a2; }
    __device__ __forceinline__ int planes(int i) const { return d[i].tz; }
    __device__ __forceinline__ long long begin(int i) const { return d[i].tile_begin; }
};

// A tile: its grid's geometry and its place in it.
struct TileGeom {
    int nx, ny, nz;
    long long sy, sz;
    int x0, y0, k0, k1;
};

template <typename Src>
__device__ __forceinline__ TileGeom tile_of(const Src& src, int gi, long long tile) {
    const Geom& G = src.geom(gi);
    TileGeom g;
    g.nx = G.nx;
    g.ny = G.ny;
    g.nz = G.nz;
    g.sy = G.sy;
    g.sz = G.sz;
    const int tz = src.planes(gi);
    const int tiles_x = (g.nx + kBlockX - 1) / kBlockX;
    const int tiles_y = (g.ny + kBlockY - 1) / kBlockY;
    const long long lt = tile - src.begin(gi);
    g.x0 = (int)(lt % tiles_x) * kBlockX;
    const long long rest = lt / tiles_x;
    g.y0 = (int)(rest % tiles_y) * kBlockY;
    g.k0 = (int)(rest / tiles_y) * tz;
    g.k1 = min(g.k0 + tz, g.nz);
    return g;
}

template <int OP, typename T, int MODE, typename Src>
__device__ __forceinline__ void pair_body(const Src& src, unsigned* flags, unsigned long long probe_ns) {
    using S = Shape<T>;
    using A = Arith<T>;
    constexpr bool kLit = OP == ET_OP_LITERAL;
    constexpr bool kTable = (MODE & kModeTable) != 0;
    constexpr int BX = S::BX, XO = S::XO;
    constexpr int kStageBytes = S::stage_bytes(kLit);
    constexpr unsigned kTx = S::tx_bytes(kLit);
    constexpr int kPrefetch = S::prefetch(kLit);
    constexpr int kStages = S::stages(kLit);
    extern __shared__ unsigned char smem_raw[];
    unsigned char* const base = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
    T* const za = reinterpret_cast<T*>(base + kStages * kStageBytes);  // [kRing][kHalo], slot = plane & 3
    uint64_t* const full = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes + kRing * kHalo * sizeof(T));
    const int t = threadIdx.x;
    if (t == 0) {
        for (int s = 0; s <= kStages; ++s) mbar_init(&full[s], 1);  // full[kStages]: the probe's
        mbar_fence_init();
    }
    __syncthreads();
    const T zero = A::zero();

    // first-term voxel of this thread on the halo plane, second-term voxel inside
    const bool has_b = t < kHalo;
    const int hx = t % kHaloX, hy = t / kHaloX;
    const int bz = (hy + 1) * BX + hx - 1 + XO;   // in a 12-row box
    const int b10 = hy * BX + hx - 1 + XO;        // in a 10-row box
    const int b11 = (hy + 1) * BX + hx - 1 + XO;  // in the 11-row box
    const bool has_c = t < kThreads;
    const int cx = t % kBlockX, cy = t / kBlockX;
    const int c10 = (cy + 1) * BX + cx + XO;
    const int c11 = (cy + 2) * BX + cx + XO;
    const int c12 = (cy + 2) * BX + cx + XO;
    const int ca = (cy + 1) * kHaloX + cx + 1;

    // ring bookkeeping, the same on every thread
    unsigned issued = 0, waited = 0;
    int islot = 0, wslot = 0;
    unsigned wpar = 0;
    const unsigned char *s3 = nullptr, *s2 = nullptr, *sp = nullptr, *sc = nullptr;  // planes L - 3 .. L
    const long long total = src.total;

    // The block's tiles (blockIdx.x, + gridDim.x, ...) form one stream of
    // stages, planes k0 - 2 .. k1 + 1 of each; loads run kPrefetch stages ahead
    // in that stream, across tile (and grid) boundaries.
    long long itile = blockIdx.x;
    const PairMaps* iM = nullptr;
    int ix0 = 0, iy0 = 0, ik1 = 0, iq = 0;
    auto issue_tile = [&]() {
        if (itile >= total) return;
        const int gi = src.find(itile);
        const TileGeom g = tile_of(src, gi, itile);
        iM = src.maps(gi);
        ix0 = g.x0;
        iy0 = g.y0;
        ik1 = g.k1;
        iq = g.k0 - 2;
    };
    issue_tile();
    auto issue_next = [&]() {
        if (itile >= total) return;
        if (t == 0) {
            unsigned char* st = base + islot * kStageBytes;
            uint64_t* bar = &full[islot];
            mbar_expect_tx(bar, kTx);
            tma_load(st + S::kZj, &iM->zj, ix0 - XO, iy0 - 2, iq, bar);
            tma_load(st + S::kW1, &iM->w1, ix0 - XO, iy0 - 2, iq, bar);
            tma_load(st + S::kW0, &iM->w0, ix0 - XO, iy0 - 1, iq, bar);
            tma_load(st + S::kW2, &iM->w2, ix0 - XO, iy0 - 1, iq, bar);
            tma_load(st + S::kDt, &iM->dt, ix0 - XO, iy0 - 1, iq, bar);
            tma_load(st + S::kB, &iM->b, ix0 - XO, iy0 - 1, iq, bar);
            if (kLit) tma_load(st + S::kW3, &iM->w3, ix0 - XO, iy0 - 1, iq, bar);
        }
        ++issued;
        if (++islot == kStages) islot = 0;
        if (++iq > ik1 + 1) {
            itile += gridDim.x;
            issue_tile();
        }
    };
    // next plane: issue one more stage of the stream, wait for this one
    auto advance = [&]() -> bool {
        issue_next();
        s3 = s2;
        s2 = sp;
        sp = sc;
        sc = base + wslot * kStageBytes;
        const bool ok = mbar_wait(&full[wslot], wpar);
        ++waited;
        if (++wslot == kStages) {
            wslot = 0;
            wpar ^= 1u;
        }
        return ok;
    };
    // true (for every thread) if some wait ran out: record it, let the copies
    // in flight land, and stop
    auto timed_out = [&](bool ok) -> bool {
        if (!__syncthreads_or(!ok)) return false;
        if (t == 0) atomicOr(flags, ET_FLAG_TIMEOUT);
        for (unsigned m = waited - 1; m < issued; ++m) mbar_wait(&full[m % kStages], (m / kStages) & 1u);
        return true;
    };

    for (int d = 0; d < kPrefetch; ++d) issue_next();
    for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int gi = src.find(tile);
        const TileGeom g = tile_of(src, gi, tile);
        const TermArgs<T>& a1 = src.first(gi);
        const TermArgs<T>& a2 = src.second(gi);
        // the terms' scalars and outputs, in registers
        const bool kHorner = kTable ? a1.horner != 0 : (MODE & kModeHorner) != 0;
        const bool kZs = kTable ? a1.has_zscale != 0 : (MODE & kModeZscale) != 0;
        const bool kBaseZ = kTable ? a1.base_mode == 2 : (MODE & kModeBaseZ) != 0;
        const T zscale1 = a1.zscale, beta1 = a1.beta, beta2 = a2.beta, g1 = a1.g, g2 = a2.g, gamma2 = a2.gamma;
        const bool hb1 = a1.has_beta != 0, hb2 = a2.has_beta != 0, last2 = a2.last != 0;
        // DF64 (bound by its pair arithmetic) skips the products of voxels
        // without off-diagonal entries; the FP32 instances evaluate every
        // voxel (the test would push the batched FP32 kernel into spills)
        const bool skip = sizeof(T) == 8 && src.maps(gi)->skip_zero != 0;
        const T* const ysrc = a1.yacc;
        T* const zfirst = kTable ? nullptr : a1.zout;  // nullptr unless the chain is recorded
        T* const zout = a2.zout;
        T* const yout = a2.yacc;
        double* const uout = a2.u;
        const int k0 = g.k0, k1 = g.k1;
        const int Llast = k1 + 1;  // planes k0 - 2 .. k1 + 1 are loaded
        const int gx = g.x0 + cx, gy = g.y0 + cy;
        const bool store_c = has_c && gx < g.nx && gy < g.ny;
        const long long pc = gx + g.sy * gy;  // column offset of the second-term voxel
        const long long sz = g.sz;

        T b_zm = zero, b_w2m = zero;  // z_j and w2 of the plane below, at the halo voxel
        T c_w2m = zero;               // w2 of the plane below, at the interior voxel

        // first term on plane q = L - 1 from stages sp (q) and sc (q + 1); returns
        // z_a at the halo voxel, with its z_j and +z weight for the carries
        auto first_val = [&](int q, T& zc, T& wzp) -> T {
            (void)q;
            const T* Zp = reinterpret_cast<const T*>(sp + S::kZj);
            const T* Zc = reinterpret_cast<const T*>(sc + S::kZj);
            const T* W0 = reinterpret_cast<const T*>(sp + S::kW0);
            const T* W1 = reinterpret_cast<const T*>(sp + S::kW1);
            const T* W2 = reinterpret_cast<const T*>(sp + S::kW2);
            const T* DT = reinterpret_cast<const T*>(sp + S::kDt);
            zc = Zp[bz];
            T wxm, wym, wzm;
            if (kLit) {
                const T w3 = reinterpret_cast<const T*>(sp + S::kW3)[b10];
                wxm = w3;
                wym = w3;
                wzm = w3;
            } else {
                wxm = W0[b10 - 1];
                wym = W1[b11 - BX];
                wzm = b_w2m;
            }
            const T bval = hb1 ? reinterpret_cast<const T*>(sp + S::kB)[b10] : zero;
            wzp = W2[b10];
            if (kZs)
                return A::template stencil<true>(DT[b10], zc, W0[b10], Zp[bz + 1], wxm, Zp[bz - 1], W1[b11],
                                                 Zp[bz + BX], wym, Zp[bz - BX], wzp, Zc[bz], wzm, b_zm, zscale1, hb1,
                                                 beta1, bval);
            return A::template stencil<false>(DT[b10], zc, W0[b10], Zp[bz + 1], wxm, Zp[bz - 1], W1[b11],
                                              Zp[bz + BX], wym, Zp[bz - BX], wzp, Zc[bz], wzm, b_zm, zscale1, hb1,
                                              beta1, bval);
        };
        auto first = [&](int q) {
            if (!has_b) return;
            T zc, wzp;
            const T v = first_val(q, zc, wzp);
            za[(q & 3) * kHalo + t] = v;
            b_zm = zc;
            b_w2m = wzp;
        };
        // second term on plane q = L - 3 from stage s3 (q) and the z_a ring;
        // returns z_b at the interior voxel (computed also for voxels past the
        // grid's edge, which are not stored)
        auto second_val = [&](int q, T& acen, T& wzp, T& bval) -> T {
            const T* Ac = za + (q & 3) * kHalo;
            const T* Ap = za + ((q + 1) & 3) * kHalo;
            const T* Am = za + ((q - 1) & 3) * kHalo;
            const T* W0 = reinterpret_cast<const T*>(s3 + S::kW0);
            const T* W1 = reinterpret_cast<const T*>(s3 + S::kW1);
            const T* DT = reinterpret_cast<const T*>(s3 + S::kDt);
            wzp = reinterpret_cast<const T*>(s3 + S::kW2)[c10];
            acen = Ac[ca];
            T wxm, wym, wzm;
            if (kLit) {
                const T w3 = reinterpret_cast<const T*>(s3 + S::kW3)[c10];
                wxm = w3;
                wym = w3;
                wzm = w3;
            } else {
                wxm = W0[c10 - 1];
                wym = W1[c11 - BX];
                wzm = c_w2m;
            }
            bval = hb2 ? reinterpret_cast<const T*>(s3 + S::kB)[c10] : zero;
            return A::template stencil<false>(DT[c10], acen, W0[c10], Ac[ca + 1], wxm, Ac[ca - 1], W1[c11],
                                              Ac[ca + kHaloX], wym, Ac[ca - kHaloX], wzp, Ap[ca], wzm, Am[ca], zero,
                                              hb2, beta2, bval);
        };
        auto second_store = [&](int q, T zb, T acen) {
            const long long p = pc + sz * q;
            if (zfirst) zfirst[p] = acen;  // a recorded chain keeps the first term too
            if (kHorner) {
                if (!last2) {
                    zout[p] = zb;
                } else {
                    const T r = A::scale(gamma2, zb);
                    if (uout) uout[p] += A::widen(r);
                    else yout[p] = r;
                }
            } else {
                const T sb0 = kBaseZ ? reinterpret_cast<const T*>(s3 + S::kZj)[c12] : ysrc[p];
                const T sa = A::axpy(g1, acen, sb0);
                T sb = A::axpy(g2, zb, sa);
                if (!last2) {
                    zout[p] = zb;
                    yout[p] = sb;
                } else {
                    sb = A::scale(gamma2, sb);
                    if (uout) uout[p] += A::widen(sb);
                    else yout[p] = sb;
                }
            }
        };
        auto second = [&](int q) {
            if (!has_c) return;
            T acen, wzp, bval;
            const T zb = second_val(q, acen, wzp, bval);
            if (store_c) second_store(q, zb, acen);
            c_w2m = wzp;
        };
        // both terms in one stretch of code (the first 8 warps), so that the
        // two independent chains of dependent additions interleave
        auto both = [&](int qb, int qc) {
            T zc, wzpb, acen, wzpc, bval;
            const T v = first_val(qb, zc, wzpb);
            const T zb = second_val(qc, acen, wzpc, bval);
            za[(qb & 3) * kHalo + t] = v;
            b_zm = zc;
            b_w2m = wzpb;
            if (store_c) second_store(qc, zb, acen);
            c_w2m = wzpc;
        };
        // Voxels without off-diagonal entries (six zero face weights; D = 0
        // around them): the term is dt z + beta b, the stencil's value up to
        // the sign of a zero.  A warp takes that path only when all its voxels
        // qualify, so the full path keeps its interleaved code.
        auto zero_first = [&]() -> bool {  // the first-term voxel on plane L - 1
            if (!has_b) return true;
            const T* W0 = reinterpret_cast<const T*>(sp + S::kW0);
            const T* W1 = reinterpret_cast<const T*>(sp + S::kW1);
            const T* W2 = reinterpret_cast<const T*>(sp + S::kW2);
            if (kLit) {
                const T w3 = reinterpret_cast<const T*>(sp + S::kW3)[b10];
                return A::zero6(W0[b10], W1[b11], W2[b10], w3, w3, w3);
            }
            return A::zero6(W0[b10], W0[b10 - 1], W1[b11], W1[b11 - BX], W2[b10], b_w2m);
        };
        auto zero_second = [&]() -> bool {  // the second-term voxel on plane L - 3
            const T* W0 = reinterpret_cast<const T*>(s3 + S::kW0);
            const T* W1 = reinterpret_cast<const T*>(s3 + S::kW1);
            const T* W2 = reinterpret_cast<const T*>(s3 + S::kW2);
            if (kLit) {
                const T w3 = reinterpret_cast<const T*>(s3 + S::kW3)[c10];
                return A::zero6(W0[c10], W1[c11], W2[c10], w3, w3, w3);
            }
            return A::zero6(W0[c10], W0[c10 - 1], W1[c11], W1[c11 - BX], W2[c10], c_w2m);
        };
        auto first_diag = [&](int q) {
            if (!has_b) return;
            const T zc = reinterpret_cast<const T*>(sp + S::kZj)[bz];
            const T dt = reinterpret_cast<const T*>(sp + S::kDt)[b10];
            const T bval = hb1 ? reinterpret_cast<const T*>(sp + S::kB)[b10] : zero;
            za[(q & 3) * kHalo + t] = kZs ? A::template diag<true>(dt, zc, zscale1, hb1, beta1, bval)
                                          : A::template diag<false>(dt, zc, zscale1, hb1, beta1, bval);
            b_zm = zc;
            b_w2m = reinterpret_cast<const T*>(sp + S::kW2)[b10];
        };
        auto second_diag = [&](int q) {
            const T acen = za[(q & 3) * kHalo + ca];
            const T dt = reinterpret_cast<const T*>(s3 + S::kDt)[c10];
            const T bval = hb2 ? reinterpret_cast<const T*>(s3 + S::kB)[c10] : zero;
            const T zb = A::template diag<false>(dt, acen, zero, hb2, beta2, bval);
            if (store_c) second_store(q, zb, acen);
            c_w2m = reinterpret_cast<const T*>(s3 + S::kW2)[c10];
        };

        // Plane L arrives: the first term runs on plane L - 1, the second on
        // plane L - 3, whose z_a neighbours were all written in earlier
        // iterations, so one barrier per plane separates the two.  Planes
        // k0 - 2 .. k0 + 2 fill the carries and the z_a ring.
        bool ok = advance();
        // test hook: a wait that nothing ends, bounded by probe_ns
        if (probe_ns && tile == blockIdx.x) ok = mbar_wait(&full[kStages], 0, probe_ns) && ok;
        if (timed_out(ok)) return;
        ok = advance();
        if (ok && has_b) {
            b_zm = reinterpret_cast<const T*>(sp + S::kZj)[bz];
            b_w2m = reinterpret_cast<const T*>(sp + S::kW2)[b10];
        }
        if (timed_out(ok)) return;
        ok = advance();
        if (ok) first(k0 - 1);
        if (timed_out(ok)) return;
        ok = advance();
        if (ok) first(k0);
        if (timed_out(ok)) return;
        ok = advance();
        if (ok) first(k0 + 1);
        if (has_c) c_w2m = reinterpret_cast<const T*>(s3 + S::kW2)[c10];  // plane k0 - 1
        if (timed_out(ok)) return;
        for (int L = k0 + 3; L <= Llast; ++L) {
            ok = advance();
            // (a first term from a stage whose load failed is never read: the
            // block stops at the vote below)
            if (has_c) {
                if (skip && __all_sync(0xffffffffu, zero_first() && zero_second())) {
                    first_diag(L - 1);
                    second_diag(L - 3);
                } else {
                    both(L - 1, L - 3);
                }
            } else if (skip && __all_sync(0xffffffffu, zero_first())) {
                first_diag(L - 1);
            } else {
                first(L - 1);
            }
            if (timed_out(ok)) return;
        }
        // plane k1 - 1: its z_a neighbours are complete
        s3 = s2;
        second(k1 - 1);
        __syncthreads();
    }
}

// Resident blocks per SM that the shared memory allows: FP32 3, DF64 2.
template <int OP, typename T, int MODE>
__global__ void __launch_bounds__(kPairThreads, sizeof(T) == 4 ? 3 : 2)
term2_kernel(const __grid_constant__ PairMaps M, const __grid_constant__ Geom G,
             const __grid_constant__ TermArgs<T> a1, const __grid_constant__ TermArgs<T> a2, int tz,
             unsigned* flags, unsigned long long probe_ns) {
    const long long total = (long long)((G.nx + kBlockX - 1) / kBlockX) * ((G.ny + kBlockY - 1) / kBlockY) *
                            ((G.nz + tz - 1) / tz);
    const OneGrid<T> src{&M, &G, &a1, &a2, tz, total};
    pair_body<OP, T, MODE>(src, flags, probe_ns);
}

template <int OP, typename T>
__global__ void __launch_bounds__(kPairThreads, sizeof(T) == 4 ? 3 : 2)
batch_term2_kernel(const BatchPair<T>* __restrict__ d, int count, long long total, unsigned* flags,
                   unsigned long long probe_ns) {
    const GridTable<T> src{d, count, total};
    pair_body<OP, T, kModeTable>(src, flags, probe_ns);
}

template <typename K>
int blocks_per_sm_of(K kernel, int smem) {
    int b = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kPairThreads, smem) != cudaSuccess || b < 1)
        b = 1;
    return b;
}

template <int OP, typename T, int MODE>
int pair_blocks_per_sm() {
    static int cached = 0;
    if (!cached) cached = blocks_per_sm_of(term2_kernel<OP, T, MODE>, Shape<T>::smem_bytes(OP == ET_OP_LITERAL));
    return cached;
}

template <int OP, typename T>
int batch_pair_blocks_per_sm() {
    static int cached = 0;
    if (!cached) cached = blocks_per_sm_of(batch_term2_kernel<OP, T>, Shape<T>::smem_bytes(OP == ET_OP_LITERAL));
    return cached;
}

// Planes per column segment: the fewest waves of segments over the resident
// blocks times the planes a segment costs (its own plus about three: the
// first term runs on two more planes than the second, and the pipeline
// fills).  Measured on 128^3 grids, long segments win over balanced ones.
// 4..64 planes.
int choose_tz(const Geom& G, long long capacity) {
    const long long cols = (long long)((G.nx + kBlockX - 1) / kBlockX) * ((G.ny + kBlockY - 1) / kBlockY);
    int best = 4;
    double best_cost = 1e300;
    for (int tz = 4; tz <= 64; ++tz) {
        const long long tiles = cols * ((G.nz + tz - 1) / tz);
        const long long waves = (tiles + capacity - 1) / capacity;
        const double cost = (double)waves * (tz + 3.0);
        if (cost < best_cost) {
            best_cost = cost;
            best = tz;
        }
        if (tz >= G.nz) break;
    }
    return best;
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool encode(CUtensorMap* m, const void* ptr, const Geom& G, int es, int bx, int rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn || !ptr || (reinterpret_cast<uintptr_t>(ptr) & 15u)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)G.nx, (cuuint64_t)G.ny, (cuuint64_t)G.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)G.nx * es, (cuuint64_t)G.nx * G.ny * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType type = es == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    return fn(m, type, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The pair kernel covers the term shapes the chain planner emits.
template <typename T>
bool pair_shape_ok(const TermArgs<T>& a1, const TermArgs<T>& a2) {
    if (a1.last || a2.has_zscale || a1.horner != a2.horner) return false;
    return a1.horner || (a2.base_mode == 0 && (a1.base_mode == 0 || a1.base_mode == 2));
}

template <int OP, typename T, int MODE>
cudaError_t launch_pair_mode(const PairMaps& M, const Geom& G, const TermArgs<T>& a1, const TermArgs<T>& a2,
                             unsigned* flags, unsigned long long probe_ns, cudaStream_t stream) {
    const long long cap = (long long)(G.sms > 0 ? G.sms : 1) * pair_blocks_per_sm<OP, T, MODE>();
    const int tz = choose_tz(G, cap);
    const long long tiles = (long long)((G.nx + kBlockX - 1) / kBlockX) * ((G.ny + kBlockY - 1) / kBlockY) *
                            ((G.nz + tz - 1) / tz);
    const int smem = Shape<T>::smem_bytes(OP == ET_OP_LITERAL);
    term2_kernel<OP, T, MODE><<<(unsigned)(tiles < cap ? tiles : cap), kPairThreads, smem, stream>>>(
        M, G, a1, a2, tz, flags, probe_ns);
    return cudaGetLastError();
}

// The kernel variant for the term shapes of a1 and a2.
template <int OP, typename T>
cudaError_t launch_pair_shape(const PairMaps& M, const Geom& G, const TermArgs<T>& a1, const TermArgs<T>& a2,
                              unsigned* flags, unsigned long long probe_ns, cudaStream_t stream) {
    if (!pair_shape_ok(a1, a2)) return cudaErrorInvalidValue;
    if (a1.horner) {
        if (a1.has_zscale)
            return launch_pair_mode<OP, T, kModeHorner | kModeZscale>(M, G, a1, a2, flags, probe_ns, stream);
        return launch_pair_mode<OP, T, kModeHorner>(M, G, a1, a2, flags, probe_ns, stream);
    }
    if (a1.has_zscale) return cudaErrorInvalidValue;  // only the chain's first (Horner) term is scaled
    if (a1.base_mode == 2) return launch_pair_mode<OP, T, kModeBaseZ>(M, G, a1, a2, flags, probe_ns, stream);
    return launch_pair_mode<OP, T, 0>(M, G, a1, a2, flags, probe_ns, stream);
}

template <int OP, typename T>
cudaError_t launch_pair_op(const PairPlan* P, const Geom& G, const TermArgs<T>& a1, const TermArgs<T>& a2,
                           unsigned* flags, unsigned long long probe_ns, cudaStream_t stream) {
    PairMaps M;
    if (!pair_maps(P, a1.zin, &M)) return cudaErrorInvalidValue;
    return launch_pair_shape<OP, T>(M, G, a1, a2, flags, probe_ns, stream);
}

template <int OP, typename T>
void prime_pair() {
    batch_pair_blocks_per_sm<OP, T>();
    pair_blocks_per_sm<OP, T, kModeHorner>();
    pair_blocks_per_sm<OP, T, kModeHorner | kModeZscale>();
    pair_blocks_per_sm<OP, T, kModeBaseZ>();
    pair_blocks_per_sm<OP, T, 0>();
}

}  // namespace

PairPlan* pair_plan_create(const Geom& G, et_precision prec, const void* const wt[4], const void* b, const void* dt,
                           const void* const yz[4]) {
    if (prec == ET_F64) return nullptr;
    const int es = prec == ET_F32 ? 4 : 8;
    if (((long long)G.nx * es) % 16 != 0) return nullptr;
    const int bx = es == 8 ? Shape<float2>::BX : Shape<float>::BX;
    PairPlan* P = new (std::nothrow) PairPlan();
    if (!P) return nullptr;
    const void* zsrc[5] = {b, yz[0], yz[1], yz[2], yz[3]};
    bool ok = true;
    for (int i = 0; i < 5; ++i) {
        ok = ok && encode(&P->zj[i], zsrc[i], G, es, bx, 12);
        P->zj_ptr[i] = zsrc[i];
    }
    ok = ok && encode(&P->w1, wt[1], G, es, bx, 11);
    ok = ok && encode(&P->w0, wt[0], G, es, bx, 10);
    ok = ok && encode(&P->w2, wt[2], G, es, bx, 10);
    ok = ok && encode(&P->w3, wt[3], G, es, bx, 10);
    ok = ok && encode(&P->dt, dt, G, es, bx, 10);
    ok = ok && encode(&P->b, b, G, es, bx, 10);
    if (!ok) {
        delete P;
        return nullptr;
    }
    return P;
}

void pair_plan_destroy(PairPlan* P) { delete P; }

void pair_plan_set_skip(PairPlan* P, bool skip) {
    if (P) P->skip_zero = skip ? 1 : 0;
}

bool pair_maps(const PairPlan* P, const void* zin, PairMaps* out) {
    if (!P) return false;
    int zi = -1;
    for (int i = 0; i < 5; ++i)
        if (P->zj_ptr[i] == zin) zi = i;
    if (zi < 0) return false;
    out->zj = P->zj[zi];
    out->skip_zero = P->skip_zero;
    out->w0 = P->w0;
    out->w1 = P->w1;
    out->w2 = P->w2;
    out->dt = P->dt;
    out->b = P->b;
    out->w3 = P->w3;
    return true;
}

bool pair_maps_for(const PairPlan* P, const Geom& G, et_precision prec, const void* zin, const void* b,
                   const void* dt, PairMaps* out) {
    if (!P || prec == ET_F64) return false;
    const int es = prec == ET_F32 ? 4 : 8;
    const int bx = es == 8 ? Shape<float2>::BX : Shape<float>::BX;
    out->w0 = P->w0;
    out->w1 = P->w1;
    out->w2 = P->w2;
    out->w3 = P->w3;
    out->skip_zero = P->skip_zero;
    return encode(&out->zj, zin, G, es, bx, 12) && encode(&out->b, b, G, es, bx, 10) &&
           encode(&out->dt, dt, G, es, bx, 10);
}

template <typename T>
cudaError_t launch_term_pair_maps(const PairMaps& M, const Geom& G, et_operator op, const TermArgs<T>& a1,
                                  const TermArgs<T>& a2, unsigned* flags, cudaStream_t stream,
                                  unsigned long long probe_ns) {
    if (op == ET_OP_CONSERVATIVE)
        return launch_pair_shape<ET_OP_CONSERVATIVE, T>(M, G, a1, a2, flags, probe_ns, stream);
    return launch_pair_shape<ET_OP_LITERAL, T>(M, G, a1, a2, flags, probe_ns, stream);
}

template cudaError_t launch_term_pair_maps<float>(const PairMaps&, const Geom&, et_operator, const TermArgs<float>&,
                                                  const TermArgs<float>&, unsigned*, cudaStream_t,
                                                  unsigned long long);
template cudaError_t launch_term_pair_maps<float2>(const PairMaps&, const Geom&, et_operator,
                                                   const TermArgs<float2>&, const TermArgs<float2>&, unsigned*,
                                                   cudaStream_t, unsigned long long);

// Batched launches hold many grids, so every block has several tiles even
// with whole columns: segments of up to 64 planes.
int batch_pair_tz(const Geom& G) { return G.nz < 64 ? (G.nz > 0 ? G.nz : 1) : 64; }

template <typename T>
cudaError_t launch_batch_term_pair(et_operator op, const BatchPair<T>* d, int count, long long tiles, int sms,
                                   unsigned* flags, cudaStream_t stream, unsigned long long probe_ns) {
    const int smem = Shape<T>::smem_bytes(op == ET_OP_LITERAL);
    const int per_sm = op == ET_OP_CONSERVATIVE ? batch_pair_blocks_per_sm<ET_OP_CONSERVATIVE, T>()
                                                : batch_pair_blocks_per_sm<ET_OP_LITERAL, T>();
    const long long cap = (long long)(sms > 0 ? sms : 1) * per_sm;
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    if (op == ET_OP_CONSERVATIVE)
        batch_term2_kernel<ET_OP_CONSERVATIVE, T><<<grid, kPairThreads, smem, stream>>>(d, count, tiles, flags,
                                                                                         probe_ns);
    else
        batch_term2_kernel<ET_OP_LITERAL, T><<<grid, kPairThreads, smem, stream>>>(d, count, tiles, flags, probe_ns);
    return cudaGetLastError();
}

template cudaError_t launch_batch_term_pair<float>(et_operator, const BatchPair<float>*, int, long long, int,
                                                   unsigned*, cudaStream_t, unsigned long long);
template cudaError_t launch_batch_term_pair<float2>(et_operator, const BatchPair<float2>*, int, long long, int,
                                                    unsigned*, cudaStream_t, unsigned long long);

template <typename T>
cudaError_t launch_term_pair(const PairPlan* P, const Geom& G, et_operator op, const TermArgs<T>& a1,
                             const TermArgs<T>& a2, unsigned* flags, cudaStream_t stream,
                             unsigned long long probe_ns) {
    if (!P) return cudaErrorInvalidValue;
    if (op == ET_OP_CONSERVATIVE)
        return launch_pair_op<ET_OP_CONSERVATIVE, T>(P, G, a1, a2, flags, probe_ns, stream);
    return launch_pair_op<ET_OP_LITERAL, T>(P, G, a1, a2, flags, probe_ns, stream);
}

bool pair_preferred(et_operator op, et_precision prec) {
    // Shared memory of the literal DF64 stage admits only one block per SM,
    // where two single-term launches are faster (measured at 128^3).
    if (prec == ET_F64) return false;
    int per_sm;
    if (prec == ET_F32)
        per_sm = op == ET_OP_CONSERVATIVE ? pair_blocks_per_sm<ET_OP_CONSERVATIVE, float, kModeHorner>()
                                          : pair_blocks_per_sm<ET_OP_LITERAL, float, kModeHorner>();
    else
        per_sm = op == ET_OP_CONSERVATIVE ? pair_blocks_per_sm<ET_OP_CONSERVATIVE, float2, kModeHorner>()
                                          : pair_blocks_per_sm<ET_OP_LITERAL, float2, kModeHorner>();
    return per_sm >= 2;
}

cudaError_t prime_launch_limits_pair() {
    prime_pair<ET_OP_CONSERVATIVE, float>();
    prime_pair<ET_OP_LITERAL, float>();
    prime_pair<ET_OP_CONSERVATIVE, float2>();
    prime_pair<ET_OP_LITERAL, float2>();
    return cudaGetLastError();
}

template cudaError_t launch_term_pair<float>(const PairPlan*, const Geom&, et_operator, const TermArgs<float>&,
                                             const TermArgs<float>&, unsigned*, cudaStream_t, unsigned long long);
template cudaError_t launch_term_pair<float2>(const PairPlan*, const Geom&, et_operator, const TermArgs<float2>&,
                                              const TermArgs<float2>&, unsigned*, cudaStream_t,
                                              unsigned long long);

}  // namespace et
