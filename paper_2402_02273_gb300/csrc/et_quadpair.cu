// Two consecutive Taylor terms of a Horner sub-step in one launch, one 16-byte
// vector of each field per thread (four FP32 voxels, or two DF64 pairs), on
// tiles that span whole rows.
//
// Terms j and j+1 of sub-step 0 (Horner's rule, Sec. 2.2 evaluated factor by
// factor) are
//     z_a = A~ z_j + beta_1 b,      z_b = A~ z_a + beta_2 b,
// and z_a never reaches memory.  Where the chain's fields exceed the L2 the
// pair is bound by HBM traffic, and a pair moves the bytes of one term: read
// z_j, the three weight fields, the diagonal and b, write z_b (28 B a voxel in
// FP32, 56 in DF64); the DF64 pair arithmetic also makes it issue-heavy, and
// whole-row tiles keep the per-voxel overhead of both small.
//
// A tile is a full-width slab of th rows (y) by a segment of planes (z).  The
// block's threads cover th + 2 rows: the first term is needed one row beyond
// the tile on both sides (the second term's y neighbours), and no column
// beyond it, since a tile holds whole rows.  Each thread owns one vector of
// one row and marches up the segment.  Its fields arrive by asynchronous
// 16-byte copies (cp.async) two planes ahead of use, into shared-memory slots:
// four planes of z_j (rows two beyond the tile on each side) and three planes
// of the weights, the diagonal and b.  Per plane L, after one barrier:
//   1. z_a on plane L from the slots (x and y neighbours; the -z plane and the
//      conservative -z weight from registers), with the per-voxel arithmetic
//      of the one-term kernels (et_arith.h), into a two-plane shared ring;
//   2. the copies of the planes two ahead, into the slots of plane L - 1;
//   3. z_b on plane L - 1 of the thread's interior row, from the ring (x and y
//      neighbours of z_a), its registers (z_a of planes L - 2, L - 1, L and the
//      operands the first term read on plane L - 1), stored to memory.
// Every slot is rewritten only after the barrier that follows its last read,
// so the one barrier per plane orders all of it.  The results are bitwise
// identical to two one-term launches.
//
// Eligible grids: FP32, nx % 4 == 0 and nx <= 256, 16-byte aligned fields,
// n < 2^31.  Running-sum pairs (sub-steps after the first) keep the TMA-fed
// two-term kernel, and so does DF64: the body is written for any 16-byte
// vector, but two DF64 voxels per thread leave a 512-thread block 8 rows (6
// interior at nx = 128) and 16 warps per SM, and the measured pair launch was
// slower than the TMA-fed one (48.6 against 40 us at 128^3).
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "et_arith.h"
#include "et_internal.h"

namespace et {
namespace {

constexpr int kQPThreads = 512;

// Voxels per 16-byte vector, and the longest row (in vectors) of a grid the
// shared-memory slots are sized for.
template <typename T>
struct VecShape {
    static constexpr int V = 16 / (int)sizeof(T);
    static constexpr int kMaxVec = std::is_same<T, float>::value ? 64 : 96;
};

template <typename T>
struct Vec {
    T e[VecShape<T>::V];
};

template <typename T>
__device__ __forceinline__ Vec<T> vzero() {
    Vec<T> r;
#pragma unroll
    for (int i = 0; i < VecShape<T>::V; ++i) r.e[i] = Arith<T>::zero();
    return r;
}
template <typename T>
__device__ __forceinline__ Vec<T> vload(const T* p) {
    const float4 raw = *reinterpret_cast<const float4*>(p);
    Vec<T> r;
    static_assert(sizeof(Vec<T>) == 16, "16-byte vectors");
    memcpy(&r, &raw, 16);
    return r;
}
template <typename T>
__device__ __forceinline__ Vec<T> vload_s(const float4* p) {
    const float4 raw = *p;
    Vec<T> r;
    memcpy(&r, &raw, 16);
    return r;
}
template <typename T>
__device__ __forceinline__ void vstore(T* p, const Vec<T>& v) {
    float4 raw;
    memcpy(&raw, &v, 16);
    *reinterpret_cast<float4*>(p) = raw;
}
template <typename T>
__device__ __forceinline__ void vstore_s(float4* p, const Vec<T>& v) {
    float4 raw;
    memcpy(&raw, &v, 16);
    *p = raw;
}
// first / last element of the vector held in a shared-memory slot
template <typename T>
__device__ __forceinline__ T vfirst_s(const float4* p) {
    return reinterpret_cast<const T*>(p)[0];
}
template <typename T>
__device__ __forceinline__ T vlast_s(const float4* p) {
    return reinterpret_cast<const T*>(p)[VecShape<T>::V - 1];
}

// One vector of one term: the stencil of the one-term kernels, element by
// element.  zl / wl: value and (conservative) weight of the -x neighbour of
// element 0; zr: value of the +x neighbour of the last element.
template <bool kCons, bool ZS, typename T>
__device__ __forceinline__ Vec<T> vec_term(const Vec<T>& dv, const Vec<T>& zc, const Vec<T>& w0v, T zr, T zl, T wl,
                                           const Vec<T>& w3v, bool has_xm, const Vec<T>& w1v, const Vec<T>& zyp,
                                           const Vec<T>& wym, const Vec<T>& zym, const Vec<T>& w2v,
                                           const Vec<T>& zp, const Vec<T>& wzm, const Vec<T>& zm, T zscale, bool hb,
                                           T beta, const Vec<T>& bq) {
    constexpr int V = VecShape<T>::V;
    Vec<T> r;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const T zxp = e + 1 < V ? zc.e[e + 1] : zr;
        const T zxm = e > 0 ? zc.e[e - 1] : zl;
        const T wxm = kCons ? (e > 0 ? w0v.e[e - 1] : wl) : ((e > 0 || has_xm) ? w3v.e[e] : Arith<T>::zero());
        r.e[e] = Arith<T>::template stencil<ZS>(dv.e[e], zc.e[e], w0v.e[e], zxp, wxm, zxm, w1v.e[e], zyp.e[e],
                                                 wym.e[e], zym.e[e], w2v.e[e], zp.e[e], wzm.e[e], zm.e[e], zscale,
                                                 hb, beta, bq.e[e]);
    }
    return r;
}

// Where the tiles of a launch come from: one grid or a table of grids.
template <typename T>
struct OneGridQ {
    const VecPairGrid<T>* d;
    long long total;
    __device__ __forceinline__ int find(long long) const { return 0; }
    __device__ __forceinline__ const VecPairGrid<T>& grid(int) const { return *d; }
};

template <typename T>
struct TableQ {
    const VecPairGrid<T>* d;
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
    __device__ __forceinline__ const VecPairGrid<T>& grid(int i) const { return d[i]; }
};

// ---- asynchronous staging (cp.async, 16 bytes a thread) ------------------------

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared-memory layout, in 16-byte units: four slots of z_j planes (rows
// gy0 - 2 .. gy0 + th + 1 of a tile whose first interior row is gy0), three
// slots of the weight fields (w0, w1, w2, the diagonal, b, and w3 for the
// literal operator; rows gy0 - 2 .. gy0 + th, the first only for w1), and two
// planes of z_a.  Row strides are those of the grid being worked on (nv
// vectors); the slot sizes are the maxima over eligible grids.
template <typename T>
struct SmemShape {
    static constexpr int kZSlot = kQPThreads + 2 * VecShape<T>::kMaxVec;  // (th + 4) nv <= 512 + 2 nv
    static constexpr int kWField = kQPThreads + VecShape<T>::kMaxVec;     // (th + 3) nv
};
constexpr int kZSlots = 4, kWSlots = 3;
enum : int { kFw0 = 0, kFw1 = 1, kFw2 = 2, kFdt = 3, kFb = 4, kFw3 = 5 };

__host__ __device__ constexpr int qp_fields(bool literal) { return literal ? 6 : 5; }
template <typename T>
__host__ __device__ constexpr int qp_smem_bytes(bool literal) {
    return 16 * (kZSlots * SmemShape<T>::kZSlot + kWSlots * qp_fields(literal) * SmemShape<T>::kWField +
                 2 * kQPThreads);
}

template <int OP, typename T, typename Src>
__device__ __forceinline__ void vec_pair_body(const Src& src) {
    using A = Arith<T>;
    constexpr bool kCons = OP == ET_OP_CONSERVATIVE;
    constexpr int NF = qp_fields(!kCons);
    constexpr int V = VecShape<T>::V;
    constexpr int kZSlot = SmemShape<T>::kZSlot, kWField = SmemShape<T>::kWField;
    extern __shared__ float4 smem4[];
    float4* const zs = smem4;                          // [kZSlots][kZSlot]
    float4* const ws = zs + kZSlots * kZSlot;          // [kWSlots][NF][kWField]
    float4* const ring = ws + kWSlots * NF * kWField;  // [2][kQPThreads]
    const int t = threadIdx.x;
    const Vec<T> zv = vzero<T>();
    const T zero = A::zero();

    for (long long tile = blockIdx.x; tile < src.total; tile += gridDim.x) {
        const VecPairGrid<T>& Q = src.grid(src.find(tile));
        const int nx = Q.G.nx, ny = Q.G.ny, nz = Q.G.nz;
        const int nv = nx / V;  // vectors per row
        const int th = Q.th;
        const int rows = th + 2;
        const int tiles_y = (ny + th - 1) / th;
        const int lt = (int)(tile - Q.tile_begin);
        const int ty = lt % tiles_y;
        const int k0 = (lt / tiles_y) * Q.tz;
        const int k1 = min(k0 + Q.tz, nz);
        // this thread's vector: row r of the block (row 0 and row th + 1 are
        // the first term's halo; grid row gy), vector c of that row
        const int r = t / nv;
        const int c = t - r * nv;
        const bool in_tile = r < rows;
        const int gy = ty * th - 1 + r;
        const bool row_ok = in_tile && gy >= 0 && gy < ny;
        const bool interior = in_tile && r >= 1 && r <= th && gy < ny;
        const bool has_xm = c > 0, has_xp = c + 1 < nv;
        const bool has_ym = gy > 0, has_yp = gy + 1 < ny;
        const int sz = nx * ny;
        const int pc = V * c + nx * (row_ok ? gy : 0);  // column offset (a valid voxel for idle threads)
        // shared-memory rows: z row r + 1 and weight row r + 1 are this thread's
        const int zo = (r + 1) * nv + c;
        const int wo = (r + 1) * nv + c;

        const T* __restrict__ z = Q.a1.zin;
        const T* const fld[6] = {Q.W.w[0], Q.W.w[1], Q.W.w[2], Q.a1.dt, Q.a1.b, Q.W.w[3]};
        const bool zs1 = Q.a1.has_zscale != 0, hb1 = Q.a1.has_beta != 0, hb2 = Q.a2.has_beta != 0;
        const bool need_b = hb1 || hb2;
        const T zscale1 = Q.a1.zscale, beta1 = Q.a1.beta, beta2 = Q.a2.beta, gamma2 = Q.a2.gamma;
        const bool last2 = Q.a2.last != 0;
        T* __restrict__ zout = Q.a2.zout;
        T* __restrict__ yout = Q.a2.yacc;
        double* __restrict__ uout = Q.a2.u;

        // copies of one plane into its slots: z_j (this thread's row, and the
        // rows two below / two above the halo rows), the weight fields
        auto copy_z = [&](int P) {
            if (P < 0 || P >= nz || P > k1 + 1 || !in_tile) return;
            float4* dst = zs + (P & 3) * kZSlot;
            const T* plane = z + (long long)sz * P;
            if (row_ok) cp_async16(dst + zo, plane + pc);
            if (r == 0 && gy - 1 >= 0 && gy - 1 < ny) cp_async16(dst + c, plane + V * c + nx * (gy - 1));
            if (r == rows - 1 && gy + 1 < ny && gy + 1 >= 0)
                cp_async16(dst + (rows + 1) * nv + c, plane + V * c + nx * (gy + 1));
        };
        auto copy_w = [&](int P) {
            if (P < 0 || P >= nz || P > k1 || !in_tile) return;
            float4* dst = ws + (P % 3) * NF * kWField;
            const int po = sz * P;
            if (row_ok) {
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    if (f != kFb || need_b) cp_async16(dst + f * kWField + wo, fld[f] + po + pc);
            }
            if (kCons && r == 0 && gy - 1 >= 0 && gy - 1 < ny)  // -y weight of the halo row
                cp_async16(dst + kFw1 * kWField + c, fld[kFw1] + po + V * c + nx * (gy - 1));
        };

        // carries: z_j and the +z weight of plane L - 1 (the conservative -z
        // weight), z_a of planes L - 2 and L - 1, and the first term's operands
        // of plane L - 1, which the second term on that plane uses again
        const int Lb = k0 - 1;
        Vec<T> zm = (row_ok && Lb - 1 >= 0) ? vload<T>(z + pc + sz * (Lb - 1)) : zv;
        Vec<T> wzc = (kCons && row_ok && Lb - 1 >= 0) ? vload<T>(fld[kFw2] + pc + sz * (Lb - 1)) : zv;
        Vec<T> am = zv, ac = zv;
        Vec<T> c_w0 = zv, c_w1 = zv, c_w2 = zv, c_d = zv, c_b = zv, c_w3 = zv, c_wym = zv, c_wzm = zv;
        T c_w0l = zero;

        // planes Lb, Lb + 1 (z_j) and Lb (weights), then Lb + 2 (z_j) and Lb + 1
        copy_z(Lb);
        copy_z(Lb + 1);
        copy_w(Lb);
        cp_async_commit();
        copy_z(Lb + 2);
        copy_w(Lb + 1);
        cp_async_commit();

        for (int L = Lb; L <= k1; ++L) {
            // z_j of plane L + 1 and the weights of plane L have landed (the
            // group committed two planes ago); the barrier makes every thread's
            // copies and the z_a plane of L - 1 visible to all
            cp_async_wait<1>();
            __syncthreads();

            // ---- first term on plane L ---------------------------------------
            const bool act = row_ok && L >= 0 && L < nz;
            Vec<T> an = zv;
            Vec<T> w0v = zv, w1v = zv, w2v = zv, dv = zv, bq = zv, w3v = zv, wym = zv, wzm = zv, zc = zv;
            T w0l = zero;
            if (act) {
                const float4* Zc = zs + (L & 3) * kZSlot;
                const float4* W = ws + (L % 3) * NF * kWField;
                zc = vload_s<T>(Zc + zo);
                const Vec<T> zp = L + 1 < nz ? vload_s<T>(zs + ((L + 1) & 3) * kZSlot + zo) : zv;
                const Vec<T> zyp = has_yp ? vload_s<T>(Zc + zo + nv) : zv;
                const Vec<T> zym = has_ym ? vload_s<T>(Zc + zo - nv) : zv;
                const T zl = has_xm ? vlast_s<T>(Zc + zo - 1) : zero;
                const T zr = has_xp ? vfirst_s<T>(Zc + zo + 1) : zero;
                w0v = vload_s<T>(W + kFw0 * kWField + wo);
                w1v = vload_s<T>(W + kFw1 * kWField + wo);
                w2v = vload_s<T>(W + kFw2 * kWField + wo);
                dv = vload_s<T>(W + kFdt * kWField + wo);
                bq = need_b ? vload_s<T>(W + kFb * kWField + wo) : zv;
                if (kCons) {
                    w0l = has_xm ? vlast_s<T>(W + kFw0 * kWField + wo - 1) : zero;
                    wym = has_ym ? vload_s<T>(W + kFw1 * kWField + wo - nv) : zv;
                    wzm = wzc;
                } else {
                    w3v = vload_s<T>(W + kFw3 * kWField + wo);
                    wym = has_ym ? w3v : zv;
                    wzm = L > 0 ? w3v : zv;
                }
                if (zs1)
                    an = vec_term<kCons, true, T>(dv, zc, w0v, zr, zl, w0l, w3v, has_xm, w1v, zyp, wym, zym, w2v, zp,
                                                  wzm, zm, zscale1, hb1, beta1, bq);
                else
                    an = vec_term<kCons, false, T>(dv, zc, w0v, zr, zl, w0l, w3v, has_xm, w1v, zyp, wym, zym, w2v,
                                                   zp, wzm, zm, zscale1, hb1, beta1, bq);
            }
            // outside the grid z_a is 0, as the one-term kernels read it
            if (in_tile) vstore_s<T>(ring + (L & 1) * kQPThreads + t, an);

            // the copies two planes ahead, into the slots of plane L - 1
            copy_z(L + 3);
            copy_w(L + 2);
            cp_async_commit();

            // ---- second term on plane q = L - 1 --------------------------------
            const int q = L - 1;
            if (q >= k0 && interior) {
                // z_a of plane q: x and y neighbours from the ring (written
                // before this plane's barrier), the centre and the planes below
                // and above from registers
                const float4* R = ring + (q & 1) * kQPThreads;
                const Vec<T> ayp = vload_s<T>(R + t + nv);  // the halo rows hold 0 outside the grid
                const Vec<T> aym = vload_s<T>(R + t - nv);
                const T al = has_xm ? vlast_s<T>(R + t - 1) : zero;
                const T ar = has_xp ? vfirst_s<T>(R + t + 1) : zero;
                const Vec<T> zb = vec_term<kCons, false, T>(c_d, ac, c_w0, ar, al, c_w0l, c_w3, has_xm, c_w1, ayp,
                                                            c_wym, aym, c_w2, an, c_wzm, am, zero, hb2, beta2, c_b);
                const int pq = pc + sz * q;
                if (!last2) {
                    vstore<T>(zout + pq, zb);
                } else {
                    Vec<T> sb;
#pragma unroll
                    for (int e = 0; e < V; ++e) sb.e[e] = A::scale(gamma2, zb.e[e]);
                    if (uout) {
#pragma unroll
                        for (int e = 0; e < V; e += 2) {
                            double2* up = reinterpret_cast<double2*>(uout + pq + e);
                            double2 uv = *up;
                            uv.x += A::widen(sb.e[e]);
                            uv.y += A::widen(sb.e[e + 1]);
                            *up = uv;
                        }
                    } else {
                        vstore<T>(yout + pq, sb);
                    }
                }
            }
            // carries for plane L + 1
            zm = zc;
            if (kCons) wzc = w2v;
            am = ac;
            ac = an;
            c_w0 = w0v;
            c_w0l = w0l;
            c_w1 = w1v;
            c_w2 = w2v;
            c_d = dv;
            c_b = bq;
            c_w3 = w3v;
            c_wym = wym;
            c_wzm = wzm;
        }
        cp_async_wait<0>();
        __syncthreads();  // the next tile's copies and z_a planes reuse the slots
    }
}

template <int OP, typename T>
__global__ void __launch_bounds__(kQPThreads, 1)
term2_quad_kernel(const __grid_constant__ VecPairGrid<T> Q, long long total) {
    pdl_begin();  // launched as a programmatic dependent launch
    const OneGridQ<T> src{&Q, total};
    vec_pair_body<OP, T>(src);
}

template <int OP, typename T>
__global__ void __launch_bounds__(kQPThreads, 1)
batch_term2_quad_kernel(const VecPairGrid<T>* __restrict__ d, int count, long long total) {
    const TableQ<T> src{d, count, total};
    vec_pair_body<OP, T>(src);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Resident blocks per SM of a kernel with its dynamic shared memory (set
// once: the opt-in above 48 KB).
template <typename K>
int blocks_per_sm_of(K kernel, int smem) {
    int b = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kQPThreads, smem) != cudaSuccess || b < 1)
        b = 1;
    return b;
}

template <int OP, typename T>
int blocks_per_sm_qp(bool batch) {
    static int cached[2] = {0, 0};
    int& c = cached[batch ? 1 : 0];
    if (!c) {
        const int smem = qp_smem_bytes<T>(OP == ET_OP_LITERAL);
        c = batch ? blocks_per_sm_of(batch_term2_quad_kernel<OP, T>, smem)
                  : blocks_per_sm_of(term2_quad_kernel<OP, T>, smem);
    }
    return c;
}

template <typename T>
int blocks_per_sm_qp(et_operator op, bool batch) {
    return op == ET_OP_CONSERVATIVE ? blocks_per_sm_qp<ET_OP_CONSERVATIVE, T>(batch)
                                    : blocks_per_sm_qp<ET_OP_LITERAL, T>(batch);
}

}  // namespace

template <typename T>
int vec_pair_rows(const Geom& G) {
    const int nv = G.nx / VecShape<T>::V;
    const int rows = kQPThreads / nv;  // block rows, halo included
    const int th = rows - 2;
    return th < G.ny ? th : G.ny;
}

template <typename T>
bool vec_pair_eligible(const Geom& G, et_operator op, const Weights<T>& W, const TermArgs<T>& a1,
                       const TermArgs<T>& a2) {
    constexpr int V = VecShape<T>::V;
    if (G.nx % V != 0 || G.nx / V > VecShape<T>::kMaxVec || G.n >= (1ll << 31)) return false;
    if (!std::is_same<T, float>::value) return false;  // DF64 keeps the TMA-fed pair kernel
    (void)op;
    if (!a1.horner || !a2.horner || a1.last || a2.has_zscale) return false;
    const void* ptrs[] = {W.w[0], W.w[1], W.w[2], W.w[3], a1.zin, a1.b, a1.dt, a2.zout, a2.yacc, a2.u};
    for (const void* p : ptrs)
        if (p && !aligned16(p)) return false;
    return a1.b == a2.b && a1.dt == a2.dt;
}

template <typename T>
VecPairGrid<T> vec_pair_grid(const Geom& G, const Weights<T>& W, const TermArgs<T>& a1, const TermArgs<T>& a2,
                             int tz, long long tile_begin) {
    VecPairGrid<T> Q;
    Q.G = G;
    Q.W = W;
    Q.a1 = a1;
    Q.a2 = a2;
    Q.th = vec_pair_rows<T>(G);
    Q.tz = tz;
    Q.tile_begin = tile_begin;
    return Q;
}

template <typename T>
long long vec_pair_tiles(const Geom& G, int tz) {
    const int th = vec_pair_rows<T>(G);
    return (long long)((G.ny + th - 1) / th) * ((G.nz + tz - 1) / tz);
}

namespace {

// Planes per segment of a single grid: the fewest waves of tiles over the
// resident blocks times the planes a segment costs (its own and the two more
// the first term runs on).
template <typename T>
int vec_pair_tz(const Geom& G, et_operator op) {
    const long long cap = (long long)(G.sms > 0 ? G.sms : 1) * blocks_per_sm_qp<T>(op, false);
    const int th = vec_pair_rows<T>(G);
    const long long ty = (G.ny + th - 1) / th;
    int best = 1;
    double best_cost = 1e300;
    for (int tz = 1; tz <= 64; ++tz) {
        const long long tiles = ty * ((G.nz + tz - 1) / tz);
        const long long waves = (tiles + cap - 1) / cap;
        const double cost = (double)waves * (tz + 2.0);
        if (cost < best_cost) {
            best_cost = cost;
            best = tz;
        }
        if (tz >= G.nz) break;
    }
    return best;
}

template <int OP, typename T>
cudaError_t launch_one(const VecPairGrid<T>& Q, long long tiles, long long cap, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tiles < cap ? tiles : cap), 1, 1);
    cfg.blockDim = dim3(kQPThreads, 1, 1);
    cfg.dynamicSmemBytes = qp_smem_bytes<T>(OP == ET_OP_LITERAL);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // programmatic dependent launch
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, term2_quad_kernel<OP, T>, Q, tiles);
}

}  // namespace

template <typename T>
cudaError_t launch_term_vec_pair(const Geom& G, et_operator op, const Weights<T>& W, const TermArgs<T>& a1,
                                 const TermArgs<T>& a2, cudaStream_t stream) {
    const int tz = vec_pair_tz<T>(G, op);
    const VecPairGrid<T> Q = vec_pair_grid<T>(G, W, a1, a2, tz, 0);
    const long long tiles = vec_pair_tiles<T>(G, tz);
    const long long cap = (long long)(G.sms > 0 ? G.sms : 1) * blocks_per_sm_qp<T>(op, false);
    if (op == ET_OP_CONSERVATIVE) return launch_one<ET_OP_CONSERVATIVE, T>(Q, tiles, cap, stream);
    return launch_one<ET_OP_LITERAL, T>(Q, tiles, cap, stream);
}

template <typename T>
cudaError_t launch_batch_term_vec_pair(et_operator op, const VecPairGrid<T>* d, int count, long long tiles, int sms,
                                       cudaStream_t stream) {
    const long long cap = (long long)(sms > 0 ? sms : 1) * blocks_per_sm_qp<T>(op, true);
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    const int smem = qp_smem_bytes<T>(op == ET_OP_LITERAL);
    if (op == ET_OP_CONSERVATIVE)
        batch_term2_quad_kernel<ET_OP_CONSERVATIVE, T><<<grid, kQPThreads, smem, stream>>>(d, count, tiles);
    else
        batch_term2_quad_kernel<ET_OP_LITERAL, T><<<grid, kQPThreads, smem, stream>>>(d, count, tiles);
    return cudaGetLastError();
}

cudaError_t prime_launch_limits_quad_pair() {
    blocks_per_sm_qp<float>(ET_OP_CONSERVATIVE, false);
    blocks_per_sm_qp<float>(ET_OP_LITERAL, false);
    blocks_per_sm_qp<float>(ET_OP_CONSERVATIVE, true);
    blocks_per_sm_qp<float>(ET_OP_LITERAL, true);
    return cudaGetLastError();
}

#define ET_VEC_PAIR_INSTANCES(T)                                                                                   \
    template int vec_pair_rows<T>(const Geom&);                                                                    \
    template bool vec_pair_eligible<T>(const Geom&, et_operator, const Weights<T>&, const TermArgs<T>&,           \
                                       const TermArgs<T>&);                                                        \
    template VecPairGrid<T> vec_pair_grid<T>(const Geom&, const Weights<T>&, const TermArgs<T>&,                  \
                                             const TermArgs<T>&, int, long long);                                  \
    template long long vec_pair_tiles<T>(const Geom&, int);                                                        \
    template cudaError_t launch_term_vec_pair<T>(const Geom&, et_operator, const Weights<T>&, const TermArgs<T>&, \
                                                 const TermArgs<T>&, cudaStream_t);                                \
    template cudaError_t launch_batch_term_vec_pair<T>(et_operator, const VecPairGrid<T>*, int, long long, int,  \
                                                       cudaStream_t);
ET_VEC_PAIR_INSTANCES(float)
#undef ET_VEC_PAIR_INSTANCES

}  // namespace et
