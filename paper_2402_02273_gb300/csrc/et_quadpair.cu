// Two consecutive Taylor terms of a Horner sub-step in one launch, FP32, four
// x-consecutive voxels ("a quad") per thread, on tiles that span whole rows.
//
// Terms j and j+1 of sub-step 0 (Horner's rule, Sec. 2.2 evaluated factor by
// factor) are
//     z_a = A~ z_j + beta_1 b,      z_b = A~ z_a + beta_2 b,
// and z_a never reaches memory.  Where the chain's fields exceed the L2 the
// pair is bound by HBM traffic, and a pair moves the bytes of one term: read
// z_j, the three weight fields, the diagonal and b, write z_b (28 B a voxel).
//
// A tile is a full-width slab of th rows (y) by a segment of planes (z).  The
// block's threads cover th + 2 rows: the first term is needed one row beyond
// the tile on both sides (the second term's y neighbours), and no column
// beyond it, since a tile holds whole rows.  Each thread owns one quad of one
// row and marches up the segment.  Its fields arrive by asynchronous 16-byte
// copies (cp.async) two planes ahead of use, into shared-memory slots: four
// planes of z_j (rows two beyond the tile on each side) and three planes of
// the weights, the diagonal and b.  Per plane L, after one barrier:
//   1. z_a on plane L from the slots (x and y neighbours; the -z plane and the
//      conservative -z weight from registers), with the operations of the
//      one-term four-voxel kernel, into a two-plane shared ring;
//   2. the copies of the planes two ahead, into the slots of plane L - 1;
//   3. z_b on plane L - 1 of the thread's interior row, from the ring (x and y
//      neighbours of z_a), its registers (z_a of planes L - 2, L - 1, L and the
//      operands the first term read on plane L - 1), stored to memory.
// Every slot is rewritten only after the barrier that follows its last read,
// so the one barrier per plane orders all of it.  The per-voxel operations
// and their order are those of the one-term kernels, so the results are
// bitwise identical to two one-term launches.
//
// Eligible grids: nx % 4 == 0 and nx <= 256, 16-byte aligned fields,
// n < 2^31.  Running-sum pairs (sub-steps after the first) keep the TMA-fed
// two-term kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "et_internal.h"

namespace et {
namespace {

constexpr int kQPThreads = 512;

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float at(const float4& v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set(float4& v, int e, float x) {
    if (e == 0) v.x = x;
    else if (e == 1) v.y = x;
    else if (e == 2) v.z = x;
    else v.w = x;
}

// One quad of one term: the stencil of the one-term kernels, element by
// element in their order.  wxm0 / zl: weight and value of the -x neighbour of
// element 0; zr: value of the +x neighbour of element 3.
template <bool kCons>
__device__ __forceinline__ float4 quad_term(const float4& dv, const float4& zc, const float4& w0v, float zr, float zl,
                                            float w0l, const float4& w3v, bool has_xm, const float4& w1v,
                                            const float4& zyp, const float4& wym, const float4& zym,
                                            const float4& w2v, const float4& zp, const float4& wzm,
                                            const float4& zm, bool zs, float zscale, bool hb, float beta,
                                            const float4& bq) {
    float4 r;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float zxp = e < 3 ? at(zc, e + 1) : zr;
        const float zxm = e > 0 ? at(zc, e - 1) : zl;
        const float wxm = kCons ? (e > 0 ? at(w0v, e - 1) : w0l) : ((e > 0 || has_xm) ? at(w3v, e) : 0.f);
        float acc = at(dv, e) * at(zc, e);
        acc = fmaf(at(w0v, e), zxp, acc);
        acc = fmaf(wxm, zxm, acc);
        acc = fmaf(at(w1v, e), at(zyp, e), acc);
        acc = fmaf(at(wym, e), at(zym, e), acc);
        acc = fmaf(at(w2v, e), at(zp, e), acc);
        acc = fmaf(at(wzm, e), at(zm, e), acc);
        if (zs) acc *= zscale;
        if (hb) acc = fmaf(beta, at(bq, e), acc);
        set(r, e, acc);
    }
    return r;
}

// Where the tiles of a launch come from: one grid or a table of grids.
struct OneGridQ {
    const QuadPairGrid* d;
    long long total;
    __device__ __forceinline__ int find(long long) const { return 0; }
    __device__ __forceinline__ const QuadPairGrid& grid(int) const { return *d; }
};

struct TableQ {
    const QuadPairGrid* d;
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
    __device__ __forceinline__ const QuadPairGrid& grid(int i) const { return d[i]; }
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

// Shared-memory layout, in float4 units: four slots of z_j planes (rows gy0 - 2
// .. gy0 + th + 1 of a tile whose first interior row is gy0), three slots of
// the weight fields (w0, w1, w2, the diagonal, b, and w3 for the literal
// operator; rows gy0 - 2 .. gy0 + th, the first only for w1), and two planes
// of z_a.  Row strides are those of the grid being worked on (qx quads); the
// slot sizes are the maxima over grids with at most kQPMaxQuads quads a row.
constexpr int kQPMaxQuads = 64;                             // nx <= 256
constexpr int kZSlot = kQPThreads + 2 * kQPMaxQuads;        // (th + 4) * qx <= 512 + 2 qx
constexpr int kWField = kQPThreads + kQPMaxQuads;           // (th + 3) * qx
constexpr int kZSlots = 4, kWSlots = 3;
enum : int { kFw0 = 0, kFw1 = 1, kFw2 = 2, kFdt = 3, kFb = 4, kFw3 = 5 };

__host__ __device__ constexpr int qp_fields(bool literal) { return literal ? 6 : 5; }
__host__ __device__ constexpr int qp_smem_bytes(bool literal) {
    return 16 * (kZSlots * kZSlot + kWSlots * qp_fields(literal) * kWField + 2 * kQPThreads);
}

template <int OP, typename Src>
__device__ __forceinline__ void quad_pair_body(const Src& src) {
    constexpr bool kCons = OP == ET_OP_CONSERVATIVE;
    constexpr int NF = qp_fields(!kCons);
    extern __shared__ float4 smem4[];
    float4* const zs = smem4;                                 // [kZSlots][kZSlot]
    float4* const ws = zs + kZSlots * kZSlot;                 // [kWSlots][NF][kWField]
    float4* const ring = ws + kWSlots * NF * kWField;         // [2][kQPThreads]
    const int t = threadIdx.x;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    for (long long tile = blockIdx.x; tile < src.total; tile += gridDim.x) {
        const QuadPairGrid& Q = src.grid(src.find(tile));
        const int nx = Q.G.nx, ny = Q.G.ny, nz = Q.G.nz;
        const int qx = nx >> 2;
        const int th = Q.th;
        const int rows = th + 2;
        const int tiles_y = (ny + th - 1) / th;
        const int lt = (int)(tile - Q.tile_begin);
        const int ty = lt % tiles_y;
        const int k0 = (lt / tiles_y) * Q.tz;
        const int k1 = min(k0 + Q.tz, nz);
        // this thread's quad: row r of the block (row 0 and row th + 1 are the
        // first term's halo; grid row gy), quad c of that row
        const int r = t / qx;
        const int c = t - r * qx;
        const bool in_tile = r < rows;
        const int gy = ty * th - 1 + r;
        const bool row_ok = in_tile && gy >= 0 && gy < ny;
        const bool interior = in_tile && r >= 1 && r <= th && gy < ny;
        const bool has_xm = c > 0, has_xp = c + 1 < qx;
        const bool has_ym = gy > 0, has_yp = gy + 1 < ny;
        const int sz = nx * ny;
        const int pc = 4 * c + nx * (row_ok ? gy : 0);  // column offset (a valid voxel for idle threads)
        // shared-memory rows: z row r + 1 and weight row r + 1 are this thread's
        const int zo = (r + 1) * qx + c;
        const int wo = (r + 1) * qx + c;

        const float* __restrict__ z = Q.a1.zin;
        const float* const fld[6] = {Q.W.w[0], Q.W.w[1], Q.W.w[2], Q.a1.dt, Q.a1.b, Q.W.w[3]};
        const bool zs1 = Q.a1.has_zscale != 0, hb1 = Q.a1.has_beta != 0, hb2 = Q.a2.has_beta != 0;
        const bool need_b = hb1 || hb2;
        const float zscale1 = Q.a1.zscale, beta1 = Q.a1.beta, beta2 = Q.a2.beta, gamma2 = Q.a2.gamma;
        const bool last2 = Q.a2.last != 0;
        float* __restrict__ zout = Q.a2.zout;
        float* __restrict__ yout = Q.a2.yacc;
        double* __restrict__ uout = Q.a2.u;

        // copies of one plane into its slots: z_j (this thread's row, and the
        // rows two below / two above the halo rows), the weight fields
        auto copy_z = [&](int P) {
            if (P < 0 || P >= nz || P > k1 + 1 || !in_tile) return;
            float4* dst = zs + (P & 3) * kZSlot;
            const float* plane = z + (long long)sz * P;
            if (row_ok) cp_async16(dst + zo, plane + pc);
            if (r == 0 && gy - 1 >= 0 && gy - 1 < ny) cp_async16(dst + c, plane + 4 * c + nx * (gy - 1));
            if (r == rows - 1 && gy + 1 < ny && gy + 1 >= 0)
                cp_async16(dst + (rows + 1) * qx + c, plane + 4 * c + nx * (gy + 1));
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
                cp_async16(dst + kFw1 * kWField + c, fld[kFw1] + po + 4 * c + nx * (gy - 1));
        };

        // carries: z_j and the +z weight of plane L - 1 (the conservative -z
        // weight), z_a of planes L - 2 and L - 1, and the first term's operands
        // of plane L - 1, which the second term on that plane uses again
        const int Lb = k0 - 1;
        float4 zm = (row_ok && Lb - 1 >= 0) ? ld4(z + pc + sz * (Lb - 1)) : zero4;
        float4 wzc = (kCons && row_ok && Lb - 1 >= 0) ? ld4(fld[kFw2] + pc + sz * (Lb - 1)) : zero4;
        float4 am = zero4, ac = zero4;
        float4 c_w0 = zero4, c_w1 = zero4, c_w2 = zero4, c_d = zero4, c_b = zero4, c_w3 = zero4, c_wym = zero4,
               c_wzm = zero4;
        float c_w0l = 0.f;

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
            float4 an = zero4;
            float4 w0v = zero4, w1v = zero4, w2v = zero4, dv = zero4, bq = zero4, w3v = zero4, wym = zero4,
                   wzm = zero4, zc = zero4;
            float w0l = 0.f;
            if (act) {
                const float4* Zc = zs + (L & 3) * kZSlot;
                const float4* W = ws + (L % 3) * NF * kWField;
                zc = Zc[zo];
                const float4 zp = L + 1 < nz ? zs[((L + 1) & 3) * kZSlot + zo] : zero4;
                const float4 zyp = has_yp ? Zc[zo + qx] : zero4;
                const float4 zym = has_ym ? Zc[zo - qx] : zero4;
                const float zl = has_xm ? Zc[zo - 1].w : 0.f;
                const float zr = has_xp ? Zc[zo + 1].x : 0.f;
                w0v = W[kFw0 * kWField + wo];
                w1v = W[kFw1 * kWField + wo];
                w2v = W[kFw2 * kWField + wo];
                dv = W[kFdt * kWField + wo];
                bq = need_b ? W[kFb * kWField + wo] : zero4;
                if (kCons) {
                    w0l = has_xm ? W[kFw0 * kWField + wo - 1].w : 0.f;
                    wym = has_ym ? W[kFw1 * kWField + wo - qx] : zero4;
                    wzm = wzc;
                } else {
                    w3v = W[kFw3 * kWField + wo];
                    wym = has_ym ? w3v : zero4;
                    wzm = L > 0 ? w3v : zero4;
                }
                an = quad_term<kCons>(dv, zc, w0v, zr, zl, w0l, w3v, has_xm, w1v, zyp, wym, zym, w2v, zp, wzm, zm,
                                      zs1, zscale1, hb1, beta1, bq);
            }
            // outside the grid z_a is 0, as the one-term kernels read it
            if (in_tile) ring[(L & 1) * kQPThreads + t] = an;

            // the copies two planes ahead, into the slots of planes L - 1
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
                const float4 ayp = R[t + qx];  // the halo rows hold 0 outside the grid
                const float4 aym = R[t - qx];
                const float al = has_xm ? R[t - 1].w : 0.f;
                const float ar = has_xp ? R[t + 1].x : 0.f;
                const float4 zb = quad_term<kCons>(c_d, ac, c_w0, ar, al, c_w0l, c_w3, has_xm, c_w1, ayp, c_wym, aym,
                                                   c_w2, an, c_wzm, am, false, 0.f, hb2, beta2, c_b);
                const int pq = pc + sz * q;
                if (!last2) {
                    st4(zout + pq, zb);
                } else if (uout) {
                    double2* up = reinterpret_cast<double2*>(uout + pq);
                    double2 u01 = up[0], u23 = up[1];
                    u01.x += (double)(zb.x * gamma2);
                    u01.y += (double)(zb.y * gamma2);
                    u23.x += (double)(zb.z * gamma2);
                    u23.y += (double)(zb.w * gamma2);
                    up[0] = u01;
                    up[1] = u23;
                } else {
                    st4(yout + pq, make_float4(zb.x * gamma2, zb.y * gamma2, zb.z * gamma2, zb.w * gamma2));
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

template <int OP>
__global__ void __launch_bounds__(kQPThreads, 1)
term2_quad_kernel(const __grid_constant__ QuadPairGrid Q, long long total) {
    pdl_begin();  // launched as a programmatic dependent launch (launch_pdl)
    const OneGridQ src{&Q, total};
    quad_pair_body<OP>(src);
}

template <int OP>
__global__ void __launch_bounds__(kQPThreads, 1)
batch_term2_quad_kernel(const QuadPairGrid* __restrict__ d, int count, long long total) {
    const TableQ src{d, count, total};
    quad_pair_body<OP>(src);
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

int blocks_per_sm_qp(et_operator op, bool batch) {
    static int cached[2][2] = {{0, 0}, {0, 0}};
    const bool cons = op == ET_OP_CONSERVATIVE;
    int& c = cached[cons ? 0 : 1][batch ? 1 : 0];
    if (!c) {
        const int smem = qp_smem_bytes(!cons);
        if (batch)
            c = cons ? blocks_per_sm_of(batch_term2_quad_kernel<ET_OP_CONSERVATIVE>, smem)
                     : blocks_per_sm_of(batch_term2_quad_kernel<ET_OP_LITERAL>, smem);
        else
            c = cons ? blocks_per_sm_of(term2_quad_kernel<ET_OP_CONSERVATIVE>, smem)
                     : blocks_per_sm_of(term2_quad_kernel<ET_OP_LITERAL>, smem);
    }
    return c;
}

}  // namespace

int quad_pair_rows(const Geom& G) {
    const int qx = G.nx / 4;
    const int rows = kQPThreads / qx;  // block rows, halo included
    const int th = rows - 2;
    return th < G.ny ? th : G.ny;
}

bool quad_pair_eligible(const Geom& G, const Weights<float>& W, const TermArgs<float>& a1,
                        const TermArgs<float>& a2) {
    if (G.nx % 4 != 0 || G.nx / 4 > kQPMaxQuads || G.n >= (1ll << 31)) return false;
    if (!a1.horner || !a2.horner || a1.last || a2.has_zscale) return false;
    const void* ptrs[] = {W.w[0], W.w[1], W.w[2], W.w[3], a1.zin, a1.b, a1.dt, a2.zout, a2.yacc, a2.u};
    for (const void* p : ptrs)
        if (p && !aligned16(p)) return false;
    return a1.b == a2.b && a1.dt == a2.dt;
}

QuadPairGrid quad_pair_grid(const Geom& G, const Weights<float>& W, const TermArgs<float>& a1,
                            const TermArgs<float>& a2, int tz, long long tile_begin) {
    QuadPairGrid Q;
    Q.G = G;
    Q.W = W;
    Q.a1 = a1;
    Q.a2 = a2;
    Q.th = quad_pair_rows(G);
    Q.tz = tz;
    Q.tile_begin = tile_begin;
    return Q;
}

long long quad_pair_tiles(const Geom& G, int tz) {
    const int th = quad_pair_rows(G);
    return (long long)((G.ny + th - 1) / th) * ((G.nz + tz - 1) / tz);
}

// Planes per segment of a single grid: the fewest waves of tiles over the
// resident blocks times the planes a segment costs (its own and the two more
// the first term runs on).
int quad_pair_tz(const Geom& G, et_operator op) {
    const long long cap = (long long)(G.sms > 0 ? G.sms : 1) * blocks_per_sm_qp(op, false);
    const int th = quad_pair_rows(G);
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

cudaError_t launch_term_quad_pair(const Geom& G, et_operator op, const Weights<float>& W, const TermArgs<float>& a1,
                                  const TermArgs<float>& a2, cudaStream_t stream) {
    const int tz = quad_pair_tz(G, op);
    const QuadPairGrid Q = quad_pair_grid(G, W, a1, a2, tz, 0);
    const long long tiles = quad_pair_tiles(G, tz);
    const long long cap = (long long)(G.sms > 0 ? G.sms : 1) * blocks_per_sm_qp(op, false);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tiles < cap ? tiles : cap), 1, 1);
    cfg.blockDim = dim3(kQPThreads, 1, 1);
    cfg.dynamicSmemBytes = qp_smem_bytes(op == ET_OP_LITERAL);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // programmatic dependent launch
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (op == ET_OP_CONSERVATIVE) return cudaLaunchKernelEx(&cfg, term2_quad_kernel<ET_OP_CONSERVATIVE>, Q, tiles);
    return cudaLaunchKernelEx(&cfg, term2_quad_kernel<ET_OP_LITERAL>, Q, tiles);
}

cudaError_t launch_batch_term_quad_pair(et_operator op, const QuadPairGrid* d, int count, long long tiles, int sms,
                                        cudaStream_t stream) {
    const long long cap = (long long)(sms > 0 ? sms : 1) * blocks_per_sm_qp(op, true);
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    const int smem = qp_smem_bytes(op == ET_OP_LITERAL);
    if (op == ET_OP_CONSERVATIVE)
        batch_term2_quad_kernel<ET_OP_CONSERVATIVE><<<grid, kQPThreads, smem, stream>>>(d, count, tiles);
    else
        batch_term2_quad_kernel<ET_OP_LITERAL><<<grid, kQPThreads, smem, stream>>>(d, count, tiles);
    return cudaGetLastError();
}

cudaError_t prime_launch_limits_quad_pair() {
    blocks_per_sm_qp(ET_OP_CONSERVATIVE, false);
    blocks_per_sm_qp(ET_OP_LITERAL, false);
    blocks_per_sm_qp(ET_OP_CONSERVATIVE, true);
    blocks_per_sm_qp(ET_OP_LITERAL, true);
    return cudaGetLastError();
}

}  // namespace et
