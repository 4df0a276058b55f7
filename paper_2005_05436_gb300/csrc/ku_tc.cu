// Tensor-core (tcgen05) form of the FP32 matrix-free operator K(xPhys) u on H8
// grids (Eqs. 4-5): the element products Ke u_e of a slab of elements run as
// TF32 MMAs with FP32 accumulation in tensor memory; the E_e-scaled corner
// rows are summed into nodes on the CUDA cores, with the smoother, residual
// and PCG-dot epilogues of the fine multigrid level fused.
//
// Blocking. A block owns a 15 x 15 column of nodes in (y, z) and LX node
// planes along x, marching along x one element plane (slab) at a time. Its
// elements are the 16 x 16 element columns touching those nodes (a one-element
// halo in -y and -z), as two M = 128 tiles of 8 (y) x 16 (z) elements. Node
// planes of 17 x 17 nodes are staged into a four-deep ring in shared memory,
// one node per 16 bytes (u_x, u_y, u_z, 0), as the TF32 high and low parts of
// u - c, where c is the displacement of one node of the block: the rows of Ke
// annihilate rigid translations, so the product is unchanged while the
// rounding acts on displacement differences (a constant added to u leaves the
// result bit-identical).
//
// Operands. In the canonical no-swizzle K-major layout a core matrix is 8 rows
// of 16 bytes, so 8 consecutive nodes along y of one staged row form a core
// matrix as they lie. For element corner offsets (gy, gz) the A operand of a
// tile is addressed directly in the staged planes: it starts at node
// (8 t + gy, gz), its 8-row groups are one staged row apart (SBO) and its two K
// halves, corners gx = 0 and gx = 1, one plane apart (LBO; for the ring slot
// pair (3, 0) the halves are swapped and so is B). One MMA per (gy, gz) and
// operand part: K = 8 (two corners x (3 components + a zero)), N = 32 (8
// output corners x 3 components, then 8 zero rows). Per slab and tile
// D = Ah Bh + Al Bh + Ah Bl, 12 MMAs, about 21 correct bits.
//
// Epilogue. A thread holds one element's 24 outputs (one TMEM lane) and scales
// them by E_e; the +x corners carry to the next slab in registers, the -y
// neighbour arrives by warp shuffle (lanes are y-consecutive in groups of 8;
// across the tile seam through shared memory), the -z neighbour through shared
// memory. Every node is written once, by its owner thread, in a fixed order.
//
// Pipeline. MMAs for slab s + 2 are issued after the barrier of slab s, into
// the TMEM buffer slab s has just been read from (two buffers of 64 columns);
// node plane s + 3 is loaded while slab s waits for its MMAs. Every mbarrier
// wait is bounded; on timeout the block sets the error word and leaves the
// loop together, waits (bounded) for the MMAs it issued and frees its TMEM.
#include <algorithm>
#include <cstring>
#include <vector>

#include "grid.h"
#include "ku_device.cuh"

namespace topo {

namespace tc {

constexpr int NT = 288;                 // eight staging / epilogue warps and one MMA warp
constexpr int NE = 256;                 // staging / epilogue threads
constexpr int TN = 15;                 // owned nodes per block along y and along z
constexpr int SN = TN + 2;             // staged nodes per row and rows per plane
constexpr int ROWB = SN * 16;          // bytes per staged row (the A operand's SBO)
constexpr int PLANEB = SN * ROWB;      // bytes per staged plane (the A operand's LBO)
constexpr int RING = 4;
constexpr int NSTG = (SN * SN + NE - 1) / NE;  // staged nodes per thread and plane
constexpr int B_HL = 64 * 8;                  // floats of the N = 64 B tile [Bh | Bl] (K = 8)
constexpr int B_H = 32 * 8;                    // floats of the N = 32 B tile Bh
constexpr int B_SET = B_HL + B_H;
constexpr int B_FLOATS = 2 * 4 * B_SET;        // [K order][(gy, gz)]
constexpr int X_FLOATS = 2 * 2 * 16 * 8 * 3;   // z exchange [parity][tile][z][y][component]
constexpr int YB_FLOATS = 2 * 16 * 6;          // tile seam [parity][z][component][gz]
constexpr int RAW = 3;                         // planes in flight as raw FP32 (cp.async ring)
constexpr int RAW_FLOATS = RAW * SN * SN * 3;
constexpr int OFF_HI = 0;
constexpr int OFF_LO = OFF_HI + RING * PLANEB;
constexpr int OFF_B = OFF_LO + RING * PLANEB;
constexpr int OFF_X = OFF_B + B_FLOATS * 4;
constexpr int OFF_YB = OFF_X + X_FLOATS * 4;
constexpr int OFF_RAW = OFF_YB + YB_FLOATS * 4;
constexpr int OFF_BAR = (OFF_RAW + RAW_FLOATS * 4 + 15) / 16 * 16;
constexpr int SMEM_BYTES = OFF_BAR + 8 * (RING + 8);  // mbarriers: full[RING], tdone[2][2], tfree[2][2]
constexpr int TMEM_COLS = 256;                 // two buffers x two tiles x 64 columns
constexpr long long WAIT_LIMIT = 1LL << 26;    // mbarrier polls before giving up
static_assert(OFF_B % 16 == 0 && OFF_BAR % 8 == 0, "operand and barrier alignment");
static_assert(3 * PLANEB / 16 < (1 << 14) && ROWB / 16 < (1 << 14), "descriptor offsets fit 14 bits");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// tcgen05 shared-memory matrix descriptor, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;                // base offset 0, LBO mode 0, layout SWIZZLE_NONE (0)
}

// Instruction descriptors: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 64 or 32.
constexpr uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
constexpr uint32_t IDESC64 = idesc_tf32(64), IDESC32 = idesc_tf32(32);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity));
        if (done) return true;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 4-byte asynchronous global -> shared copy, zero-filled when !pred.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool pred) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "r"(pred ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Offset (floats) of the B tiles of (K order, (gy, gz)) -- the N = 64 tile
// [Bh | Bl] first, the N = 32 tile Bh after it -- and of entry (n, k) inside a
// tile: core matrices (n / 8, k / 4) of 8 rows x 4 floats, K-adjacent ones 128
// bytes apart (LBO), N-adjacent ones 256 bytes apart (SBO).
__host__ __device__ constexpr int b_set(int order, int m) { return (order * 4 + m) * B_SET; }
__host__ __device__ constexpr int b_off(int n, int k) { return ((n >> 3) * 2 + (k >> 2)) * 32 + (n & 7) * 4 + (k & 3); }

}  // namespace tc

template <int MODE, bool PCG>
__global__ void __launch_bounds__(tc::NT, 2)
    k_ku_tc(Dims d, int LX, int ntY, int ntZ, const float* __restrict__ E, const float* __restrict__ u,
            const float* __restrict__ r, const float* __restrict__ dinv, float* __restrict__ out,
            const uint8_t* __restrict__ fixed, float omega, const float* __restrict__ Bpack, const int* skip,
            PcgScalars* pcg, double* partials, unsigned* counter, int* err) {
    using namespace tc;
    pdl_begin();
    if (skip && *skip) return;  // uniform, before any tensor-memory use
    extern __shared__ __align__(1024) unsigned char smem[];
    float* X = reinterpret_cast<float*>(smem + OFF_X);
    float* YB = reinterpret_cast<float*>(smem + OFF_YB);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + OFF_BAR);  // [RING] plane staged (NE arrivals)
    uint64_t* tdone = full + RING;                                  // [buffer][tile] MMAs complete (commit)
    uint64_t* tfree = tdone + 4;                                    // [buffer][tile] TMEM read (128 arrivals)
    __shared__ uint32_t tmem_base;
    __shared__ int fail[2];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool epi = tid < NE;  // staging / epilogue threads; warp NE / 32 issues the MMAs
    int bid = blockIdx.x;
    const int tY = bid % ntY;
    bid /= ntY;
    const int tZ = bid % ntZ;
    const int X0 = (bid / ntZ) * LX;
    const int Y0 = tY * TN, Z0 = tZ * TN;  // first owned node
    const int nny = d.nny, nnz = d.nnz, nnx = d.nnx;
    const int nsteps = min(LX, nnx - X0);  // output planes X0 .. X0 + nsteps - 1
    const int nslab = nsteps + 1;          // element planes X0 - 1 .. X0 + nsteps - 1

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < RING; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(full + i)), "r"(NE));
        for (int i = 0; i < 4; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(tdone + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(tfree + i)), "r"(NE / 2));
        }
        fail[0] = fail[1] = 0;
    }
    for (int i = tid; i < B_FLOATS / 4; i += NT)
        reinterpret_cast<float4*>(smem + OFF_B)[i] = reinterpret_cast<const float4*>(Bpack)[i];
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    fence_before_sync();
    __syncthreads();  // barriers, B tiles and the TMEM address published
    fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t s_hi = smem_u32(smem + OFF_HI), s_lo = smem_u32(smem + OFF_LO), s_b = smem_u32(smem + OFF_B);

    double dot_out = 0.0;  // this thread's share of the PCG dot product
    if (!epi) {
        // ---- MMA issue warp: slab s (planes s, s + 1) into TMEM buffer s & 1,
        // tile t at 64 columns: Ah [Bh | Bl] + Al [Bh | 0]; completion on tdone[2 (s & 1) + t]
        if (lane == 0) {
            bool ok = true;
            int issued = -1;
            for (int s = 0; s < nslab && ok; ++s) {
                for (int jp = s == 0 ? 0 : s + 1; jp <= s + 1 && ok; ++jp)
                    ok = mbar_wait(smem_u32(full + (jp & (RING - 1))), (uint32_t)((jp >> 2) & 1));
                if (ok && s >= 2)
                    for (int tt = 0; tt < 2 && ok; ++tt)
                        ok = mbar_wait(smem_u32(tfree + 2 * (s & 1) + tt), (uint32_t)(((s - 2) >> 1) & 1));
                if (!ok) break;
                fence_after_sync();
                const int slot = s & (RING - 1);
                const int order = slot == RING - 1 ? 1 : 0;  // ring pair (3, 0): K halves swapped
                const uint32_t kslot = order ? 0u : (uint32_t)slot;
                const uint32_t lbo = order ? (uint32_t)((RING - 1) * PLANEB) : (uint32_t)PLANEB;
#pragma unroll
                for (int tt = 0; tt < 2; ++tt) {
                    const uint32_t dcol = tmem + (uint32_t)((s & 1) * 128 + tt * 64);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int gy = m >> 1, gz = m & 1;
                        const uint32_t aoff = kslot * PLANEB + (uint32_t)((gz * SN + 8 * tt + gy) * 16);
                        const uint64_t bhl = make_desc(s_b + 4u * b_set(order, m), 128, 256);
                        const uint64_t bh = make_desc(s_b + 4u * (b_set(order, m) + B_HL), 128, 256);
                        mma_tf32(dcol, make_desc(s_hi + aoff, lbo, ROWB), bhl, IDESC64, m > 0 ? 1u : 0u);
                        mma_tf32(dcol, make_desc(s_lo + aoff, lbo, ROWB), bh, IDESC32, 1u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                     smem_u32(tdone + 2 * (s & 1) + tt))
                                 : "memory");
                }
                issued = s;
            }
            if (!ok && err) atomicExch(err, (int)TO_ETIMEOUT);
            // nothing may be in flight when the block frees its tensor memory
            if (issued >= 0) (void)mbar_wait(smem_u32(tdone + 2 * (issued & 1) + 1), (uint32_t)((issued >> 1) & 1));
        }
    } else {
        // ---- staging and epilogue warps
        // the block's reference displacement c
        const long long cref = 3 * (min(Y0, nny - 1) + (long long)nny * (min(Z0, nnz - 1) + (long long)nnz * min(X0, nnx - 1)));
        const float c0 = u[cref], c1 = u[cref + 1], c2 = u[cref + 2];
        // staged nodes of this thread: k = tid + j NE -> (ys, zs) = (k % SN, k / SN)
        const long long pstride = 3LL * nny * nnz;
        int goff[NSTG], soff[NSTG];
#pragma unroll
        for (int j = 0; j < NSTG; ++j) {
            const int k = tid + j * NE;
            const int ys = k % SN, zs = k / SN;
            const int gy = Y0 - 1 + ys, gz = Z0 - 1 + zs;
            goff[j] = (k < SN * SN && gy >= 0 && gy < nny && gz >= 0 && gz < nnz) ? 3 * (gy + nny * gz) : -1;
            soff[j] = k < SN * SN ? (zs * SN + ys) * 16 : -1;
        }
        // Node plane jp: raw FP32 values by cp.async into raw slot jp % RAW (one
        // commit group per call, empty past the last plane), then, once landed,
        // u - c split into the TF32 parts of ring slot jp % RING, and an arrival
        // on full[jp % RING]. Each thread converts only the values it copied.
        float* raw = reinterpret_cast<float*>(smem + OFF_RAW);
        auto raw_issue = [&](int jp) {
            if (jp <= nslab) {
                const int nx = X0 - 1 + jp;
                const bool pv = nx >= 0 && nx < nnx;
                float* dst = raw + (jp % RAW) * (SN * SN * 3);
#pragma unroll
                for (int j = 0; j < NSTG; ++j) {
                    if (soff[j] < 0) continue;
                    const bool ok = pv && goff[j] >= 0;
                    const float* src = u + (ok ? nx * pstride + goff[j] : 0);
#pragma unroll
                    for (int i = 0; i < 3; ++i) cp_async4(dst + 3 * (tid + j * NE) + i, src + (ok ? i : 0), ok);
                }
            }
            cp_async_commit();
        };
        auto store_plane = [&](int jp) {
            if (jp > nslab) return;
            const int slot = jp & (RING - 1);
            const int nx = X0 - 1 + jp;
            const bool pv = nx >= 0 && nx < nnx;
            const float* src = raw + (jp % RAW) * (SN * SN * 3);
#pragma unroll
            for (int j = 0; j < NSTG; ++j) {
                if (soff[j] < 0) continue;
                const bool ok = pv && goff[j] >= 0;  // outside the grid: 0, not -c
                const float* w = src + 3 * (tid + j * NE);
                const float v0 = ok ? w[0] - c0 : 0.f, v1 = ok ? w[1] - c1 : 0.f, v2 = ok ? w[2] - c2 : 0.f;
                float4 h, l;
                h.x = to_tf32(v0);
                h.y = to_tf32(v1);
                h.z = to_tf32(v2);
                h.w = 0.f;
                l.x = to_tf32(v0 - h.x);
                l.y = to_tf32(v1 - h.y);
                l.z = to_tf32(v2 - h.z);
                l.w = 0.f;
                *reinterpret_cast<float4*>(smem + OFF_HI + slot * PLANEB + soff[j]) = h;
                *reinterpret_cast<float4*>(smem + OFF_LO + slot * PLANEB + soff[j]) = l;
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(full + slot)) : "memory");
        };

        // this thread's element column: tile t, TMEM lane row; (yl, zl) in the block's element frame
        const int t = warp >> 2, row = 32 * (warp & 3) + lane;
        const int yq = row & 7, zl = row >> 3, yl = 8 * t + yq;
        const int ey = Y0 - 1 + yl, ez = Z0 - 1 + zl;
        const bool eyz = ey >= 0 && ey < d.nely && ez >= 0 && ez < d.nelz;
        const long long eoff = ey + (long long)d.nely * ez, estride = (long long)d.nely * d.nelz;
        auto loadE = [&](int s) {
            const int ex = X0 - 1 + s;
            return (eyz && ex >= 0 && ex < d.nelx) ? E[eoff + ex * estride] : 0.f;
        };
        const bool owner = yl >= 1 && zl >= 1 && ey < nny && ez < nnz;  // node (ey, ez) of each plane

        // prologue: planes 0, 1, 2 staged, 3 and 4 in flight
        raw_issue(0);
        raw_issue(1);
        raw_issue(2);
        cp_async_wait<0>();
        store_plane(0);
        store_plane(1);
        store_plane(2);
        raw_issue(3);
        raw_issue(4);

        float Enext = loadE(0);
        float cin[3][4];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) cin[i][q] = 0.f;
        // epilogue operands of the owned node in output plane X0 - 1 + s, fetched one slab ahead
        float rn[3], dn[3], un[3];
        unsigned fn[3];  // the raw flags: tested where used, so the load does not stall the fetch
        auto fetch = [&](int s1) {
            const bool em = s1 > 0 && s1 < nslab && owner;
            const long long g1 = 3 * (ey + (long long)nny * (ez + (long long)nnz * (X0 - 1 + s1)));
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                rn[i] = (MODE != 0 && em) ? r[g1 + i] : 0.f;
                dn[i] = (MODE == 1 && em) ? dinv[g1 + i] : 0.f;
                un[i] = ((MODE == 1 || PCG) && em) ? u[g1 + i] : 0.f;
                fn[i] = em ? (unsigned)fixed[g1 + i] : 0u;
            }
        };
        fetch(1);
        DotAcc<float> dot;
        for (int s = 0; s < nslab; ++s) {
            raw_issue(s + 5);  // two slabs of slack for the copy
            const float Es = Enext;
            if (s + 1 < nslab) Enext = loadE(s + 1);
            const bool emit = s > 0 && owner;  // output node plane X0 - 1 + s
            const long long gn = 3 * (ey + (long long)nny * (ez + (long long)nnz * (X0 - 1 + s)));
            float rr[3], di[3], uo[3];
            unsigned fx[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                rr[i] = rn[i];
                di[i] = dn[i];
                uo[i] = un[i];
                fx[i] = fn[i];
            }
            if (s > 0) fetch(s + 1);  // (at s = 0 the registers already hold slab 1)
            const int par = s & 1;
            if (!mbar_wait(smem_u32(tdone + 2 * par + t), (uint32_t)((s >> 1) & 1))) {
                fail[par] = 1;
                if (err) atomicExch(err, (int)TO_ETIMEOUT);
            }
            fence_after_sync();
            float D[24];
            {
                float Dl[24];
                const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(par * 128 + t * 64);
                tmem_ld16(taddr, D);
                tmem_ld8(taddr + 16, D + 16);
                tmem_ld16(taddr + 32, Dl);
                tmem_ld8(taddr + 48, Dl + 16);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int n = 0; n < 24; ++n) D[n] += Dl[n];  // (Ah Bh + Al Bh) + Ah Bl
            }
            fence_before_sync();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(tfree + 2 * par + t)) : "memory");
            // x: the gx = 0 corners of this slab plus the carried gx = 1 corners of the previous one;
            // corner q = 2 hy + hz of output row 3 (4 hx + q) + i
            float p[3][4];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    p[i][q] = fmaf(Es, D[3 * q + i], cin[i][q]);
                    cin[i][q] = Es * D[3 * (4 + q) + i];
                }
            // y: the hy = 1 corners of the element column at yl - 1 (lane - 1 inside a group of 8)
            float q0[3], q1[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float y0 = __shfl_up_sync(0xffffffffu, p[i][2], 1, 8);
                const float y1 = __shfl_up_sync(0xffffffffu, p[i][3], 1, 8);
                q0[i] = p[i][0] + (yq ? y0 : 0.f);
                q1[i] = p[i][1] + (yq ? y1 : 0.f);
            }
            float* Xp = X + par * (X_FLOATS / 2);
            float* Yp = YB + par * (YB_FLOATS / 2);
#pragma unroll
            for (int i = 0; i < 3; ++i) Xp[((t * 16 + zl) * 8 + yq) * 3 + i] = q1[i];
            if (t == 0 && yq == 7) {  // the tile seam: tile 1's first y row needs these
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    Yp[(zl * 3 + i) * 2] = p[i][2];
                    Yp[(zl * 3 + i) * 2 + 1] = p[i][3];
                }
            }
            // plane s + 3 goes to the ring slot of plane s - 1, which the MMAs of slab s - 1
            // (both tiles, issued before those of slab s this thread waited for) no longer read
            cp_async_wait<2>();  // plane s + 3 has landed (s + 4, s + 5 may be in flight)
            store_plane(s + 3);
            asm volatile("bar.sync 1, %0;\n" ::"n"(NE) : "memory");  // the staging / epilogue warps only
            if (fail[par]) break;  // the same value in every thread: written before this barrier only
            if (emit) {
                // z: the gz = 1 corners of the element column at zl - 1
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float o = q0[i] + Xp[((t * 16 + zl - 1) * 8 + yq) * 3 + i];
                    if (t == 1 && yq == 0) o += Yp[(zl * 3 + i) * 2] + Yp[((zl - 1) * 3 + i) * 2 + 1];
                    if (MODE == 1) o = uo[i] + omega * di[i] * (rr[i] - o);
                    if (MODE == 2) o = rr[i] - o;
                    if (fx[i] != 0u) o = 0.f;
                    out[gn + i] = o;
                    if (PCG) dot.add(MODE == 1 ? rr[i] : uo[i], o);
                }
            }
        }
        cp_async_wait<0>();
        if (PCG) dot_out = dot.value();
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
    }
    if (PCG) {
        double vv[1] = {dot_out}, tot[1];
        if (last_block_totals<NT, 1>(vv, partials, counter, tot) && threadIdx.x == 0) {
            if (MODE == 1) {  // last V-cycle sweep: rz = r.z, beta = rz / rz_old
                pcg->beta = tot[0] / pcg->rz;
                pcg->rz = tot[0];
            } else {          // K p: alpha = rz / p.Ap
                pcg->pAp = tot[0];
                pcg->alpha = pcg->rz / tot[0];
            }
        }
    }
}

// Round to TF32 as cvt.rna does (nearest, ties away from zero).
static float tf32_host(float v) {
    uint32_t b;
    std::memcpy(&b, &v, 4);
    if ((b & 0x7f800000u) != 0x7f800000u) b = (b + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

// Pack Ke (rounded to FP32) as the B operand tiles of the tensor-core operator.
// For each K order (gx = 0 then 1, or swapped) and element corner offsets
// (gy, gz): an N = 64 tile whose rows n < 24 hold the TF32 high part of
// B[n][k] = Ke[3 Lo + co][3 Li + ci] and rows 32 + n its TF32 low part, and an
// N = 32 tile of the high part alone; n = 3 (4 hx + 2 hy + hz) + co, k =
// 4 (gx or 1 - gx) + ci (ci = 3 and the other rows zero); Lo, Li the local node
// numbers of the output corner (hx, hy, hz) and the input corner (gx, gy, gz)
// of the element in grid orientation.
void tc_pack_ke(const std::vector<double>& Ke, std::vector<float>& pack) {
    using namespace tc;
    pack.assign(B_FLOATS, 0.f);
    auto lof = [](int gx, int gy, int gz) { return local_node(gx, 1 - gy, gz); };
    for (int order = 0; order < 2; ++order)
        for (int m = 0; m < 4; ++m) {
            const int gy = m >> 1, gz = m & 1;
            float* hl = pack.data() + b_set(order, m);
            float* h_only = hl + B_HL;
            for (int n = 0; n < 24; ++n) {
                const int go = n / 3, co = n % 3;
                const int Lo = lof(go >> 2, (go >> 1) & 1, go & 1);
                for (int k = 0; k < 8; ++k) {
                    const int ci = k & 3;
                    if (ci == 3) continue;
                    const int gx = order ? 1 - (k >> 2) : (k >> 2);
                    const float v = (float)Ke[(size_t)(3 * Lo + co) * 24 + 3 * lof(gx, gy, gz) + ci];
                    const float h = tf32_host(v);
                    hl[b_off(n, k)] = h;
                    hl[b_off(32 + n, k)] = tf32_host(v - h);
                    h_only[b_off(n, k)] = h;
                }
            }
        }
}

template <int MODE, bool PCG>
static void tc_dispatch(const to_grid* g, const float* E, const float* u, const float* r, const float* dinv, float* out,
                        float omega, const int* skip, PcgScalars* pcg, cudaStream_t st) {
    using namespace tc;
    static bool attr_set = false;  // the same attribute value on every call
    if (!attr_set) {
        TOPO_CUDA(cudaFuncSetAttribute(k_ku_tc<MODE, PCG>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        attr_set = true;
    }
    const Dims& d = g->d;
    const int ntY = div_up(d.nny, TN), ntZ = div_up(d.nnz, TN);
    const long long tiles = (long long)ntY * ntZ;
    const int nsm = g->nsm > 0 ? g->nsm : 148;
    // about four blocks per SM over the launch, at least four planes per block
    // (the first element plane of a block only carries into the next)
    const long long chunks = std::max<long long>(1, 4LL * nsm / tiles);
    int LX = std::max(4, div_up(d.nnx, chunks));
    long long nb = tiles * div_up(d.nnx, LX);
    while (PCG && nb > g->npartials) {  // one partial per block
        LX *= 2;
        nb = tiles * div_up(d.nnx, LX);
    }
    launch_k(k_ku_tc<MODE, PCG>, (unsigned)nb, NT, SMEM_BYTES, st, d, LX, ntY, ntZ, E, u, r, dinv, out,
             (const uint8_t*)g->fixed, omega, (const float*)g->ke_tc, skip, pcg, g->partials, g->counter, g->tc_err);
}

void launch_fine_op_tc(const to_grid* g, int mode, const float* E, const float* u, const float* r, const float* dinv,
                       float* out, float omega, const int* skip, PcgScalars* pcg, cudaStream_t st) {
    TOPO_REQUIRE(g->d.dim == 3 && g->ke_tc, "tensor-core operator needs a 3D grid and packed Ke");
    if (mode == 0 && pcg)
        tc_dispatch<0, true>(g, E, u, r, dinv, out, omega, skip, pcg, st);
    else if (mode == 0)
        tc_dispatch<0, false>(g, E, u, r, dinv, out, omega, skip, nullptr, st);
    else if (mode == 1 && pcg)
        tc_dispatch<1, true>(g, E, u, r, dinv, out, omega, skip, pcg, st);
    else if (mode == 1)
        tc_dispatch<1, false>(g, E, u, r, dinv, out, omega, skip, nullptr, st);
    else
        tc_dispatch<2, false>(g, E, u, r, dinv, out, omega, skip, nullptr, st);
}

}  // namespace topo
