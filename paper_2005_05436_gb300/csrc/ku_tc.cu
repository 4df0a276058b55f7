// Tensor-core (tcgen05) form of the FP32 matrix-free operator K(xPhys) u on H8
// grids: the element contraction Ke u_e of Eqs. 4-5, batched over the elements
// of a brick, runs as TF32 MMAs with FP32 accumulation in tensor memory.
//
// A CTA owns an 8 x 4 x 4 (y, z, x) brick of nodes and computes the 9 x 5 x 5
// elements touching it (two M = 128 row tiles, rows 225..255 zero):
//   A[e][k] = u_e[k] - u_e[node 0 of e][k % 3]    (24 columns, K = 24)
//   B[j][k] = Ke[j][k]                             (N = 32, rows 24..31 zero)
//   D = A B^T  ->  D[e][j] = (Ke u_e)_j, exact for the translation shift because
//   the rows of Ke annihilate rigid translations.
// A and B are split into TF32 high and low parts and D = Ah Bh + Al Bh + Ah Bl,
// which carries about 21 bits, close to FP32. Each owned node then sums, from
// shared memory, the E_e-scaled rows of its 8 elements, so every output is
// written by exactly one thread and the smoother / residual / PCG-dot epilogues
// of the CUDA-core operator stay fused.
//
// Operands use the canonical no-swizzle K-major layout: 8-row x 16-byte core
// matrices, LBO = 128 B between core matrices along K, SBO = 768 B between
// 8-row groups (6 core matrices of K per row group).
#include <cstring>
#include <vector>

#include "grid.h"
#include "ku_device.cuh"
#include "mg.h"

namespace topo {

namespace tc {

constexpr int OY = 8, OZ = 4, OX = 4;              // owned nodes per CTA
constexpr int EY = OY + 1, EZ = OZ + 1, EX = OX + 1;  // elements touching them
constexpr int NEL = EY * EZ * EX;                  // 225
constexpr int PY = OY + 2, PZ = OZ + 2, PX = OX + 2;  // input node patch
constexpr int NPATCH = PY * PZ * PX;               // 360
constexpr int ROWS = 256;                          // two M = 128 tiles
constexpr int KDIM = 24, NDIM = 32, KG = KDIM / 4;  // K in 4-element (16 B) core columns
constexpr int RSTRIDE = 25;                        // element-result row stride (floats)
constexpr int NT = 256;
constexpr int TMEM_COLS = 64;                      // two tiles x 32 columns
constexpr long long WAIT_LIMIT = 1LL << 26;        // mbarrier polls before giving up

// shared-memory layout (bytes)
constexpr int A_BYTES = ROWS * KDIM * 4;           // 24576
constexpr int B_BYTES = NDIM * KDIM * 4;           // 3072
constexpr int OFF_AHI = 0;
constexpr int OFF_ALO = OFF_AHI + A_BYTES;
constexpr int OFF_BHI = OFF_ALO + A_BYTES;
constexpr int OFF_BLO = OFF_BHI + B_BYTES;
constexpr int OFF_E = OFF_BLO + B_BYTES;           // 256 floats
constexpr int OFF_U = OFF_E + 256 * 4;             // NPATCH * 3 floats
constexpr int OFF_BAR = OFF_U + ((NPATCH * 3 * 4 + 15) / 16) * 16;
constexpr int SMEM_BYTES = OFF_BAR + 16;
static_assert(NEL * RSTRIDE * 4 <= A_BYTES, "element results reuse the A(hi) buffer");

// Float offset of element (row r, column k) in the core-matrix layout.
__host__ __device__ constexpr int core_off(int r, int k) { return ((r >> 3) * KG + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }

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

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, N = 32, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NDIM >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc));
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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc

template <int MODE, bool PCG>
__global__ void __launch_bounds__(tc::NT, 2) k_fine_op3_tc(Dims d, const float* __restrict__ E,
                                                           const float* __restrict__ u, const float* __restrict__ r,
                                                           const float* __restrict__ dinv, float* __restrict__ out,
                                                           const uint8_t* __restrict__ fixed, float omega,
                                                           const float* __restrict__ Bpack, const int* skip,
                                                           PcgScalars* pcg, double* partials, unsigned* counter,
                                                           int* err) {
    using namespace tc;
    if (skip && *skip) return;  // uniform, before any tensor-memory use
    extern __shared__ __align__(1024) unsigned char smem[];
    float* Ahi = (float*)(smem + OFF_AHI);
    float* Alo = (float*)(smem + OFF_ALO);
    float* Bhi = (float*)(smem + OFF_BHI);
    float* Blo = (float*)(smem + OFF_BLO);
    float* Es = (float*)(smem + OFF_E);
    float* pu = (float*)(smem + OFF_U);
    uint64_t* bar = (uint64_t*)(smem + OFF_BAR);
    __shared__ uint32_t tmem_base;
    __shared__ int wait_ok;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int by0 = blockIdx.x * OY, bz0 = blockIdx.y * OZ, bx0 = blockIdx.z * OX;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)));
        wait_ok = 1;
    }
    // node patch (0 outside the grid), element moduli (0 outside), packed Ke halves
    for (int i = tid; i < NPATCH * 3; i += NT) {
        const int p = i / 3, c = i % 3;
        const int py = p % PY, pz = (p / PY) % PZ, px = p / (PY * PZ);
        const int gy = by0 - 1 + py, gz = bz0 - 1 + pz, gx = bx0 - 1 + px;
        float v = 0.f;
        if (gy >= 0 && gy < d.nny && gz >= 0 && gz < d.nnz && gx >= 0 && gx < d.nnx)
            v = u[3 * (gy + (long long)d.nny * (gz + (long long)d.nnz * gx)) + c];
        pu[i] = v;
    }
    for (int i = tid; i < ROWS; i += NT) {
        float v = 0.f;
        if (i < NEL) {
            const int ly = i % EY, lz = (i / EY) % EZ, lx = i / (EY * EZ);
            const int ey = by0 - 1 + ly, ez = bz0 - 1 + lz, ex = bx0 - 1 + lx;
            if (ey >= 0 && ey < d.nely && ez >= 0 && ez < d.nelz && ex >= 0 && ex < d.nelx)
                v = E[ey + (long long)d.nely * (ez + (long long)d.nelz * ex)];
        }
        Es[i] = v;
    }
    for (int i = tid; i < 2 * NDIM * KDIM; i += NT) (i < NDIM * KDIM ? Bhi : Blo)[i % (NDIM * KDIM)] = Bpack[i];
    __syncthreads();
    // A rows: thread tid builds row tid (rows >= NEL are zero)
    {
        const int row = tid;
        float vals[KDIM];
        if (row < NEL) {
            const int ly = row % EY, lz = (row / EY) % EZ, lx = row / (EY * EZ);
            float ref[3];
#pragma unroll
            for (int M = 0; M < 8; ++M) {
                const int p = (ly + 1 - lny(M)) + PY * ((lz + lnz(M)) + PZ * (lx + lnx(M)));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float v = pu[3 * p + c];
                    if (M == 0) ref[c] = v;
                    vals[3 * M + c] = v - ref[c];
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < KDIM; ++k) vals[k] = 0.f;
        }
#pragma unroll
        for (int kg = 0; kg < KG; ++kg) {
            float4 h, l;
            h.x = to_tf32(vals[4 * kg + 0]);
            h.y = to_tf32(vals[4 * kg + 1]);
            h.z = to_tf32(vals[4 * kg + 2]);
            h.w = to_tf32(vals[4 * kg + 3]);
            l.x = to_tf32(vals[4 * kg + 0] - h.x);
            l.y = to_tf32(vals[4 * kg + 1] - h.y);
            l.z = to_tf32(vals[4 * kg + 2] - h.z);
            l.w = to_tf32(vals[4 * kg + 3] - h.w);
            *(float4*)(Ahi + core_off(row, 4 * kg)) = h;
            *(float4*)(Alo + core_off(row, 4 * kg)) = l;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (tid == 0) {
        const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo), bhi = smem_u32(Bhi), blo = smem_u32(Blo);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const uint32_t dt = tmem + 32 * t;                 // column offset of tile t
            const uint32_t arow = (uint32_t)(t * 16 * KG * 128);  // 16 row groups per tile
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const uint32_t kofs = (uint32_t)(2 * s * 128);      // two core columns per K step
                const uint64_t dah = make_desc(ahi + arow + kofs, 128, KG * 128);
                const uint64_t dal = make_desc(alo + arow + kofs, 128, KG * 128);
                const uint64_t dbh = make_desc(bhi + kofs, 128, KG * 128);
                const uint64_t dbl = make_desc(blo + kofs, 128, KG * 128);
                mma_tf32(dt, dah, dbh, s > 0 ? 1u : 0u);
                mma_tf32(dt, dal, dbh, 1u);
                mma_tf32(dt, dah, dbl, 1u);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(bar))
                     : "memory");
    }
    if (!mbar_wait(smem_u32(bar), 0)) {
        wait_ok = 0;
        if (err) atomicExch(err, (int)TO_ETIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // D rows back to registers: warp w reads tile w / 4, lanes 32 (w % 4) ...
    float dv[KDIM];
    {
        const int t = warp >> 2, q = warp & 3;
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * t);
        float v8[8];
#pragma unroll
        for (int c8 = 0; c8 < 3; ++c8) {
            tc::tmem_ld8(taddr + 8 * c8, v8);
#pragma unroll
            for (int i = 0; i < 8; ++i) dv[8 * c8 + i] = v8[i];
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // all MMAs consumed: A(hi) becomes the element-result buffer
    {
        const int row = 128 * (warp >> 2) + 32 * (warp & 3) + lane;
        float* R = Ahi;
        if (row < NEL) {
            const float s = wait_ok ? Es[row] : 0.f;
#pragma unroll
            for (int j = 0; j < KDIM; ++j) R[row * RSTRIDE + j] = s * dv[j];
        }
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
    }
    // owned nodes: sum the rows of their 8 elements, fused epilogue
    DotAcc<float> dot;
    const float* R = Ahi;
    for (int item = tid; item < OY * OZ * OX * 3; item += NT) {
        const int o = item / 3, c = item % 3;
        const int oy = o % OY, oz = (o / OY) % OZ, ox = o / (OY * OZ);
        const int iy = by0 + oy, iz = bz0 + oz, ix = bx0 + ox;
        if (iy >= d.nny || iz >= d.nnz || ix >= d.nnx) continue;
        float a = 0.f;
#pragma unroll
        for (int e8 = 0; e8 < 8; ++e8) {
            const int exo = e8 >> 2, ezo = (e8 >> 1) & 1, eyo = e8 & 1;
            const int row = (oy + eyo) + EY * ((oz + ezo) + EZ * (ox + exo));
            const int L = local_node(1 - exo, eyo, 1 - ezo);
            a += R[row * RSTRIDE + 3 * L + c];
        }
        const long long i = 3 * (iy + (long long)d.nny * (iz + (long long)d.nnz * ix)) + c;
        float o_ = a;
        if (MODE == 1) o_ = u[i] + omega * dinv[i] * (r[i] - a);
        if (MODE == 2) o_ = r[i] - a;
        if (fixed[i]) o_ = 0.f;
        out[i] = o_;
        if (PCG) dot.add(u[i], o_);
    }
    if (PCG) {
        double v[1] = {dot.value()}, tot[1];
        if (last_block_totals<tc::NT, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
            pcg->pAp = tot[0];
            pcg->alpha = pcg->rz / tot[0];
        }
    }
}

// Pack Ke (FP32) into the B operand: high and low TF32 halves, N = 32 rows
// (24..31 zero), core-matrix layout; [2][32 * 24] floats.
static float tf32_host(float v) {
    uint32_t b;
    std::memcpy(&b, &v, 4);
    if ((b & 0x7f800000u) != 0x7f800000u) b = (b + 0x1000u) & 0xffffe000u;  // round half away from zero
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

void tc_pack_ke(const std::vector<double>& Ke, std::vector<float>& pack) {
    using namespace tc;
    pack.assign(2 * NDIM * KDIM, 0.f);
    for (int j = 0; j < NDIM; ++j)
        for (int k = 0; k < KDIM; ++k) {
            const float v = j < 24 ? (float)Ke[(size_t)j * 24 + k] : 0.f;
            const float h = tf32_host(v);
            pack[core_off(j, k)] = h;
            pack[NDIM * KDIM + core_off(j, k)] = tf32_host(v - h);
        }
}

template <int MODE, bool PCG>
static void tc_dispatch(const to_grid* g, const float* E, const float* u, const float* r, const float* dinv, float* out,
                        float omega, const int* skip, PcgScalars* pcg, cudaStream_t st) {
    using namespace tc;
    static bool attr_set = false;
    if (!attr_set) {
        TOPO_CUDA(cudaFuncSetAttribute(k_fine_op3_tc<MODE, PCG>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        attr_set = true;
    }
    const Dims& d = g->d;
    dim3 grid(div_up(d.nny, OY), div_up(d.nnz, OZ), div_up(d.nnx, OX));
    k_fine_op3_tc<MODE, PCG><<<grid, NT, SMEM_BYTES, st>>>(d, E, u, r, dinv, out, g->fixed, omega, g->ke_tc, skip, pcg,
                                                         g->partials, g->counter, g->tc_err);
    TOPO_CHECK_LAUNCH();
}

void launch_fine_op_tc(const to_grid* g, int mode, const float* E, const float* u, const float* r, const float* dinv,
                       float* out, float omega, const int* skip, PcgScalars* pcg, cudaStream_t st) {
    TOPO_REQUIRE(g->d.dim == 3 && g->ke_tc, "tensor-core operator needs a 3D grid and packed Ke");
    if (mode == 0 && pcg)
        tc_dispatch<0, true>(g, E, u, r, dinv, out, omega, skip, pcg, st);
    else if (mode == 0)
        tc_dispatch<0, false>(g, E, u, r, dinv, out, omega, skip, nullptr, st);
    else if (mode == 1)
        tc_dispatch<1, false>(g, E, u, r, dinv, out, omega, skip, nullptr, st);
    else
        tc_dispatch<2, false>(g, E, u, r, dinv, out, omega, skip, nullptr, st);
}

}  // namespace topo
