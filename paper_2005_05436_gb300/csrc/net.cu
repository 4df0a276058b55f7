// The learned warm start of the state solve (no counterpart in the paper): a
// small 3D convolutional encoder-decoder that maps node fields (the physical
// density averaged to the nodes and the load) to a displacement direction, with
// its own forward and backward kernels and an Adam optimiser.
//
// Architecture (levels 3, base channels c; every conv is 3x3x3, zero padding 1):
//   e0 = relu(conv(relu(conv(x, 4->c)), c->c))
//   e1 = relu(conv(relu(conv(pool(e0), c->2c)), 2c->2c))
//   e2 = relu(conv(relu(conv(pool(e1), 2c->4c)), 4c->4c))
//   d1 = relu(conv(relu(conv(up(e2), 4c->2c)) + e1, 2c->2c))
//   d0 = relu(conv(relu(conv(up(d1), 2c->c)) + e0, c->c))
//   y  = conv(d0, c->3)
// pool = 2x2x2 mean, up = nearest 2x. Tensors are [N][D][H][W][C] (channels
// last); the spatial sizes must be multiples of 4. Activations and the weights
// the convolutions read are BF16 (or FP32 for exact gradient checks); every
// product is accumulated in FP32; master weights, gradients and Adam moments
// are FP32. Parameters are one flat vector, layer by layer W[27][cin][cout]
// then b[cout], tap t = (dx+1)*9 + (dy+1)*3 + (dz+1) over (D, H, W).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <vector>

#include "grid.h"

namespace topo {
namespace nn {
namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float tof(float v) { return v; }
__device__ __forceinline__ float tof(bf16 v) { return __bfloat162float(v); }
template <typename T>
__device__ __forceinline__ T fromf(float v);
template <>
__device__ __forceinline__ float fromf<float>(float v) { return v; }
template <>
__device__ __forceinline__ bf16 fromf<bf16>(float v) { return __float2bfloat16_rn(v); }

// Four consecutive channels (Cin % 4 == 0; 8- or 16-byte aligned).
__device__ __forceinline__ void load4(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
__device__ __forceinline__ void load4(const bf16* p, float (&o)[4]) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&v.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&v.y);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    o[0] = fa.x;
    o[1] = fa.y;
    o[2] = fb.x;
    o[3] = fb.y;
}

struct Shape {
    int N, D, H, W;
    __host__ __device__ long long vox() const { return (long long)N * D * H * W; }
};

__device__ __forceinline__ void decode(const Shape& s, long long v, int& n, int& d, int& h, int& w) {
    w = (int)(v % s.W);
    long long t = v / s.W;
    h = (int)(t % s.H);
    t /= s.H;
    d = (int)(t % s.D);
    n = (int)(t / s.D);
}

constexpr int CT = 128;  // threads of the convolution kernels

// y[v][co] = b[co] + sum_t sum_ci x[v + tap t][ci] W[t][ci][co]  (+ relu)
template <typename TI, typename TO, int COB>
__global__ void __launch_bounds__(CT) kn_conv_fwd(const TI* __restrict__ x, const TI* __restrict__ Wt,
                                                  const float* __restrict__ bias, TO* __restrict__ y, Shape s,
                                                  int Cin, int Cout, int relu) {
    extern __shared__ float ws[];  // [Cin][COB] of the current tap
    const long long V = s.vox();
    const long long v = (long long)blockIdx.x * CT + threadIdx.x;
    const int co0 = blockIdx.y * COB;
    int n = 0, d = 0, h = 0, w = 0;
    if (v < V) decode(s, v, n, d, h, w);
    float acc[COB];
#pragma unroll
    for (int j = 0; j < COB; ++j) acc[j] = co0 + j < Cout ? bias[co0 + j] : 0.f;
    for (int t = 0; t < 27; ++t) {
        __syncthreads();
        for (int i = threadIdx.x; i < Cin * COB; i += CT) {
            const int ci = i / COB, j = i % COB;
            ws[i] = co0 + j < Cout ? tof(Wt[((long long)t * Cin + ci) * Cout + co0 + j]) : 0.f;
        }
        __syncthreads();
        if (v >= V) continue;
        const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
        const int dd = d + dx, hh = h + dy, ww = w + dz;
        if (dd < 0 || dd >= s.D || hh < 0 || hh >= s.H || ww < 0 || ww >= s.W) continue;
        const TI* xp = x + (v + ((long long)dx * s.H + dy) * s.W + dz) * Cin;
        for (int ci = 0; ci < Cin; ci += 4) {
            float xv[4];
            load4(xp + ci, xv);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int j = 0; j < COB; ++j) acc[j] += xv[q] * ws[(ci + q) * COB + j];
        }
    }
    if (v >= V) return;
#pragma unroll
    for (int j = 0; j < COB; ++j) {
        if (co0 + j >= Cout) continue;
        const float o = relu ? fmaxf(acc[j], 0.f) : acc[j];
        y[v * Cout + co0 + j] = fromf<TO>(o);
    }
}

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05, kind::f16) forward convolution for BF16 layers with
// Cin, Cout in {16, 32, 64}: an implicit GEMM with M = 128 voxels per CTA,
// N = Cout and K = 27 taps x Cin. For each tap the CTA stages the 128 shifted
// input rows (Cin BF16 values, zero outside the volume) and the tap's weights
// (packed once per weight update into the same layout) into shared memory with
// 16-byte cp.async, NSTAGE taps in flight; one thread issues the Cin/16 MMAs
// of the tap (BF16 A and B, FP32 accumulation in tensor memory) and commits
// them to the buffer's mbarrier, whose completion frees the buffer for the tap
// NSTAGE - 1 later.
// Operands use the canonical no-swizzle K-major layout: 8-row x 16-byte core
// matrices, LBO = 128 B along K, SBO = 128 Cin / 8 B between 8-row groups.
namespace tcc {
constexpr int MT = 128;                      // voxels (rows) per CTA
constexpr int NTH = 128;                     // threads: one per row
constexpr long long WAIT_LIMIT = 1LL << 26;  // mbarrier polls before giving up
constexpr int NSTAGE = 4;                    // tap buffers in flight

__host__ __device__ constexpr int core_byte(int r, int k, int KG) {
    return ((r >> 3) * KG + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; base offset 0, no swizzle
    return d;
}
// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
                 "r"(pred ? 16 : 0)
                 : "memory");
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
}  // namespace tcc

// Packed weights of one layer: per tap, Cout rows x Cin columns in the core layout.
__global__ void kn_pack_w(const bf16* __restrict__ W, bf16* __restrict__ Bp, int cin, int cout) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = 27LL * cin * cout;
    if (i >= n) return;
    const int co = (int)(i % cout);
    const long long r = i / cout;
    const int ci = (int)(r % cin), t = (int)(r / cin);  // W[t][ci][co]
    Bp[(long long)t * cin * cout + tcc::core_byte(co, ci, cin / 8) / 2] = W[i];
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(tcc::NTH) kn_conv_fwd_tc(const bf16* __restrict__ x, const bf16* __restrict__ Bp,
                                                           const float* __restrict__ bias, bf16* __restrict__ y,
                                                           Shape s, int relu, int* err) {
    using namespace tcc;
    constexpr int KG = CIN / 8;
    constexpr int A_BYTES = MT * CIN * 2, B_BYTES = COUT * CIN * 2, S_BYTES = A_BYTES + B_BYTES;
    constexpr int TCOLS = COUT < 32 ? 32 : COUT;
    constexpr uint32_t IDESC = idesc_bf16(COUT);
    extern __shared__ __align__(1024) unsigned char smc[];
    uint64_t* bar = (uint64_t*)(smc + NSTAGE * S_BYTES);  // one per stage
    __shared__ uint32_t tmem_base;
    __shared__ int ok_s;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long V = s.vox();
    const long long v = (long long)blockIdx.x * MT + tid;  // this thread's row
    const bool vin = v < V;
    int n_ = 0, d_ = 0, h_ = 0, w_ = 0;
    if (vin) decode(s, v, n_, d_, h_, w_);
    (void)n_;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < NSTAGE; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar[b])));
        ok_s = 1;
    }
    // one commit group per call (empty past the last tap)
    auto stage = [&](int t) {
        if (t < 27) {
            const int buf = t % NSTAGE;
            const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
            const int dd = d_ + dx, hh = h_ + dy, ww = w_ + dz;
            const bool ok = vin && dd >= 0 && dd < s.D && hh >= 0 && hh < s.H && ww >= 0 && ww < s.W;
            const bf16* src = ok ? x + (v + ((long long)dx * s.H + dy) * s.W + dz) * CIN : x;
            unsigned char* A = smc + buf * S_BYTES;
#pragma unroll
            for (int kc = 0; kc < KG; ++kc) cp_async16(A + core_byte(tid, 8 * kc, KG), ok ? src + 8 * kc : x, ok);
            const unsigned char* bsrc = (const unsigned char*)(Bp + (long long)t * CIN * COUT);
            unsigned char* B = A + A_BYTES;
            for (int c = tid; c < B_BYTES / 16; c += NTH) cp_async16(B + 16 * c, bsrc + 16 * c, true);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
#pragma unroll
    for (int t = 0; t < NSTAGE - 1; ++t) stage(t);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool ok = true;
    for (int t = 0; t < 27; ++t) {
        asm volatile("cp.async.wait_group %0;\n" ::"n"(NSTAGE - 2) : "memory");  // tap t has landed
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int buf = t % NSTAGE;
            const uint32_t a0 = smem_u32(smc + buf * S_BYTES), b0 = a0 + A_BYTES;
#pragma unroll
            for (int k = 0; k < CIN / 16; ++k) {
                const uint64_t da = make_desc(a0 + 256 * k, 128, KG * 128);
                const uint64_t db = make_desc(b0 + 256 * k, 128, KG * 128);
                const uint32_t acc = (t > 0 || k > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&bar[buf]))
                         : "memory");
        }
        // with tap t queued behind it, wait for tap t - 1 and reuse its buffer for tap t + NSTAGE - 1
        const int tn = t + NSTAGE - 1;
        if (tn < 27 && t >= 1 && ok &&
            !mbar_wait(smem_u32(&bar[(t - 1) % NSTAGE]), (uint32_t)(((t - 1) / NSTAGE) & 1)))
            ok = false;
        stage(tn);
    }
    // the taps whose commits were not awaited in the loop, in order
    for (int t = 27 - NSTAGE; t < 27; ++t)
        if (ok && !mbar_wait(smem_u32(&bar[t % NSTAGE]), (uint32_t)((t / NSTAGE) & 1))) ok = false;
    if (!ok) {
        ok_s = 0;
        if (err) atomicExch(err, (int)TO_ETIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float acc[COUT];
    {
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int c8 = 0; c8 < COUT / 8; ++c8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(taddr + 8 * c8));
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[8 * c8 + i] = __uint_as_float(r[i]);
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS));
    }
    if (!vin || !ok_s) return;
    bf16* yo = y + v * COUT;
#pragma unroll
    for (int c8 = 0; c8 < COUT / 8; ++c8) {
        __nv_bfloat162 q[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float a = acc[8 * c8 + 2 * i] + bias[8 * c8 + 2 * i];
            float b = acc[8 * c8 + 2 * i + 1] + bias[8 * c8 + 2 * i + 1];
            if (relu) {
                a = fmaxf(a, 0.f);
                b = fmaxf(b, 0.f);
            }
            q[i] = __floats2bfloat162_rn(a, b);
        }
        *reinterpret_cast<uint4*>(yo + 8 * c8) = *reinterpret_cast<const uint4*>(q);
    }
}

// gx[v][ci] = sum_t sum_co gz[v - tap t][co] W[t][ci][co]
template <typename TW, int CIB>
__global__ void __launch_bounds__(CT) kn_conv_bwd_data(const float* __restrict__ gz, const TW* __restrict__ Wt,
                                                       float* __restrict__ gx, Shape s, int Cin, int Cout) {
    extern __shared__ float ws[];  // [Cout][CIB] of the current tap
    const long long V = s.vox();
    const long long v = (long long)blockIdx.x * CT + threadIdx.x;
    const int ci0 = blockIdx.y * CIB;
    int n = 0, d = 0, h = 0, w = 0;
    if (v < V) decode(s, v, n, d, h, w);
    float acc[CIB];
#pragma unroll
    for (int j = 0; j < CIB; ++j) acc[j] = 0.f;
    for (int t = 0; t < 27; ++t) {
        __syncthreads();
        for (int i = threadIdx.x; i < Cout * CIB; i += CT) {
            const int co = i / CIB, j = i % CIB;
            ws[i] = ci0 + j < Cin ? tof(Wt[((long long)t * Cin + ci0 + j) * Cout + co]) : 0.f;
        }
        __syncthreads();
        if (v >= V) continue;
        const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
        const int dd = d - dx, hh = h - dy, ww = w - dz;
        if (dd < 0 || dd >= s.D || hh < 0 || hh >= s.H || ww < 0 || ww >= s.W) continue;
        const float* gp = gz + (v - ((long long)dx * s.H + dy) * s.W - dz) * Cout;
        for (int co = 0; co < Cout; ++co) {
            const float g = gp[co];
#pragma unroll
            for (int j = 0; j < CIB; ++j) acc[j] += g * ws[co * CIB + j];
        }
    }
    if (v >= V) return;
#pragma unroll
    for (int j = 0; j < CIB; ++j)
        if (ci0 + j < Cin) gx[v * Cin + ci0 + j] = acc[j];
}

// Partial weight gradients of one voxel chunk: part[chunk][t][ci][co] =
// sum_{v in chunk} x[v + tap t][ci] gz[v][co]; one 16 x 16 (ci, co) tile per CTA.
template <typename TI>
__global__ void __launch_bounds__(256) kn_conv_bwd_w(const TI* __restrict__ x, const float* __restrict__ gz,
                                                     float* __restrict__ part, Shape s, int Cin, int Cout,
                                                     long long chunk, int nco_tiles) {
    __shared__ float xs[32][17];
    __shared__ float gs[32][17];
    const int t = blockIdx.x;
    const long long c = blockIdx.y;
    const int ci0 = (blockIdx.z / nco_tiles) * 16, co0 = (blockIdx.z % nco_tiles) * 16;
    const int ti = threadIdx.x >> 4, to = threadIdx.x & 15;
    const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
    const long long V = s.vox();
    const long long v0 = c * chunk, v1 = std::min(V, v0 + chunk);
    float acc = 0.f;
    for (long long vb = v0; vb < v1; vb += 32) {
        for (int i = threadIdx.x; i < 32 * 16; i += 256) {
            const int k = i >> 4, q = i & 15;
            const long long v = vb + k;
            float xv = 0.f, gv = 0.f;
            if (v < v1) {
                int n, d, h, w;
                decode(s, v, n, d, h, w);
                const int dd = d + dx, hh = h + dy, ww = w + dz;
                if (ci0 + q < Cin && dd >= 0 && dd < s.D && hh >= 0 && hh < s.H && ww >= 0 && ww < s.W)
                    xv = tof(x[(v + ((long long)dx * s.H + dy) * s.W + dz) * Cin + ci0 + q]);
                if (co0 + q < Cout) gv = gz[v * Cout + co0 + q];
            }
            xs[k][q] = xv;
            gs[k][q] = gv;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) acc += xs[k][ti] * gs[k][to];
        __syncthreads();
    }
    if (ci0 + ti < Cin && co0 + to < Cout)
        part[((c * 27 + t) * Cin + ci0 + ti) * Cout + co0 + to] = acc;
}

// Partial bias gradients: part[chunk][co] = sum_{v in chunk} gz[v][co].
__global__ void kn_bias_part(const float* __restrict__ gz, float* __restrict__ part, long long V, int Cout,
                             long long chunk) {
    const int co = threadIdx.x;
    if (co >= Cout) return;
    const long long v0 = (long long)blockIdx.x * chunk, v1 = std::min(V, v0 + chunk);
    float a = 0.f;
    for (long long v = v0; v < v1; ++v) a += gz[v * Cout + co];
    part[(long long)blockIdx.x * Cout + co] = a;
}

// grad[i] += sum over chunks of part[chunk][i] (chunk order).
__global__ void kn_reduce_chunks(const float* __restrict__ part, float* __restrict__ grad, long long n, int nchunk) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a = 0.f;
    for (int c = 0; c < nchunk; ++c) a += part[(long long)c * n + i];
    grad[i] += a;
}

template <typename T>
__global__ void kn_pool(const T* __restrict__ x, T* __restrict__ y, Shape so, int C) {
    // so: the output (half) shape
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= so.vox() * C) return;
    const int c = (int)(i % C);
    int n, d, h, w;
    decode(so, i / C, n, d, h, w);
    const int D = 2 * so.D, H = 2 * so.H, W = 2 * so.W;
    float a = 0.f;
    for (int q = 0; q < 8; ++q) {
        const long long v = (((long long)n * D + 2 * d + (q >> 2)) * H + 2 * h + ((q >> 1) & 1)) * W + 2 * w + (q & 1);
        a += tof(x[v * C + c]);
    }
    y[i] = fromf<T>(a * 0.125f);
}

template <typename T>
__global__ void kn_up(const T* __restrict__ x, T* __restrict__ y, Shape so, int C) {
    // so: the output (double) shape
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= so.vox() * C) return;
    const int c = (int)(i % C);
    int n, d, h, w;
    decode(so, i / C, n, d, h, w);
    const long long v = (((long long)n * (so.D / 2) + d / 2) * (so.H / 2) + h / 2) * (so.W / 2) + w / 2;
    y[i] = x[v * C + c];
}

// gx = up(g) / 8 (the adjoint of the mean pooling), added into gx.
__global__ void kn_pool_bwd_add(const float* __restrict__ g, float* __restrict__ gx, Shape sf, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sf.vox() * C) return;
    const int c = (int)(i % C);
    int n, d, h, w;
    decode(sf, i / C, n, d, h, w);
    const long long v = (((long long)n * (sf.D / 2) + d / 2) * (sf.H / 2) + h / 2) * (sf.W / 2) + w / 2;
    gx[i] += 0.125f * g[v * C + c];
}

// gx = sum of g over the 2x2x2 children (the adjoint of nearest upsampling).
__global__ void kn_up_bwd(const float* __restrict__ g, float* __restrict__ gx, Shape sc, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.vox() * C) return;
    const int c = (int)(i % C);
    int n, d, h, w;
    decode(sc, i / C, n, d, h, w);
    const int D = 2 * sc.D, H = 2 * sc.H, W = 2 * sc.W;
    float a = 0.f;
    for (int q = 0; q < 8; ++q) {
        const long long v = (((long long)n * D + 2 * d + (q >> 2)) * H + 2 * h + ((q >> 1) & 1)) * W + 2 * w + (q & 1);
        a += g[v * C + c];
    }
    gx[i] = a;
}

template <typename T>
__global__ void kn_add(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ y, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fromf<T>(tof(a[i]) + tof(b[i]));
}

// g <- g * (y > 0) (relu'), or into out when out != g.
template <typename T>
__global__ void kn_relu_mask(const float* __restrict__ g, const T* __restrict__ y, float* __restrict__ out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = tof(y[i]) > 0.f ? g[i] : 0.f;
}

template <typename T>
__global__ void kn_cast(const float* __restrict__ a, T* __restrict__ y, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fromf<T>(a[i]);
}

// Masked squared error: totals (sum of squares, count of valid entries).
__global__ void __launch_bounds__(256) kn_mse_sum(const float* __restrict__ y, const float* __restrict__ tgt,
                                                  const uint8_t* __restrict__ mask, long long V, int C,
                                                  double* partials, unsigned* counter, double* out) {
    double v[2] = {0.0, 0.0}, tot[2];
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < V * C; i += (long long)gridDim.x * 256) {
        if (!mask[i / C]) continue;
        const double e = (double)y[i] - (double)tgt[i];
        v[0] += e * e;
        v[1] += 1.0;
    }
    if (last_block_totals<256, 2>(v, partials, counter, tot) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
    }
}

// dL/dy = 2 m (y - t) / count.
__global__ void kn_mse_grad(const float* __restrict__ y, const float* __restrict__ tgt,
                            const uint8_t* __restrict__ mask, float* __restrict__ g, long long V, int C,
                            const double* sums) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V * C) return;
    const double cnt = sums[1] > 0.0 ? sums[1] : 1.0;
    g[i] = mask[i / C] ? (float)(2.0 * ((double)y[i] - (double)tgt[i]) / cnt) : 0.f;
}

// Adam with bias correction; the weights the convolutions read are refreshed.
template <typename T>
__global__ void kn_adam(float* __restrict__ theta, T* __restrict__ wact, float* __restrict__ grad,
                        float* __restrict__ m, float* __restrict__ v, long long n, float lr_t, float b1, float b2,
                        float eps, float gscale) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i] * gscale;
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr_t * mi / (sqrtf(vi) + eps);
    theta[i] = th;
    wact[i] = fromf<T>(th);
    grad[i] = 0.f;
}

inline int nb(long long n, int t = 256) { return (int)std::max<long long>(1, (n + t - 1) / t); }

}  // namespace
}  // namespace nn
}  // namespace topo

// ------------------------------------------------------------------- host

using namespace topo;
using namespace topo::nn;

struct NLayer {
    int cin, cout;
    long long woff, boff;
};

struct to_net {
    to_net_cfg cfg{};
    cudaStream_t ust = nullptr, st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<NLayer> L;
    long long np = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    void* wact = nullptr;  // weights in the activation type
    long long step = 0;
    std::vector<void*> allocs;  // parameter-sized
    // workspace for one shape
    Shape shp{0, 0, 0, 0};
    std::vector<void*> ws;
    void *xa = nullptr, *a0 = nullptr, *e0 = nullptr, *p0 = nullptr, *a2 = nullptr, *e1 = nullptr, *p1 = nullptr,
         *a4 = nullptr, *e2 = nullptr, *u2 = nullptr, *a6 = nullptr, *s1 = nullptr, *d1 = nullptr, *u1 = nullptr,
         *a8 = nullptr, *s0 = nullptr, *d0 = nullptr;
    float *y = nullptr, *gy = nullptr, *A0 = nullptr, *B0 = nullptr, *C0 = nullptr, *D0 = nullptr, *A1 = nullptr,
          *B1 = nullptr, *C1 = nullptr, *D1 = nullptr, *A2 = nullptr, *B2 = nullptr, *C2 = nullptr, *part = nullptr;
    long long part_cap = 0;
    double* sums = nullptr;     // [2] loss totals
    double* partials = nullptr; // reduction scratch
    unsigned* counter = nullptr;
    double* hsums = nullptr;    // pinned
    // tensor-core forward: weights packed per tap (BF16 layers with Cin, Cout in {16, 32, 64})
    bf16* wpack = nullptr;
    long long wver = 0, pver = -1;  // weight version and the version packed
    int* tc_err = nullptr;          // device error word of the tensor-core kernels
};

namespace {

template <typename T>
T* nalloc(std::vector<void*>& list, long long count) {
    void* p = nullptr;
    TOPO_CUDA(cudaMalloc(&p, std::max<long long>(count, 1) * sizeof(T)));
    list.push_back(p);
    return (T*)p;
}

void free_ws(to_net* n) {
    for (void* p : n->ws) cudaFree(p);
    n->ws.clear();
    n->shp = Shape{0, 0, 0, 0};
}

size_t act_size(const to_net* n) { return n->cfg.bf16 ? sizeof(bf16) : sizeof(float); }

void* aalloc(to_net* n, long long count) {
    void* p = nullptr;
    TOPO_CUDA(cudaMalloc(&p, std::max<long long>(count, 1) * act_size(n)));
    n->ws.push_back(p);
    return p;
}

void ensure_ws(to_net* n, const Shape& s) {
    if (s.N == n->shp.N && s.D == n->shp.D && s.H == n->shp.H && s.W == n->shp.W) return;
    free_ws(n);
    const int c = n->cfg.base;
    const long long V0 = s.vox(), V1 = V0 / 8, V2 = V1 / 8;
    n->xa = aalloc(n, V0 * 4);
    n->a0 = aalloc(n, V0 * c);
    n->e0 = aalloc(n, V0 * c);
    n->p0 = aalloc(n, V1 * c);
    n->a2 = aalloc(n, V1 * 2 * c);
    n->e1 = aalloc(n, V1 * 2 * c);
    n->p1 = aalloc(n, V2 * 2 * c);
    n->a4 = aalloc(n, V2 * 4 * c);
    n->e2 = aalloc(n, V2 * 4 * c);
    n->u2 = aalloc(n, V1 * 4 * c);
    n->a6 = aalloc(n, V1 * 2 * c);
    n->s1 = aalloc(n, V1 * 2 * c);
    n->d1 = aalloc(n, V1 * 2 * c);
    n->u1 = aalloc(n, V0 * 2 * c);
    n->a8 = aalloc(n, V0 * c);
    n->s0 = aalloc(n, V0 * c);
    n->d0 = aalloc(n, V0 * c);
    n->y = nalloc<float>(n->ws, V0 * 3);
    n->gy = nalloc<float>(n->ws, V0 * 3);
    n->A0 = nalloc<float>(n->ws, V0 * c);
    n->B0 = nalloc<float>(n->ws, V0 * c);
    n->C0 = nalloc<float>(n->ws, V0 * c);
    n->D0 = nalloc<float>(n->ws, V0 * 2 * c);
    n->A1 = nalloc<float>(n->ws, V1 * 2 * c);
    n->B1 = nalloc<float>(n->ws, V1 * 2 * c);
    n->C1 = nalloc<float>(n->ws, V1 * 2 * c);
    n->D1 = nalloc<float>(n->ws, V1 * 4 * c);
    n->A2 = nalloc<float>(n->ws, V2 * 4 * c);
    n->B2 = nalloc<float>(n->ws, V2 * 4 * c);
    n->C2 = nalloc<float>(n->ws, V2 * 2 * c);
    long long cap = 0;
    const Shape lv[3] = {s, Shape{s.N, s.D / 2, s.H / 2, s.W / 2}, Shape{s.N, s.D / 4, s.H / 4, s.W / 4}};
    const int lev_of[11] = {0, 0, 1, 1, 2, 2, 1, 1, 0, 0, 0};
    for (int k = 0; k < 11; ++k) {
        const long long V = lv[lev_of[k]].vox();
        const long long nch = (V + 2047) / 2048;
        cap = std::max(cap, nch * 27 * n->L[k].cin * n->L[k].cout);
        cap = std::max(cap, nch * n->L[k].cout);
    }
    n->part = nalloc<float>(n->ws, cap);
    n->part_cap = cap;
    n->shp = s;
}

bool tc_layer(const to_net* n, int k) {
    const bool on = n->cfg.cuda_cores_only == 0;
    const NLayer& Lk = n->L[k];
    auto ok = [](int c) { return c == 16 || c == 32 || c == 64; };
    // 16-byte cp.async of the packed weights: the layer's offset must be a multiple of 8 BF16 values
    return on && n->cfg.bf16 && ok(Lk.cin) && ok(Lk.cout) && Lk.woff % 8 == 0;
}

template <int CIN, int COUT>
void launch_conv_tc(to_net* n, const NLayer& Lk, const void* x, void* y, const Shape& s, int relu) {
    constexpr int smem = tcc::NSTAGE * (tcc::MT * CIN * 2 + COUT * CIN * 2) + 8 * tcc::NSTAGE;
    static bool attr = false;
    if (!attr) {
        TOPO_CUDA(cudaFuncSetAttribute(kn_conv_fwd_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    const unsigned blocks = (unsigned)((s.vox() + tcc::MT - 1) / tcc::MT);
    kn_conv_fwd_tc<CIN, COUT><<<blocks, tcc::NTH, smem, n->st>>>((const bf16*)x, n->wpack + Lk.woff,
                                                                 n->theta + Lk.boff, (bf16*)y, s, relu, n->tc_err);
    TOPO_CHECK_LAUNCH();
}

void conv_fwd_tc(to_net* n, int k, const void* x, void* y, const Shape& s, int relu) {
    const NLayer& Lk = n->L[k];
#define TOPO_CT(CI, CO)                                          \
    if (Lk.cin == CI && Lk.cout == CO) {                          \
        launch_conv_tc<CI, CO>(n, Lk, x, y, s, relu);            \
        return;                                                  \
    }
    TOPO_CT(16, 16) TOPO_CT(16, 32) TOPO_CT(32, 16) TOPO_CT(32, 32) TOPO_CT(32, 64) TOPO_CT(64, 32)
    TOPO_CT(64, 64) TOPO_CT(16, 64) TOPO_CT(64, 16)
#undef TOPO_CT
    throw Error(TO_EINVAL, "tensor-core convolution: unsupported channel counts");
}

// Pack the weights of the tensor-core layers after every weight update.
void pack_weights(to_net* n) {
    if (n->pver == n->wver) return;
    for (int k = 0; k < (int)n->L.size(); ++k) {
        if (!tc_layer(n, k)) continue;
        const NLayer& Lk = n->L[k];
        const long long cnt = 27LL * Lk.cin * Lk.cout;
        kn_pack_w<<<nb(cnt), 256, 0, n->st>>>((const bf16*)n->wact + Lk.woff, n->wpack + Lk.woff, Lk.cin, Lk.cout);
        TOPO_CHECK_LAUNCH();
    }
    n->pver = n->wver;
}

template <typename TI, typename TO>
void conv_fwd(to_net* n, int k, const void* x, void* y, const Shape& s, int relu) {
    const NLayer& Lk = n->L[k];
    if constexpr (sizeof(TI) == 2 && sizeof(TO) == 2) {
        if (tc_layer(n, k)) {
            conv_fwd_tc(n, k, x, y, s, relu);
            return;
        }
    }
    const TI* W = (const TI*)n->wact + Lk.woff;
    const float* b = n->theta + Lk.boff;
    const int blocks = nb(s.vox(), CT);
    if (Lk.cout >= 8) {
        dim3 g(blocks, (Lk.cout + 7) / 8);
        kn_conv_fwd<TI, TO, 8><<<g, CT, Lk.cin * 8 * sizeof(float), n->st>>>((const TI*)x, W, b, (TO*)y, s, Lk.cin,
                                                                             Lk.cout, relu);
    } else {
        dim3 g(blocks, (Lk.cout + 3) / 4);
        kn_conv_fwd<TI, TO, 4><<<g, CT, Lk.cin * 4 * sizeof(float), n->st>>>((const TI*)x, W, b, (TO*)y, s, Lk.cin,
                                                                             Lk.cout, relu);
    }
    TOPO_CHECK_LAUNCH();
}

template <typename TI>
void conv_bwd(to_net* n, int k, const void* x, const float* gz, float* gx, const Shape& s) {
    const NLayer& Lk = n->L[k];
    const long long V = s.vox();
    const TI* W = (const TI*)n->wact + Lk.woff;
    if (gx) {
        dim3 g(nb(V, CT), (Lk.cin + 7) / 8);
        kn_conv_bwd_data<TI, 8><<<g, CT, Lk.cout * 8 * sizeof(float), n->st>>>(gz, W, gx, s, Lk.cin, Lk.cout);
        TOPO_CHECK_LAUNCH();
    }
    const long long chunk = 2048, nch = (V + chunk - 1) / chunk;
    const int nco = (Lk.cout + 15) / 16, nci = (Lk.cin + 15) / 16;
    TOPO_REQUIRE(nch * 27 * Lk.cin * Lk.cout <= n->part_cap, "network workspace");
    dim3 gw(27, (unsigned)nch, nci * nco);
    kn_conv_bwd_w<TI><<<gw, 256, 0, n->st>>>((const TI*)x, gz, n->part, s, Lk.cin, Lk.cout, chunk, nco);
    TOPO_CHECK_LAUNCH();
    const long long nw = 27LL * Lk.cin * Lk.cout;
    kn_reduce_chunks<<<nb(nw), 256, 0, n->st>>>(n->part, n->grad + Lk.woff, nw, (int)nch);
    TOPO_CHECK_LAUNCH();
    kn_bias_part<<<(unsigned)nch, 256, 0, n->st>>>(gz, n->part, V, Lk.cout, chunk);
    TOPO_CHECK_LAUNCH();
    kn_reduce_chunks<<<nb(Lk.cout), 256, 0, n->st>>>(n->part, n->grad + Lk.boff, Lk.cout, (int)nch);
    TOPO_CHECK_LAUNCH();
}

template <typename T>
void pool(to_net* n, const void* x, void* y, const Shape& so, int C) {
    kn_pool<T><<<nb(so.vox() * C), 256, 0, n->st>>>((const T*)x, (T*)y, so, C);
    TOPO_CHECK_LAUNCH();
}
template <typename T>
void up(to_net* n, const void* x, void* y, const Shape& so, int C) {
    kn_up<T><<<nb(so.vox() * C), 256, 0, n->st>>>((const T*)x, (T*)y, so, C);
    TOPO_CHECK_LAUNCH();
}
template <typename T>
void add(to_net* n, const void* a, const void* b, void* y, long long cnt) {
    kn_add<T><<<nb(cnt), 256, 0, n->st>>>((const T*)a, (const T*)b, (T*)y, cnt);
    TOPO_CHECK_LAUNCH();
}
template <typename T>
void mask(to_net* n, const float* g, const void* y, float* out, long long cnt) {
    kn_relu_mask<T><<<nb(cnt), 256, 0, n->st>>>(g, (const T*)y, out, cnt);
    TOPO_CHECK_LAUNCH();
}

template <typename T>
void forward(to_net* n, const float* x, const Shape& s) {
    const int c = n->cfg.base;
    const Shape s1{s.N, s.D / 2, s.H / 2, s.W / 2}, s2{s.N, s.D / 4, s.H / 4, s.W / 4};
    if (sizeof(T) == 2) pack_weights(n);
    kn_cast<T><<<nb(s.vox() * 4), 256, 0, n->st>>>(x, (T*)n->xa, s.vox() * 4);
    TOPO_CHECK_LAUNCH();
    conv_fwd<T, T>(n, 0, n->xa, n->a0, s, 1);
    conv_fwd<T, T>(n, 1, n->a0, n->e0, s, 1);
    pool<T>(n, n->e0, n->p0, s1, c);
    conv_fwd<T, T>(n, 2, n->p0, n->a2, s1, 1);
    conv_fwd<T, T>(n, 3, n->a2, n->e1, s1, 1);
    pool<T>(n, n->e1, n->p1, s2, 2 * c);
    conv_fwd<T, T>(n, 4, n->p1, n->a4, s2, 1);
    conv_fwd<T, T>(n, 5, n->a4, n->e2, s2, 1);
    up<T>(n, n->e2, n->u2, s1, 4 * c);
    conv_fwd<T, T>(n, 6, n->u2, n->a6, s1, 1);
    add<T>(n, n->a6, n->e1, n->s1, s1.vox() * 2 * c);
    conv_fwd<T, T>(n, 7, n->s1, n->d1, s1, 1);
    up<T>(n, n->d1, n->u1, s, 2 * c);
    conv_fwd<T, T>(n, 8, n->u1, n->a8, s, 1);
    add<T>(n, n->a8, n->e0, n->s0, s.vox() * c);
    conv_fwd<T, T>(n, 9, n->s0, n->d0, s, 1);
    conv_fwd<T, float>(n, 10, n->d0, n->y, s, 0);
}

// Backward from gy (dL/dy) into n->grad (accumulated).
template <typename T>
void backward(to_net* n, const Shape& s) {
    const int c = n->cfg.base;
    const Shape s1{s.N, s.D / 2, s.H / 2, s.W / 2}, s2{s.N, s.D / 4, s.H / 4, s.W / 4};
    const long long V0 = s.vox(), V1 = s1.vox(), V2 = s2.vox();
    conv_bwd<T>(n, 10, n->d0, n->gy, n->A0, s);                       // gd0
    mask<T>(n, n->A0, n->d0, n->A0, V0 * c);                           // gz9
    conv_bwd<T>(n, 9, n->s0, n->A0, n->B0, s);                        // gs0 = ge0 (skip) = ga8
    mask<T>(n, n->B0, n->a8, n->C0, V0 * c);                           // gz8
    conv_bwd<T>(n, 8, n->u1, n->C0, n->D0, s);                        // gu1
    kn_up_bwd<<<nb(V1 * 2 * c), 256, 0, n->st>>>(n->D0, n->A1, s1, 2 * c);  // gd1
    TOPO_CHECK_LAUNCH();
    mask<T>(n, n->A1, n->d1, n->A1, V1 * 2 * c);                       // gz7
    conv_bwd<T>(n, 7, n->s1, n->A1, n->B1, s1);                       // gs1 = ge1 (skip) = ga6
    mask<T>(n, n->B1, n->a6, n->C1, V1 * 2 * c);                       // gz6
    conv_bwd<T>(n, 6, n->u2, n->C1, n->D1, s1);                       // gu2
    kn_up_bwd<<<nb(V2 * 4 * c), 256, 0, n->st>>>(n->D1, n->A2, s2, 4 * c);  // ge2
    TOPO_CHECK_LAUNCH();
    mask<T>(n, n->A2, n->e2, n->A2, V2 * 4 * c);                       // gz5
    conv_bwd<T>(n, 5, n->a4, n->A2, n->B2, s2);                       // ga4
    mask<T>(n, n->B2, n->a4, n->B2, V2 * 4 * c);                       // gz4
    conv_bwd<T>(n, 4, n->p1, n->B2, n->C2, s2);                       // gp1
    kn_pool_bwd_add<<<nb(V1 * 2 * c), 256, 0, n->st>>>(n->C2, n->B1, s1, 2 * c);  // ge1 += pool'(gp1)
    TOPO_CHECK_LAUNCH();
    mask<T>(n, n->B1, n->e1, n->B1, V1 * 2 * c);                       // gz3
    conv_bwd<T>(n, 3, n->a2, n->B1, n->A1, s1);                       // ga2
    mask<T>(n, n->A1, n->a2, n->A1, V1 * 2 * c);                       // gz2
    conv_bwd<T>(n, 2, n->p0, n->A1, n->C1, s1);                       // gp0
    kn_pool_bwd_add<<<nb(V0 * c), 256, 0, n->st>>>(n->C1, n->B0, s, c);  // ge0 += pool'(gp0)
    TOPO_CHECK_LAUNCH();
    mask<T>(n, n->B0, n->e0, n->B0, V0 * c);                           // gz1
    conv_bwd<T>(n, 1, n->a0, n->B0, n->A0, s);                        // ga0
    mask<T>(n, n->A0, n->a0, n->A0, V0 * c);                           // gz0
    conv_bwd<T>(n, 0, n->xa, n->A0, nullptr, s);
}

void check_shape(const to_net* n, int N, int D, int H, int W) {
    (void)n;
    TOPO_REQUIRE(N >= 1 && D >= 4 && H >= 4 && W >= 4 && D % 4 == 0 && H % 4 == 0 && W % 4 == 0,
                 "network input: N >= 1 and D, H, W multiples of 4 (>= 4)");
}

void sync_in(to_net* n) {
    TOPO_CUDA(cudaEventRecord(n->ev_in, n->ust));
    TOPO_CUDA(cudaStreamWaitEvent(n->st, n->ev_in, 0));
}
void sync_out(to_net* n) {
    TOPO_CUDA(cudaEventRecord(n->ev_out, n->st));
    TOPO_CUDA(cudaStreamWaitEvent(n->ust, n->ev_out, 0));
}

void destroy_net(to_net* n) {
    if (!n) return;
    free_ws(n);
    for (void* p : n->allocs) cudaFree(p);
    if (n->hsums) cudaFreeHost(n->hsums);
    if (n->ev_in) cudaEventDestroy(n->ev_in);
    if (n->ev_out) cudaEventDestroy(n->ev_out);
    if (n->st) cudaStreamDestroy(n->st);
    delete n;
}

}  // namespace

namespace topo {
// Forward pass on the caller's stream (for the warm start inside to_step).
void net_forward_on(to_net* n, const float* x, int N, int D, int H, int W, float* y, cudaStream_t st) {
    check_shape(n, N, D, H, W);
    const Shape s{N, D, H, W};
    TOPO_CUDA(cudaEventRecord(n->ev_in, st));
    TOPO_CUDA(cudaStreamWaitEvent(n->st, n->ev_in, 0));
    ensure_ws(n, s);
    if (n->cfg.bf16)
        forward<bf16>(n, x, s);
    else
        forward<float>(n, x, s);
    TOPO_CUDA(cudaMemcpyAsync(y, n->y, s.vox() * 3 * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
    TOPO_CUDA(cudaEventRecord(n->ev_out, n->st));
    TOPO_CUDA(cudaStreamWaitEvent(st, n->ev_out, 0));
}
}  // namespace topo

#define TOPO_NET_BEGIN try {
#define TOPO_NET_END                                                                       \
    }                                                                                      \
    catch (const topo::Error& e) { return topo::api_fail(e.code, e.what()); }              \
    catch (const std::bad_alloc&) { return topo::api_fail(TO_ENOMEM, "host allocation failed"); } \
    catch (const std::exception& e) { return topo::api_fail(TO_ECUDA, e.what()); }         \
    return TO_OK;

extern "C" {

to_status to_net_create(const to_net_cfg* cfg, void* stream, to_net** out) {
    if (!cfg || !out) return api_fail(TO_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->base < 1 || cfg->base > 64 || cfg->in_ch != 4 || cfg->out_ch != 3)
        return api_fail(TO_EINVAL, "network: base in [1, 64], in_ch 4, out_ch 3");
    to_net* n = new to_net();
    TOPO_NET_BEGIN
    try {
        n->cfg = *cfg;
        n->ust = (cudaStream_t)stream;
        TOPO_CUDA(cudaStreamCreateWithFlags(&n->st, cudaStreamNonBlocking));
        TOPO_CUDA(cudaEventCreateWithFlags(&n->ev_in, cudaEventDisableTiming));
        TOPO_CUDA(cudaEventCreateWithFlags(&n->ev_out, cudaEventDisableTiming));
        const int c = cfg->base;
        const int shapes[11][2] = {{4, c}, {c, c}, {c, 2 * c}, {2 * c, 2 * c}, {2 * c, 4 * c}, {4 * c, 4 * c},
                                   {4 * c, 2 * c}, {2 * c, 2 * c}, {2 * c, c}, {c, c}, {c, 3}};
        long long off = 0;
        for (auto& sh : shapes) {
            NLayer Lk{sh[0], sh[1], off, off + 27LL * sh[0] * sh[1]};
            off = Lk.boff + sh[1];
            n->L.push_back(Lk);
        }
        // the convolutions load 4 channels at a time: every W block must stay aligned
        TOPO_REQUIRE(c % 4 == 0, "network base channels must be a multiple of 4");
        n->np = off;
        n->theta = nalloc<float>(n->allocs, off);
        n->grad = nalloc<float>(n->allocs, off);
        n->m = nalloc<float>(n->allocs, off);
        n->v = nalloc<float>(n->allocs, off);
        void* w = nullptr;
        TOPO_CUDA(cudaMalloc(&w, off * (cfg->bf16 ? sizeof(bf16) : sizeof(float))));
        n->allocs.push_back(w);
        n->wact = w;
        if (cfg->bf16) n->wpack = nalloc<bf16>(n->allocs, off);
        n->tc_err = nalloc<int>(n->allocs, 1);
        TOPO_CUDA(cudaMemsetAsync(n->tc_err, 0, sizeof(int), n->st));
        n->sums = nalloc<double>(n->allocs, 2);
        n->partials = nalloc<double>(n->allocs, 2 * 4096);
        n->counter = nalloc<unsigned>(n->allocs, 1);
        TOPO_CUDA(cudaMallocHost(&n->hsums, 2 * sizeof(double)));
        for (float* p : {n->theta, n->grad, n->m, n->v}) TOPO_CUDA(cudaMemsetAsync(p, 0, off * sizeof(float), n->st));
        TOPO_CUDA(cudaMemsetAsync(n->wact, 0, off * (cfg->bf16 ? sizeof(bf16) : sizeof(float)), n->st));
        TOPO_CUDA(cudaMemsetAsync(n->counter, 0, sizeof(unsigned), n->st));
        TOPO_CUDA(cudaStreamSynchronize(n->st));
        *out = n;
    } catch (...) {
        destroy_net(n);
        throw;
    }
    TOPO_NET_END
}

int64_t to_net_param_count(const to_net* n) { return n ? n->np : 0; }

to_status to_net_set_params(to_net* n, const float* theta) {
    if (!n || !theta) return api_fail(TO_EINVAL, "NULL argument");
    TOPO_NET_BEGIN
    sync_in(n);
    TOPO_CUDA(cudaMemcpyAsync(n->theta, theta, n->np * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
    if (n->cfg.bf16)
        kn_cast<bf16><<<nb(n->np), 256, 0, n->st>>>(n->theta, (bf16*)n->wact, n->np);
    else
        kn_cast<float><<<nb(n->np), 256, 0, n->st>>>(n->theta, (float*)n->wact, n->np);
    TOPO_CHECK_LAUNCH();
    for (float* p : {n->grad, n->m, n->v}) TOPO_CUDA(cudaMemsetAsync(p, 0, n->np * sizeof(float), n->st));
    n->step = 0;
    n->wver += 1;
    sync_out(n);
    TOPO_NET_END
}

to_status to_net_get_params(const to_net* n, float* theta) {
    if (!n || !theta) return api_fail(TO_EINVAL, "NULL argument");
    TOPO_NET_BEGIN
    TOPO_CUDA(cudaMemcpyAsync(theta, n->theta, n->np * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
    TOPO_CUDA(cudaStreamSynchronize(n->st));
    TOPO_NET_END
}

to_status to_net_forward(to_net* n, const float* x, int32_t N, int32_t D, int32_t H, int32_t W, float* y) {
    if (!n || !x || !y) return api_fail(TO_EINVAL, "NULL argument");
    TOPO_NET_BEGIN
    check_shape(n, N, D, H, W);
    const Shape s{N, D, H, W};
    sync_in(n);
    ensure_ws(n, s);
    if (n->cfg.bf16)
        forward<bf16>(n, x, s);
    else
        forward<float>(n, x, s);
    TOPO_CUDA(cudaMemcpyAsync(y, n->y, s.vox() * 3 * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
    sync_out(n);
    TOPO_NET_END
}

to_status to_net_accumulate(to_net* n, const float* x, const float* target, const uint8_t* mask_v, int32_t N,
                            int32_t D, int32_t H, int32_t W, double* loss) {
    if (!n || !x || !target || !mask_v) return api_fail(TO_EINVAL, "NULL argument");
    TOPO_NET_BEGIN
    check_shape(n, N, D, H, W);
    const Shape s{N, D, H, W};
    sync_in(n);
    ensure_ws(n, s);
    if (n->cfg.bf16)
        forward<bf16>(n, x, s);
    else
        forward<float>(n, x, s);
    const long long V = s.vox();
    kn_mse_sum<<<std::min(nb(V * 3), 4096), 256, 0, n->st>>>(n->y, target, mask_v, V, 3, n->partials, n->counter,
                                                             n->sums);
    TOPO_CHECK_LAUNCH();
    kn_mse_grad<<<nb(V * 3), 256, 0, n->st>>>(n->y, target, mask_v, n->gy, V, 3, n->sums);
    TOPO_CHECK_LAUNCH();
    if (n->cfg.bf16)
        backward<bf16>(n, s);
    else
        backward<float>(n, s);
    if (loss) {
        TOPO_CUDA(cudaMemcpyAsync(n->hsums, n->sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, n->st));
        TOPO_CUDA(cudaStreamSynchronize(n->st));
        *loss = n->hsums[1] > 0.0 ? n->hsums[0] / n->hsums[1] : 0.0;
    }
    sync_out(n);
    TOPO_NET_END
}

to_status to_net_backward(to_net* n, const float* gy, int32_t N, int32_t D, int32_t H, int32_t W) {
    if (!n || !gy) return api_fail(TO_EINVAL, "NULL argument");
    TOPO_NET_BEGIN
    check_shape(n, N, D, H, W);
    TOPO_REQUIRE(n->shp.N == N && n->shp.D == D && n->shp.H == H && n->shp.W == W,
                 "to_net_backward: the last forward pass had another shape");
    const Shape s{N, D, H, W};
    sync_in(n);
    TOPO_CUDA(cudaMemcpyAsync(n->gy, gy, s.vox() * 3 * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
    if (n->cfg.bf16)
        backward<bf16>(n, s);
    else
        backward<float>(n, s);
    sync_out(n);
    TOPO_NET_END
}

to_status to_net_get_grad(const to_net* n, float* g) {
    if (!n || !g) return api_fail(TO_EINVAL, "NULL argument");
    TOPO_NET_BEGIN
    TOPO_CUDA(cudaMemcpyAsync(g, n->grad, n->np * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
    TOPO_CUDA(cudaStreamSynchronize(n->st));
    TOPO_NET_END
}

to_status to_net_zero_grad(to_net* n) {
    if (!n) return api_fail(TO_EINVAL, "NULL argument");
    TOPO_NET_BEGIN
    TOPO_CUDA(cudaMemsetAsync(n->grad, 0, n->np * sizeof(float), n->st));
    TOPO_NET_END
}

to_status to_net_adam(to_net* n, double lr, double beta1, double beta2, double eps, double grad_scale) {
    if (!n || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return api_fail(TO_EINVAL, "bad Adam arguments");
    TOPO_NET_BEGIN
    n->step += 1;
    n->wver += 1;
    const double lr_t = lr * std::sqrt(1.0 - std::pow(beta2, (double)n->step)) / (1.0 - std::pow(beta1, (double)n->step));
    if (n->cfg.bf16)
        kn_adam<bf16><<<nb(n->np), 256, 0, n->st>>>(n->theta, (bf16*)n->wact, n->grad, n->m, n->v, n->np, (float)lr_t,
                                                    (float)beta1, (float)beta2, (float)eps, (float)grad_scale);
    else
        kn_adam<float><<<nb(n->np), 256, 0, n->st>>>(n->theta, (float*)n->wact, n->grad, n->m, n->v, n->np,
                                                     (float)lr_t, (float)beta1, (float)beta2, (float)eps,
                                                     (float)grad_scale);
    TOPO_CHECK_LAUNCH();
    TOPO_NET_END
}

void to_net_destroy(to_net* n) { destroy_net(n); }

size_t to_sizeof_net_cfg(void) { return sizeof(to_net_cfg); }

}  // extern "C"
