// Instrumentation (no counterpart in the paper): the cost of one tcgen05.mma of
// kind::tf32 (K = 8, FP32 accumulation in tensor memory) for a given M and N,
// number of issuing threads per block and blocks per SM. Each issuing thread
// (lane 0 of warps 0 .. issuers - 1) issues `reps` MMAs into its own
// accumulator from zero-filled shared-memory operands, commits them to its own
// mbarrier and waits (bounded); the block records the clock64 cycles of its
// first issuer. This is the measurement behind the choice of the FP32 fine
// operator: small-N MMAs cost the same per instruction as large-N ones.
#include <algorithm>
#include <vector>

#include "grid.h"

namespace topo {

namespace {

constexpr int PROBE_SMEM = 24 * 1024;  // A: 16 x 256 B (M = 128); B: N / 8 x 256 B at 8 KB (N <= 256)
constexpr long long PROBE_WAIT = 1LL << 26;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc_nosw(uint32_t a, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((a & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__global__ void __launch_bounds__(256) k_probe_mma(int M, int N, int issuers, int ncols, int reps, long long* cyc,
                                                   int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint32_t tbase;
    __shared__ uint64_t bars[8];
    const int tid = threadIdx.x, w = tid >> 5;
    for (int i = tid; i < PROBE_SMEM / 4; i += blockDim.x) reinterpret_cast<float*>(sm)[i] = 0.f;
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tbase)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0)
        for (int i = 0; i < 8; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&bars[i])));
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t t = tbase;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
    if ((tid & 31) == 0 && w < issuers) {
        const uint64_t ad = desc_nosw(su32(sm), 128, 256), bd = desc_nosw(su32(sm + 8192), 128, 256);
        const uint32_t d = t + (uint32_t)(w * N);
        const long long t0 = clock64();
        for (int r = 0; r < reps; ++r)
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
                "l"(ad), "l"(bd), "r"(idesc), "r"(r > 0 ? 1u : 0u));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(&bars[w]))
                     : "memory");
        uint32_t done = 0;
        for (long long it = 0; it < PROBE_WAIT && !done; ++it)
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
                : "=r"(done)
                : "r"(su32(&bars[w])));
        if (!done) atomicExch(err, 1);
        if (w == 0) cyc[blockIdx.x] = clock64() - t0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (w == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(t), "r"(ncols));
    }
}

}  // namespace

}  // namespace topo

using namespace topo;

extern "C" to_status to_time_tf32_mma(int32_t m, int32_t n, int32_t issuers, int32_t blocks_per_sm, int32_t reps,
                                      double* cycles, double* mac_per_cycle) {
    if (!cycles || !mac_per_cycle || (m != 64 && m != 128) || n < 8 || n > 256 || n % (m == 128 ? 16 : 8) != 0 ||
        issuers < 1 || issuers > 8 || (blocks_per_sm != 1 && blocks_per_sm != 2 && blocks_per_sm != 4) || reps < 1)
        return api_fail(TO_EINVAL, "to_time_tf32_mma: m 64 or 128, n 8..256 (multiple of 16 for m = 128), "
                                   "issuers 1..8, blocks_per_sm 1, 2 or 4");
    const int ncols = 512 / blocks_per_sm;  // the block's tensor-memory columns
    if ((long long)issuers * n > ncols) return api_fail(TO_EINVAL, "to_time_tf32_mma: issuers x n exceeds the block's columns");
    long long* cyc = nullptr;
    int* err = nullptr;
    try {
        int dev = 0, nsm = 0;
        TOPO_CUDA(cudaGetDevice(&dev));
        TOPO_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int nb = nsm * blocks_per_sm;
        TOPO_CUDA(cudaMalloc(&cyc, nb * sizeof(long long)));
        TOPO_CUDA(cudaMalloc(&err, sizeof(int)));
        TOPO_CUDA(cudaMemset(err, 0, sizeof(int)));
        TOPO_CUDA(cudaFuncSetAttribute(k_probe_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM));
        k_probe_mma<<<nb, 256, PROBE_SMEM>>>(m, n, issuers, ncols, reps, cyc, err);
        TOPO_CHECK_LAUNCH();
        TOPO_CUDA(cudaStreamSynchronize(0));
        std::vector<long long> h(nb);
        int herr = 0;
        TOPO_CUDA(cudaMemcpy(h.data(), cyc, nb * sizeof(long long), cudaMemcpyDeviceToHost));
        TOPO_CUDA(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr) throw Error(TO_ETIMEOUT, "to_time_tf32_mma: an mbarrier wait passed its limit");
        double s = 0.0;
        for (long long v : h) s += (double)v;
        *cycles = s / nb / reps;  // per MMA, as seen by one issuing thread
        // the blocks of one SM run together: its multiply-adds over the mean block cycles
        *mac_per_cycle = (double)m * n * 8.0 * reps * issuers * blocks_per_sm / (s / nb);
    } catch (const Error& e) {
        if (cyc) cudaFree(cyc);
        if (err) cudaFree(err);
        return api_fail(e.code, e.what());
    }
    cudaFree(cyc);
    cudaFree(err);
    return TO_OK;
}
