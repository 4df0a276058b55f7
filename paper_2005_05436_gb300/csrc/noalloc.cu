// OC update that allocates no device memory (see to_oc_update_noalloc in
// include/topopt.h). Its scratch is one file-scope device array; the update
// itself is the same cooperative kernel that to_oc_update launches.
#include <mutex>
#include <new>
#include <string>

#include "grid.h"
#include "kernels.h"

namespace topo {

constexpr long long NOALLOC_MAX_NEL = 1LL << 20;  // elements
constexpr int NOALLOC_MAX_BLOCKS = 1024;          // cooperative blocks
constexpr int NOALLOC_NV = 16;                    // reduction values per block (OC uses <= 15)

// Layout: ocP[MAX_NEL] | partials[2 * NV * MAX_BLOCKS] | GridBarrier | OcOut | active count
constexpr size_t NOALLOC_OCP = 0;
constexpr size_t NOALLOC_PART = NOALLOC_OCP + sizeof(double) * NOALLOC_MAX_NEL;
constexpr size_t NOALLOC_BAR = NOALLOC_PART + sizeof(double) * 2 * NOALLOC_NV * NOALLOC_MAX_BLOCKS;
constexpr size_t NOALLOC_OUT = NOALLOC_BAR + 256;
constexpr size_t NOALLOC_CNT = NOALLOC_OUT + 256;
constexpr size_t NOALLOC_BYTES = NOALLOC_CNT + 256;

// Held by every GPU that loads the library, for the life of the process.
static __device__ __align__(256) unsigned char g_oc_scratch[NOALLOC_BYTES];

__global__ void k_count_active(long long n, const int8_t* __restrict__ passive,
                               unsigned long long* count) {
    unsigned long long c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        c += passive[i] == 0;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Device address of g_oc_scratch, resolved once per device with that device
// current (in host code the symbol's name is only a host-side stand-in). The
// first resolution on a device loads the module that holds the array (CUDA
// loads modules lazily), which is when the array's memory is reserved.
static unsigned char* scratch_address(int dev) {
    static std::mutex mu;
    static unsigned char* addr[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    TOPO_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
    if (!addr[dev]) {
        void* p = nullptr;
        TOPO_CUDA(cudaGetSymbolAddress(&p, g_oc_scratch));
        addr[dev] = (unsigned char*)p;
    }
    return addr[dev];
}

}  // namespace topo

using namespace topo;

extern "C" to_status to_oc_update_noalloc(int64_t nel, double* x, const double* dc, const double* dV0,
                                          const int8_t* passive, double volfrac, double move,
                                          double oc_tol, int32_t oc_maxit, int64_t deadline_cycles,
                                          void* stream, double* lm_out) {
    if (!x || !dc || !dV0) return api_fail(TO_EINVAL, "to_oc_update_noalloc: NULL x, dc or dV0");
    if (nel < 1 || nel > NOALLOC_MAX_NEL)
        return api_fail(TO_EINVAL, "to_oc_update_noalloc: nel must lie in [1, 1048576] (the size of its "
                                   "static scratch array)");
    if (!(volfrac > 0.0 && volfrac < 1.0) || !(move > 0.0 && move <= 1.0) || !(oc_tol > 0.0) ||
        oc_maxit < 1 || deadline_cycles <= 0)
        return api_fail(TO_EINVAL, "to_oc_update_noalloc: need 0 < volfrac < 1, 0 < move <= 1, oc_tol > 0, "
                                   "oc_maxit >= 1, deadline_cycles > 0");
    try {
        cudaStream_t st = (cudaStream_t)stream;
        int dev = 0;
        TOPO_CUDA(cudaGetDevice(&dev));
        unsigned char* base = scratch_address(dev);
        double* ocp = (double*)(base + NOALLOC_OCP);
        double* partials = (double*)(base + NOALLOC_PART);
        GridBarrier* bar = (GridBarrier*)(base + NOALLOC_BAR);
        OcOut* out = (OcOut*)(base + NOALLOC_OUT);
        unsigned long long* cnt = (unsigned long long*)(base + NOALLOC_CNT);

        long long nact = nel;
        if (passive) {
            unsigned long long h = 0;
            TOPO_CUDA(cudaMemsetAsync(cnt, 0, sizeof(*cnt), st));
            k_count_active<<<div_up(nel, 256 * 8) < 1024 ? div_up(nel, 256 * 8) : 1024, 256, 0, st>>>(
                nel, passive, cnt);
            TOPO_CHECK_LAUNCH();
            TOPO_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
            TOPO_CUDA(cudaStreamSynchronize(st));
            nact = (long long)h;
            if (nact < 1) return api_fail(TO_EINVAL, "to_oc_update_noalloc: no active element");
        }
        int nblocks = oc_max_blocks();
        if (nblocks > NOALLOC_MAX_BLOCKS) nblocks = NOALLOC_MAX_BLOCKS;
        TOPO_CUDA(cudaMemsetAsync(out, 0, sizeof(OcOut), st));
        // launch_oc clears the grid barrier before its cooperative launch
        launch_oc(nel, x, dc, dV0, passive, nact, move, volfrac, oc_tol, oc_maxit, deadline_cycles, ocp,
                  partials, bar, out, nblocks, st);
        OcOut h_out{};
        GridBarrier h_bar{};
        TOPO_CUDA(cudaMemcpyAsync(&h_out, out, sizeof(h_out), cudaMemcpyDeviceToHost, st));
        TOPO_CUDA(cudaMemcpyAsync(&h_bar, bar, sizeof(h_bar), cudaMemcpyDeviceToHost, st));
        TOPO_CUDA(cudaStreamSynchronize(st));
        if (h_bar.error) return api_fail(TO_ETIMEOUT, "to_oc_update_noalloc: grid barrier deadline passed");
        if (lm_out) *lm_out = h_out.lm;
        if (h_out.status != TO_OK)
            return api_fail(TO_ENOTCONV, "to_oc_update_noalloc: the multiplier search stopped at oc_maxit "
                                         "before the bracket met oc_tol (x holds the last candidate)");
    } catch (const topo::Error& e) {
        return api_fail(e.code, e.what());
    } catch (const std::bad_alloc&) {
        return api_fail(TO_ENOMEM, "to_oc_update_noalloc: host allocation failed");
    } catch (const std::exception& e) {
        return api_fail(TO_ECUDA, e.what());
    }
    return TO_OK;
}
