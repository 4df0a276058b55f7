// Instrumentation entry points (no counterpart in the paper): kernel-launch
// accounting, the programmatic-dependent-launch switch of the calling thread
// and CUDA-event timing of the matrix-free operator kernel.
#include <atomic>
#include <string>

#include "grid.h"

namespace topo {

static std::atomic<long long> g_launches{0};
static thread_local bool g_capturing = false;
static thread_local long long g_captured = 0;

void count_launches(long long n) {
    if (g_capturing)
        g_captured += n;
    else
        g_launches.fetch_add(n, std::memory_order_relaxed);
}
long long captured_launches_reset() {
    const long long c = g_captured;
    g_captured = 0;
    return c;
}
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }
void set_capturing(bool on) { g_capturing = on; }

static thread_local bool g_pdl = false;
bool pdl_on() { return g_pdl; }
void set_pdl(bool on) { g_pdl = on; }

}  // namespace topo

using namespace topo;

extern "C" {

int64_t to_kernel_launches(void) { return (int64_t)launches_total(); }

to_status to_apply_K_fp32(to_grid* g, const double* xPhys, const double* u, double* y, int32_t impl) {
    if (!g || !xPhys || !u || !y || u == y) return TO_EINVAL;
    try {
        grid_sync_in(g);
        apply_K_fp32(g, xPhys, u, y, impl);
        grid_sync_out(g);
    } catch (const topo::Error& e) {
        return e.code;
    }
    return TO_OK;
}

to_status to_time_apply_K(to_grid* g, const double* xPhys, int32_t precision, int32_t reps, double* us) {
    if (!g || !xPhys || !us || reps < 1) return TO_EINVAL;
    try {
        const Dims& d = g->d;
        cudaStream_t st = g->st;
        grid_sync_in(g);
        double* u = g->v[6];
        double* y = g->v[5];
        launch_fill(d.ndof, u, 1.0, st);
        cudaEvent_t e0, e1;
        TOPO_CUDA(cudaEventCreate(&e0));
        TOPO_CUDA(cudaEventCreate(&e1));
        float ms = 0.f;
        if (precision == TO_FP64) {
            launch_modulus<double>(d.nel, xPhys, g->penal, g->p.E0, g->p.Emin, g->E, st);
            launch_apply_K<double>(d, g->ke3, g->ke2, g->wk, g->node_centric, g->E, u, y, g->fixed,
                               true, st);
            TOPO_CUDA(cudaEventRecord(e0, st));
            for (int r = 0; r < reps; ++r)
                launch_apply_K<double>(d, g->ke3, g->ke2, g->wk, g->node_centric, g->E, u, y, g->fixed,
                               true, st);
            TOPO_CUDA(cudaEventRecord(e1, st));
        } else {
            time_apply_K_mixed(g, xPhys, reps, e0, e1);
        }
        TOPO_CUDA(cudaEventSynchronize(e1));
        TOPO_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        grid_sync_out(g);
        *us = 1000.0 * ms / reps;
    } catch (const topo::Error& e) {
        return e.code;
    }
    return TO_OK;
}

}  // extern "C"
