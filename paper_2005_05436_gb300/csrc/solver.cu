// State solve K(xPhys)(free, free) U = F (Eq. 4) by preconditioned CG on the
// matrix-free operator. The PCG iteration body is captured once per handle as
// a CUDA graph of CHUNK iterations; the kernels become no-ops once the device
// flag `done` is set, so the host only polls the scalars between chunks.
#include <cmath>

#include "grid.h"

namespace topo {

struct Solver {
    // FP64 Jacobi-PCG vectors (nDof)
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr, *b = nullptr,
           *dinv = nullptr;
    cudaGraphExec_t chunk = nullptr;
    int chunk_iters = 0;
};

static constexpr int CHUNK = 16;

void solver_init(to_grid* g) {
    Solver* s = new Solver();
    g->solver = s;
    // v[0..5] are the handle's nDof vectors; v[6] stays free for to_apply_K masking
    s->x = g->v[0];
    s->r = g->v[1];
    s->z = g->v[2];
    s->p = g->v[3];
    s->Ap = g->v[4];
    s->b = g->v[5];
    TOPO_CUDA(cudaMalloc(&s->dinv, g->d.ndof * sizeof(double)));
}

void solver_free(to_grid* g) {
    Solver* s = g->solver;
    if (!s) return;
    if (s->chunk) cudaGraphExecDestroy(s->chunk);
    if (s->dinv) cudaFree(s->dinv);
    delete s;
    g->solver = nullptr;
}

static void enqueue_iteration(to_grid* g, Solver* s) {
    const Dims& d = g->d;
    PcgScalars* sc = &g->ds->pcg;
    launch_apply_K<double>(d, g->ke3, g->ke2, g->E, s->p, s->Ap, g->fixed, true, sc, g->partials,
                           g->counter, g->st);
    launch_pcg_update(d.ndof, s->x, s->r, s->z, s->p, s->Ap, s->dinv, sc, g->partials, g->counter, g->st);
    launch_pcg_dir(d.ndof, s->z, s->p, sc, g->st);
}

static void build_chunk_graph(to_grid* g, Solver* s) {
    cudaGraph_t graph;
    TOPO_CUDA(cudaStreamBeginCapture(g->st, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    try {
        for (int i = 0; i < CHUNK; ++i) enqueue_iteration(g, s);
    } catch (...) {
        set_capturing(false);
        cudaStreamEndCapture(g->st, &graph);
        throw;
    }
    set_capturing(false);
    TOPO_CUDA(cudaStreamEndCapture(g->st, &graph));
    TOPO_CUDA(cudaGraphInstantiate(&s->chunk, graph, 0));
    TOPO_CUDA(cudaGraphDestroy(graph));
    s->chunk_iters = CHUNK;
}

to_status solve_state(to_grid* g, const double* b, double* U, to_solve_info* info) {
    Solver* s = g->solver;
    const Dims& d = g->d;
    cudaStream_t st = g->st;
    if (!s->chunk) build_chunk_graph(g, s);
    // b = F (masked inside pcg_init), x = U warm start
    TOPO_CUDA(cudaMemcpyAsync(s->b, b, d.ndof * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_mask_copy(d.ndof, U, s->x, g->fixed, st);
    launch_diag_inv<double>(d, g->ke3, g->ke2, g->E, g->fixed, s->dinv, st);
    PcgScalars init{};
    init.rtol2 = g->p.cg_rtol * g->p.cg_rtol;
    init.maxit = g->p.cg_maxit;
    TOPO_CUDA(cudaMemcpyAsync(&g->ds->pcg, &init, sizeof(PcgScalars), cudaMemcpyHostToDevice, st));
    launch_apply_K<double>(d, g->ke3, g->ke2, g->E, s->x, s->Ap, g->fixed, true, nullptr, nullptr,
                           nullptr, st);
    launch_pcg_init(d.ndof, s->b, s->Ap, s->x, s->r, s->z, s->p, s->dinv, g->fixed, &g->ds->pcg,
                    g->partials, g->counter, st);
    PcgScalars h{};
    for (;;) {
        TOPO_CUDA(cudaMemcpyAsync(&g->hs->pcg, &g->ds->pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
        TOPO_CUDA(cudaStreamSynchronize(st));
        h = g->hs->pcg;
        if (h.done) break;
        TOPO_CUDA(cudaGraphLaunch(s->chunk, st));
        count_launches(3LL * s->chunk_iters);
    }
    TOPO_CUDA(cudaMemcpyAsync(U, s->x, d.ndof * sizeof(double), cudaMemcpyDeviceToDevice, st));
    to_status status = TO_OK;
    if (h.done == 2) status = TO_ENOTCONV;
    if (h.done == 3) status = TO_ENAN;
    if (info) {
        info->iters = h.iters;
        info->refinements = 0;
        info->rel_res = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
        info->status = (int)status;
    }
    return status;
}

void time_apply_K_mixed(to_grid*, const double*, int, cudaEvent_t, cudaEvent_t) {
    throw Error(TO_EINVAL, "mixed-precision operator not available");
}

}  // namespace topo
