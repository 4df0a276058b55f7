// State solve K(xPhys)(free, free) U = F (Eq. 4) by preconditioned CG on the
// matrix-free operator, with a Jacobi or geometric-multigrid preconditioner.
//
// Each PCG solve is a handful of set-up kernels followed by ONE launch of a
// CUDA graph holding a conditional WHILE node: its body is one PCG iteration
// and its last kernel clears the condition once the device-side residual test
// (or the iteration cap) sets `done`. The host does not poll.
//
// TO_FP64: the PCG and the preconditioner run in FP64.
// TO_MIXED: the FP32 PCG (FP32 operator and V-cycle, float-float dot
// products) works on corrections of the FP64 iterate U, and the true FP64
// residual r = F - K U decides convergence, ||r|| <= cg_rtol ||F||. Two ways
// of joining them (to_params.refine): reliable updates, in which one PCG runs
// in segments; after each segment (residual fallen by inner_rtol) U += its
// FP32 correction in FP64 and the FP64 residual replaces the recursive one
// while the search direction carries on, so the Krylov space is not restarted;
// or flexible CG, in which each FP32 solve to inner_rtol starts from scratch
// and is followed by one FP64 CG step along its result, K-orthogonal to the
// previous step, with the exact line search.
#include <algorithm>
#include <cmath>

#include "grid.h"
#include "mg.h"

namespace topo {

// ------------------------------------------------------------------ kernels

constexpr int KNT = 256;
// iteration cap of one reliable-update segment (a segment of the 96x48x48
// cantilever takes about 40 iterations, of the 1200x400 MBB beam about 60)
constexpr int RELIABLE_SEG_MAX = 400;

static int kblocks(long long n) {
    int nb = div_up(n, KNT * 4);
    return nb < 1 ? 1 : (nb > 1024 ? 1024 : nb);
}

template <typename Tin, typename Tout>
__global__ void k_cast_mask(long long n, const Tin* __restrict__ in, Tout* __restrict__ out,
                            const uint8_t* __restrict__ fixed) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (fixed && fixed[i]) ? Tout(0) : (Tout)in[i];
}

// rr = r.r, bb = b.b over free DOFs; start the PCG scalars.
template <typename T>
__global__ void __launch_bounds__(KNT) k_gpcg_init(long long n, const T* __restrict__ b, const T* __restrict__ r,
                                                   const uint8_t* __restrict__ fixed, PcgScalars* s,
                                                   double* partials, unsigned* counter) {
    double v[2] = {0.0, 0.0}, tot[2];
    for (long long i = (long long)blockIdx.x * KNT + threadIdx.x; i < n; i += (long long)gridDim.x * KNT) {
        const double ri = r[i], bi = fixed[i] ? 0.0 : (double)b[i];
        v[0] += ri * ri;
        v[1] += bi * bi;
    }
    if (last_block_totals<KNT, 2>(v, partials, counter, tot) && threadIdx.x == 0) {
        s->rr = tot[0];
        s->bb = tot[1];
        s->iters = 0;
        s->done = (tot[0] <= s->rtol2 * tot[1]) ? 1 : 0;
        if (!isfinite(tot[0])) s->done = 3;
    }
}

// rz = r.z (Jacobi: z = dinv r computed here); FIRST: p = z, else beta = rz / rz_old.
template <typename T, bool FIRST, bool JAC>
__global__ void __launch_bounds__(KNT) k_gpcg_rz(long long n, const T* __restrict__ r, T* __restrict__ z,
                                                 const T* __restrict__ dinv, T* __restrict__ p, PcgScalars* s,
                                                 double* partials, unsigned* counter) {
    pdl_begin();
    const int dn = s->done;  // tested before the stores, so its load overlaps the others
    DotAcc<T> acc;
    double tot[1];
    for (long long i = (long long)blockIdx.x * KNT + threadIdx.x; i < n; i += (long long)gridDim.x * KNT) {
        const T ri = r[i];
        const T zi = JAC ? dinv[i] * ri : z[i];
        if (dn) return;
        if (JAC) z[i] = zi;
        if (FIRST) p[i] = zi;
        acc.add(ri, zi);
    }
    if (dn) return;
    double v[1] = {acc.value()};
    if (last_block_totals<KNT, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
        if (FIRST) {
            s->rz = tot[0];
        } else {
            s->beta = tot[0] / s->rz;
            s->rz = tot[0];
        }
    }
}

// x += alpha p; r -= alpha Ap; rr; iteration count and the stopping tests.
// With dinv0 (multigrid): also the V-cycle's first fine-level iterate
// z0 = omega dinv0 r (the k_jacobi_first of level 0, fused).
// The iterate x is FP64 in either precision. Rounding x to FP32 at every
// update would add an error of about eps_32 |x| per DOF that the recursion
// for r never sees; its image under K, about eps_32 || |K| |x| ||, is then
// a floor for the true residual far above the FP32 residual recursion's own
// (it grows with the size of the displacements, i.e. with the grid and the
// softness of the design). Kept in FP64, x carries exactly the steps
// alpha p whose K-images the recursion subtracted.
template <typename T>
__global__ void __launch_bounds__(KNT) k_gpcg_xr(long long n, double* __restrict__ x, T* __restrict__ r,
                                                 const T* __restrict__ p, const T* __restrict__ Ap, PcgScalars* s,
                                                 double* partials, unsigned* counter, const T* __restrict__ dinv0,
                                                 T* __restrict__ z0, T omega) {
    pdl_begin();
    const int dn = s->done;  // tested before the stores, so its load overlaps the others
    const T alpha = (T)s->alpha;
    DotAcc<T> acc;
    double tot[1];
    const long long stride = (long long)gridDim.x * KNT;
    long long i = (long long)blockIdx.x * KNT + threadIdx.x;
    // four strided elements per trip with every load issued before the first
    // use, so that a thread waits for memory once rather than four times
    for (; i + 3 * stride < n; i += 4 * stride) {
        double xv[4];
        T pv[4], rv[4], av[4], dv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long j = i + k * stride;
            xv[k] = x[j];
            pv[k] = p[j];
            rv[k] = r[j];
            av[k] = Ap[j];
            dv[k] = dinv0 ? dinv0[j] : T(0);
        }
        if (dn) return;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long j = i + k * stride;
            x[j] = xv[k] + (double)alpha * (double)pv[k];
            const T ri = rv[k] - alpha * av[k];
            r[j] = ri;
            if (dinv0) z0[j] = omega * dv[k] * ri;
            acc.add(ri, ri);
        }
    }
    if (dn) return;
    for (; i < n; i += stride) {
        x[i] += (double)alpha * (double)p[i];
        const T ri = r[i] - alpha * Ap[i];
        r[i] = ri;
        if (dinv0) z0[i] = omega * dinv0[i] * ri;
        acc.add(ri, ri);
    }
    double v[1] = {acc.value()};
    if (last_block_totals<KNT, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
        s->iters += 1;
        s->rr = tot[0];
        if (!isfinite(tot[0]) || !isfinite(s->alpha))
            s->done = 3;
        else if (tot[0] <= s->rtol2 * s->bb)
            s->done = 1;
        else if (s->iters >= s->maxit)
            s->done = 2;
    }
}

// p = z + beta p, then set the WHILE condition of the enclosing graph.
template <typename T>
__global__ void k_gpcg_p(long long n, const T* __restrict__ z, T* __restrict__ p, const PcgScalars* s,
                         cudaGraphConditionalHandle cond, int set_cond) {
    pdl_begin();
    const int done = s->done;  // tested before the stores, so its load overlaps the others
    const T beta = (T)s->beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T zi = z[i], pi = p[i];
        if (!done) p[i] = zi + beta * pi;
    }
    if (set_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, done ? 0u : 1u);
}

// Mixed refinement: r64 = b - y (0 at fixed DOFs), r32 = (float) r64, rr, bb.
__global__ void __launch_bounds__(KNT) k_refine_resid(long long n, const double* __restrict__ b,
                                                      const double* __restrict__ y, double* __restrict__ r64,
                                                      float* __restrict__ r32, const uint8_t* __restrict__ fixed,
                                                      double* res, double* partials, unsigned* counter) {
    double v[2] = {0.0, 0.0}, tot[2];
    for (long long i = (long long)blockIdx.x * KNT + threadIdx.x; i < n; i += (long long)gridDim.x * KNT) {
        const bool f = fixed[i] != 0;
        const double bi = f ? 0.0 : b[i];
        const double ri = f ? 0.0 : bi - y[i];
        r64[i] = ri;
        if (r32) r32[i] = (float)ri;
        v[0] += ri * ri;
        v[1] += bi * bi;
    }
    if (last_block_totals<KNT, 2>(v, partials, counter, tot) && threadIdx.x == 0) {
        res[0] = tot[0];
        res[1] = tot[1];
    }
}

// New stopping data of a resumed PCG segment; rz and p of the previous segment stay.
__global__ void k_pcg_resume(PcgScalars* s, double rtol2, int maxit) {
    s->rtol2 = rtol2;
    s->maxit = maxit;
    s->done = 0;
}

__global__ void k_refine_update(long long n, double* __restrict__ x64, const double* __restrict__ d) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x64[i] += d[i];
}

template <typename T>
__global__ void k_zero(long long n, T* __restrict__ a) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = T(0);
}

// FP64 outer iteration of the mixed path as a flexible CG with one previous
// direction: the FP32 inner solution d is K-orthogonalised against the previous
// direction (beta = -(d . K p_prev) / (p_prev . K p_prev)), and the step along
// p = d + beta p_prev is the exact FP64 line search alpha = (p . r) / (p . K p).
// Each step minimises the energy norm of the error along p, so it cannot grow
// when an inner FP32 solve is poor (plain refinement x += d diverges once the
// design's condition number is far beyond the reach of FP32).
struct FcgS {
    double beta, alpha, pkp;
    int has_prev, pad;
};

__global__ void __launch_bounds__(KNT) k_fcg_beta(long long n, const double* __restrict__ d,
                                                  const double* __restrict__ Kp, FcgS* s, double* partials,
                                                  unsigned* counter) {
    if (!s->has_prev) return;  // uniform
    double v[1] = {0.0}, tot[1];
    for (long long i = (long long)blockIdx.x * KNT + threadIdx.x; i < n; i += (long long)gridDim.x * KNT)
        v[0] += d[i] * Kp[i];
    if (last_block_totals<KNT, 1>(v, partials, counter, tot) && threadIdx.x == 0)
        s->beta = s->pkp > 0.0 ? -tot[0] / s->pkp : 0.0;
}

__global__ void k_fcg_dir(long long n, const double* __restrict__ d, double* __restrict__ p, const FcgS* s) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double beta = s->has_prev ? s->beta : 0.0;
    p[i] = d[i] + beta * p[i];
}

__global__ void __launch_bounds__(KNT) k_fcg_alpha(long long n, const double* __restrict__ p,
                                                   const double* __restrict__ r, const double* __restrict__ Kp,
                                                   FcgS* s, double* partials, unsigned* counter) {
    double v[2] = {0.0, 0.0}, tot[2];
    for (long long i = (long long)blockIdx.x * KNT + threadIdx.x; i < n; i += (long long)gridDim.x * KNT) {
        v[0] += p[i] * r[i];
        v[1] += p[i] * Kp[i];
    }
    if (last_block_totals<KNT, 2>(v, partials, counter, tot) && threadIdx.x == 0) {
        const bool ok = tot[1] > 0.0 && isfinite(tot[0]) && isfinite(tot[1]);
        s->alpha = ok ? tot[0] / tot[1] : 0.0;
        s->pkp = ok ? tot[1] : 0.0;
        s->has_prev = ok ? 1 : 0;
    }
}

// x += alpha p, r -= alpha K p, r32 = (float) r, res[0] = r.r.
__global__ void __launch_bounds__(KNT) k_fcg_update(long long n, double* __restrict__ x, double* __restrict__ r,
                                                    const double* __restrict__ p, const double* __restrict__ Kp,
                                                    float* __restrict__ r32, const FcgS* s, double* res,
                                                    double* partials, unsigned* counter) {
    const double alpha = s->alpha;
    double v[1] = {0.0}, tot[1];
    for (long long i = (long long)blockIdx.x * KNT + threadIdx.x; i < n; i += (long long)gridDim.x * KNT) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * Kp[i];
        r[i] = ri;
        r32[i] = (float)ri;
        v[0] += ri * ri;
    }
    if (last_block_totals<KNT, 1>(v, partials, counter, tot) && threadIdx.x == 0) res[0] = tot[0];
}

// ------------------------------------------------------------------ PCG

template <typename T>
struct Pcg {
    double* x = nullptr;         // iterate, FP64 in either precision (k_gpcg_xr)
    T *r = nullptr, *p = nullptr, *Ap = nullptr, *zj = nullptr, *dinv_j = nullptr, *b = nullptr;
    T* E = nullptr;              // modulus in T
    MG<T>* mg = nullptr;         // nullptr: Jacobi
    PcgScalars* s = nullptr;     // device
    cudaGraphExec_t loop = nullptr;
    long long body_kernels = 0;  // kernels per loop iteration
    bool pdl = false;            // the body's kernels use programmatic dependent launch
    T* z = nullptr;              // preconditioner output buffer (fixed at capture)
};

struct Solver {
    Pcg<double> p64;
    Pcg<float> p32;
    double* y64 = nullptr;       // FP64 K U of the refinement
    double *fp = nullptr, *fKp = nullptr;  // outer flexible-CG direction and its K product (mixed)
    FcgS* fs = nullptr;
    double* res = nullptr;       // device refinement sums [4]
    double* hres = nullptr;      // pinned mirror
    PcgScalars* hpcg = nullptr;  // pinned mirror
    std::vector<void*> allocs;
    cudaEvent_t ev[3] = {};      // phase timers
    cudaEvent_t ev_setup[2] = {};  // solver_setup's own timers
    bool setup_done = false;       // solver_setup ran for the coming solve
    double t_setup = 0, t_krylov = 0, t_resid = 0;
};

static float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    TOPO_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
}

template <typename T>
static T* salloc(Solver* s, size_t count) {
    void* p = nullptr;
    TOPO_CUDA(cudaMalloc(&p, count * sizeof(T) + 16));
    s->allocs.push_back(p);
    return (T*)p;
}

template <typename T>
static void pcg_alloc(to_grid* g, Solver* sv, Pcg<T>& P, bool gmg) {
    const long long n = g->d.ndof;
    P.x = salloc<double>(sv, n);
    P.r = salloc<T>(sv, n);
    P.p = salloc<T>(sv, n);
    P.Ap = salloc<T>(sv, n);
    P.zj = salloc<T>(sv, n);
    P.b = salloc<T>(sv, n);
    P.dinv_j = salloc<T>(sv, n);
    P.E = sizeof(T) == 8 ? (T*)g->E : salloc<T>(sv, g->d.nel);
    P.s = salloc<PcgScalars>(sv, 1);
    if (gmg) {
        P.mg = mg_create<T>(g, g->p.mg_levels, g->p.mg_nu, g->p.mg_omega);
        P.mg->coarse_every = g->p.mg_coarse_every;
        P.mg->nu_fine = g->p.mg_nu_fine;
    }
}

// The body of one PCG iteration, captured into the WHILE node's body graph.
template <typename T>
static void enqueue_body(to_grid* g, Pcg<T>& P, cudaGraphConditionalHandle cond, int set_cond, cudaStream_t st) {
    const long long n = g->d.ndof;
    const int* skip = &P.s->done;
    launch_fine_op<T>(g, 0, P.E, P.p, nullptr, nullptr, P.Ap, T(0), skip, P.s, st);
    const MGLevel<T>* L0 = P.mg ? &P.mg->lev[0] : nullptr;
    launch_k(k_gpcg_xr<T>, kblocks(n), KNT, 0, st, n, P.x, P.r, P.p, P.Ap, P.s, g->partials, g->counter,
             L0 ? L0->dinv : nullptr, L0 ? L0->z : nullptr, P.mg ? P.mg->omega : T(0));
    if (P.mg) {
        bool fused = false;
        P.z = mg_vcycle<T>(g, P.mg, P.r, skip, st, P.s, &fused, true);
        if (!fused)
            launch_k(k_gpcg_rz<T, false, false>, kblocks(n), KNT, 0, st, n, P.r, P.z, (const T*)nullptr,
                     (T*)nullptr, P.s, g->partials, g->counter);
    } else {
        P.z = P.zj;
        launch_k(k_gpcg_rz<T, false, true>, kblocks(n), KNT, 0, st, n, P.r, P.z, P.dinv_j, (T*)nullptr, P.s,
                 g->partials, g->counter);
    }
    launch_k(k_gpcg_p<T>, div_up(n, 256) < 2048 ? div_up(n, 256) : 2048, 256, 0, st, n, P.z, P.p, P.s, cond,
             set_cond);
}

template <typename T>
static void build_loop_graph(to_grid* g, Pcg<T>& P, bool pdl) {
    PdlScope pdl_scope(pdl);
    cudaGraph_t graph = nullptr;
    TOPO_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    TOPO_CUDA(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    TOPO_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    TOPO_CUDA(cudaStreamBeginCaptureToGraph(g->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    try {
        enqueue_body<T>(g, P, cond, 1, g->st);
    } catch (...) {
        set_capturing(false);
        cudaStreamEndCapture(g->st, &body);
        cudaGraphDestroy(graph);
        throw;
    }
    set_capturing(false);
    TOPO_CUDA(cudaStreamEndCapture(g->st, &body));
    const cudaError_t e = cudaGraphInstantiate(&P.loop, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        P.loop = nullptr;
        (void)cudaGetLastError();
        if (pdl) {  // programmatic edges refused in the body: plain launches
            captured_launches_reset();
            build_loop_graph<T>(g, P, false);
            return;
        }
        TOPO_CUDA(e);
    }
    P.pdl = pdl;
}

// Set up the preconditioner from P.E (when `setup`), r = b - K x (or r = b for
// x = 0), and run the loop.
// The preconditioner for the current modulus P.E: multigrid hierarchy or Jacobi diagonal.
template <typename T>
static void precond_setup(to_grid* g, Pcg<T>& P, cudaStream_t st) {
    if (P.mg)
        mg_setup<T>(g, P.mg, P.E, st);
    else
        launch_diag_inv<T>(g->d, grid_ke3<T>(g), grid_ke2<T>(g), P.E, g->fixed, P.dinv_j, st);
}

// resume (with x0_zero): continue the previous segment's iteration from the
// residual now in P.b: its search direction p and r.z are kept, and the new
// direction is p = z + (r.z / r.z_old) p instead of p = z.
template <typename T>
static PcgScalars run_pcg(to_grid* g, Solver* sv, Pcg<T>& P, double rtol, int maxit, bool x0_zero, bool setup,
                          bool resume = false) {
    const Dims& d = g->d;
    const long long n = d.ndof;
    cudaStream_t st = g->st;
    TOPO_CUDA(cudaEventRecord(sv->ev[0], st));
    if (setup) precond_setup<T>(g, P, st);
    if (P.mg) mg_wait_coarse<T>(P.mg, st);
    if (!P.loop) {
        build_loop_graph<T>(g, P, g->p.pdl_off == 0);
        P.body_kernels = captured_launches_reset();
    }
    PdlScope pdl_scope(P.pdl);
    TOPO_CUDA(cudaEventRecord(sv->ev[1], st));
    if (resume) {
        k_pcg_resume<<<1, 1, 0, st>>>(P.s, rtol * rtol, maxit);
        TOPO_CHECK_LAUNCH();
    } else {
        PcgScalars init{};
        init.rtol2 = rtol * rtol;
        init.maxit = maxit;
        TOPO_CUDA(cudaMemcpyAsync(P.s, &init, sizeof(PcgScalars), cudaMemcpyHostToDevice, st));
    }
    if (x0_zero) {
        k_zero<double><<<div_up(n, 256), 256, 0, st>>>(n, P.x);
        TOPO_CUDA(cudaMemcpyAsync(P.r, P.b, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
        count_launches(1);
    } else {
        // only the FP64 solve starts from a nonzero x; the FP32 one solves for a correction
        if constexpr (sizeof(T) == 8) {
            launch_fine_op<T>(g, 2, P.E, P.x, P.b, nullptr, P.r, T(0), nullptr, nullptr, st);
        } else {
            TOPO_REQUIRE(false, "the FP32 PCG starts from x = 0");
        }
    }
    k_gpcg_init<T><<<kblocks(n), KNT, 0, st>>>(n, P.b, P.r, g->fixed, P.s, g->partials, g->counter);
    TOPO_CHECK_LAUNCH();
    if (P.mg) {
        T* z = mg_vcycle<T>(g, P.mg, P.r, &P.s->done, st);
        (void)z;  // the same buffer the captured body uses
        if (resume)
            k_gpcg_rz<T, false, false><<<kblocks(n), KNT, 0, st>>>(n, P.r, P.z, nullptr, nullptr, P.s, g->partials,
                                                                   g->counter);
        else
            k_gpcg_rz<T, true, false><<<kblocks(n), KNT, 0, st>>>(n, P.r, P.z, nullptr, P.p, P.s, g->partials,
                                                                  g->counter);
    } else {
        if (resume)
            k_gpcg_rz<T, false, true><<<kblocks(n), KNT, 0, st>>>(n, P.r, P.zj, P.dinv_j, nullptr, P.s,
                                                                  g->partials, g->counter);
        else
            k_gpcg_rz<T, true, true><<<kblocks(n), KNT, 0, st>>>(n, P.r, P.zj, P.dinv_j, P.p, P.s, g->partials,
                                                                 g->counter);
    }
    TOPO_CHECK_LAUNCH();
    if (resume) {
        k_gpcg_p<T><<<div_up(n, 256) < 2048 ? div_up(n, 256) : 2048, 256, 0, st>>>(
            n, P.mg ? P.z : P.zj, P.p, P.s, cudaGraphConditionalHandle{}, 0);
        TOPO_CHECK_LAUNCH();
    }
    if (g->p.loop_mode == 0) {
        TOPO_CUDA(cudaGraphLaunch(P.loop, st));
    } else {
        // the same body kernels from a host loop, polled every 8 iterations
        for (;;) {
            for (int k = 0; k < 8; ++k) enqueue_body<T>(g, P, cudaGraphConditionalHandle{}, 0, st);
            TOPO_CUDA(cudaMemcpyAsync(sv->hpcg, P.s, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
            TOPO_CUDA(cudaStreamSynchronize(st));
            if (sv->hpcg->done) break;
        }
    }
    TOPO_CUDA(cudaEventRecord(sv->ev[2], st));
    TOPO_CUDA(cudaMemcpyAsync(sv->hpcg, P.s, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
    TOPO_CUDA(cudaStreamSynchronize(st));
    sv->t_setup += elapsed_ms(sv->ev[0], sv->ev[1]);
    sv->t_krylov += elapsed_ms(sv->ev[1], sv->ev[2]);
    PcgScalars h = *sv->hpcg;
    if (g->p.loop_mode == 0) count_launches((long long)(h.iters > 0 ? h.iters : 1) * P.body_kernels);
    return h;
}

// ------------------------------------------------------------------ entry

void solver_init(to_grid* g) {
    Solver* s = new Solver();
    g->solver = s;
    try {
        const bool gmg = g->p.precond == TO_PC_GMG;
        if (g->p.precision == TO_FP64) {
            pcg_alloc<double>(g, s, s->p64, gmg);
        } else {
            pcg_alloc<float>(g, s, s->p32, gmg);
            s->p64.x = salloc<double>(s, g->d.ndof);
            s->p64.r = salloc<double>(s, g->d.ndof);
            s->fp = salloc<double>(s, g->d.ndof);
            s->fKp = salloc<double>(s, g->d.ndof);
            s->fs = salloc<FcgS>(s, 1);
        }
        s->y64 = salloc<double>(s, g->d.ndof);
        s->res = salloc<double>(s, 4);
        for (int i = 0; i < 3; ++i) TOPO_CUDA(cudaEventCreate(&s->ev[i]));
        for (int i = 0; i < 2; ++i) TOPO_CUDA(cudaEventCreate(&s->ev_setup[i]));
        TOPO_CUDA(cudaMallocHost(&s->hres, 4 * sizeof(double)));
        TOPO_CUDA(cudaMallocHost(&s->hpcg, sizeof(PcgScalars)));
    } catch (...) {
        solver_free(g);
        throw;
    }
}

void solver_free(to_grid* g) {
    Solver* s = g->solver;
    if (!s) return;
    if (s->p64.loop) cudaGraphExecDestroy(s->p64.loop);
    if (s->p32.loop) cudaGraphExecDestroy(s->p32.loop);
    if (s->p64.mg) mg_destroy(s->p64.mg);
    if (s->p32.mg) mg_destroy(s->p32.mg);
    for (void* p : s->allocs) cudaFree(p);
    for (int i = 0; i < 3; ++i)
        if (s->ev[i]) cudaEventDestroy(s->ev[i]);
    for (int i = 0; i < 2; ++i)
        if (s->ev_setup[i]) cudaEventDestroy(s->ev_setup[i]);
    if (s->hres) cudaFreeHost(s->hres);
    if (s->hpcg) cudaFreeHost(s->hpcg);
    delete s;
    g->solver = nullptr;
}

// ||b - K x|| and ||b|| in FP64 (x, b FP64), into hres[0..1].
static void true_residual(to_grid* g, Solver* sv, const double* b, const double* x, double* r64, float* r32) {
    const long long n = g->d.ndof;
    TOPO_CUDA(cudaEventRecord(sv->ev[0], g->st));
    launch_apply_K<double>(g->d, g->ke3, g->ke2, g->wk, g->node_centric, g->E, x, sv->y64, g->fixed,
                               true, g->st);
    k_refine_resid<<<kblocks(n), KNT, 0, g->st>>>(n, b, sv->y64, r64, r32, g->fixed, sv->res, g->partials,
                                                   g->counter);
    TOPO_CHECK_LAUNCH();
    TOPO_CUDA(cudaEventRecord(sv->ev[1], g->st));
    TOPO_CUDA(cudaMemcpyAsync(sv->hres, sv->res, 2 * sizeof(double), cudaMemcpyDeviceToHost, g->st));
    TOPO_CUDA(cudaStreamSynchronize(g->st));
    sv->t_resid += elapsed_ms(sv->ev[0], sv->ev[1]);
}

// Preconditioner set-up for the modulus in g->E, enqueued on the grid stream
// ahead of the next solve_state (which then skips it), so that independent work
// on another stream (the learned warm start) can overlap it.
void solver_setup(to_grid* g) {
    Solver* sv = g->solver;
    cudaStream_t st = g->st;
    TOPO_CUDA(cudaEventRecord(sv->ev_setup[0], st));
    if (g->p.precision == TO_FP64) {
        precond_setup<double>(g, sv->p64, st);
    } else {
        k_cast_mask<double, float><<<div_up(g->d.nel, 256), 256, 0, st>>>(g->d.nel, g->E, sv->p32.E, nullptr);
        TOPO_CHECK_LAUNCH();
        precond_setup<float>(g, sv->p32, st);
    }
    TOPO_CUDA(cudaEventRecord(sv->ev_setup[1], st));
    sv->setup_done = true;
}

void solver_discard_setup(to_grid* g) {
    if (g->solver) g->solver->setup_done = false;
}

// The FP64 PCG of a TO_MIXED handle, allocated the first time the mixed solve
// hands over to it (its iterate and residual are the refinement's x64, r64).
static void ensure_fp64_pcg(to_grid* g, Solver* sv) {
    Pcg<double>& P = sv->p64;
    if (P.b) return;
    const long long n = g->d.ndof;
    P.p = salloc<double>(sv, n);
    P.Ap = salloc<double>(sv, n);
    P.zj = salloc<double>(sv, n);
    P.b = salloc<double>(sv, n);
    P.dinv_j = salloc<double>(sv, n);
    P.E = g->E;
    P.s = salloc<PcgScalars>(sv, 1);
    if (g->p.precond == TO_PC_GMG) {
        P.mg = mg_create<double>(g, g->p.mg_levels, g->p.mg_nu, g->p.mg_omega);
        P.mg->coarse_every = g->p.mg_coarse_every;
        P.mg->nu_fine = g->p.mg_nu_fine;
    }
}

// FP64 PCG from x = P.x on P.b: the recursive CG residual can drift below the
// true one, so the true FP64 residual decides, and the PCG restarts from the
// current x if needed (restarts counted in *restarts).
static to_status fp64_pcg(to_grid* g, Solver* sv, bool setup, int& iters, int& restarts, double& rel) {
    Pcg<double>& P = sv->p64;
    for (int restart = 0;; ++restart) {
        const PcgScalars h =
            run_pcg<double>(g, sv, P, g->p.cg_rtol, g->p.cg_maxit - iters, false, restart == 0 && setup);
        iters += h.iters;
        true_residual(g, sv, P.b, P.x, P.r, nullptr);
        rel = sv->hres[1] > 0 ? std::sqrt(sv->hres[0] / sv->hres[1]) : 0.0;
        if (h.done == 3 || !std::isfinite(rel)) return TO_ENAN;
        if (rel <= g->p.cg_rtol) return TO_OK;
        if (h.done == 2 || restart >= 8 || iters >= g->p.cg_maxit) return TO_ENOTCONV;
        restarts = restart + 1;
    }
}

to_status solve_state(to_grid* g, const double* b, double* U, to_solve_info* info) {
    Solver* sv = g->solver;
    const Dims& d = g->d;
    const long long n = d.ndof;
    cudaStream_t st = g->st;
    to_status status = TO_OK;
    int iters = 0, refinements = 0;
    double rel = 0.0;
    sv->t_setup = sv->t_krylov = sv->t_resid = 0.0;
    const bool pre = sv->setup_done;  // the preconditioner is already set up for this modulus
    sv->setup_done = false;
    bool fallback = false;
    if (g->p.precision == TO_FP64) {
        Pcg<double>& P = sv->p64;
        TOPO_CUDA(cudaMemcpyAsync(P.b, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        k_cast_mask<double, double><<<div_up(n, 256), 256, 0, st>>>(n, U, P.x, g->fixed);
        TOPO_CHECK_LAUNCH();
        status = fp64_pcg(g, sv, !pre, iters, refinements, rel);  // restarts reported as refinements
        TOPO_CUDA(cudaMemcpyAsync(U, P.x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
        Pcg<float>& P = sv->p32;
        double* x64 = sv->p64.x;
        double* r64 = sv->p64.r;
        if (!pre) {  // set up first: the coarsest factorization then overlaps the true residual
            solver_setup(g);
            sv->setup_done = false;
        }
        k_cast_mask<double, double><<<div_up(n, 256), 256, 0, st>>>(n, U, x64, g->fixed);
        TOPO_CHECK_LAUNCH();
        bool prepared = true;
        const int max_ref = 60;
        true_residual(g, sv, b, x64, r64, P.b);
        rel = sv->hres[1] > 0 ? std::sqrt(sv->hres[0] / sv->hres[1]) : 0.0;
        bool confirmed = true;  // rel is the true FP64 residual (not the recursive one)
        TOPO_CUDA(cudaMemsetAsync(sv->fs, 0, sizeof(FcgS), st));
        bool reliable = g->p.refine == TO_REFINE_RELIABLE;
        bool have_dir = false;  // a previous segment left its search direction
        double per_decade = 0.0;  // PCG iterations per decade of residual drop in the first segment
        for (;;) {
            if (!std::isfinite(rel)) {
                status = TO_ENAN;
                break;
            }
            if (rel <= g->p.cg_rtol) {
                if (confirmed) break;
                // the recursive residual says converged: the true FP64 residual decides
                true_residual(g, sv, b, x64, r64, P.b);
                rel = sv->hres[1] > 0 ? std::sqrt(sv->hres[0] / sv->hres[1]) : 0.0;
                confirmed = true;
                TOPO_CUDA(cudaMemsetAsync(sv->fs, 0, sizeof(FcgS), st));  // restart from the true residual
                continue;
            }
            if (refinements >= max_ref || iters >= g->p.cg_maxit) {
                status = TO_ENOTCONV;
                break;
            }
            if (reliable) {
                // one segment of the FP32 PCG until its residual has fallen by inner_rtol (or by
                // less, when less reaches cg_rtol with a margin for the drift of the FP32
                // recursion), then U += the FP32 correction in FP64 and the true FP64 residual
                // replaces the recursive one; the next segment keeps the search direction
                const double drop = std::max(g->p.inner_rtol, std::min(0.5, 0.3 * g->p.cg_rtol / rel));
                const double decades = std::max(std::log10(1.0 / drop), 0.3);
                // a segment that needs more than RELIABLE_SEG_MAX iterations, or four times the
                // first segment's rate, has stalled in FP32
                int cap = std::min({g->p.inner_maxit, RELIABLE_SEG_MAX, g->p.cg_maxit - iters});
                if (per_decade > 0.0) cap = std::min(cap, 16 + (int)std::ceil(4.0 * per_decade * decades));
                const PcgScalars h = run_pcg<float>(g, sv, P, drop, cap, true, !prepared, have_dir);
                prepared = true;
                iters += h.iters;
                if (h.done == 3) {
                    status = TO_ENAN;
                    break;
                }
                k_refine_update<<<div_up(n, 256), 256, 0, st>>>(n, x64, P.x);
                TOPO_CHECK_LAUNCH();
                count_launches(1);
                if (per_decade == 0.0 && h.done == 1 && h.iters > 0) per_decade = h.iters / decades;
                const double rel_prev = rel;
                true_residual(g, sv, b, x64, r64, P.b);
                rel = sv->hres[1] > 0 ? std::sqrt(sv->hres[0] / sv->hres[1]) : 0.0;
                confirmed = true;
                ++refinements;
                // the next segment keeps the search direction only while the FP32 recursion
                // tracks the true residual: where the true residual fell far less than the
                // recursive one (the FP32 operator's accuracy limit), beta = r.z / r.z_old
                // would scale the old direction up by the mismatch and the resumed iteration
                // stalls; it then restarts from the true residual instead
                const double rec = h.bb > 0.0 ? std::sqrt(h.rr / h.bb) : 0.0;
                have_dir = std::isfinite(rel) && rel <= 4.0 * rec * rel_prev;
                // the FP32 recursion stalled (segment cap) or no longer tracks the FP64
                // residual: continue with the flexible-CG steps, whose exact FP64 line search
                // cannot raise the energy
                if (h.done == 2 || (std::isfinite(rel) && rel > 0.5 * rel_prev)) reliable = false;
                continue;
            }
            // the preconditioner is set up once per solve
            // each inner solve is capped: a stalled FP32 run still hands the FP64 step a direction
            const PcgScalars h = run_pcg<float>(g, sv, P, g->p.inner_rtol,
                                                std::min(g->p.inner_maxit, g->p.cg_maxit - iters), true, !prepared);
            prepared = true;
            iters += h.iters;
            if (h.done == 3) {
                status = TO_ENAN;
                break;
            }
            // one flexible-CG step in FP64 along the inner solution
            TOPO_CUDA(cudaEventRecord(sv->ev[0], st));
            k_fcg_beta<<<kblocks(n), KNT, 0, st>>>(n, P.x, sv->fKp, sv->fs, g->partials, g->counter);
            k_fcg_dir<<<div_up(n, 256), 256, 0, st>>>(n, P.x, sv->fp, sv->fs);
            launch_apply_K<double>(d, g->ke3, g->ke2, g->wk, g->node_centric, g->E, sv->fp, sv->fKp, g->fixed,
                               true, st);
            k_fcg_alpha<<<kblocks(n), KNT, 0, st>>>(n, sv->fp, r64, sv->fKp, sv->fs, g->partials, g->counter);
            k_fcg_update<<<kblocks(n), KNT, 0, st>>>(n, x64, r64, sv->fp, sv->fKp, P.b, sv->fs, sv->res,
                                                    g->partials, g->counter);
            TOPO_CHECK_LAUNCH();
            count_launches(3);
            TOPO_CUDA(cudaEventRecord(sv->ev[1], st));
            TOPO_CUDA(cudaMemcpyAsync(sv->hres, sv->res, sizeof(double), cudaMemcpyDeviceToHost, st));
            TOPO_CUDA(cudaStreamSynchronize(st));
            sv->t_resid += elapsed_ms(sv->ev[0], sv->ev[1]);
            rel = sv->hres[1] > 0 ? std::sqrt(sv->hres[0] / sv->hres[1]) : 0.0;
            confirmed = false;
            ++refinements;
        }
        // The FP32 iteration failed (a non-finite value, or the refinement cap with
        // iterations left): the design is beyond FP32's reach (a condition number far
        // above 1 / eps_32, e.g. a load path through near-void elements or a few
        // clamped nodes). The FP64 PCG finishes the solve, from the refined iterate,
        // or from the caller's start after a non-finite value.
        if ((status == TO_ENAN || status == TO_ENOTCONV) && iters < g->p.cg_maxit) {
            ensure_fp64_pcg(g, sv);
            Pcg<double>& Q = sv->p64;  // Q.x is x64, Q.r is r64
            TOPO_CUDA(cudaMemcpyAsync(Q.b, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            if (status == TO_ENAN) {
                k_cast_mask<double, double><<<div_up(n, 256), 256, 0, st>>>(n, U, x64, g->fixed);
                TOPO_CHECK_LAUNCH();
            }
            int restarts = 0;
            status = fp64_pcg(g, sv, true, iters, restarts, rel);
            fallback = true;
        }
        TOPO_CUDA(cudaMemcpyAsync(U, x64, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (g->tc_err) {
            int herr = 0;
            TOPO_CUDA(cudaMemcpyAsync(&herr, g->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
            TOPO_CUDA(cudaStreamSynchronize(st));
            if (herr) status = TO_ETIMEOUT;
        }
    }
    // the stream has drained
    if (pre || g->p.precision != TO_FP64) sv->t_setup += elapsed_ms(sv->ev_setup[0], sv->ev_setup[1]);
    if (info) {
        info->iters = iters;
        info->refinements = refinements;
        info->rel_res = rel;
        info->status = (int)status;
        info->fallback = fallback ? 1 : 0;
        info->t_setup_ms = sv->t_setup;
        info->t_krylov_ms = sv->t_krylov;
        info->t_resid_ms = sv->t_resid;
    }
    return status;
}

// y = K u with the FP32 operator of the mixed path (impl 1: node-centric dense Ke, 2: tensor cores,
// 3: Walsh-factored element tiles).
void apply_K_fp32(to_grid* g, const double* xPhys, const double* u, double* y, int impl) {
    Solver* sv = g->solver;
    TOPO_REQUIRE(g->p.precision == TO_MIXED, "handle was created for TO_FP64");
    TOPO_REQUIRE(impl == 1 || (impl == 2 && g->ke_tc) || (impl == 3 && g->d.dim == 3) ||
                     (impl == 4 && g->d.dim == 3 && walsh_pair_supported(g->d)),
                 "impl must be 1, or 2, 3 or 4 on a 3D grid");
    const Dims& d = g->d;
    const long long n = d.ndof;
    cudaStream_t st = g->st;
    Pcg<float>& P = sv->p32;
    launch_modulus<float>(d.nel, xPhys, g->penal, g->p.E0, g->p.Emin, P.E, st);
    k_cast_mask<double, float><<<div_up(n, 256), 256, 0, st>>>(n, u, P.p, g->fixed);
    TOPO_CHECK_LAUNCH();
    const bool saved = g->use_tc, saved_nc = g->node_centric, saved_wp = g->walsh_pair;
    g->use_tc = impl == 2;
    g->node_centric = impl == 1;
    g->walsh_pair = impl == 4;
    try {
        launch_fine_op<float>(g, 0, P.E, P.p, nullptr, nullptr, P.Ap, 0.f, nullptr, nullptr, st);
    } catch (...) {
        g->use_tc = saved;
        g->node_centric = saved_nc;
        g->walsh_pair = saved_wp;
        throw;
    }
    g->use_tc = saved;
    g->node_centric = saved_nc;
    g->walsh_pair = saved_wp;
    k_cast_mask<float, double><<<div_up(n, 256), 256, 0, st>>>(n, P.Ap, y, nullptr);
    TOPO_CHECK_LAUNCH();
    if (g->tc_err) {
        int h = 0;
        TOPO_CUDA(cudaMemcpyAsync(&h, g->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        TOPO_CUDA(cudaStreamSynchronize(st));
        if (h) throw Error(TO_ETIMEOUT, "tensor-core operator: mbarrier wait passed its limit");
    }
}

void time_apply_K_mixed(to_grid* g, const double* xPhys, int reps, cudaEvent_t e0, cudaEvent_t e1) {
    Solver* sv = g->solver;
    TOPO_REQUIRE(g->p.precision == TO_MIXED, "handle was created for TO_FP64");
    const Dims& d = g->d;
    cudaStream_t st = g->st;
    Pcg<float>& P = sv->p32;
    launch_modulus<float>(d.nel, xPhys, g->penal, g->p.E0, g->p.Emin, P.E, st);
    k_zero<float><<<div_up(d.ndof, 256), 256, 0, st>>>(d.ndof, P.p);
    TOPO_CHECK_LAUNCH();
    launch_fine_op<float>(g, 0, P.E, P.p, nullptr, nullptr, P.Ap, 0.f, nullptr, nullptr, st);
    TOPO_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r)
        launch_fine_op<float>(g, 0, P.E, P.p, nullptr, nullptr, P.Ap, 0.f, nullptr, nullptr, st);
    TOPO_CUDA(cudaEventRecord(e1, st));
}

}  // namespace topo
