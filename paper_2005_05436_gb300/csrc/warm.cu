// The learned warm start inside the design iteration (no counterpart in the
// paper): node features -> network -> displacement direction U_h, and the
// starting point of the state solve is the minimiser of the potential energy
// 1/2 U^T K U - F^T U over span{U_prev, U_h} (a 2 x 2 Rayleigh-Ritz step; its
// operator products in FP32 for the mixed solve, FP64 otherwise). Its energy
// never exceeds that of U_prev, and the solve that follows runs to the same
// tolerance, so the solution does not depend on the network; only the
// iteration count can. It runs on a stream of its own while the grid stream
// sets up the preconditioner.
#include <algorithm>
#include <cmath>

#include "grid.h"
#include "mg.h"

namespace topo {

void net_forward_on(to_net* n, const float* x, int N, int D, int H, int W, float* y, cudaStream_t st);  // net.cu

namespace {

// The network works on the node grid coarsened by S (1 or 2): coarse node
// (I, J, K) sits on fine node (S I, S J, S K) (the last coarse node of an odd
// axis lies one node past the grid). Load-like fields are restricted by full
// weighting (the transpose of the trilinear prolongation, which conserves the
// total load); the network output is prolongated trilinearly to the fine nodes.
struct CGrid {
    int S, Nx, Ny, Nz, D, H, W;  // coarse node counts and the padded tensor dims
};

struct WarmWS {
    int D = 0, H = 0, W = 0;
    CGrid cg{};
    float *x = nullptr, *y = nullptr;
    double *Uh = nullptr, *KUh = nullptr, *Up = nullptr, *KUp = nullptr, *dots = nullptr, *hdots = nullptr;
    unsigned* fmax = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // the warm start runs on its own stream, beside the preconditioner set-up
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, ready = nullptr, join = nullptr;
    float *E32 = nullptr, *u32 = nullptr, *y32 = nullptr;  // FP32 operator products (mixed path)
    double* partials = nullptr;                            // reduction scratch of its own
    unsigned* counter = nullptr;
};

inline int pad4(int n) { return (n + 3) / 4 * 4; }

__global__ void kw_absmax(long long n, const double* __restrict__ F, unsigned* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(out, __float_as_uint((float)fabs(F[i])));  // non-negative floats order as integers
}

__host__ __device__ inline int coarse_n(int nn, int S) { return S == 1 ? nn : (nn - 1 + 1) / 2 + 1; }

// sum_{o} w(o) f(S I + o) along three axes (w = 1 at o = 0, 1/2 at o = +-1 for S = 2).
template <typename Fn>
__device__ __forceinline__ void restrict3(const Dims& d, const CGrid& c, int I, int J, int K, Fn&& add) {
    const int r = c.S == 2 ? 1 : 0;
    for (int ox = -r; ox <= r; ++ox)
        for (int oz = -r; oz <= r; ++oz)
            for (int oy = -r; oy <= r; ++oy) {
                const int ix = c.S * I + ox, iz = c.S * K + oz, iy = c.S * J + oy;
                if (ix < 0 || ix >= d.nnx || iz < 0 || iz >= d.nnz || iy < 0 || iy >= d.nny) continue;
                const double w = (ox ? 0.5 : 1.0) * (oz ? 0.5 : 1.0) * (oy ? 0.5 : 1.0);
                add(iy + (long long)d.nny * (iz + (long long)d.nnz * ix), w);
            }
}

__device__ __forceinline__ void decode_v(const CGrid& c, long long v, int& I, int& K, int& J) {
    J = (int)(v % c.W);
    K = (int)((v / c.W) % c.H);
    I = (int)(v / ((long long)c.W * c.H));
}

// Network input on the padded coarse node grid [D][H][W] (x, z, y: the node
// numbering's order): the mean physical density of the elements around the
// node (-1 at nodes with a Dirichlet DOF, so that supports are visible to the
// network) and the restricted load scaled by 1 / max |F|; zero in the padding.
__global__ void kw_features(Dims d, CGrid c, const double* __restrict__ xPhys, const double* __restrict__ F,
                            const uint8_t* __restrict__ fixed, const unsigned* __restrict__ fmax,
                            float* __restrict__ x) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)c.D * c.H * c.W) return;
    int I, K, J;
    decode_v(c, v, I, K, J);
    float f[4] = {0.f, 0.f, 0.f, 0.f};
    if (I < c.Nx && K < c.Nz && J < c.Ny) {
        const int ix = min(c.S * I, d.nnx - 1), iz = min(c.S * K, d.nnz - 1), iy = min(c.S * J, d.nny - 1);
        double s = 0.0;
        int cnt = 0;
        for (int o = 0; o < 8; ++o) {
            const int ex = ix - 1 + (o >> 2), ez = iz - 1 + ((o >> 1) & 1), ey = iy - 1 + (o & 1);
            if (ex < 0 || ex >= d.nelx || ey < 0 || ey >= d.nely || ez < 0 || ez >= d.nelz) continue;
            s += xPhys[ey + (long long)d.nely * (ez + (long long)d.nelz * ex)];
            ++cnt;
        }
        const long long n = iy + (long long)d.nny * (iz + (long long)d.nnz * ix);
        const bool sup = fixed[3 * n] || fixed[3 * n + 1] || fixed[3 * n + 2];
        f[0] = sup ? -1.f : (cnt ? (float)(s / cnt) : 0.f);
        const float fm = __uint_as_float(*fmax);
        const double sc = fm > 0.f ? 1.0 / fm : 0.0;
        double a[3] = {0.0, 0.0, 0.0};
        restrict3(d, c, I, J, K, [&](long long m, double w) {
            for (int q = 0; q < 3; ++q) a[q] += w * F[3 * m + q];
        });
        for (int q = 0; q < 3; ++q) f[1 + q] = (float)(a[q] * sc);
    }
    for (int q = 0; q < 4; ++q) x[v * 4 + q] = f[q];
}

// Training target: U / rms(U) at the coarse nodes (fine node S I, clamped) and
// the coarse node mask.
__global__ void kw_target(Dims d, CGrid c, const double* __restrict__ U, const double* __restrict__ sumsq,
                          float* __restrict__ t, uint8_t* __restrict__ mask) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)c.D * c.H * c.W) return;
    int I, K, J;
    decode_v(c, v, I, K, J);
    const bool in = I < c.Nx && K < c.Nz && J < c.Ny;
    const double ss = *sumsq;
    const double inv = ss > 0.0 ? 1.0 / sqrt(ss / (double)d.ndof) : 0.0;
    const int ix = min(c.S * I, d.nnx - 1), iz = min(c.S * K, d.nnz - 1), iy = min(c.S * J, d.nny - 1);
    const long long n = iy + (long long)d.nny * (iz + (long long)d.nnz * ix);
    for (int q = 0; q < 3; ++q) t[v * 3 + q] = in ? (float)(U[3 * n + q] * inv) : 0.f;
    mask[v] = in ? 1 : 0;
}

// U_h at the fine nodes: trilinear prolongation of the coarse output; 0 at
// Dirichlet DOFs.
__global__ void kw_crop(Dims d, CGrid c, const float* __restrict__ y, const uint8_t* __restrict__ fixed,
                        double* __restrict__ Uh) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.nnodes) return;
    const int iy = (int)(n % d.nny), iz = (int)((n / d.nny) % d.nnz), ix = (int)(n / ((long long)d.nny * d.nnz));
    double a[3] = {0.0, 0.0, 0.0};
    const int I0 = ix / c.S, K0 = iz / c.S, J0 = iy / c.S;
    const int nI = (c.S == 2 && (ix & 1)) ? 2 : 1, nK = (c.S == 2 && (iz & 1)) ? 2 : 1,
              nJ = (c.S == 2 && (iy & 1)) ? 2 : 1;
    const double w = 1.0 / (nI * nK * nJ);
    for (int p = 0; p < nI; ++p)
        for (int q = 0; q < nK; ++q)
            for (int r = 0; r < nJ; ++r) {
                const long long v = ((long long)(I0 + p) * c.H + (K0 + q)) * c.W + (J0 + r);
                for (int k = 0; k < 3; ++k) a[k] += w * (double)y[v * 3 + k];
            }
    for (int k = 0; k < 3; ++k) Uh[3 * n + k] = fixed[3 * n + k] ? 0.0 : a[k];
}

// Output gradient of the energy objective: g = ga F + gb K U_h on the free fine
// DOFs, taken to the coarse grid by the transpose of the prolongation.
__global__ void kw_energy_grad(Dims d, CGrid c, const double* __restrict__ F, const double* __restrict__ KUh,
                               const uint8_t* __restrict__ fixed, double ga, double gb, float* __restrict__ gy) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)c.D * c.H * c.W) return;
    int I, K, J;
    decode_v(c, v, I, K, J);
    double a[3] = {0.0, 0.0, 0.0};
    if (I < c.Nx && K < c.Nz && J < c.Ny) {
        restrict3(d, c, I, J, K, [&](long long m, double w) {
            // the prolongation weight of fine node m from this coarse node is w / (its stencil size)
            const int ix = (int)(m / ((long long)d.nny * d.nnz)), iz = (int)((m / d.nny) % d.nnz), iy = (int)(m % d.nny);
            const int cnt = ((c.S == 2 && (ix & 1)) ? 2 : 1) * ((c.S == 2 && (iz & 1)) ? 2 : 1) *
                            ((c.S == 2 && (iy & 1)) ? 2 : 1);
            const double pw = 1.0 / cnt;
            for (int q = 0; q < 3; ++q)
                if (!fixed[3 * m + q]) a[q] += pw * (ga * F[3 * m + q] + gb * KUh[3 * m + q]);
            (void)w;
        });
    }
    for (int q = 0; q < 3; ++q) gy[v * 3 + q] = (float)a[q];
}

// The sums both combination rules need, in one pass over F, U_prev (Up, zero at
// fixed DOFs), U_h and their operator products: dots[0] F.Up, [1] F.Uh,
// [2] Up.KUp, [3] Up.KUh, [4] Uh.KUh, [8] KUp.KUp, [9] KUp.KUh, [10] KUh.KUh,
// [11] F.KUp, [12] F.KUh and [13] ||F||^2 over the free DOFs (K U is 0 at fixed
// DOFs, so the sums with it run over the free DOFs). Block partials are summed
// in block order by the last block (deterministic).
constexpr int WNT = 256;
constexpr int WDOTS = 11;
__global__ void __launch_bounds__(WNT) kw_dots(long long n, const double* __restrict__ F,
                                               const uint8_t* __restrict__ fixed, const double* __restrict__ Up,
                                               const double* __restrict__ Uh, const double* __restrict__ KUp,
                                               const double* __restrict__ KUh, double* dots, double* partials,
                                               unsigned* counter) {
    double v[WDOTS] = {}, tot[WDOTS];
    for (long long i = (long long)blockIdx.x * WNT + threadIdx.x; i < n; i += (long long)gridDim.x * WNT) {
        const double f = F[i], up = Up[i], uh = Uh[i], kp = KUp[i], kh = KUh[i];
        const double ff = fixed[i] ? 0.0 : f;
        v[0] += f * up;
        v[1] += f * uh;
        v[2] += up * kp;
        v[3] += up * kh;
        v[4] += uh * kh;
        v[5] += kp * kp;
        v[6] += kp * kh;
        v[7] += kh * kh;
        v[8] += f * kp;
        v[9] += f * kh;
        v[10] += ff * ff;
    }
    if (last_block_totals<WNT, WDOTS>(v, partials, counter, tot) && threadIdx.x == 0) {
        constexpr int slot[WDOTS] = {0, 1, 2, 3, 4, 8, 9, 10, 11, 12, 13};
#pragma unroll
        for (int k = 0; k < WDOTS; ++k) dots[slot[k]] = tot[k];
    }
}

__global__ void kw_combine(long long n, double a, const double* __restrict__ Up, double b,
                           const double* __restrict__ Uh, double* __restrict__ U) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) U[i] = a * Up[i] + b * Uh[i];
}

__global__ void kw_to_f32(long long n, const double* __restrict__ a, const uint8_t* __restrict__ fixed,
                          float* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (fixed && fixed[i]) ? 0.f : (float)a[i];
}

__global__ void kw_to_f64(long long n, const float* __restrict__ a, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)a[i];
}

template <typename T>
T* walloc(to_grid* g, long long count) {
    void* p = nullptr;
    TOPO_CUDA(cudaMalloc(&p, std::max<long long>(count, 1) * sizeof(T)));
    g->allocs.push_back(p);
    return (T*)p;
}

WarmWS* warm_ws(to_grid* g) {
    if (g->warm && ((WarmWS*)g->warm)->cg.S == g->warm_stride) return (WarmWS*)g->warm;
    TOPO_REQUIRE(!g->warm, "the warm-start coarsening cannot change after first use");
    TOPO_REQUIRE(g->d.dim == 3, "the learned warm start works on 3D grids");
    WarmWS* w = new WarmWS();
    g->warm = w;
    w->cg.S = g->warm_stride;
    w->cg.Nx = coarse_n(g->d.nnx, w->cg.S);
    w->cg.Ny = coarse_n(g->d.nny, w->cg.S);
    w->cg.Nz = coarse_n(g->d.nnz, w->cg.S);
    w->D = w->cg.D = pad4(w->cg.Nx);
    w->H = w->cg.H = pad4(w->cg.Nz);
    w->W = w->cg.W = pad4(w->cg.Ny);
    const long long V = (long long)w->D * w->H * w->W;
    w->x = walloc<float>(g, V * 4);
    w->y = walloc<float>(g, V * 3);
    for (double** a : {&w->Uh, &w->KUh, &w->Up, &w->KUp}) *a = walloc<double>(g, g->d.ndof);
    w->dots = walloc<double>(g, 16);
    w->fmax = walloc<unsigned>(g, 1);
    TOPO_CUDA(cudaMallocHost(&w->hdots, 16 * sizeof(double)));
    TOPO_CUDA(cudaEventCreate(&w->e0));
    TOPO_CUDA(cudaEventCreate(&w->e1));
    TOPO_CUDA(cudaStreamCreateWithFlags(&w->aux, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&w->fork, &w->ready, &w->join})
        TOPO_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    if (g->p.precision == TO_MIXED) {
        w->E32 = walloc<float>(g, g->d.nel);
        w->u32 = walloc<float>(g, g->d.ndof);
        w->y32 = walloc<float>(g, g->d.ndof);
    }
    w->partials = walloc<double>(g, g->npartials);
    w->counter = walloc<unsigned>(g, 16);
    TOPO_CUDA(cudaMemsetAsync(w->counter, 0, 16 * sizeof(unsigned), g->st));
    TOPO_CUDA(cudaStreamSynchronize(g->st));
    return w;
}

// KU = K U with the grid's FP32 operator (the one of the mixed solve) and the FP32 modulus in w->E32.
void product32(to_grid* g, WarmWS* w, const double* U, double* KU, cudaStream_t st) {
    const long long n = g->d.ndof;
    kw_to_f32<<<div_up(n, 256), 256, 0, st>>>(n, U, g->fixed, w->u32);
    TOPO_CHECK_LAUNCH();
    launch_fine_op<float>(g, 0, w->E32, w->u32, nullptr, nullptr, w->y32, 0.f, nullptr, nullptr, st);
    kw_to_f64<<<div_up(n, 256), 256, 0, st>>>(n, w->y32, KU);
    TOPO_CHECK_LAUNCH();
}

void features(to_grid* g, WarmWS* w, const double* xPhys, float* x, cudaStream_t st) {
    const Dims& d = g->d;
    TOPO_CUDA(cudaMemsetAsync(w->fmax, 0, sizeof(unsigned), st));
    kw_absmax<<<div_up(d.ndof, 256), 256, 0, st>>>(d.ndof, g->F, w->fmax);
    TOPO_CHECK_LAUNCH();
    const long long V = (long long)w->D * w->H * w->W;
    kw_features<<<div_up(V, 256), 256, 0, st>>>(d, w->cg, xPhys, g->F, g->fixed, w->fmax, x);
    TOPO_CHECK_LAUNCH();
}

}  // namespace

void warm_free(to_grid* g) {
    WarmWS* w = (WarmWS*)g->warm;
    if (!w) return;
    if (w->hdots) cudaFreeHost(w->hdots);
    if (w->e0) cudaEventDestroy(w->e0);
    if (w->e1) cudaEventDestroy(w->e1);
    for (cudaEvent_t e : {w->fork, w->ready, w->join})
        if (e) cudaEventDestroy(e);
    if (w->aux) {
        cudaStreamSynchronize(w->aux);
        cudaStreamDestroy(w->aux);
    }
    delete w;
    g->warm = nullptr;
}

// Makes the grid stream wait for everything enqueued on the warm-start stream,
// also when the warm start ends by an exception (the grid stream then never
// runs ahead of kernels still reading U or the grid's buffers).
struct AuxJoin {
    WarmWS* w;
    cudaStream_t st;
    bool done = false;
    ~AuxJoin() {
        if (done) return;
        cudaEventRecord(w->join, w->aux);
        cudaStreamWaitEvent(st, w->join, 0);
    }
};

// U <- argmin of the energy over span{U, U_h}; E(xPhys) in g->E (FP64).
void learned_warm_start(to_grid* g, const double* xPhys, double* U, double* coef, double* ms, double* energy,
                        double* resid) {
    WarmWS* w = warm_ws(g);
    const Dims& d = g->d;
    cudaStream_t st = g->st, ax = w->aux;
    // xPhys, E and U are ready in the grid stream's order; the warm start forks
    // onto its own stream, and the preconditioner set-up for this design runs on
    // the grid stream meanwhile (the two share no buffer that either writes).
    TOPO_CUDA(cudaEventRecord(w->fork, st));
    TOPO_CUDA(cudaStreamWaitEvent(ax, w->fork, 0));
    AuxJoin joiner{w, st};
    TOPO_CUDA(cudaEventRecord(w->e0, ax));
    features(g, w, xPhys, w->x, ax);
    net_forward_on(g->net, w->x, 1, w->D, w->H, w->W, w->y, ax);
    kw_crop<<<div_up(d.nnodes, 256), 256, 0, ax>>>(d, w->cg, w->y, g->fixed, w->Uh);
    TOPO_CHECK_LAUNCH();
    launch_mask_copy(d.ndof, U, w->Up, g->fixed, ax);
    if (g->p.precision == TO_MIXED) {
        // the products only choose a starting point: the FP32 operator is enough
        launch_modulus<float>(d.nel, xPhys, g->penal, g->p.E0, g->p.Emin, w->E32, ax);
        product32(g, w, w->Uh, w->KUh, ax);
        product32(g, w, w->Up, w->KUp, ax);
    } else {
        launch_apply_K<double>(d, g->ke3, g->ke2, g->wk, g->node_centric, g->E, w->Uh, w->KUh, g->fixed,
                               true, ax);
        launch_apply_K<double>(d, g->ke3, g->ke2, g->wk, g->node_centric, g->E, w->Up, w->KUp, g->fixed,
                               true, ax);
    }
    // the energy rule's Gram matrix and products with F, the residual rule's
    // (the two residual directions K U), and ||F||^2, in one pass
    {
        const long long nb = std::min<long long>({(d.ndof + 4LL * WNT - 1) / (4LL * WNT), 1024LL,
                                                  g->npartials / WDOTS});
        kw_dots<<<(unsigned)std::max<long long>(nb, 1), WNT, 0, ax>>>(d.ndof, g->F, g->fixed, w->Up, w->Uh, w->KUp,
                                                                      w->KUh, w->dots, w->partials, w->counter);
        TOPO_CHECK_LAUNCH();
    }
    const bool by_residual = g->warm_rule == TO_WARM_RESIDUAL;
    TOPO_CUDA(cudaMemcpyAsync(w->hdots, w->dots, 14 * sizeof(double), cudaMemcpyDeviceToHost, ax));
    TOPO_CUDA(cudaEventRecord(w->ready, ax));
    solver_setup(g);
    TOPO_CUDA(cudaEventSynchronize(w->ready));
    const double fp = w->hdots[0], fh = w->hdots[1], pp = w->hdots[2], ph = w->hdots[3], hh = w->hdots[4];
    double a = 1.0, b = 0.0;  // keep U when the network direction adds nothing
    const bool hok = hh > 0.0 && std::isfinite(hh) && std::isfinite(fh);
    if (by_residual) {
        // minimiser of ||F - K (a U_prev + b U_h)||_2 over the free DOFs: the
        // stopping test's norm, so the start is never worse than U_prev in it
        const double rpp = w->hdots[8], rph = w->hdots[9], rhh = w->hdots[10], rfp = w->hdots[11],
                     rfh = w->hdots[12];
        const bool rok = rhh > 0.0 && std::isfinite(rhh) && std::isfinite(rfh) && std::isfinite(rph);
        if (rok && !(rpp > 0.0)) {
            a = 0.0;
            b = rfh / rhh;
        } else if (rok && std::isfinite(rpp) && std::isfinite(rfp)) {
            const double det = rpp * rhh - rph * rph;
            if (det > 1e-12 * rpp * rhh) {
                a = (rfp * rhh - rfh * rph) / det;
                b = (rpp * rfh - rph * rfp) / det;
            }
        }
    } else if (hok && !(pp > 0.0)) {  // no previous solution: the energy-optimal multiple of U_h
        a = 0.0;
        b = fh / hh;
    } else if (hok && std::isfinite(pp) && std::isfinite(ph) && std::isfinite(fp)) {
        const double det = pp * hh - ph * ph;
        if (det > 1e-12 * pp * hh) {
            a = (fp * hh - fh * ph) / det;
            b = (pp * fh - ph * fp) / det;
        }
    }
    if (!(a == 1.0 && b == 0.0)) {
        kw_combine<<<div_up(d.ndof, 256), 256, 0, ax>>>(d.ndof, a, w->Up, b, w->Uh, U);
        TOPO_CHECK_LAUNCH();
    }
    TOPO_CUDA(cudaEventRecord(w->e1, ax));
    TOPO_CUDA(cudaEventRecord(w->join, ax));
    TOPO_CUDA(cudaStreamWaitEvent(st, w->join, 0));
    joiner.done = true;
    TOPO_CUDA(cudaEventSynchronize(w->e1));
    float t = 0.f;
    TOPO_CUDA(cudaEventElapsedTime(&t, w->e0, w->e1));
    if (coef) {
        coef[0] = a;
        coef[1] = b;
    }
    if (ms) *ms = t;
    if (energy) {  // potential energy 1/2 U^T K U - F^T U of U_prev and of the new start
        energy[0] = 0.5 * pp - fp;
        energy[1] = 0.5 * (a * a * pp + 2.0 * a * b * ph + b * b * hh) - (a * fp + b * fh);
    }
    if (resid) {  // ||F - K U|| / ||F|| of U_prev and of the new start
        const double ff = w->hdots[13], rpp = w->hdots[8], rph = w->hdots[9], rhh = w->hdots[10],
                     rfp = w->hdots[11], rfh = w->hdots[12];
        auto r2 = [&](double ca, double cb) {
            return std::fmax(0.0, ff - 2.0 * (ca * rfp + cb * rfh) + ca * ca * rpp + 2.0 * ca * cb * rph + cb * cb * rhh);
        };
        resid[0] = ff > 0.0 ? std::sqrt(r2(1.0, 0.0) / ff) : 0.0;
        resid[1] = ff > 0.0 ? std::sqrt(r2(a, b) / ff) : 0.0;
    }
}

}  // namespace topo

using namespace topo;

extern "C" {

to_status to_set_warm_start(to_grid* g, to_net* net, int32_t stride) {
    if (!g) return api_fail(TO_EINVAL, "NULL handle");
    if (net && g->d.dim != 3) return api_fail(TO_EINVAL, "the learned warm start works on 3D grids");
    if (stride != 1 && stride != 2) return api_fail(TO_EINVAL, "stride must be 1 or 2");
    if (g->warm && ((WarmWS*)g->warm)->cg.S != stride)
        return api_fail(TO_EINVAL, "the warm-start coarsening cannot change after first use");
    g->net = net;
    g->warm_stride = stride;
    return TO_OK;
}

to_status to_set_warm_start_rule(to_grid* g, int32_t rule) {
    if (!g) return api_fail(TO_EINVAL, "NULL handle");
    if (rule != TO_WARM_ENERGY && rule != TO_WARM_RESIDUAL) return api_fail(TO_EINVAL, "rule must be TO_WARM_ENERGY or TO_WARM_RESIDUAL");
    g->warm_rule = rule;
    return TO_OK;
}

to_status to_learned_features(to_grid* g, const double* xPhys, float* x, int32_t* dims) {
    if (!g) return api_fail(TO_EINVAL, "NULL handle");
    try {
        WarmWS* w = warm_ws(g);
        if (dims) {
            dims[0] = w->D;
            dims[1] = w->H;
            dims[2] = w->W;
        }
        if (!x) return TO_OK;
        if (!xPhys) return api_fail(TO_EINVAL, "NULL xPhys");
        grid_sync_in(g);
        features(g, w, xPhys, x, g->st);
        grid_sync_out(g);
    } catch (const topo::Error& e) {
        return api_fail(e.code, e.what());
    }
    return TO_OK;
}

to_status to_learned_target(to_grid* g, const double* U, float* t, uint8_t* mask) {
    if (!g || !U || !t || !mask) return api_fail(TO_EINVAL, "NULL argument");
    try {
        WarmWS* w = warm_ws(g);
        grid_sync_in(g);
        const Dims& d = g->d;
        launch_dot(d.ndof, U, nullptr, w->dots + 5, g->partials, g->counter, g->st);
        const long long V = (long long)w->D * w->H * w->W;
        kw_target<<<div_up(V, 256), 256, 0, g->st>>>(d, w->cg, U, w->dots + 5, t, mask);
        TOPO_CHECK_LAUNCH();
        grid_sync_out(g);
    } catch (const topo::Error& e) {
        return api_fail(e.code, e.what());
    }
    return TO_OK;
}

to_status to_learned_energy_grad(to_grid* g, const double* xPhys, const float* y, double c_star, float* gy,
                                 double* loss) {
    if (!g || !xPhys || !y || !gy || !(c_star > 0.0)) return api_fail(TO_EINVAL, "NULL argument or c <= 0");
    try {
        WarmWS* w = warm_ws(g);
        grid_sync_in(g);
        const Dims& d = g->d;
        cudaStream_t st = g->st;
        launch_modulus<double>(d.nel, xPhys, g->penal, g->p.E0, g->p.Emin, g->E, st);
        kw_crop<<<div_up(d.nnodes, 256), 256, 0, st>>>(d, w->cg, y, g->fixed, w->Uh);
        TOPO_CHECK_LAUNCH();
        launch_apply_K<double>(d, g->ke3, g->ke2, g->wk, g->node_centric, g->E, w->Uh, w->KUh, g->fixed,
                               true, st);
        launch_dot(d.ndof, g->F, w->Uh, w->dots + 6, g->partials, g->counter, st);
        launch_dot(d.ndof, w->Uh, w->KUh, w->dots + 7, g->partials, g->counter, st);
        TOPO_CUDA(cudaMemcpyAsync(w->hdots + 6, w->dots + 6, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        TOPO_CUDA(cudaStreamSynchronize(st));
        const double fh = w->hdots[6], hh = w->hdots[7];
        double ga = 0.0, gb = 0.0, L = 1.0;
        if (hh > 0.0 && std::isfinite(hh) && std::isfinite(fh)) {
            // L = 1 - fh^2 / (hh c): the relative energy error of the best multiple of U_h
            L = 1.0 - fh * fh / (hh * c_star);
            ga = -2.0 * fh / (hh * c_star);
            gb = 2.0 * fh * fh / (hh * hh * c_star);
        }
        const long long V = (long long)w->D * w->H * w->W;
        kw_energy_grad<<<div_up(V, 256), 256, 0, st>>>(d, w->cg, g->F, w->KUh, g->fixed, ga, gb, gy);
        TOPO_CHECK_LAUNCH();
        grid_sync_out(g);
        if (loss) *loss = L;
    } catch (const topo::Error& e) {
        return api_fail(e.code, e.what());
    }
    return TO_OK;
}

}  // extern "C"
