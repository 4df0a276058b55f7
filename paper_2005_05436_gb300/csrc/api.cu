// C ABI of the topopt CUDA path: the grid handle and the entry points declared
// in include/topopt.h. Host orchestration only; all arithmetic of the method
// runs in the kernels of kernels_ku.cu, kernels_design.cu and solver.cu.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "grid.h"

using namespace topo;

static thread_local std::string g_last_error;

static to_status fail(to_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

namespace topo {
to_status api_fail(to_status s, const std::string& msg) { return fail(s, msg); }
}  // namespace topo

#define TOPO_API_BEGIN try {
#define TOPO_API_END                                                  \
    }                                                                 \
    catch (const topo::Error& e) { return fail(e.code, e.what()); }  \
    catch (const std::bad_alloc&) { return fail(TO_ENOMEM, "host allocation failed"); } \
    catch (const std::exception& e) { return fail(TO_ECUDA, e.what()); } \
    return TO_OK;

namespace topo {

// Unit-element stiffness by Gauss quadrature (2x2 / 2x2x2 points): bilinear Q4 in
// plane stress, trilinear H8 isotropic; local node order of local_node().
void element_matrix(int dim, double nu, std::vector<double>& K) {
    const int nn = dim == 2 ? 4 : 8, D = dim * nn;
    K.assign((size_t)D * D, 0.0);
    int X[8][3];
    for (int M = 0; M < nn; ++M) {
        const int q = M & 3;
        X[M][0] = (q == 1 || q == 2) ? 1 : 0;
        X[M][1] = q >= 2 ? 1 : 0;
        X[M][2] = M >> 2;
    }
    double C[6][6] = {};
    int ns;
    if (dim == 2) {
        const double f = 1.0 / (1.0 - nu * nu);
        C[0][0] = C[1][1] = f;
        C[0][1] = C[1][0] = f * nu;
        C[2][2] = f * (1.0 - nu) / 2.0;
        ns = 3;
    } else {
        const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) C[a][b] = lam + (a == b ? 2.0 * mu : 0.0);
        C[3][3] = C[4][4] = C[5][5] = mu;
        ns = 6;
    }
    const double g[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
    const double w = 1.0 / (dim == 2 ? 4.0 : 8.0);
    const int npts = dim == 2 ? 4 : 8;
    std::vector<double> B((size_t)ns * D);
    for (int qp = 0; qp < npts; ++qp) {
        double xi[3] = {g[qp & 1], g[(qp >> 1) & 1], g[(qp >> 2) & 1]};
        std::fill(B.begin(), B.end(), 0.0);
        for (int M = 0; M < nn; ++M) {
            double G[3];
            for (int k = 0; k < dim; ++k) {
                double v = 1.0;
                for (int m = 0; m < dim; ++m) {
                    const double lin = X[M][m] ? xi[m] : 1.0 - xi[m];
                    v *= (m == k) ? (X[M][m] ? 1.0 : -1.0) : lin;
                }
                G[k] = v;
            }
            if (dim == 2) {
                B[0 * D + 2 * M] = G[0];
                B[1 * D + 2 * M + 1] = G[1];
                B[2 * D + 2 * M] = G[1];
                B[2 * D + 2 * M + 1] = G[0];
            } else {
                B[0 * D + 3 * M] = G[0];
                B[1 * D + 3 * M + 1] = G[1];
                B[2 * D + 3 * M + 2] = G[2];
                B[3 * D + 3 * M] = G[1];
                B[3 * D + 3 * M + 1] = G[0];
                B[4 * D + 3 * M + 1] = G[2];
                B[4 * D + 3 * M + 2] = G[1];
                B[5 * D + 3 * M] = G[2];
                B[5 * D + 3 * M + 2] = G[0];
            }
        }
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                double s = 0.0;
                for (int a = 0; a < ns; ++a)
                    for (int b = 0; b < ns; ++b) s += B[a * D + i] * C[a][b] * B[b * D + j];
                K[(size_t)i * D + j] += w * s;
            }
    }
}

void grid_sync_in(to_grid* g) {
    if (g->ust != g->st) {
        TOPO_CUDA(cudaEventRecord(g->ev_in, g->ust));
        TOPO_CUDA(cudaStreamWaitEvent(g->st, g->ev_in, 0));
    }
}
void grid_sync_out(to_grid* g) {
    if (g->ust != g->st) {
        TOPO_CUDA(cudaEventRecord(g->ev_out, g->st));
        TOPO_CUDA(cudaStreamWaitEvent(g->ust, g->ev_out, 0));
    }
}

template <typename T>
static T* dalloc(to_grid* g, size_t count) {
    void* p = nullptr;
    TOPO_CUDA(cudaMalloc(&p, count * sizeof(T) + 16));
    g->allocs.push_back(p);
    return (T*)p;
}

static void validate(const to_params* p) {
    TOPO_REQUIRE(p != nullptr, "params is NULL");
    TOPO_REQUIRE(p->dim == 2 || p->dim == 3, "dim must be 2 or 3");
    TOPO_REQUIRE(p->nelx >= 1 && p->nely >= 1, "nelx, nely must be >= 1");
    TOPO_REQUIRE(p->dim == 2 ? p->nelz == 0 : p->nelz >= 1, "nelz must be 0 in 2D and >= 1 in 3D");
    TOPO_REQUIRE(p->volfrac > 0.0 && p->volfrac < 1.0, "volfrac must be in (0, 1)");
    TOPO_REQUIRE(p->penal >= 1.0, "penal must be >= 1");
    TOPO_REQUIRE(p->rmin > 0.0 && p->rmin < 200.0, "rmin must be in (0, 200)");
    TOPO_REQUIRE(p->ft >= 1 && p->ft <= 3, "ft must be 1, 2 or 3");
    TOPO_REQUIRE(p->ftBC == 'N' || p->ftBC == 'D', "ftBC must be 'N' or 'D'");
    TOPO_REQUIRE(p->eta >= 0.0 && p->eta <= 1.0 && p->beta > 0.0, "eta in [0,1], beta > 0");
    TOPO_REQUIRE(p->move > 0.0 && p->move <= 1.0, "move must be in (0, 1]");
    TOPO_REQUIRE(p->E0 > p->Emin && p->Emin >= 0.0, "need E0 > Emin >= 0");
    TOPO_REQUIRE(p->nu > -1.0 && p->nu < 0.5, "nu must be in (-1, 0.5)");
    TOPO_REQUIRE(p->cg_rtol > 0.0 && p->cg_maxit >= 1, "cg_rtol > 0, cg_maxit >= 1");
    TOPO_REQUIRE(p->oc_tol > 0.0 && p->oc_maxit >= 1 && p->newton_tol > 0.0 && p->newton_maxit >= 0,
                 "tolerances must be positive");
    TOPO_REQUIRE(p->precision == TO_FP64 || p->precision == TO_MIXED, "precision");
    TOPO_REQUIRE(p->precond == TO_PC_JACOBI || p->precond == TO_PC_GMG, "precond");
    TOPO_REQUIRE(p->deadline_cycles > 0, "deadline_cycles must be > 0");
    TOPO_REQUIRE(p->inner_rtol > 0.0 && p->inner_rtol < 1.0, "inner_rtol must be in (0, 1)");
    TOPO_REQUIRE(p->mg_coarse_every >= 1 && p->mg_coarse_every <= 1000, "mg_coarse_every must be in [1, 1000]");
    TOPO_REQUIRE(p->mg_omega > 0.0 && p->mg_omega < 2.0 && p->mg_nu >= 1 && p->mg_nu <= 16,
                 "mg_omega in (0, 2), mg_nu in [1, 16]");
    TOPO_REQUIRE(p->mg_nu_fine >= 0 && p->mg_nu_fine <= 16, "mg_nu_fine must be in [0, 16]");
    TOPO_REQUIRE(p->mg_omega_coarse == 0.0 || (p->mg_omega_coarse > 0.0 && p->mg_omega_coarse < 2.0),
                 "mg_omega_coarse must be 0 or in (0, 2)");
    TOPO_REQUIRE(p->ku_impl >= 0 && p->ku_impl <= 4, "ku_impl must be 0, 1, 2, 3 or 4");
    TOPO_REQUIRE(p->pae_q0 >= 0 && p->pae_q >= 1 && p->pae_m >= 1 && p->pae_m <= 4 && p->pae_alpha > 0.0 &&
                     p->pae_alpha <= 1.0 && p->pae_zeta >= 0.0 && p->pae_zeta <= 1.0,
                 "Anderson extrapolation: pae_q0 >= 0, pae_q >= 1, pae_m in 1..4, pae_alpha in (0, 1], "
                 "pae_zeta in [0, 1]");
    TOPO_REQUIRE(p->inner_maxit >= 1, "inner_maxit must be >= 1");
    TOPO_REQUIRE(p->refine == TO_REFINE_RELIABLE || p->refine == TO_REFINE_FLEXIBLE,
                 "refine must be TO_REFINE_RELIABLE or TO_REFINE_FLEXIBLE");
    TOPO_REQUIRE(p->oc_method == TO_OC_BISECTION || p->oc_method == TO_OC_PRIMAL_DUAL ||
                     p->oc_method == TO_OC_PHYSICAL_VOLUME,
                 "oc_method must be TO_OC_BISECTION, TO_OC_PRIMAL_DUAL or TO_OC_PHYSICAL_VOLUME");
    TOPO_REQUIRE(!(p->ku_impl == 2 && p->dim != 3), "the tensor-core operator is 3D only");
    const long long nnodes = (long long)(p->nelx + 1) * (p->nely + 1) * (p->dim == 3 ? p->nelz + 1 : 1);
    TOPO_REQUIRE(nnodes * p->dim < (1LL << 31) - 1, "grid too large for 32-bit DOF indices");
}

}  // namespace topo

extern "C" {

const char* to_last_error(void) { return g_last_error.c_str(); }
size_t to_sizeof_params(void) { return sizeof(to_params); }
size_t to_sizeof_state(void) { return sizeof(to_state); }
size_t to_sizeof_iter_info(void) { return sizeof(to_iter_info); }

to_status to_params_init(to_params* p, int32_t dim, int32_t nelx, int32_t nely, int32_t nelz) {
    if (!p) return fail(TO_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->dim = dim;
    p->nelx = nelx;
    p->nely = nely;
    p->nelz = dim == 3 ? nelz : 0;
    p->E0 = 1.0;
    p->Emin = 1e-9;
    p->nu = 0.3;
    p->volfrac = 0.5;
    p->penal = 3.0;
    p->rmin = dim == 3 ? std::sqrt(3.0) : 1.5;
    p->ft = 3;
    p->ftBC = 'N';
    p->eta = 0.5;
    p->beta = 2.0;
    p->move = 0.2;
    p->penal_cnt = to_continuation{1, 25, 3.0, 0.25, TO_CNT_ADD, 0};
    p->beta_cnt = to_continuation{1, 25, 2.0, 2.0, TO_CNT_ADD, 0};
    p->newton_tol = 1e-6;
    p->newton_maxit = 50;
    p->oc_maxit = 200;
    p->oc_tol = 1e-4;
    p->cg_rtol = 1e-8;
    p->cg_maxit = 20000;
    p->precision = TO_FP64;
    p->precond = TO_PC_JACOBI;
    p->mg_levels = 0;
    p->deadline_cycles = 2000000000LL;
    p->inner_rtol = 1e-3;
    p->mg_omega = 1.8;
    p->mg_nu = 2;
    p->mg_coarse_every = 1;
    p->oc_method = TO_OC_BISECTION;
    p->pae_q0 = 0;
    p->pae_q = 4;
    p->pae_m = 4;
    p->pae_alpha = 0.9;
    p->pae_zeta = 1.0;
    p->inner_maxit = 2000;
    p->refine = TO_REFINE_RELIABLE;
    return TO_OK;
}

to_status to_init_grid(const to_params* p, const double* F, const uint8_t* fixed, const int8_t* passive,
                       void* stream, to_grid** out) {
    if (!out) return fail(TO_EINVAL, "out is NULL");
    *out = nullptr;
    to_grid* g = nullptr;
    TOPO_API_BEGIN
    validate(p);
    TOPO_REQUIRE(F && fixed, "F and fixed must be device pointers");
    g = new to_grid();
    g->p = *p;
    g->d = make_dims(p->dim, p->nelx, p->nely, p->nelz);
    g->ust = (cudaStream_t)stream;
    TOPO_CUDA(cudaGetDevice(&g->dev));
    TOPO_CUDA(cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, g->dev));
    // Work goes on the caller's stream; a private stream is made only for the
    // legacy default stream (NULL), which cannot be captured into CUDA graphs.
    if (g->ust) {
        g->st = g->ust;
    } else {
        TOPO_CUDA(cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking));
        g->own_stream = true;
    }
    TOPO_CUDA(cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming));
    TOPO_CUDA(cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming));
    for (int i = 0; i < 5; ++i) TOPO_CUDA(cudaEventCreate(&g->ev_t[i]));
    grid_sync_in(g);
    const Dims& d = g->d;
    g->penal = p->penal;
    g->beta = p->beta;
    g->eta = p->eta;

    // Ke (Appendix B/C element matrices, by quadrature)
    std::vector<double> K;
    element_matrix(d.dim, p->nu, K);
    const int D = d.dim == 2 ? 8 : 24;
    for (int i = 0; i < D * D; ++i) {
        if (D == 24) {
            g->ke3.k[i] = K[i];
            g->ke3f.k[i] = (float)K[i];
        } else {
            g->ke2.k[i] = K[i];
            g->ke2f.k[i] = (float)K[i];
        }
    }
    if (D == 24) {
        double dev = 0.0;
        if (!walsh_constants(K.data(), g->wk, &dev))
            throw std::runtime_error("element matrix is not block diagonal in the Walsh basis (deviation " +
                                     std::to_string(dev) + ")");
        const WalshK<double>& w = g->wk;
        g->wkf = WalshK<float>{(float)w.amb, (float)w.b, (float)w.c, (float)w.d,
                               (float)w.f, (float)w.g, (float)w.pmq, (float)w.q};
    }
    g->node_centric = p->ku_impl == 1;
    if (d.dim == 3 && p->ku_impl == 4) {
        TOPO_REQUIRE(walsh_pair_supported(d), "no element-pair tile shape fits this grid (ku_impl 4)");
        g->walsh_pair = true;
    }
    g->Ke_host = K;
    g->Ke_dev = dalloc<double>(g, K.size());
    TOPO_CUDA(cudaMemcpyAsync(g->Ke_dev, K.data(), K.size() * sizeof(double), cudaMemcpyHostToDevice, g->st));
    if (p->precision == TO_MIXED && d.dim == 3) {
        std::vector<float> pack;
        tc_pack_ke(K, pack);
        g->ke_tc = dalloc<float>(g, pack.size());
        TOPO_CUDA(cudaMemcpy(g->ke_tc, pack.data(), pack.size() * sizeof(float), cudaMemcpyHostToDevice));
        g->tc_err = dalloc<int>(g, 1);
        TOPO_CUDA(cudaMemset(g->tc_err, 0, sizeof(int)));
        g->use_tc = p->ku_impl == 2;  // auto: the CUDA-core operator (faster so far)
    }

    // problem data
    g->F = dalloc<double>(g, d.ndof);
    g->fixed = dalloc<uint8_t>(g, d.ndof);
    TOPO_CUDA(cudaMemcpyAsync(g->F, F, d.ndof * sizeof(double), cudaMemcpyDeviceToDevice, g->st));
    TOPO_CUDA(cudaMemcpyAsync(g->fixed, fixed, d.ndof, cudaMemcpyDeviceToDevice, g->st));
    std::vector<int8_t> pas_h(d.nel, 0);
    g->passive = nullptr;
    if (passive) {
        g->passive = dalloc<int8_t>(g, d.nel);
        TOPO_CUDA(cudaMemcpyAsync(g->passive, passive, d.nel, cudaMemcpyDeviceToDevice, g->st));
        TOPO_CUDA(cudaMemcpyAsync(pas_h.data(), passive, d.nel, cudaMemcpyDeviceToHost, g->st));
        TOPO_CUDA(cudaStreamSynchronize(g->st));
    }
    g->nsolid = g->nvoid = 0;
    for (long long e = 0; e < d.nel; ++e) {
        TOPO_REQUIRE(pas_h[e] >= -1 && pas_h[e] <= 1, "passive values must be -1, 0 or 1");
        g->nsolid += pas_h[e] == 1;
        g->nvoid += pas_h[e] == -1;
    }
    g->nact = d.nel - g->nsolid - g->nvoid;
    TOPO_REQUIRE(g->nact > 0, "no active elements");

    // filter taps (Eq. 2): offsets -ceil(rmin)+1 .. ceil(rmin)-1, cone weights
    {
        const int R = (int)std::ceil(p->rmin) - 1;
        std::vector<int> off;
        std::vector<double> w;
        std::vector<float> wf;
        double wsum = 0.0;
        const int Rz = d.dim == 3 ? R : 0;
        for (int ox = -R; ox <= R; ++ox)
            for (int oz = -Rz; oz <= Rz; ++oz)
                for (int oy = -R; oy <= R; ++oy) {
                    const double wt = std::fmax(0.0, p->rmin - std::sqrt((double)(ox * ox + oy * oy + oz * oz)));
                    if (wt <= 0.0) continue;
                    off.push_back(ox);
                    off.push_back(oy);
                    off.push_back(oz);
                    w.push_back(wt);
                    wf.push_back((float)wt);
                    wsum += wt;
                }
        g->taps.nw = (int)w.size();
        int* doff = dalloc<int>(g, off.size());
        double* dw = dalloc<double>(g, w.size());
        float* dwf = dalloc<float>(g, wf.size());
        TOPO_CUDA(cudaMemcpyAsync(doff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, g->st));
        TOPO_CUDA(cudaMemcpyAsync(dw, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, g->st));
        TOPO_CUDA(cudaMemcpyAsync(dwf, wf.data(), wf.size() * sizeof(float), cudaMemcpyHostToDevice, g->st));
        TOPO_CUDA(cudaStreamSynchronize(g->st));  // host vectors go out of scope
        g->taps.off = doff;
        g->taps.w = dw;
        g->taps.wf = dwf;
        g->Hs_const = wsum;
        g->rHs_const = 1.0 / wsum;
        // the same window as rows along x, padded to whole chunks (tiled filter)
        std::vector<int> rows;
        std::vector<double> rw;
        std::vector<float> rwh, rwl;
        for (int oz = -Rz; oz <= Rz; ++oz)
            for (int oy = -R; oy <= R; ++oy) {
                int dmax = -1;
                for (int ox = 0; ox <= R; ++ox)
                    if (p->rmin - std::sqrt((double)(ox * ox + oy * oy + oz * oz)) > 0.0) dmax = ox;
                if (dmax < 0) continue;
                const int nch = (2 * dmax + 1 + FILTER_K - 1) / FILTER_K;
                rows.insert(rows.end(), {oy, oz, -dmax, nch});
                for (int i = 0; i < nch * FILTER_K; ++i) {
                    const int ox = -dmax + i;
                    const double wt =
                        ox <= dmax ? std::fmax(0.0, p->rmin - std::sqrt((double)(ox * ox + oy * oy + oz * oz))) : 0.0;
                    rw.push_back(wt);
                    const float h = (float)wt;
                    rwh.push_back(h);
                    rwl.push_back((float)(wt - (double)h));
                }
            }
        g->taps.R = R;
        g->taps.Rz = Rz;
        g->taps.nrows = (int)rows.size() / 4;
        int* drows = dalloc<int>(g, rows.size());
        double* drw = dalloc<double>(g, rw.size());
        float* drwh = dalloc<float>(g, rw.size());
        float* drwl = dalloc<float>(g, rw.size());
        TOPO_CUDA(cudaMemcpyAsync(drows, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice, g->st));
        TOPO_CUDA(cudaMemcpyAsync(drw, rw.data(), rw.size() * sizeof(double), cudaMemcpyHostToDevice, g->st));
        TOPO_CUDA(cudaMemcpyAsync(drwh, rwh.data(), rwh.size() * sizeof(float), cudaMemcpyHostToDevice, g->st));
        TOPO_CUDA(cudaMemcpyAsync(drwl, rwl.data(), rwl.size() * sizeof(float), cudaMemcpyHostToDevice, g->st));
        TOPO_CUDA(cudaStreamSynchronize(g->st));
        g->taps.rows = drows;
        g->taps.rw = drw;
        g->taps.rwh = drwh;
        g->taps.rwl = drwl;
    }

    // workspaces
    g->E = dalloc<double>(g, d.nel);
    g->Ef = dalloc<float>(g, d.nel);
    g->xt = dalloc<double>(g, d.nel);
    g->dprj = dalloc<double>(g, d.nel);
    g->dc = dalloc<double>(g, d.nel);
    g->dcf = dalloc<double>(g, d.nel);
    g->dV = dalloc<double>(g, d.nel);
    g->dV0 = dalloc<double>(g, d.nel);
    g->ocp = dalloc<double>(g, d.nel);
    for (int i = 0; i < 7; ++i) g->v[i] = dalloc<double>(g, d.ndof);
    g->Hs = nullptr;
    if (p->ftBC == 'D') {
        g->Hs = dalloc<double>(g, d.nel);
        launch_fill(d.nel, g->dc, 1.0, g->st);
        launch_filter(d, g->taps, 'D', nullptr, 1.0, g->dc, nullptr, g->Hs, nullptr, nullptr, g->st);
        g->rHs = dalloc<double>(g, d.nel);
        launch_recip(d.nel, g->Hs, g->rHs, g->st);
    }
    g->proj_blocks = project_max_blocks();
    g->oc_blocks = oc_max_blocks();
    const long long pn = std::max<long long>(std::initializer_list<long long>
        {d.nnodes / 256 + 2, d.nel / 256 + 2, 4096, 2LL * 16 * std::max(g->proj_blocks, g->oc_blocks)});
    g->partials = dalloc<double>(g, pn * 4);
    g->npartials = pn * 4;
    g->counter = dalloc<unsigned>(g, 16);
    TOPO_CUDA(cudaMemsetAsync(g->counter, 0, 16 * sizeof(unsigned), g->st));
    g->bar = dalloc<GridBarrier>(g, 1);
    g->ds = dalloc<DevScalars>(g, 1);
    TOPO_CUDA(cudaMemsetAsync(g->ds, 0, sizeof(DevScalars), g->st));
    TOPO_CUDA(cudaMallocHost(&g->hs, sizeof(DevScalars)));
    solver_init(g);
    TOPO_CUDA(cudaStreamSynchronize(g->st));
    grid_sync_out(g);
    *out = g;
    g = nullptr;
    }
    catch (const topo::Error& e) {
        if (g) to_destroy(g);
        return fail(e.code, e.what());
    }
    catch (const std::exception& e) {
        if (g) to_destroy(g);
        return fail(TO_ECUDA, e.what());
    }
    return TO_OK;
}

void to_destroy(to_grid* g) {
    if (!g) return;
    if (g->st) cudaStreamSynchronize(g->st);
    solver_free(g);
    warm_free(g);
    pae_free(g);
    for (void* p : g->allocs) cudaFree(p);
    if (g->hs) cudaFreeHost(g->hs);
    if (g->ev_in) cudaEventDestroy(g->ev_in);
    if (g->ev_out) cudaEventDestroy(g->ev_out);
    for (int i = 0; i < 5; ++i)
        if (g->ev_t[i]) cudaEventDestroy(g->ev_t[i]);
    if (g->st && g->own_stream) cudaStreamDestroy(g->st);
    delete g;
}

to_status to_set_scalars(to_grid* g, double penal, double beta, double eta) {
    if (!g) return fail(TO_EINVAL, "grid is NULL");
    if (!(penal >= 1.0 && beta > 0.0 && eta >= 0.0 && eta <= 1.0)) return fail(TO_EINVAL, "bad scalars");
    g->penal = penal;
    g->beta = beta;
    g->eta = eta;
    return TO_OK;
}

to_status to_apply_K(to_grid* g, const double* xPhys, const double* u, double* y, int32_t masked) {
    if (!g || !xPhys || !u || !y) return fail(TO_EINVAL, "NULL argument");
    if (u == y) return fail(TO_EINVAL, "y must not alias u");
    TOPO_API_BEGIN
    grid_sync_in(g);
    const Dims& d = g->d;
    launch_modulus<double>(d.nel, xPhys, g->penal, g->p.E0, g->p.Emin, g->E, g->st);
    const double* src = u;
    if (masked) {
        launch_mask_copy(d.ndof, u, g->v[6], g->fixed, g->st);
        src = g->v[6];
    }
    launch_apply_K<double>(d, g->ke3, g->ke2, g->wk, g->node_centric, g->E, src, y, g->fixed, masked != 0,
                           g->st);
    grid_sync_out(g);
    TOPO_API_END
}

to_status to_filter(to_grid* g, const double* in, double* out, const double* dprj) {
    if (!g || !in || !out) return fail(TO_EINVAL, "NULL argument");
    if (in == out) return fail(TO_EINVAL, "out must not alias in");
    TOPO_API_BEGIN
    grid_sync_in(g);
    launch_filter(g->d, g->taps, (char)g->p.ftBC, g->rHs, g->rHs_const, in, dprj, out, nullptr, nullptr, g->st,
                  g->p.precision == TO_MIXED);
    grid_sync_out(g);
    TOPO_API_END
}

to_status to_project(to_grid* g, const double* xTilde, double* xPhys, double* dprj, double* eta_inout,
                     int32_t volume_preserving) {
    if (!g || !xTilde || !xPhys || !dprj || !eta_inout) return fail(TO_EINVAL, "NULL argument");
    TOPO_API_BEGIN
    grid_sync_in(g);
    DevScalars* ds = g->ds;
    launch_project(g->d.nel, xTilde, xPhys, dprj, g->beta, *eta_inout, g->p.volfrac, volume_preserving,
                   g->p.newton_tol, g->p.newton_maxit, g->p.deadline_cycles, g->partials, g->bar,
                   &ds->po, g->proj_blocks, g->st);
    TOPO_CUDA(cudaMemcpyAsync(g->hs, ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, g->st));
    TOPO_CUDA(cudaMemcpyAsync(&g->hbar, g->bar, sizeof(GridBarrier), cudaMemcpyDeviceToHost, g->st));
    TOPO_CUDA(cudaStreamSynchronize(g->st));
    grid_sync_out(g);
    if (g->hbar.error) return fail(TO_ETIMEOUT, "projection: grid barrier deadline passed");
    *eta_inout = g->hs->po.eta;
    if (g->hs->po.status) return fail((to_status)g->hs->po.status, "projection: eta search did not converge");
    TOPO_API_END
}

to_status to_sensitivity(to_grid* g, const double* xPhys, const double* U, double* dc, double* c_out) {
    if (!g || !xPhys || !U || !dc) return fail(TO_EINVAL, "NULL argument");
    TOPO_API_BEGIN
    grid_sync_in(g);
    launch_sensitivity(g->d, g->ke3, g->ke2, g->wk, g->node_centric, xPhys, U, g->passive, g->penal, g->p.E0, g->p.Emin, dc,
                       &g->ds->esum, g->partials, g->counter, g->st);
    if (c_out) {
        launch_dot(g->d.ndof, g->F, U, &g->ds->c, g->partials, g->counter, g->st);
        TOPO_CUDA(cudaMemcpyAsync(g->hs, g->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, g->st));
        TOPO_CUDA(cudaStreamSynchronize(g->st));
        *c_out = g->hs->c;
    }
    grid_sync_out(g);
    TOPO_API_END
}

// Stop test of the OC search: the relative bracket width oc_tol (bisection) or
// the absolute change 1e-10 of sqrt(lambda) between primal-dual iterates.
static double oc_tol_of(const to_params& p) { return p.oc_method == TO_OC_PRIMAL_DUAL ? 1e-10 : p.oc_tol; }

to_status to_oc_update(to_grid* g, double* x, const double* dc, const double* dV0, double* lm_out) {
    if (!g || !x || !dc || !dV0) return fail(TO_EINVAL, "NULL argument");
    TOPO_API_BEGIN
    grid_sync_in(g);
    if (g->p.oc_method == TO_OC_PHYSICAL_VOLUME) {
        TOPO_CUDA(cudaMemsetAsync(g->bar, 0, sizeof(GridBarrier), g->st));
        launch_oc_filtered(g->d, g->taps, (char)g->p.ftBC, g->rHs, g->rHs_const, x, dc, dV0, g->passive, g->nact,
                           g->p.move, g->p.volfrac, g->p.ft, g->eta, nullptr, g->beta, g->p.oc_tol, g->p.oc_maxit, g->ocp,
                           g->dV, g->dc, &g->ds->ocf, &g->hs->ocf, g->partials, g->counter, &g->ds->oo, g->st);
    } else {
        launch_oc(g->d.nel, x, dc, dV0, g->passive, g->nact, g->p.move, g->p.volfrac, oc_tol_of(g->p),
                  g->p.oc_maxit, g->p.deadline_cycles, g->ocp, g->partials, g->bar, &g->ds->oo,
                  g->oc_blocks, g->st, g->p.oc_method);
    }
    TOPO_CUDA(cudaMemcpyAsync(g->hs, g->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, g->st));
    TOPO_CUDA(cudaMemcpyAsync(&g->hbar, g->bar, sizeof(GridBarrier), cudaMemcpyDeviceToHost, g->st));
    TOPO_CUDA(cudaStreamSynchronize(g->st));
    grid_sync_out(g);
    if (g->hbar.error) return fail(TO_ETIMEOUT, "OC: grid barrier deadline passed");
    if (lm_out) *lm_out = g->hs->oo.lm;
    if (g->hs->oo.status != TO_OK)
        return fail(TO_ENOTCONV, "OC: the multiplier search stopped at oc_maxit before meeting oc_tol "
                                 "(x holds the last candidate)");
    TOPO_API_END
}

to_status to_solve(to_grid* g, const double* xPhys, const double* F, double* U, to_solve_info* info) {
    if (!g || !xPhys || !U) return fail(TO_EINVAL, "NULL argument");
    to_solve_info si{};
    to_status st = TO_OK;
    TOPO_API_BEGIN
    grid_sync_in(g);
    solver_discard_setup(g);
    launch_modulus<double>(g->d.nel, xPhys, g->penal, g->p.E0, g->p.Emin, g->E, g->st);
    st = solve_state(g, F ? F : g->F, U, &si);
    grid_sync_out(g);
    if (info) *info = si;
    if (st != TO_OK) return fail(st, "state solve did not reach cg_rtol");
    TOPO_API_END
}

to_status to_assemble_lower(to_grid* g, const double* xPhys, int64_t* nnz, int32_t* row_ptr, int32_t* col,
                            double* val) {
    if (!g || !nnz) return fail(TO_EINVAL, "NULL argument");
    TOPO_API_BEGIN
    grid_sync_in(g);
    const Dims& d = g->d;
    int32_t* counts = (int32_t*)g->v[0];  // ndof int32 fit in ndof doubles
    int32_t* rp = row_ptr ? row_ptr : (int32_t*)g->v[3];  // ndof + 1 int32 fit as well
    if (!g->scan_tmp) {
        TOPO_CUDA(cudaMalloc(&g->scan_tmp, scan_tmp_size(d.ndof)));
        g->allocs.push_back(g->scan_tmp);
    }
    void* tmp = g->scan_tmp;
    launch_lower_row_counts(d, counts, g->st);
    launch_exclusive_scan(counts, rp, d.ndof, tmp, &g->ds->nnz, g->st);
    TOPO_CUDA(cudaMemcpyAsync(g->hs, g->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, g->st));
    TOPO_CUDA(cudaStreamSynchronize(g->st));
    const long long total = g->hs->nnz;
    TOPO_REQUIRE(total < (1LL << 31), "nnz exceeds int32 indices");
    if (val) {
        TOPO_REQUIRE(row_ptr && col && xPhys, "row_ptr, col and xPhys required when val != NULL");
        TOPO_REQUIRE(*nnz >= total, "nnz capacity too small");
        launch_modulus<double>(d.nel, xPhys, g->penal, g->p.E0, g->p.Emin, g->E, g->st);
        launch_lower_fill_dev(d, g->Ke_dev, g->E, row_ptr, col, val, g->st);
    }
    *nnz = total;
    grid_sync_out(g);
    TOPO_API_END
}

to_status to_step(to_grid* g, to_state* s, to_iter_info* info) {
    if (!g || !s || !s->x || !s->xPhys || !s->xOld || !s->U) return fail(TO_EINVAL, "NULL argument");
    to_iter_info it{};
    TOPO_API_BEGIN
    grid_sync_in(g);
    solver_discard_setup(g);
    const Dims& d = g->d;
    const to_params& p = g->p;
    cudaStream_t st = g->st;
    g->penal = s->penal;
    g->beta = s->beta;
    g->eta = s->eta;
    s->loop += 1;
    TOPO_CUDA(cudaEventRecord(g->ev_t[0], st));
    // RL.1 physical density: xPhys(act) = xTilde(act), passive keep x
    const bool ffilt = p.precision == TO_MIXED;  // the mixed path filters in float-float arithmetic
    launch_filter(d, g->taps, (char)p.ftBC, g->rHs, g->rHs_const, s->x, nullptr, g->xt, g->passive, s->x, st,
                  ffilt);
    if (p.ft > 1) {
        launch_project(d.nel, g->xt, s->xPhys, g->dprj, s->beta, s->eta, p.volfrac, p.ft == 3,
                       p.newton_tol, p.newton_maxit, p.deadline_cycles, g->partials, g->bar,
                       &g->ds->po, g->proj_blocks, st);
    } else {
        TOPO_CUDA(cudaMemcpyAsync(s->xPhys, g->xt, d.nel * sizeof(double), cudaMemcpyDeviceToDevice, st));
        launch_fill(d.nel, g->dprj, 1.0, st);
    }
    launch_change(d.nel, s->xPhys, s->xOld, g->ds->change, 1, g->partials, g->counter, st);
    TOPO_CUDA(cudaEventRecord(g->ev_t[1], st));
    // RL.2 modulus and state solve (warm start from s->U)
    launch_modulus<double>(d.nel, s->xPhys, s->penal, p.E0, p.Emin, g->E, st);
    double wen[2] = {0.0, 0.0};
    if (g->net) {
        double coef[2] = {1.0, 0.0}, wms = 0.0;
        double wres[2] = {0.0, 0.0};
        learned_warm_start(g, s->xPhys, s->U, coef, &wms, wen, wres);
        it.warm_a = coef[0];
        it.warm_b = coef[1];
        it.t_warm_ms = wms;
        it.warm_res_prev = wres[0];
        it.warm_res = wres[1];
    }
    to_solve_info si{};
    const to_status sst = solve_state(g, g->F, s->U, &si);
    TOPO_CUDA(cudaEventRecord(g->ev_t[2], st));
    // RL.3 sensitivities and chain rule through projection and filter
    launch_sensitivity(d, g->ke3, g->ke2, g->wk, g->node_centric, s->xPhys, s->U, g->passive, s->penal, p.E0, p.Emin, g->dc,
                       &g->ds->esum, g->partials, g->counter, st);
    launch_dot(d.ndof, g->F, s->U, &g->ds->c, g->partials, g->counter, st);
    launch_dv(d.nel, g->passive, 1.0 / ((double)d.nel * p.volfrac), g->dV, st);
    launch_filter(d, g->taps, (char)p.ftBC, g->rHs, g->rHs_const, g->dc, g->dprj, g->dcf, nullptr, nullptr, st,
                  ffilt);
    launch_filter(d, g->taps, (char)p.ftBC, g->rHs, g->rHs_const, g->dV, g->dprj, g->dV0, nullptr, nullptr, st,
                  ffilt);
    TOPO_CUDA(cudaEventRecord(g->ev_t[3], st));
    // RL.4 OC update
    const bool pae_on = p.pae_q0 > 0 && s->loop >= p.pae_q0;
    if (pae_on) pae_before_oc(g, s->x, st);
    if (p.oc_method == TO_OC_PHYSICAL_VOLUME) {
        // the physical field of each candidate, with the step's threshold and sharpness
        launch_oc_filtered(d, g->taps, (char)p.ftBC, g->rHs, g->rHs_const, s->x, g->dcf, g->dV0, g->passive, g->nact,
                           p.move, p.volfrac, p.ft, s->eta, p.ft == 3 ? &g->ds->po.eta : nullptr, s->beta, p.oc_tol,
                           p.oc_maxit, g->ocp, g->dV, g->dc,
                           &g->ds->ocf, &g->hs->ocf, g->partials, g->counter, &g->ds->oo, st);
    } else {
        launch_oc(d.nel, s->x, g->dcf, g->dV0, g->passive, g->nact, p.move, p.volfrac, oc_tol_of(p), p.oc_maxit,
                  p.deadline_cycles, g->ocp, g->partials, g->bar, &g->ds->oo, g->oc_blocks, st, p.oc_method);
    }
    const int pae_kind = pae_on ? pae_after_oc(g, s->x, s->loop - p.pae_q0, st) : 0;
    TOPO_CUDA(cudaEventRecord(g->ev_t[4], st));
    TOPO_CUDA(cudaMemcpyAsync(g->hs, g->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
    TOPO_CUDA(cudaMemcpyAsync(&g->hbar, g->bar, sizeof(GridBarrier), cudaMemcpyDeviceToHost, st));
    TOPO_CUDA(cudaStreamSynchronize(st));
    const DevScalars& h = *g->hs;
    if (g->hbar.error) return fail(TO_ETIMEOUT, "design step: grid barrier deadline passed");
    it.loop = s->loop;
    it.n_cg = si.iters;
    it.n_refine = si.refinements;
    it.fallback = si.fallback;
    it.rel_res = si.rel_res;
    it.c = h.c;
    if (g->net && h.c > 0.0) {  // energy errors relative to the zero start: (E(U) - E*) / (-E*), E* = -c / 2
        it.warm_err_prev = (wen[0] + 0.5 * h.c) / (0.5 * h.c);
        it.warm_err = (wen[1] + 0.5 * h.c) / (0.5 * h.c);
    }
    it.V = h.change[1] / (double)d.nel;
    it.ch = std::sqrt(h.change[0]) / std::sqrt((double)d.nel);
    if (p.ft > 1) {
        s->eta = h.po.eta;
        it.n_newton = h.po.newton;
    }
    it.lm = h.oo.lm;
    it.pae = pae_kind == 2 ? (h.pae_ok ? 2 : 1) : pae_kind;
    it.n_bisect = h.oo.steps;
    float ms[4];
    for (int i = 0; i < 4; ++i) TOPO_CUDA(cudaEventElapsedTime(&ms[i], g->ev_t[i], g->ev_t[i + 1]));
    it.t_filter_ms = ms[0];
    it.t_solve_ms = ms[1];
    it.t_setup_ms = si.t_setup_ms;
    it.t_krylov_ms = si.t_krylov_ms;
    it.t_resid_ms = si.t_resid_ms;
    it.t_sens_ms = ms[2];
    it.t_oc_ms = ms[3];
    // continuation (Sec. 3), post-increment loop counter
    auto cnt = [&](double v, const to_continuation& c) {
        if (s->loop >= c.istart && v < c.maxpar && c.isteps > 0 && s->loop % c.isteps == 0)
            v = c.kind == TO_CNT_MUL ? std::fmin(c.maxpar, v * c.delta) : v + c.delta;
        return v;
    };
    s->penal = cnt(s->penal, p.penal_cnt);
    s->beta = cnt(s->beta, p.beta_cnt);
    g->penal = s->penal;
    g->beta = s->beta;
    g->eta = s->eta;
    it.penal = s->penal;
    it.beta = s->beta;
    it.eta = s->eta;
    it.status = (int)sst;
    if (it.status == TO_OK && h.oo.status != TO_OK) it.status = TO_ENOTCONV;
    if (!std::isfinite(it.c)) it.status = TO_ENAN;
    grid_sync_out(g);
    if (info) *info = it;
    if (it.status == TO_ENAN) return fail(TO_ENAN, "compliance is not finite");
    if (sst != TO_OK) return fail(sst, "state solve did not reach cg_rtol");
    if (h.oo.status != TO_OK)
        return fail(TO_ENOTCONV, "OC: the multiplier search stopped at oc_maxit before meeting oc_tol");
    TOPO_API_END
}

}  // extern "C"
