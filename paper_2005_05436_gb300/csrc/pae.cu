// Periodic Anderson extrapolation of the OC fixed-point iteration (Sec. 3.6):
// the OC step is a fixed-point map x -> U(x) with residual r = U(x) - x on the
// active elements; from loop q0 on, the differences of x and r between
// consecutive design iterations are kept in m cyclic slots, and every q-th
// step (reading R23: when it + 1, it = loop - q0, is a multiple of q) the
// design jumps to x + zeta r - (X + zeta R) gamma, gamma minimising
// ||r - R gamma||_2 (normal equations, solved in FP64 by the last block of the
// Gram reduction); the other steps are x + alpha r. The result is clipped to
// [0, 1]; passive elements are not touched.
#include <cmath>

#include "grid.h"

namespace topo {

constexpr int PAE_MMAX = 4;
constexpr int PAE_NV = PAE_MMAX * (PAE_MMAX + 1) / 2 + PAE_MMAX;  // Gram entries + right-hand side

struct PaeWS {
    double *X = nullptr, *R = nullptr;        // [m][nEl] cyclic slots
    double *xold = nullptr, *rold = nullptr;  // previous x and r
    double *xprev = nullptr, *rcur = nullptr;  // this step's x before the OC and its residual
    double* gam = nullptr;                     // [m]
    int m = 0, filled = 0;
};

// r = U(x) - x; slot k receives x - xold and r - rold (it >= 1).
__global__ void k_pae_hist(long long n, const double* __restrict__ xprev, const double* __restrict__ xoc,
                           const int8_t* __restrict__ passive, const double* __restrict__ xold,
                           const double* __restrict__ rold, double* __restrict__ Xk, double* __restrict__ Rk,
                           double* __restrict__ rcur, int store) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool act = !passive || passive[i] == 0;
    const double r = act ? xoc[i] - xprev[i] : 0.0;
    rcur[i] = r;
    if (store) {
        Xk[i] = act ? xprev[i] - xold[i] : 0.0;
        Rk[i] = act ? r - rold[i] : 0.0;
    }
}

// G = R^T R, b = R^T r over the f filled slots; the last block solves G gamma = b
// by Gaussian elimination with partial pivoting (a pivot below 1e-14 of the
// largest diagonal entry marks the system singular: ok = 0).
__global__ void __launch_bounds__(256) k_pae_gram(long long n, const double* __restrict__ R, int f,
                                                  const double* __restrict__ r, double* __restrict__ gam, int* ok,
                                                  double* partials, unsigned* counter) {
    double v[PAE_NV], tot[PAE_NV];
#pragma unroll
    for (int k = 0; k < PAE_NV; ++k) v[k] = 0.0;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        double ra[PAE_MMAX];
#pragma unroll
        for (int a = 0; a < PAE_MMAX; ++a) ra[a] = a < f ? R[(long long)a * n + i] : 0.0;
        const double ri = r[i];
        int k = 0;
#pragma unroll
        for (int a = 0; a < PAE_MMAX; ++a) {
#pragma unroll
            for (int b = 0; b <= a; ++b) v[k++] += ra[a] * ra[b];
        }
#pragma unroll
        for (int a = 0; a < PAE_MMAX; ++a) v[k++] += ra[a] * ri;
    }
    if (last_block_totals<256, PAE_NV>(v, partials, counter, tot) && threadIdx.x == 0) {
        double G[PAE_MMAX][PAE_MMAX], b[PAE_MMAX];
        int k = 0;
        for (int a = 0; a < PAE_MMAX; ++a)
            for (int c = 0; c <= a; ++c) {
                G[a][c] = G[c][a] = tot[k];
                ++k;
            }
        for (int a = 0; a < PAE_MMAX; ++a) b[a] = tot[k++];
        double scale = 0.0;
        for (int a = 0; a < f; ++a) scale = fmax(scale, fabs(G[a][a]));
        scale = fmax(scale, 1e-300);
        int good = 1;
        for (int c = 0; c < f && good; ++c) {
            int piv = c;
            for (int i = c + 1; i < f; ++i)
                if (fabs(G[i][c]) > fabs(G[piv][c])) piv = i;
            if (!(fabs(G[piv][c]) > 1e-14 * scale)) {
                good = 0;
                break;
            }
            if (piv != c) {
                for (int j = 0; j < f; ++j) {
                    const double t = G[c][j];
                    G[c][j] = G[piv][j];
                    G[piv][j] = t;
                }
                const double t = b[c];
                b[c] = b[piv];
                b[piv] = t;
            }
            for (int i = c + 1; i < f; ++i) {
                const double fac = G[i][c] / G[c][c];
                for (int j = c; j < f; ++j) G[i][j] -= fac * G[c][j];
                b[i] -= fac * b[c];
            }
        }
        if (good) {
            for (int i = f - 1; i >= 0; --i) {
                double s = b[i];
                for (int j = i + 1; j < f; ++j) s -= G[i][j] * gam[j];
                gam[i] = s / G[i][i];
            }
        }
        *ok = good;
    }
}

// x = clip(x_prev + zeta r - (X + zeta R) gamma) when ok, else clip(x_prev + alpha r);
// then xold = x_prev, rold = r.
__global__ void k_pae_update(long long n, double* __restrict__ x, const double* __restrict__ xprev,
                             const double* __restrict__ rcur, const double* __restrict__ X,
                             const double* __restrict__ R, int f, const double* __restrict__ gam, const int* ok,
                             double alpha, double zeta, const int8_t* __restrict__ passive, double* __restrict__ xold,
                             double* __restrict__ rold) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xp = xprev[i], r = rcur[i];
    xold[i] = xp;
    rold[i] = r;
    if (passive && passive[i] != 0) return;
    double xn;
    if (ok && *ok) {
        double d = 0.0;
        for (int a = 0; a < f; ++a) d += (X[(long long)a * n + i] + zeta * R[(long long)a * n + i]) * gam[a];
        xn = xp + zeta * r - d;
    } else {
        xn = xp + alpha * r;
    }
    x[i] = fmin(fmax(xn, 0.0), 1.0);
}

static PaeWS* pae_ws(to_grid* g) {
    if (!g->pae) {
        PaeWS* w = new PaeWS();
        const long long n = g->d.nel;
        w->m = g->p.pae_m;
        for (double** p : {&w->xold, &w->rold, &w->xprev, &w->rcur}) TOPO_CUDA(cudaMalloc(p, n * sizeof(double)));
        TOPO_CUDA(cudaMalloc(&w->X, (size_t)w->m * n * sizeof(double)));
        TOPO_CUDA(cudaMalloc(&w->R, (size_t)w->m * n * sizeof(double)));
        TOPO_CUDA(cudaMalloc(&w->gam, PAE_MMAX * sizeof(double)));
        g->pae = w;
    }
    return (PaeWS*)g->pae;
}

void pae_free(to_grid* g) {
    PaeWS* w = (PaeWS*)g->pae;
    if (!w) return;
    for (double* p : {w->X, w->R, w->xold, w->rold, w->xprev, w->rcur, w->gam}) cudaFree(p);
    delete w;
    g->pae = nullptr;
}

void pae_before_oc(to_grid* g, const double* x, cudaStream_t st) {
    PaeWS* w = pae_ws(g);
    TOPO_CUDA(cudaMemcpyAsync(w->xprev, x, g->d.nel * sizeof(double), cudaMemcpyDeviceToDevice, st));
}

int pae_after_oc(to_grid* g, double* x, int it, cudaStream_t st) {
    PaeWS* w = pae_ws(g);
    const long long n = g->d.nel;
    const int m = w->m, q = g->p.pae_q;
    const int nb = div_up(n, 256);
    if (it == 0) w->filled = 0;
    const int slot = it >= 1 ? (it - 1) % m : 0;
    k_pae_hist<<<nb, 256, 0, st>>>(n, w->xprev, x, g->passive, w->xold, w->rold, w->X + (size_t)slot * n,
                                   w->R + (size_t)slot * n, w->rcur, it >= 1 ? 1 : 0);
    TOPO_CHECK_LAUNCH();
    if (it >= 1) w->filled = std::min(w->filled + 1, m);
    const bool extrapolate = it >= 1 && (it + 1) % q == 0;
    int* ok = nullptr;
    if (extrapolate) {
        ok = &g->ds->pae_ok;
        k_pae_gram<<<std::min(nb, 1024), 256, 0, st>>>(n, w->R, w->filled, w->rcur, w->gam, ok, g->partials,
                                                        g->counter);
        TOPO_CHECK_LAUNCH();
    }
    k_pae_update<<<nb, 256, 0, st>>>(n, x, w->xprev, w->rcur, w->X, w->R, w->filled, w->gam, ok, g->p.pae_alpha,
                                     g->p.pae_zeta, g->passive, w->xold, w->rold);
    TOPO_CHECK_LAUNCH();
    return extrapolate ? 2 : 1;
}

}  // namespace topo
