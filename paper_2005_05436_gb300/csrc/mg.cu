// Geometric multigrid: fine-level fused operators, Galerkin coarsening, node
// stencils, transfer operators, coarsest dense inverse and the V-cycle.
#include <cstdlib>
#include <algorithm>
#include <cmath>

#include "grid.h"
#include "ku_device.cuh"
#include "mg.h"

namespace topo {

// Operators take displacements relative to the centre node (see ku_device.cuh).
template <typename T>
__host__ __device__ constexpr bool rel_form() { return true; }

// ------------------------------------------------------ fine level (matrix-free)

template <typename T, int MODE, bool PCG>
__global__ void __launch_bounds__(256) k_fine_op3(Dims d, const KeP<T, 24> ke, const T* __restrict__ E,
                                                  const T* __restrict__ u, const T* __restrict__ r,
                                                  const T* __restrict__ dinv, T* __restrict__ out,
                                                  const uint8_t* __restrict__ fixed, T omega,
                                                  const int* skip, PcgScalars* pcg, double* partials,
                                                  unsigned* counter) {
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested before the stores, so its load overlaps the others
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = n < d.nnodes;
    DotAcc<T> dot;
    // the epilogue's operands depend on nothing computed here: fetched first
    T r_i[3], d_i[3], u_i[3];
    unsigned f_i[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long i = 3 * n + c;
        r_i[c] = (MODE != 0 && in) ? r[i] : T(0);
        d_i[c] = (MODE == 1 && in) ? dinv[i] : T(0);
        u_i[c] = ((MODE == 1 || PCG) && in) ? u[i] : T(0);
        f_i[c] = in ? (unsigned)fixed[i] : 0u;
    }
    T a[3] = {};
    if (in) ku3_node_clamped<T>(ke, E, u, (int)n, d, a[0], a[1], a[2]);  // register-cached, branch-free
    if (sk) return;
    if (in) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long i = 3 * n + c;
            T o = a[c];
            if (MODE == 1) o = u_i[c] + omega * d_i[c] * (r_i[c] - a[c]);
            if (MODE == 2) o = r_i[c] - a[c];
            if (f_i[c]) o = T(0);
            out[i] = o;
            if (PCG) dot.add(MODE == 1 ? r_i[c] : u_i[c], o);
        }
    }
    if (PCG) {
        double v[1] = {dot.value()}, tot[1];
        if (last_block_totals<256, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
            if (MODE == 1) {  // last V-cycle sweep: rz = r.z, beta = rz / rz_old
                pcg->beta = tot[0] / pcg->rz;
                pcg->rz = tot[0];
            } else {          // K p: alpha = rz / p.Ap
                pcg->pAp = tot[0];
                pcg->alpha = pcg->rz / tot[0];
            }
        }
    }
}

template <typename T, int MODE, bool PCG>
__global__ void __launch_bounds__(256) k_fine_op2(Dims d, const KeP<T, 8> ke, const T* __restrict__ E,
                                                  const T* __restrict__ u, const T* __restrict__ r,
                                                  const T* __restrict__ dinv, T* __restrict__ out,
                                                  const uint8_t* __restrict__ fixed, T omega,
                                                  const int* skip, PcgScalars* pcg, double* partials,
                                                  unsigned* counter) {
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested before the stores, so its load overlaps the others
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = n < d.nnodes;
    DotAcc<T> dot;
    // the epilogue's operands depend on nothing computed here: fetched first
    T r_i[2], d_i[2], u_i[2];
    unsigned f_i[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const long long i = 2 * n + c;
        r_i[c] = (MODE != 0 && in) ? r[i] : T(0);
        d_i[c] = (MODE == 1 && in) ? dinv[i] : T(0);
        u_i[c] = ((MODE == 1 || PCG) && in) ? u[i] : T(0);
        f_i[c] = in ? (unsigned)fixed[i] : 0u;
    }
    T a[2] = {};
    if (in) ku2_node<T, rel_form<T>()>(ke, E, u, n, d, a[0], a[1]);
    if (sk) return;
    if (in) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const long long i = 2 * n + c;
            T o = a[c];
            if (MODE == 1) o = u_i[c] + omega * d_i[c] * (r_i[c] - a[c]);
            if (MODE == 2) o = r_i[c] - a[c];
            if (f_i[c]) o = T(0);
            out[i] = o;
            if (PCG) dot.add(MODE == 1 ? r_i[c] : u_i[c], o);
        }
    }
    if (PCG) {
        double v[1] = {dot.value()}, tot[1];
        if (last_block_totals<256, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
            if (MODE == 1) {  // last V-cycle sweep: rz = r.z, beta = rz / rz_old
                pcg->beta = tot[0] / pcg->rz;
                pcg->rz = tot[0];
            } else {          // K p: alpha = rz / p.Ap
                pcg->pAp = tot[0];
                pcg->alpha = pcg->rz / tot[0];
            }
        }
    }
}

template <typename T, int MODE, bool PCG>
static void fine_op_dispatch(const to_grid* g, const T* E, const T* u, const T* r, const T* dinv, T* out,
                             T omega, const int* skip, PcgScalars* pcg, cudaStream_t st) {
    const Dims& d = g->d;
    const int nb = div_up(d.nnodes, 256);
    if (d.dim == 3 && !g->node_centric) {
        if constexpr (sizeof(T) == 4) {
            if (g->walsh_pair) {
                launch_walsh_pair3(d, g->wkf, MODE, E, u, r, dinv, out, g->fixed, true, omega, skip, pcg,
                                   g->partials, g->npartials, g->counter, g->nsm, st);
                return;
            }
        }
        launch_walsh_op3<T>(d, grid_wk<T>(g), MODE, E, u, r, dinv, out, g->fixed, true, omega, skip, pcg,
                            g->partials, g->npartials, g->counter, g->nsm, st);
        return;
    }
    if (d.dim == 3)
        launch_k(k_fine_op3<T, MODE, PCG>, nb, 256, 0, st, d, grid_ke3<T>(g), E, u, r, dinv, out, g->fixed, omega,
                 skip, pcg, g->partials, g->counter);
    else
        launch_k(k_fine_op2<T, MODE, PCG>, nb, 256, 0, st, d, grid_ke2<T>(g), E, u, r, dinv, out, g->fixed, omega,
                 skip, pcg, g->partials, g->counter);
}

template <typename T>
void launch_fine_op(const to_grid* g, int mode, const T* E, const T* u, const T* r, const T* dinv, T* out,
                    T omega, const int* skip, PcgScalars* pcg, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (g->use_tc) {
            launch_fine_op_tc(g, mode, E, u, r, dinv, out, omega, skip, pcg, st);
            return;
        }
    }
    if (mode == 0 && pcg)
        fine_op_dispatch<T, 0, true>(g, E, u, r, dinv, out, omega, skip, pcg, st);
    else if (mode == 1 && pcg)
        fine_op_dispatch<T, 1, true>(g, E, u, r, dinv, out, omega, skip, pcg, st);
    else if (mode == 0)
        fine_op_dispatch<T, 0, false>(g, E, u, r, dinv, out, omega, skip, nullptr, st);
    else if (mode == 1)
        fine_op_dispatch<T, 1, false>(g, E, u, r, dinv, out, omega, skip, nullptr, st);
    else
        fine_op_dispatch<T, 2, false>(g, E, u, r, dinv, out, omega, skip, nullptr, st);
}
template void launch_fine_op<double>(const to_grid*, int, const double*, const double*, const double*,
                                     const double*, double*, double, const int*, PcgScalars*, cudaStream_t);
template void launch_fine_op<float>(const to_grid*, int, const float*, const float*, const float*,
                                    const float*, float*, float, const int*, PcgScalars*, cudaStream_t);

// ------------------------------------------------------------ Galerkin

// Weight of coarse corner B at the position of child j's corner b (trilinear /
// bilinear interpolation; positions in half-element units 0, 1, 2).
template <int DIM>
__device__ __forceinline__ float pn_weight(int j, int b, int B) {
    float w = 1.f;
    const int p[3] = {lnx(j) + lnx(b), lny(j) + lny(b), lnz(j) + lnz(b)};
    const int q[3] = {lnx(B), lny(B), lnz(B)};
#pragma unroll
    for (int a = 0; a < DIM; ++a) w *= q[a] ? 0.5f * p[a] : 0.5f * (2 - p[a]);
    return w;
}

// One CTA per coarse element: Kc = sum_j P_j^T K_j P_j over the children j.
// FROM_FINE: K_j = M_j (E_j Ke) M_j with M_j zeroing fine Dirichlet DOFs. When
// no fine DOF of the coarse element is fixed this is sum_j E_j C_j with the
// constant C_j = P_j^T Ke P_j (Cj, precomputed), 16x fewer multiply-adds.
// touched_c[ec] = 1 if a fine Dirichlet DOF lies under the coarse element
// (FROM_FINE: among its 3^dim fine nodes; else: under one of its children,
// touched_f). An untouched element matrix annihilates the rigid translations
// exactly: K_j does, and the interpolation P_j maps a coarse translation to the
// same fine translation.
template <typename T, int DIM, bool FROM_FINE>
__global__ void __launch_bounds__(256) k_galerkin(Dims dc, Dims df, const T* __restrict__ Ef,
                                                  const double* __restrict__ Ke, const T* __restrict__ Cj,
                                                  const T* __restrict__ Kf, const uint8_t* __restrict__ fixed_f,
                                                  const uint8_t* __restrict__ touched_f, T* __restrict__ Kc,
                                                  uint8_t* __restrict__ touched_c) {
    constexpr int NN = DIM == 3 ? 8 : 4, D = DIM * NN, DD = D * D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ks = (T*)smem_raw;  // [NN children][D*D]
    T* Ts = Ks + NN * DD;  // [NN children][NN a][NN B][DIM][DIM]
    __shared__ T pw[NN * NN * NN];  // pn weights [j][b][B]
    __shared__ T Ej[NN];
    __shared__ int any_fixed, has_fixed;
    const long long ec = blockIdx.x;
    const int ey = (int)(ec % dc.nely);
    const long long t0 = ec / dc.nely;
    const int ez = (int)(t0 % dc.nelz);
    const int ex = (int)(t0 / dc.nelz);
    for (int i = threadIdx.x; i < NN * NN * NN; i += blockDim.x)
        pw[i] = (T)pn_weight<DIM>(i / (NN * NN), (i / NN) % NN, i % NN);
    // children beyond an odd fine grid (ceil coarsening) contribute nothing
    const bool all_inside = 2 * ex + 1 < df.nelx && 2 * ey + 1 < df.nely && (DIM == 2 || 2 * ez + 1 < df.nelz);
    if (FROM_FINE) {
        if (threadIdx.x == 0) has_fixed = 0;
        if (threadIdx.x < NN) {
            const int j = threadIdx.x;
            const int exf = 2 * ex + lnx(j), eyf = 2 * ey + (1 - lny(j)), ezf = DIM == 3 ? 2 * ez + lnz(j) : 0;
            const bool in = exf < df.nelx && eyf < df.nely && ezf < df.nelz;
            Ej[j] = in ? Ef[eyf + (long long)df.nely * (ezf + (long long)df.nelz * exf)] : T(0);
        }
        __syncthreads();
        // the 3^dim fine nodes of the coarse element
        for (int i = threadIdx.x; i < (DIM == 3 ? 27 : 9) * DIM; i += blockDim.x) {
            const int c = i % DIM, q = i / DIM;
            const int ox = DIM == 3 ? q / 9 : q / 3, oz = DIM == 3 ? (q / 3) % 3 : 0, oy = q % 3;
            const int fy = 2 * ey + oy, fz = DIM == 3 ? 2 * ez + oz : 0, fx = 2 * ex + ox;
            if (fy >= df.nny || fz >= df.nnz || fx >= df.nnx) continue;
            const long long nf = fy + (long long)df.nny * (fz + (long long)df.nnz * fx);
            if (fixed_f[DIM * nf + c]) has_fixed = 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            touched_c[ec] = (uint8_t)has_fixed;
            any_fixed = has_fixed || !all_inside;  // partial coarse elements take the general path
        }
        __syncthreads();
        if (!any_fixed) {
            for (int idx = threadIdx.x; idx < DD; idx += blockDim.x) {
                T s = T(0);
#pragma unroll
                for (int j = 0; j < NN; ++j) s += Ej[j] * Cj[j * DD + idx];
                Kc[ec * DD + idx] = s;
            }
            return;
        }
    } else if (threadIdx.x == 0) {
        int tch = 0;
        for (int j = 0; j < NN; ++j) {
            const int exf = 2 * ex + lnx(j), eyf = 2 * ey + (1 - lny(j)), ezf = DIM == 3 ? 2 * ez + lnz(j) : 0;
            if (exf < df.nelx && eyf < df.nely && ezf < df.nelz)
                tch |= touched_f[eyf + (long long)df.nely * (ezf + (long long)df.nelz * exf)];
        }
        touched_c[ec] = (uint8_t)tch;
    }
    for (int idx = threadIdx.x; idx < NN * DD; idx += blockDim.x) {
        const int j = idx / DD, rem = idx % DD, row = rem / D, col = rem % D;
        const int exf = 2 * ex + lnx(j), eyf = 2 * ey + (1 - lny(j)), ezf = DIM == 3 ? 2 * ez + lnz(j) : 0;
        const long long ef = eyf + (long long)df.nely * (ezf + (long long)df.nelz * exf);
        T v;
        if (exf >= df.nelx || eyf >= df.nely || ezf >= df.nelz) {
            v = T(0);
        } else if (FROM_FINE) {
            const int a = row / DIM, c = row % DIM, b = col / DIM, k = col % DIM;
            const long long na = (eyf + 1 - lny(a)) + (long long)df.nny * ((ezf + lnz(a)) + (long long)df.nnz * (exf + lnx(a)));
            const long long nb = (eyf + 1 - lny(b)) + (long long)df.nny * ((ezf + lnz(b)) + (long long)df.nnz * (exf + lnx(b)));
            const bool masked = fixed_f[DIM * na + c] || fixed_f[DIM * nb + k];
            v = masked ? T(0) : (T)((double)Ef[ef] * Ke[rem]);
        } else {
            v = Kf[ef * DD + rem];
        }
        Ks[idx] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < NN * NN * NN * DIM * DIM; idx += blockDim.x) {
        const int k = idx % DIM, c = (idx / DIM) % DIM, B = (idx / (DIM * DIM)) % NN,
                  a = (idx / (DIM * DIM * NN)) % NN, j = idx / (DIM * DIM * NN * NN);
        const T* kr = Ks + j * DD + (a * DIM + c) * D + k;
        const T* w = pw + j * NN * NN + B;
        T s = T(0);
#pragma unroll
        for (int b = 0; b < NN; ++b) s += kr[b * DIM] * w[b * NN];
        Ts[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < DD; idx += blockDim.x) {
        const int row = idx / D, col = idx % D, A = row / DIM, c = row % DIM, B = col / DIM, k = col % DIM;
        T s = T(0);
        for (int j = 0; j < NN; ++j)
#pragma unroll
            for (int a = 0; a < NN; ++a) s += pw[(j * NN + a) * NN + A] * Ts[(((j * NN + a) * NN + B) * DIM + c) * DIM + k];
        Kc[ec * DD + idx] = s;
    }
}

// Host copy of the interpolation weight (the same as pn_weight).
static double pn_weight_host(int dim, int j, int b, int B) {
    auto bx = [](int M) { return ((M & 3) == 1 || (M & 3) == 2) ? 1 : 0; };
    auto by = [](int M) { return (M & 3) >= 2 ? 1 : 0; };
    auto bz = [](int M) { return M >> 2; };
    const int p[3] = {bx(j) + bx(b), by(j) + by(b), bz(j) + bz(b)};
    const int q[3] = {bx(B), by(B), bz(B)};
    double w = 1.0;
    for (int a = 0; a < dim; ++a) w *= q[a] ? 0.5 * p[a] : 0.5 * (2 - p[a]);
    return w;
}

// Level-0 element matrices E_e Ke (only for a dense solve of a tiny fine grid).
template <typename T, int DIM>
__global__ void k_elem_from_E(Dims d, const T* __restrict__ E, const double* __restrict__ Ke, T* __restrict__ Kel) {
    constexpr int D = DIM == 3 ? 24 : 8, DD = D * D;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.nel * DD) return;
    Kel[i] = (T)((double)E[i / DD] * Ke[i % DD]);
}

// ------------------------------------------------------------- stencils

template <int DIM>
__host__ __device__ constexpr int n_stencil() { return DIM == 3 ? 27 : 9; }

// Whether a coarse node's row sums can be nonzero: one of its (up to 2^dim)
// elements is touched by a fine Dirichlet DOF (touched == nullptr: all are).
template <int DIM>
__device__ __forceinline__ bool node_touched(const Dims& d, const uint8_t* __restrict__ touched, int ix, int iy,
                                             int iz) {
    if (!touched) return true;
    bool t = false;
#pragma unroll
    for (int o = 0; o < (DIM == 3 ? 8 : 4); ++o) {
        const int ex = ix - 1 + (DIM == 3 ? (o >> 2) & 1 : (o >> 1) & 1), ey = iy - 1 + (o & 1);
        const int ez = DIM == 3 ? iz - 1 + ((o >> 1) & 1) : 0;
        if (ex < 0 || ex >= d.nelx || ey < 0 || ey >= d.nely || ez < 0 || ez >= d.nelz) continue;
        t |= touched[ey + (long long)d.nely * (ez + (long long)d.nelz * ex)] != 0;
    }
    return t;
}

// Node stencil S[n][s] = sum over the elements containing n and n + s of the
// element-matrix block (n, n + s); R[n] = sum_s S[n][s], the operator applied
// to the unit translations. SoA layout. At a node none of whose elements is
// touched R is exactly 0 and is stored so: summed in the level's precision it
// would instead hold the rounding of the cancelling blocks, which in the
// relative form of the operator (R_n u_n) acts on absolute displacements and
// perturbs the smooth modes the coarse correction exists for.
template <typename T, int DIM>
__global__ void k_stencil_build(Dims d, const T* __restrict__ Kel, const uint8_t* __restrict__ touched,
                                T* __restrict__ S, T* __restrict__ R) {
    constexpr int NS = n_stencil<DIM>(), D = DIM == 3 ? 24 : 8, DD = D * D, Q = DIM * DIM;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.nnodes) return;
    const int iy = (int)(n % d.nny);
    const long long t = n / d.nny;
    const int iz = (int)(t % d.nnz);
    const int ix = (int)(t / d.nnz);
    T rs[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) rs[q] = T(0);
    for (int s = 0; s < NS; ++s) {
        const int dx = DIM == 3 ? s / 9 - 1 : s / 3 - 1;
        const int dz = DIM == 3 ? (s / 3) % 3 - 1 : 0;
        const int dy = s % 3 - 1;
        const int mx = ix + dx, my = iy + dy, mz = iz + dz;
        T blk[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) blk[q] = T(0);
        if (mx >= 0 && mx < d.nnx && my >= 0 && my < d.nny && mz >= 0 && mz < d.nnz) {
            for (int o = 0; o < (DIM == 3 ? 8 : 4); ++o) {
                const int exo = DIM == 3 ? (o >> 2) & 1 : (o >> 1) & 1, ezo = DIM == 3 ? (o >> 1) & 1 : 1,
                          eyo = o & 1;
                const int ex = ix - 1 + exo, ey = iy - 1 + eyo, ez = DIM == 3 ? iz - 1 + ezo : 0;
                if (ex < 0 || ex >= d.nelx || ey < 0 || ey >= d.nely || ez < 0 || ez >= d.nelz) continue;
                const int bx = mx - ex, brow = my - ey, bz = mz - ez;
                if (bx < 0 || bx > 1 || brow < 0 || brow > 1 || bz < 0 || bz > 1) continue;
                const int Ln = local_node(1 - exo, eyo, DIM == 3 ? 1 - ezo : 0);
                const int Lm = local_node(bx, 1 - brow, bz);
                const T* Ke = Kel + (ey + (long long)d.nely * (ez + (long long)d.nelz * ex)) * DD;
#pragma unroll
                for (int c = 0; c < DIM; ++c)
#pragma unroll
                    for (int k = 0; k < DIM; ++k) blk[c * DIM + k] += Ke[(Ln * DIM + c) * D + Lm * DIM + k];
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            S[((long long)s * Q + q) * d.nnodes + n] = blk[q];
            rs[q] += blk[q];
        }
    }
    const bool tch = node_touched<DIM>(d, touched, ix, iy, iz);
#pragma unroll
    for (int q = 0; q < Q; ++q) R[(long long)q * d.nnodes + n] = tch ? rs[q] : T(0);
}

// 3D stencils with one thread per (node, stencil block): block (SB_NODES, 27),
// each thread sums its block over the (up to 8) shared elements as
// k_stencil_build does, and nine threads per node then add the 27 blocks in
// stencil order for R, so S and R are those of k_stencil_build.
template <typename T>
struct StencilNodes {
    static constexpr int v = sizeof(T) == 8 ? 16 : 32;
};

template <typename T>
__global__ void __launch_bounds__(27 * StencilNodes<T>::v) k_stencil_build3s(Dims d, const T* __restrict__ Kel,
                                                                          const uint8_t* __restrict__ touched,
                                                                          T* __restrict__ S, T* __restrict__ R) {
    constexpr int NB = StencilNodes<T>::v, D = 24, DD = D * D, Q = 9;
    __shared__ T part[27][NB][Q];
    const int tx = threadIdx.x, s = threadIdx.y;
    const long long n = (long long)blockIdx.x * NB + tx;
    const bool valid = n < d.nnodes;
    T blk[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) blk[q] = T(0);
    if (valid) {
        const int iy = (int)(n % d.nny);
        const long long t = n / d.nny;
        const int iz = (int)(t % d.nnz);
        const int ix = (int)(t / d.nnz);
        const int dx = s / 9 - 1, dz = (s / 3) % 3 - 1, dy = s % 3 - 1;
        const int mx = ix + dx, my = iy + dy, mz = iz + dz;
        if (mx >= 0 && mx < d.nnx && my >= 0 && my < d.nny && mz >= 0 && mz < d.nnz) {
            for (int o = 0; o < 8; ++o) {
                const int exo = (o >> 2) & 1, ezo = (o >> 1) & 1, eyo = o & 1;
                const int ex = ix - 1 + exo, ey = iy - 1 + eyo, ez = iz - 1 + ezo;
                if (ex < 0 || ex >= d.nelx || ey < 0 || ey >= d.nely || ez < 0 || ez >= d.nelz) continue;
                const int bx = mx - ex, brow = my - ey, bz = mz - ez;
                if (bx < 0 || bx > 1 || brow < 0 || brow > 1 || bz < 0 || bz > 1) continue;
                const int Ln = local_node(1 - exo, eyo, 1 - ezo);
                const int Lm = local_node(bx, 1 - brow, bz);
                const T* Ke = Kel + (ey + (long long)d.nely * (ez + (long long)d.nelz * ex)) * DD;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int k = 0; k < 3; ++k) blk[c * 3 + k] += Ke[(Ln * 3 + c) * D + Lm * 3 + k];
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) S[((long long)s * Q + q) * d.nnodes + n] = blk[q];
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) part[s][tx][q] = blk[q];
    __syncthreads();
    if (s < Q && valid) {
        T rs = T(0);
        for (int k = 0; k < 27; ++k) rs += part[k][tx][s];
        const int iy = (int)(n % d.nny);
        const long long t = n / d.nny;
        R[(long long)s * d.nnodes + n] =
            node_touched<3>(d, touched, (int)(t / d.nnz), iy, (int)(t % d.nnz)) ? rs : T(0);
    }
}

// l1-Jacobi smoother weights: dinv = 1 / sum_j |A_ij| (row sums of absolute
// values), so that lambda_max(D^-1 A) <= 1 (Gershgorin) for any modulus
// contrast and the damped sweep contracts; coarse DOFs whose diagonal is zero
// (all their fine DOFs are fixed) become fixed.
template <typename T, int DIM>
__global__ void k_stencil_diag(Dims d, const T* __restrict__ S, T* __restrict__ dinv, uint8_t* __restrict__ fixed) {
    constexpr int NS = n_stencil<DIM>(), Q = DIM * DIM;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.nnodes) return;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        const T diag = S[((long long)(NS / 2) * Q + c * DIM + c) * d.nnodes + n];
        T l1 = T(0);
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int k = 0; k < DIM; ++k) l1 += fabs(S[((long long)s * Q + c * DIM + k) * d.nnodes + n]);
        const bool f = !(diag > T(0));
        fixed[DIM * n + c] = f;
        dinv[DIM * n + c] = f ? T(0) : T(1) / l1;
    }
}

// Level 0: l1 row sums sum_e E_e sum_j |Ke[row, j]| from the per-row absolute
// sums of Ke (arow); 0 at fixed DOFs.
template <typename T, int DIM>
struct RowAbs {
    T a[DIM == 3 ? 24 : 8];
};

template <typename T, int DIM>
__global__ void k_l1_inv(Dims d, const RowAbs<T, DIM> ra, const T* __restrict__ E, const uint8_t* __restrict__ fixed,
                         T* __restrict__ dinv) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.nnodes) return;
    const int iy = (int)(n % d.nny);
    const long long t = n / d.nny;
    const int iz = (int)(t % d.nnz);
    const int ix = (int)(t / d.nnz);
    T acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] = T(0);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int exo = (o >> 2) & 1, ezo = (o >> 1) & 1, eyo = o & 1;
        if (DIM == 2 && ezo) continue;
        const int ex = ix - 1 + exo, ey = iy - 1 + eyo, ez = DIM == 3 ? iz - 1 + ezo : 0;
        if (ex < 0 || ex >= d.nelx || ey < 0 || ey >= d.nely || ez < 0 || ez >= d.nelz) continue;
        const T Ee = E[ey + (long long)d.nely * (ez + (long long)d.nelz * ex)];
        const int L = local_node(1 - exo, eyo, DIM == 3 ? 1 - ezo : 0);
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] += Ee * ra.a[DIM * L + c];
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) dinv[DIM * n + c] = fixed[DIM * n + c] ? T(0) : T(1) / acc[c];
}

// Coarse-level operator: modes as the fine level. FP32 uses the relative form
// sum_{m != n} S_nm (u_m - u_n) + R_n u_n (exact rewriting of sum_m S_nm u_m).
template <typename T, int DIM, int MODE>
__global__ void __launch_bounds__(256) k_stencil_op(Dims d, const T* __restrict__ S, const T* __restrict__ R,
                                                    const T* __restrict__ u, const T* __restrict__ r,
                                                    const T* __restrict__ dinv, T* __restrict__ out,
                                                    const uint8_t* __restrict__ fixed, T omega,
                                                    const int* skip) {
    constexpr int NS = n_stencil<DIM>(), Q = DIM * DIM;
    constexpr bool REL = rel_form<T>();
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested before the stores, so its load overlaps the others
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.nnodes) return;
    const int iy = (int)(n % d.nny);
    const long long t = n / d.nny;
    const int iz = (int)(t % d.nnz);
    const int ix = (int)(t / d.nnz);
    T r_i[DIM], d_i[DIM];
    unsigned f_i[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        r_i[c] = MODE != 0 ? r[DIM * n + c] : T(0);
        d_i[c] = MODE == 1 ? dinv[DIM * n + c] : T(0);
        f_i[c] = fixed[DIM * n + c];
    }
    T uc[DIM], acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) uc[c] = u[DIM * n + c];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        acc[c] = T(0);
        if (REL) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) acc[c] += R[(long long)(c * DIM + k) * d.nnodes + n] * uc[k];
        }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (REL && s == NS / 2) continue;
        const int dx = DIM == 3 ? s / 9 - 1 : s / 3 - 1;
        const int dz = DIM == 3 ? (s / 3) % 3 - 1 : 0;
        const int dy = s % 3 - 1;
        const int mx = ix + dx, my = iy + dy, mz = iz + dz;
        if (mx < 0 || mx >= d.nnx || my < 0 || my >= d.nny || mz < 0 || mz >= d.nnz) continue;
        const long long m = my + (long long)d.nny * (mz + (long long)d.nnz * mx);
        T um[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) um[k] = REL ? u[DIM * m + k] - uc[k] : u[DIM * m + k];
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
            for (int k = 0; k < DIM; ++k) acc[c] += S[((long long)s * Q + c * DIM + k) * d.nnodes + n] * um[k];
    }
    if (sk) return;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        const long long i = DIM * n + c;
        T o = acc[c];
        if (MODE == 1) o = uc[c] + omega * d_i[c] * (r_i[c] - acc[c]);
        if (MODE == 2) o = r_i[c] - acc[c];
        if (f_i[c]) o = T(0);
        out[i] = o;
    }
}

// 3D coarse-level operator with nine threads per node: thread (tx, ty) serves
// node blockIdx.x*32 + tx, output component c = ty / 3 and the stencil plane
// dx = ty % 3 - 1 (9 of the 27 blocks). The three plane partials are summed in
// plane order in shared memory, so the result does not depend on scheduling.
// A single thread per node issues 243 dependent-latency loads; splitting them
// gives the small coarse grids enough warps in flight.
// The body of one 32-node block vb (the kernel's blockIdx.x); 288 threads (32, 9).
template <typename T, int MODE>
__device__ __forceinline__ void stencil_op3s_body(int vb, const Dims& d, const T* __restrict__ S,
                                                  const T* __restrict__ R, const T* __restrict__ u,
                                                  const T* __restrict__ r, const T* __restrict__ dinv,
                                                  T* __restrict__ out, const uint8_t* __restrict__ fixed, T omega,
                                                  int skip_now = 0) {
    constexpr int Q = 9;
    constexpr bool REL = rel_form<T>();
    __shared__ T part[9][32];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int c = ty / 3, pl = ty % 3;
    const long long n = (long long)vb * 32 + tx;
    // the epilogue's operands depend on nothing computed here: fetched first
    const bool outp = pl == 0 && n < d.nnodes;
    const long long i = 3 * n + c;
    const T r_i = (MODE != 0 && outp) ? r[i] : T(0), d_i = (MODE == 1 && outp) ? dinv[i] : T(0);
    const unsigned f_i = outp ? (unsigned)fixed[i] : 0u;
    T acc = T(0);
    if (n < d.nnodes) {
        const int iy = (int)(n % d.nny);
        const long long t = n / d.nny;
        const int iz = (int)(t % d.nnz);
        const int ix = (int)(t / d.nnz);
        T uc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) uc[k] = u[3 * n + k];
        if (REL && pl == 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) acc += R[(long long)(c * 3 + k) * d.nnodes + n] * uc[k];
        }
        const int mx = ix + pl - 1;
        if (mx >= 0 && mx < d.nnx) {
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const int s = pl * 9 + j;
                if (REL && s == 13) continue;
                const int dz = j / 3 - 1, dy = j % 3 - 1;
                const int my = iy + dy, mz = iz + dz;
                if (my < 0 || my >= d.nny || mz < 0 || mz >= d.nnz) continue;
                const long long m = my + (long long)d.nny * (mz + (long long)d.nnz * mx);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const T um = REL ? u[3 * m + k] - uc[k] : u[3 * m + k];
                    acc += S[((long long)s * Q + c * 3 + k) * d.nnodes + n] * um;
                }
            }
        }
    }
    part[ty][tx] = acc;
    __syncthreads();
    if (skip_now || !outp) return;
    const T a = (part[ty][tx] + part[ty + 1][tx]) + part[ty + 2][tx];
    T o = a;
    if (MODE == 1) o = u[i] + omega * d_i * (r_i - a);
    if (MODE == 2) o = r_i - a;
    if (f_i) o = T(0);
    out[i] = o;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(288) k_stencil_op3s(Dims d, const T* __restrict__ S, const T* __restrict__ R,
                                                      const T* __restrict__ u, const T* __restrict__ r,
                                                      const T* __restrict__ dinv, T* __restrict__ out,
                                                      const uint8_t* __restrict__ fixed, T omega,
                                                      const int* skip) {
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested before the stores, so its load overlaps the others
    stencil_op3s_body<T, MODE>(blockIdx.x, d, S, R, u, r, dinv, out, fixed, omega, sk);
}

// ------------------------------------------------------- transfer operators

// With dinv_c: also the coarse level's first damped Jacobi iterate
// z_c = omega dinv_c r_c (its k_jacobi_first, fused).
template <typename T, int DIM>
__global__ void k_restrict(Dims dc, Dims df, const T* __restrict__ rf, T* __restrict__ rc,
                           const uint8_t* __restrict__ fixed_c, const int* skip, const T* __restrict__ dinv_c,
                           T* __restrict__ z_c, T omega) {
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested before the stores, so its load overlaps the others
    const long long N = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (N >= dc.nnodes) return;
    unsigned f_N[DIM];
    T d_N[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        f_N[c] = fixed_c[DIM * N + c];
        d_N[c] = dinv_c ? dinv_c[DIM * N + c] : T(0);
    }
    const int NY = (int)(N % dc.nny);
    const long long t = N / dc.nny;
    const int NZ = (int)(t % dc.nnz);
    const int NX = (int)(t / dc.nnz);
    T acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] = T(0);
    for (int ox = -1; ox <= 1; ++ox)
        for (int oz = (DIM == 3 ? -1 : 0); oz <= (DIM == 3 ? 1 : 0); ++oz)
            for (int oy = -1; oy <= 1; ++oy) {
                const int fx = 2 * NX + ox, fy = 2 * NY + oy, fz = DIM == 3 ? 2 * NZ + oz : 0;
                if (fx < 0 || fx >= df.nnx || fy < 0 || fy >= df.nny || fz < 0 || fz >= df.nnz) continue;
                const T w = (ox ? T(0.5) : T(1)) * (oy ? T(0.5) : T(1)) * (oz ? T(0.5) : T(1));
                const long long f = fy + (long long)df.nny * (fz + (long long)df.nnz * fx);
#pragma unroll
                for (int c = 0; c < DIM; ++c) acc[c] += w * rf[DIM * f + c];
            }
    if (sk) return;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        const T v = f_N[c] ? T(0) : acc[c];
        rc[DIM * N + c] = v;
        if (dinv_c) z_c[DIM * N + c] = omega * d_N[c] * v;
    }
}

// 3D restriction with nine threads per coarse node: thread (tx, ty) sums the
// nine fine nodes of plane ox = ty % 3 - 1 for component c = ty / 3; the plane
// partials are added in plane order in shared memory (same result as k_restrict
// up to the order of the three plane sums, fixed for every launch).
template <typename T>
__device__ __forceinline__ void restrict3s_body(int vb, const Dims& dc, const Dims& df, const T* __restrict__ rf,
                                                T* __restrict__ rc, const uint8_t* __restrict__ fixed_c,
                                                const T* __restrict__ dinv_c, T* __restrict__ z_c, T omega,
                                                int skip_now = 0) {
    __shared__ T part[9][32];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int c = ty / 3, ox = ty % 3 - 1;
    const long long N = (long long)vb * 32 + tx;
    const bool outp = ty % 3 == 0 && N < dc.nnodes;
    const unsigned f_N = outp ? (unsigned)fixed_c[3 * N + c] : 0u;
    const T d_N = (outp && dinv_c) ? dinv_c[3 * N + c] : T(0);
    T acc = T(0);
    if (N < dc.nnodes) {
        const int NY = (int)(N % dc.nny);
        const long long t = N / dc.nny;
        const int NZ = (int)(t % dc.nnz);
        const int NX = (int)(t / dc.nnz);
        const int fx = 2 * NX + ox;
        if (fx >= 0 && fx < df.nnx) {
            const T wx = ox ? T(0.5) : T(1);
#pragma unroll
            for (int oz = -1; oz <= 1; ++oz)
#pragma unroll
                for (int oy = -1; oy <= 1; ++oy) {
                    const int fy = 2 * NY + oy, fz = 2 * NZ + oz;
                    if (fy < 0 || fy >= df.nny || fz < 0 || fz >= df.nnz) continue;
                    const T w = wx * (oy ? T(0.5) : T(1)) * (oz ? T(0.5) : T(1));
                    const long long f = fy + (long long)df.nny * (fz + (long long)df.nnz * fx);
                    acc += w * rf[3 * f + c];
                }
        }
    }
    part[ty][tx] = acc;
    __syncthreads();
    if (skip_now || !outp) return;
    const T a = (part[ty][tx] + part[ty + 1][tx]) + part[ty + 2][tx];
    const T v = f_N ? T(0) : a;
    rc[3 * N + c] = v;
    if (dinv_c) z_c[3 * N + c] = omega * d_N * v;
}

template <typename T>
__global__ void __launch_bounds__(288) k_restrict3s(Dims dc, Dims df, const T* __restrict__ rf,
                                                    T* __restrict__ rc, const uint8_t* __restrict__ fixed_c,
                                                    const int* skip, const T* __restrict__ dinv_c,
                                                    T* __restrict__ z_c, T omega) {
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested before the stores, so its load overlaps the others
    restrict3s_body<T>(blockIdx.x, dc, df, rf, rc, fixed_c, dinv_c, z_c, omega, sk);
}

template <typename T, int DIM>
__global__ void k_prolong_add(Dims df, Dims dc, const T* __restrict__ zc, T* __restrict__ zf,
                              const uint8_t* __restrict__ fixed_f, const int* skip) {
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested before the stores, so its load overlaps the others
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= df.nnodes) return;
    unsigned fl[DIM];
    T zv[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        fl[c] = fixed_f[DIM * f + c];
        zv[c] = zf[DIM * f + c];
    }
    const int fy = (int)(f % df.nny);
    const long long t = f / df.nny;
    const int fz = (int)(t % df.nnz);
    const int fx = (int)(t / df.nnz);
    T acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] = T(0);
    const int nx = (fx & 1) ? 2 : 1, ny = (fy & 1) ? 2 : 1, nz = (fz & 1) ? 2 : 1;
    for (int a = 0; a < nx; ++a)
        for (int b = 0; b < nz; ++b)
            for (int e = 0; e < ny; ++e) {
                const int NX = (fx >> 1) + a, NZ = (fz >> 1) + b, NY = (fy >> 1) + e;
                const T w = (nx == 2 ? T(0.5) : T(1)) * (ny == 2 ? T(0.5) : T(1)) * (nz == 2 ? T(0.5) : T(1));
                const long long N = NY + (long long)dc.nny * (NZ + (long long)dc.nnz * NX);
#pragma unroll
                for (int c = 0; c < DIM; ++c) acc[c] += w * zc[DIM * N + c];
            }
    if (sk) return;
#pragma unroll
    for (int c = 0; c < DIM; ++c)
        if (!fl[c]) zf[DIM * f + c] = zv[c] + acc[c];
}

// Prolongation fused into the first post-smoothing sweep of a 3D coarse level:
// out = u + omega dinv (r - K u) with u = cur + P zc (P zc added on free DOFs),
// u never written to memory. A CTA covers a TY x TZ tile of nodes at one x
// (TY * TZ = 32) with nine threads per node as k_stencil_op3s; it first forms
// u on the tile and its one-node halo in shared memory, summing P zc in
// k_prolong_add's order, then sweeps the stencil in k_stencil_op3s's order,
// so the result is that of the two kernels in sequence.
template <typename T, int TY>
__device__ __forceinline__ void prolong_smooth3s_body(int vb, const Dims& d, const Dims& dc, const T* __restrict__ zc,
                                                      const T* __restrict__ cur, const T* __restrict__ S,
                                                      const T* __restrict__ R, const T* __restrict__ r,
                                                      const T* __restrict__ dinv, T* __restrict__ out,
                                                      const uint8_t* __restrict__ fixed, T omega,
                                                      int skip_now = 0) {
    constexpr int TZ = 32 / TY, HY = TY + 2, HZ = TZ + 2, NH = 3 * HZ * HY, Q = 9;
    constexpr bool REL = rel_form<T>();
    __shared__ T us[3 * NH];
    __shared__ T part[9][32];
    const int nty = (d.nny + TY - 1) / TY, ntz = (d.nnz + TZ - 1) / TZ;
    const int by = vb % nty, bz = (vb / nty) % ntz, ix = vb / (nty * ntz);
    const int iy0 = by * TY, iz0 = bz * TZ;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int c = ty / 3, pl = ty % 3;
    const int ly = tx % TY, lz = tx / TY;
    const int iy = iy0 + ly, iz = iz0 + lz;
    const bool valid = iy < d.nny && iz < d.nnz;
    const long long n = iy + (long long)d.nny * (iz + (long long)d.nnz * ix);
    const int mx = ix + pl - 1;
    const bool plane = valid && mx >= 0 && mx < d.nnx;
    // the epilogue's operands and this thread's stencil blocks do not depend on u: their loads go out first
    const bool outp = pl == 0 && valid;
    const long long i = 3 * n + c;
    const T r_i = outp ? r[i] : T(0), d_i = outp ? dinv[i] : T(0);
    const unsigned f_i = outp ? (unsigned)fixed[i] : 0u;
    T sv[27], rv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) rv[k] = (REL && pl == 1 && valid) ? R[(long long)(c * 3 + k) * d.nnodes + n] : T(0);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int s = pl * 9 + j;
        const int my = iy + j % 3 - 1, mz = iz + j / 3 - 1;
        const bool in = plane && !(REL && s == 13) && my >= 0 && my < d.nny && mz >= 0 && mz < d.nnz;
#pragma unroll
        for (int k = 0; k < 3; ++k) sv[3 * j + k] = in ? S[((long long)s * Q + c * 3 + k) * d.nnodes + n] : T(0);
    }
    for (int v = tid; v < 3 * NH; v += 288) {
        const int h = v / 3, k = v % 3;
        const int hy = h % HY, hz = (h / HY) % HZ, hx = h / (HY * HZ);
        const int fx = ix - 1 + hx, fz = iz0 - 1 + hz, fy = iy0 - 1 + hy;
        T val = T(0);
        if (fx >= 0 && fx < d.nnx && fy >= 0 && fy < d.nny && fz >= 0 && fz < d.nnz) {
            const long long f = fy + (long long)d.nny * (fz + (long long)d.nnz * fx);
            const T cv = cur[3 * f + k];
            const unsigned fv = fixed[3 * f + k];
            // P zc is formed before the free-DOF test so that its loads go out with cur's
            T acc = T(0);
            const int nx = (fx & 1) ? 2 : 1, ny = (fy & 1) ? 2 : 1, nz = (fz & 1) ? 2 : 1;
            for (int a = 0; a < nx; ++a)
                for (int b = 0; b < nz; ++b)
                    for (int e = 0; e < ny; ++e) {
                        const int NX = (fx >> 1) + a, NZ = (fz >> 1) + b, NY = (fy >> 1) + e;
                        const T w = (nx == 2 ? T(0.5) : T(1)) * (ny == 2 ? T(0.5) : T(1)) *
                                    (nz == 2 ? T(0.5) : T(1));
                        const long long N = NY + (long long)dc.nny * (NZ + (long long)dc.nnz * NX);
                        acc += w * zc[3 * N + k];
                    }
            val = fv ? cv : cv + acc;
        }
        us[v] = val;
    }
    __syncthreads();
    const int hc = (ly + 1) + HY * ((lz + 1) + HZ * 1);
    T acc = T(0);
    if (valid) {
        T uc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) uc[k] = us[3 * hc + k];
        if (REL && pl == 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) acc += rv[k] * uc[k];
        }
        if (plane) {
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const int s = pl * 9 + j;
                if (REL && s == 13) continue;
                const int dz = j / 3 - 1, dy = j % 3 - 1;
                const int my = iy + dy, mz = iz + dz;
                if (my < 0 || my >= d.nny || mz < 0 || mz >= d.nnz) continue;
                const int hm = (ly + 1 + dy) + HY * ((lz + 1 + dz) + HZ * pl);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const T um = REL ? us[3 * hm + k] - uc[k] : us[3 * hm + k];
                    acc += sv[3 * j + k] * um;
                }
            }
        }
    }
    part[ty][tx] = acc;
    __syncthreads();
    if (skip_now || !outp) return;
    const T a = (part[ty][tx] + part[ty + 1][tx]) + part[ty + 2][tx];
    T o = us[3 * hc + c] + omega * d_i * (r_i - a);
    if (f_i) o = T(0);
    out[i] = o;
}

template <typename T, int TY>
__global__ void __launch_bounds__(288, 2) k_prolong_smooth3s(Dims d, Dims dc, const T* __restrict__ zc,
                                                          const T* __restrict__ cur, const T* __restrict__ S,
                                                          const T* __restrict__ R, const T* __restrict__ r,
                                                          const T* __restrict__ dinv, T* __restrict__ out,
                                                          const uint8_t* __restrict__ fixed, T omega,
                                                          const int* skip) {
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested before the stores, so its load overlaps the others
    prolong_smooth3s_body<T, TY>(blockIdx.x, d, dc, zc, cur, S, R, r, dinv, out, fixed, omega, sk);
}

// Tile height (nodes along y) of k_prolong_smooth3s with the fewest idle lanes.
inline int prolong_smooth_ty(const Dims& d) {
    int best = 8;
    double bu = -1.0;
    for (int ty : {8, 16, 32}) {
        const int tz = 32 / ty;
        const double u = (double)d.nny / (((d.nny + ty - 1) / ty) * ty) * ((double)d.nnz / (((d.nnz + tz - 1) / tz) * tz));
        if (u > bu + 1e-9) {
            bu = u;
            best = ty;
        }
    }
    return best;
}

template <typename T>
__global__ void k_jacobi_first(long long n, const T* __restrict__ dinv, const T* __restrict__ r, T* __restrict__ z,
                               T omega, const int* skip) {
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested before the store, so its load overlaps the others
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T v = omega * dinv[i] * r[i];
    if (!sk) z[i] = v;
}

// ------------------------------------------------------- coarsest level

// The coarsest operator as a dense FP64 matrix: the off-diagonal blocks are the
// stencil's, the diagonal block of node n is R_n - sum_{m != n} S_nm, i.e. the
// operator of the relative form k_stencil_op applies (exact for the rigid
// translations however S was rounded), summed in FP64. Fixed DOFs get
// identity rows and columns. A (and A32) arrive zeroed: only the nonzeros are
// written.
template <typename T, int DIM>
__global__ void k_dense_assemble(Dims d, const T* __restrict__ S, const T* __restrict__ R,
                                 const uint8_t* __restrict__ fixed, double* __restrict__ A,
                                 float* __restrict__ A32) {
    constexpr int NS = n_stencil<DIM>(), Q = DIM * DIM;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.nnodes) return;
    const long long nc = d.ndof;
    const int iy = (int)(n % d.nny);
    const long long t = n / d.nny;
    const int iz = (int)(t % d.nnz);
    const int ix = (int)(t / d.nnz);
    for (int c = 0; c < DIM; ++c) {
        const long long i = DIM * n + c;
        double* row = A + i * nc;
        float* row32 = A32 ? A32 + i * nc : nullptr;
        if (fixed[i]) {
            row[i] = 1.0;
            if (row32) row32[i] = 1.f;
            continue;
        }
        double dg[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) dg[k] = (double)R[(long long)(c * DIM + k) * d.nnodes + n];
        for (int s = 0; s < NS; ++s) {
            if (s == NS / 2) continue;
            const int dx = DIM == 3 ? s / 9 - 1 : s / 3 - 1;
            const int dz = DIM == 3 ? (s / 3) % 3 - 1 : 0;
            const int dy = s % 3 - 1;
            const int mx = ix + dx, my = iy + dy, mz = iz + dz;
            if (mx < 0 || mx >= d.nnx || my < 0 || my >= d.nny || mz < 0 || mz >= d.nnz) continue;
            const long long m = my + (long long)d.nny * (mz + (long long)d.nnz * mx);
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const double v = (double)S[((long long)s * Q + c * DIM + k) * d.nnodes + n];
                dg[k] -= v;
                if (!fixed[DIM * m + k]) {
                    row[DIM * m + k] = v;
                    if (row32) row32[DIM * m + k] = (float)v;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < DIM; ++k)
            if (!fixed[DIM * n + k]) {
                row[DIM * n + k] = dg[k];
                if (row32) row32[DIM * n + k] = (float)dg[k];
            }
    }
}

// Coarsest-level dense inverse in four kernels (below). The FP64 solve factors in
// FP64. The FP32 solve factors in FP32, and again in FP64 only where the FP32
// factorization met a pivot below 1e-4 of its original diagonal (four of FP32's
// seven digits cancelled): the coarsest operator of a weakly supported or
// high-contrast design can be far too ill-conditioned for FP32, while FP64 runs
// at a small fraction of the FP32 rate on this part. The choice is made on the
// device: every kernel takes a gate (the FP32 factorization's flag) and the
// branch it belongs to, and returns at once on the other branch. The inverse is
// stored in the solve's precision T.
//  1. blocked right-looking Cholesky A = L L^T by one CTA: the NB x NB diagonal
//     block is factored in shared memory by the whole CTA (one thread per
//     element, three barriers per column), the column panel below it is solved
//     row by row (reciprocal pivots) and staged in shared memory, then the
//     trailing lower triangle is updated from the staged panel in 4 x 4
//     register tiles (n/NB panel phases instead of 3 n). A pivot below 1e-6 of the original diagonal is floored there and
//     flagged, which keeps the factor that of an SPD matrix.
//  2. inverses of the diagonal blocks of L (one CTA each);
//  3. W = L^{-1} block column by block column (one CTA per block column);
//  4. A^{-1} = W^T W, zero on fixed rows and columns.
template <typename T>
struct CholNB {
    static constexpr int v = sizeof(T) == 8 ? 16 : 32;
};

// True when the kernel belongs to the branch the gate selects (no gate: always).
__device__ __forceinline__ bool gate_open(const int* gate, int want) { return !gate || ((*gate != 0) == (want != 0)); }

// status: set to 1 if a pivot fell to flag_ratio of its original diagonal or below.
template <typename T>
__global__ void __launch_bounds__(1024) k_chol_blocked(int n, T* A, T* diag0, int* status, T flag_ratio,
                                                       const int* gate, int want) {
    constexpr int NB = CholNB<T>::v, LD = NB + 1;
    extern __shared__ __align__(16) unsigned char chol_smem[];
    T* Dg = (T*)chol_smem;  // NB x LD diagonal block
    T* Pn = Dg + NB * LD;   // up to n x LD panel
    __shared__ T rdiag[NB];  // reciprocals of the factored diagonal
    if (!gate_open(gate, want)) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) *status = 0;
    for (int k = tid; k < n; k += nt) diag0[k] = A[(long long)k * n + k];
    __syncthreads();
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int kw = min(NB, n - k0), k1 = k0 + kw, m = n - k1;
        for (int i = tid; i < kw * kw; i += nt) {
            const int r = i / kw, c = i % kw;
            Dg[r * LD + c] = c <= r ? A[(long long)(k0 + r) * n + k0 + c] : T(0);
        }
        __syncthreads();
        // the diagonal block, one thread per element (r, c), column by column
        for (int j = 0; j < kw; ++j) {
            if (tid == 0) {
                T p = Dg[j * LD + j];
                const T fl = T(1e-6) * diag0[k0 + j];
                if (!(p > flag_ratio * diag0[k0 + j])) *status = 1;
                if (!(p > fl)) p = fl > T(0) ? fl : T(1);
                Dg[j * LD + j] = sqrt(p);
            }
            __syncthreads();
            if (tid > j && tid < kw) Dg[tid * LD + j] /= Dg[j * LD + j];
            __syncthreads();
            for (int q = tid; q < kw * kw; q += nt) {
                const int r = q / kw, c = q % kw;
                if (c > j && c <= r) Dg[r * LD + c] -= Dg[r * LD + j] * Dg[c * LD + j];
            }
            __syncthreads();
        }
        for (int i = tid; i < kw * kw; i += nt) {
            const int r = i / kw, c = i % kw;
            if (c <= r) A[(long long)(k0 + r) * n + k0 + c] = Dg[r * LD + c];
        }
        if (tid < kw) rdiag[tid] = T(1) / Dg[tid * LD + tid];
        __syncthreads();
        // panel rows k1..n-1: x L_kk^T = a  (forward substitution per row)
        for (int i = tid; i < m; i += nt) {
            T x[NB];
            const long long row = (long long)(k1 + i) * n + k0;
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                if (j < kw) {
                    T s = A[row + j];
#pragma unroll
                    for (int l = 0; l < j; ++l) s -= x[l] * Dg[j * LD + l];
                    x[j] = s * rdiag[j];
                    Pn[i * LD + j] = x[j];
                    A[row + j] = x[j];
                }
            }
        }
        __syncthreads();
        // trailing update of the lower triangle from the staged panel, 4 x 4
        // register tiles (ti >= tj) over the m x m trailing block
        const int mt = (m + 3) / 4;
        const int ntile = mt * (mt + 1) / 2;
        for (int t = tid; t < ntile; t += nt) {
            int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
            while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
            while (ti * (ti + 1) / 2 > t) --ti;
            const int tj = t - ti * (ti + 1) / 2;
            T acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
            int ri[4], ci[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                ri[r] = min(4 * ti + r, m - 1);
                ci[r] = min(4 * tj + r, m - 1);
            }
            for (int l = 0; l < kw; ++l) {
                T a[4], b[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    a[r] = Pn[ri[r] * LD + l];
                    b[r] = Pn[ci[r] * LD + l];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int gi = 4 * ti + r, gj = 4 * tj + c;
                    if (gi < m && gj <= gi) A[(long long)(k1 + gi) * n + k1 + gj] -= acc[r][c];
                }
        }
        __syncthreads();
    }
}

// Inverse of diagonal block b of the lower-triangular L: one CTA per block,
// thread c solves column c.
template <typename T>
__global__ void k_chol_diag_inv(int n, const T* __restrict__ L, T* __restrict__ Dinv, const int* gate, int want) {
    constexpr int NB = CholNB<T>::v;
    if (!gate_open(gate, want)) return;
    const int b = blockIdx.x, k0 = b * NB, kw = min(NB, n - k0), c = threadIdx.x;
    if (c >= NB) return;
    T* out = Dinv + (long long)b * NB * NB;
    T x[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        T s = T(0);
        if (r < kw && c < kw) {
            s = (r == c) ? T(1) : T(0);
            for (int l = 0; l < r; ++l) s -= L[(long long)(k0 + r) * n + k0 + l] * x[l];
            s /= L[(long long)(k0 + r) * n + k0 + r];
        }
        x[r] = s;
        out[r * NB + c] = s;
    }
}

// Block column jb of W = L^{-1}: W_jj = inv(L_jj); W_ij = -inv(L_ii) sum_{k=j}^{i-1} L_ik W_kj.
template <typename T>
__global__ void __launch_bounds__(1024) k_chol_trinv(int n, const T* __restrict__ L, const T* __restrict__ Dinv,
                                                     T* __restrict__ W, const int* gate, int want) {
    constexpr int NB = CholNB<T>::v, LD = NB + 1;
    if (!gate_open(gate, want)) return;
    extern __shared__ __align__(16) unsigned char trinv_smem[];
    const int nblk = (n + NB - 1) / NB, jb = blockIdx.x;
    T* Wc = (T*)trinv_smem;        // [nblk][NB][LD] blocks of this column
    T* S = Wc + nblk * NB * LD;    // NB x LD
    const int r = threadIdx.x / NB, c = threadIdx.x % NB;  // NB x NB threads
    const bool act = threadIdx.x < NB * NB;
    if (act) Wc[(jb * NB + r) * LD + c] = Dinv[(long long)jb * NB * NB + r * NB + c];
    __syncthreads();
    for (int ib = jb + 1; ib < nblk; ++ib) {
        if (act) {
            T s = T(0);
            const int gi = ib * NB + r;
            if (gi < n)
                for (int kb = jb; kb < ib; ++kb)
                    for (int mm = 0; mm < NB; ++mm) {
                        const int gk = kb * NB + mm;
                        if (gk < n) s += L[(long long)gi * n + gk] * Wc[(kb * NB + mm) * LD + c];
                    }
            S[r * LD + c] = s;
        }
        __syncthreads();
        if (act) {
            T s = T(0);
            for (int mm = 0; mm < NB; ++mm) s += Dinv[(long long)ib * NB * NB + r * NB + mm] * S[mm * LD + c];
            Wc[(ib * NB + r) * LD + c] = -s;
        }
        __syncthreads();
    }
    // write the column of blocks: W[gi][jb*NB + c]
    for (int i = threadIdx.x; i < nblk * NB * NB; i += blockDim.x) {
        const int bi = i / (NB * NB), rr = (i / NB) % NB, cc = i % NB;
        const int gi = bi * NB + rr, gj = jb * NB + cc;
        if (gi < n && gj < n) W[(long long)gi * n + gj] = (bi >= jb) ? Wc[(bi * NB + rr) * LD + cc] : T(0);
    }
}

// A^{-1} = W^T W (W = L^{-1} lower triangular, type TW), stored in T; fixed
// rows and columns zero.
template <typename TW, typename T>
__global__ void k_chol_wtw(int n, const TW* __restrict__ W, const uint8_t* __restrict__ fixed,
                           T* __restrict__ Ainv, const int* gate, int want) {
    if (!gate_open(gate, want)) return;
    const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    TW s = TW(0);
    if (!fixed[i] && !fixed[j])
        for (int k = max(i, j); k < n; ++k) s += W[(long long)k * n + i] * W[(long long)k * n + j];
    Ainv[(long long)i * n + j] = (T)s;
}

// One factorization branch: Cholesky of A (type TF), diagonal-block inverses,
// W = L^{-1} and Ainv = W^T W. flag: the Cholesky's status word.
template <typename TF, typename T>
static void chol_inverse(int nc, TF* A, TF* work, TF* dblk, int* flag, TF flag_ratio, const uint8_t* fixed,
                         T* Ainv, const int* gate, int want, cudaStream_t st) {
    constexpr int NB = CholNB<TF>::v;
    const int nblk = (nc + NB - 1) / NB;
    const int smem_chol = (NB * (NB + 1) + nc * (NB + 1)) * (int)sizeof(TF);
    const int smem_trinv = (nblk * NB * (NB + 1) + NB * (NB + 1)) * (int)sizeof(TF);
    TOPO_CUDA(cudaFuncSetAttribute(k_chol_blocked<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_chol));
    TOPO_CUDA(cudaFuncSetAttribute(k_chol_trinv<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_trinv));
    k_chol_blocked<TF><<<1, 1024, smem_chol, st>>>(nc, A, work, flag, flag_ratio, gate, want);
    TOPO_CHECK_LAUNCH();
    k_chol_diag_inv<TF><<<nblk, 32, 0, st>>>(nc, A, dblk, gate, want);
    TOPO_CHECK_LAUNCH();
    k_chol_trinv<TF><<<nblk, NB * NB, smem_trinv, st>>>(nc, A, dblk, work, gate, want);
    TOPO_CHECK_LAUNCH();
    k_chol_wtw<TF, T><<<dim3(div_up(nc, 128), nc), 128, 0, st>>>(nc, work, fixed, Ainv, gate, want);
    TOPO_CHECK_LAUNCH();
}

template <typename T>
__global__ void k_dense_apply(int n, const T* __restrict__ Ainv, const T* __restrict__ r, T* __restrict__ z,
                              const int* skip) {
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested before the store, so its load overlaps the others
    const int lane = threadIdx.x & 31;
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    double s = 0.0;
    for (int k = lane; k < n; k += 32) s += (double)Ainv[i * n + k] * (double)r[k];
    s = warp_sum(s);
    if (lane == 0 && !sk) z[i] = (T)s;
}

// ------------------------------------------------------------ host side

static constexpr long long DENSE_MAX = 1024;
static constexpr long long FUSE_MAX_NODES = 16384;  // coarse levels with the fused prolongation
static constexpr long long COARSE_TARGET = 1500;

template <typename U, typename T>
static U* mg_alloc(MG<T>* mg, size_t bytes) {
    void* p = nullptr;
    TOPO_CUDA(cudaMalloc(&p, bytes + 16));
    mg->allocs.push_back(p);
    return (U*)p;
}

template <typename T>
MG<T>* mg_create(to_grid* g, int max_levels, int nu, double omega) {
    MG<T>* mg = new MG<T>();
    try {
        mg->fuse_up = g->p.mg_unfused == 0;
        mg->nu = nu;
        mg->omega = (T)omega;
        mg->omega_c = (T)(g->p.mg_omega_coarse > 0.0 ? g->p.mg_omega_coarse : omega);
        Dims d = g->d;
        const int dim = d.dim;
        mg->lev.push_back(MGLevel<T>());
        mg->lev[0].d = d;
        for (;;) {
            const Dims& c = mg->lev.back().d;
            if (c.ndof <= COARSE_TARGET) break;
            if (max_levels > 0 && (int)mg->lev.size() >= max_levels) break;
            if (c.nelx < 2 && c.nely < 2 && (dim == 2 || c.nelz < 2)) break;
            // ceil(n / 2): an odd grid coarsens too, its last coarse element covering one fine layer
            MGLevel<T> L;
            L.d = make_dims(dim, (c.nelx + 1) / 2, (c.nely + 1) / 2, dim == 3 ? (c.nelz + 1) / 2 : 0);
            mg->lev.push_back(L);
        }
        mg->nlev = (int)mg->lev.size();
        const int D = dim == 3 ? 24 : 8, NS = dim == 3 ? 27 : 9;
        for (int l = 0; l < mg->nlev; ++l) {
            MGLevel<T>& L = mg->lev[l];
            const long long nd = L.d.ndof;
            L.dinv = mg_alloc<T>(mg, nd * sizeof(T));
            L.z = mg_alloc<T>(mg, nd * sizeof(T));
            L.t = mg_alloc<T>(mg, nd * sizeof(T));
            L.w = mg_alloc<T>(mg, nd * sizeof(T));
            L.r = l > 0 ? mg_alloc<T>(mg, nd * sizeof(T)) : nullptr;
            L.fixed = l > 0 ? mg_alloc<uint8_t>(mg, nd) : g->fixed;
            const bool need_stencil = l > 0 || (mg->nlev == 1 && nd <= DENSE_MAX);
            if (need_stencil) {
                L.Kel = mg_alloc<T>(mg, L.d.nel * D * D * sizeof(T));
                L.S = mg_alloc<T>(mg, (size_t)NS * dim * dim * L.d.nnodes * sizeof(T));
                L.R = mg_alloc<T>(mg, (size_t)dim * dim * L.d.nnodes * sizeof(T));
                if (l > 0) L.touched = mg_alloc<uint8_t>(mg, L.d.nel);
            }
        }
        const Dims& dc = mg->lev.back().d;
        if (dc.ndof <= DENSE_MAX) {
            mg->nc = (int)dc.ndof;
            mg->A = mg_alloc<double>(mg, (size_t)mg->nc * mg->nc * sizeof(double));
            mg->A_work = mg_alloc<double>(mg, (size_t)mg->nc * mg->nc * sizeof(double));
            mg->Dblk = mg_alloc<double>(mg, (size_t)(mg->nc + CholNB<double>::v) * CholNB<double>::v * sizeof(double));
            if (sizeof(T) == 4) {
                mg->A32 = mg_alloc<float>(mg, (size_t)mg->nc * mg->nc * sizeof(float));
                mg->A32_work = mg_alloc<float>(mg, (size_t)mg->nc * mg->nc * sizeof(float));
                mg->Dblk32 = mg_alloc<float>(mg, (size_t)(mg->nc + CholNB<float>::v) * CholNB<float>::v * sizeof(float));
            }
            mg->Ainv = mg_alloc<T>(mg, (size_t)mg->nc * mg->nc * sizeof(T));
            mg->status = mg_alloc<int>(mg, 2 * sizeof(int));
            TOPO_CUDA(cudaMemset(mg->status, 0, 2 * sizeof(int)));
        }
        if (mg->nlev > 1) {
            // C_j = P_j^T Ke P_j for the children j of a coarse element (level-1 fast path)
            const int NN = dim == 3 ? 8 : 4, DD = D * D;
            std::vector<T> C((size_t)NN * DD);
            for (int j = 0; j < NN; ++j)
                for (int A = 0; A < NN; ++A)
                    for (int c = 0; c < dim; ++c)
                        for (int B = 0; B < NN; ++B)
                            for (int k = 0; k < dim; ++k) {
                                double s = 0.0;
                                for (int a = 0; a < NN; ++a)
                                    for (int b = 0; b < NN; ++b)
                                        s += pn_weight_host(dim, j, a, A) * g->Ke_host[(size_t)(a * dim + c) * D + b * dim + k] *
                                             pn_weight_host(dim, j, b, B);
                                C[(size_t)j * DD + (A * dim + c) * D + B * dim + k] = (T)s;
                            }
            mg->Cj = mg_alloc<T>(mg, C.size() * sizeof(T));
            TOPO_CUDA(cudaMemcpy(mg->Cj, C.data(), C.size() * sizeof(T), cudaMemcpyHostToDevice));
        }
        if (dim == 3) {
            const int smem = 2 * 8 * 24 * 24 * (int)sizeof(T);
            TOPO_CUDA(cudaFuncSetAttribute(k_galerkin<T, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            TOPO_CUDA(cudaFuncSetAttribute(k_galerkin<T, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        }
    } catch (...) {
        mg_destroy(mg);
        throw;
    }
    return mg;
}

template <typename T>
void mg_destroy(MG<T>* mg) {
    if (!mg) return;
    if (mg->side) {
        cudaStreamSynchronize(mg->side);
        cudaStreamDestroy(mg->side);
    }
    if (mg->fork) cudaEventDestroy(mg->fork);
    if (mg->ready) cudaEventDestroy(mg->ready);
    for (void* p : mg->allocs) cudaFree(p);
    delete mg;
}

template <typename T>
void mg_wait_coarse(MG<T>* mg, cudaStream_t st) {
    if (!mg->pending) return;
    TOPO_CUDA(cudaStreamWaitEvent(st, mg->ready, 0));
    mg->pending = false;
}

template <typename T, int DIM>
static void setup_dim(to_grid* g, MG<T>* mg, const T* E, cudaStream_t st) {
    constexpr int D = DIM == 3 ? 24 : 8;
    const int smem = 2 * (DIM == 3 ? 8 : 4) * D * D * (int)sizeof(T);
    RowAbs<T, DIM> ra;
    for (int r = 0; r < D; ++r) {
        double s = 0.0;
        for (int j = 0; j < D; ++j) s += std::fabs(g->Ke_host[(size_t)r * D + j]);
        ra.a[r] = (T)s;
    }
    k_l1_inv<T, DIM><<<div_up(g->d.nnodes, 256), 256, 0, st>>>(g->d, ra, E, g->fixed, mg->lev[0].dinv);
    TOPO_CHECK_LAUNCH();
    for (int l = 0; l < mg->nlev; ++l) {
        MGLevel<T>& L = mg->lev[l];
        if (!L.S) continue;
        if (l == 0) {
            k_elem_from_E<T, DIM><<<div_up(L.d.nel * D * D, 256), 256, 0, st>>>(L.d, E, g->Ke_dev, L.Kel);
        } else if (l == 1) {
            k_galerkin<T, DIM, true><<<(unsigned)L.d.nel, 256, smem, st>>>(L.d, mg->lev[0].d, E, g->Ke_dev, mg->Cj,
                                                                       nullptr, g->fixed, nullptr, L.Kel,
                                                                       L.touched);
        } else {
            k_galerkin<T, DIM, false><<<(unsigned)L.d.nel, 256, smem, st>>>(
                L.d, mg->lev[l - 1].d, nullptr, nullptr, nullptr, mg->lev[l - 1].Kel, nullptr,
                mg->lev[l - 1].touched, L.Kel, L.touched);
        }
        TOPO_CHECK_LAUNCH();
        if (DIM == 3) {
            constexpr int NB = StencilNodes<T>::v;
            k_stencil_build3s<T><<<div_up(L.d.nnodes, NB), dim3(NB, 27), 0, st>>>(L.d, L.Kel, L.touched, L.S, L.R);
        } else {
            k_stencil_build<T, DIM><<<div_up(L.d.nnodes, 128), 128, 0, st>>>(L.d, L.Kel, L.touched, L.S, L.R);
        }
        TOPO_CHECK_LAUNCH();
        if (l > 0) {
            k_stencil_diag<T, DIM><<<div_up(L.d.nnodes, 256), 256, 0, st>>>(L.d, L.S, L.dinv, L.fixed);
            TOPO_CHECK_LAUNCH();
        }
    }
    const bool refactor = mg->setups++ % mg->coarse_every == 0;
    if (mg->nc > 0 && refactor) {
        MGLevel<T>& L = mg->lev.back();
        if (!mg->side) {
            TOPO_CUDA(cudaStreamCreateWithFlags(&mg->side, cudaStreamNonBlocking));
            TOPO_CUDA(cudaEventCreateWithFlags(&mg->fork, cudaEventDisableTiming));
            TOPO_CUDA(cudaEventCreateWithFlags(&mg->ready, cudaEventDisableTiming));
        }
        // the rest of this set-up runs on the side stream; mg_wait_coarse joins it
        TOPO_CUDA(cudaEventRecord(mg->fork, st));
        TOPO_CUDA(cudaStreamWaitEvent(mg->side, mg->fork, 0));
        st = mg->side;
        const size_t nn2 = (size_t)mg->nc * mg->nc;
        TOPO_CUDA(cudaMemsetAsync(mg->A, 0, nn2 * sizeof(double), st));
        if (mg->A32) TOPO_CUDA(cudaMemsetAsync(mg->A32, 0, nn2 * sizeof(float), st));
        k_dense_assemble<T, DIM><<<div_up(L.d.nnodes, 64), 64, 0, st>>>(L.d, L.S, L.R, L.fixed, mg->A, mg->A32);
        TOPO_CHECK_LAUNCH();
        // work holds the original diagonal during a factorization, then W = L^{-1};
        // dblk the inverses of L's diagonal blocks
        if (mg->A32) {
            chol_inverse<float, T>(mg->nc, mg->A32, mg->A32_work, mg->Dblk32, mg->status, 1e-4f, L.fixed,
                                   mg->Ainv, nullptr, 1, st);
            chol_inverse<double, T>(mg->nc, mg->A, mg->A_work, mg->Dblk, mg->status + 1, 1e-6, L.fixed, mg->Ainv,
                                    mg->status, 1, st);
        } else {
            chol_inverse<double, T>(mg->nc, mg->A, mg->A_work, mg->Dblk, mg->status + 1, 1e-6, L.fixed, mg->Ainv,
                                    nullptr, 1, st);
        }
        TOPO_CUDA(cudaEventRecord(mg->ready, st));
        mg->pending = true;
    }
}

template <typename T>
void mg_setup(to_grid* g, MG<T>* mg, const T* E, cudaStream_t st) {
    // the previous factorization may still read the coarsest stencils when no V-cycle joined it
    mg_wait_coarse<T>(mg, st);
    mg->E = E;
    if (g->d.dim == 3)
        setup_dim<T, 3>(g, mg, E, st);
    else
        setup_dim<T, 2>(g, mg, E, st);
}

template <typename T>
static void level_op(to_grid* g, MG<T>* mg, int l, int mode, const T* E, const T* u, const T* r, T* out,
                     const int* skip, cudaStream_t st, PcgScalars* pcg = nullptr) {
    MGLevel<T>& L = mg->lev[l];
    if (l == 0) {
        launch_fine_op<T>(g, mode, E, u, r, L.dinv, out, mg->omega, skip, pcg, st);
        return;
    }
    const int nb = div_up(L.d.nnodes, 256);
    const T w = mg->omega_c;
#define TOPO_SOP(DIMV, MODEV) \
    launch_k(k_stencil_op<T, DIMV, MODEV>, nb, 256, 0, st, L.d, L.S, L.R, u, r, L.dinv, out, L.fixed, w, skip)
#define TOPO_SOP3(MODEV)                                                                                  \
    launch_k(k_stencil_op3s<T, MODEV>, div_up(L.d.nnodes, 32), dim3(32, 9), 0, st, L.d, L.S, L.R, u, r, \
             L.dinv, out, L.fixed, w, skip)
    if (L.d.dim == 3) {
        if (mode == 1) TOPO_SOP3(1); else if (mode == 2) TOPO_SOP3(2); else TOPO_SOP3(0);
    } else {
        if (mode == 1) TOPO_SOP(2, 1); else if (mode == 2) TOPO_SOP(2, 2); else TOPO_SOP(2, 0);
    }
#undef TOPO_SOP3
#undef TOPO_SOP
}

template <typename T>
static T* vcycle_level(to_grid* g, MG<T>* mg, int l, const T* E, const T* rhs, const int* skip, cudaStream_t st,
                       PcgScalars* fuse_rz = nullptr, bool* fused = nullptr, bool first_done = false) {
    MGLevel<T>& L = mg->lev[l];
    const bool coarsest = l == mg->nlev - 1;
    if (coarsest && mg->nc > 0) {
        launch_k(k_dense_apply<T>, div_up((long long)mg->nc * 32, 256), 256, 0, st, mg->nc, (const T*)mg->Ainv,
                 rhs, L.z, skip);
        return L.z;
    }
    if (!first_done)
        launch_k(k_jacobi_first<T>, div_up(L.d.ndof, 256), 256, 0, st, L.d.ndof, (const T*)L.dinv, rhs, L.z,
                 l == 0 ? mg->omega : mg->omega_c, skip);
    T* cur = L.z;
    T* oth = L.t;
    const int nu = coarsest ? 4 * mg->nu : (l == 0 && mg->nu_fine > 0 ? mg->nu_fine : mg->nu);
    int s0 = 0;  // post-smoothing sweeps already done (1 when fused with the prolongation)
    for (int s = 1; s < nu; ++s) {
        level_op<T>(g, mg, l, 1, E, cur, rhs, oth, skip, st);
        std::swap(cur, oth);
    }
    if (!coarsest) {
        level_op<T>(g, mg, l, 2, E, cur, rhs, L.w, skip, st);
        MGLevel<T>& C = mg->lev[l + 1];
        const int nbc = div_up(C.d.nnodes, 256), nbf = div_up(L.d.nnodes, 256);
        // the coarse level's first Jacobi iterate is formed by the restriction
        // unless that level is the dense coarsest
        const bool jf = !(l + 1 == mg->nlev - 1 && mg->nc > 0);
        const T* dc_inv = jf ? C.dinv : nullptr;
        if (L.d.dim == 3)
            launch_k(k_restrict3s<T>, div_up(C.d.nnodes, 32), dim3(32, 9), 0, st, C.d, L.d, (const T*)L.w, C.r,
                     (const uint8_t*)C.fixed, skip, dc_inv, C.z, mg->omega_c);
        else
            launch_k(k_restrict<T, 2>, nbc, 256, 0, st, C.d, L.d, (const T*)L.w, C.r, (const uint8_t*)C.fixed,
                     skip, dc_inv, C.z, mg->omega_c);
        T* zc = vcycle_level<T>(g, mg, l + 1, E, C.r, skip, st, nullptr, nullptr, jf);
        // small levels only: on a large one the halo's repeated prolongation costs
        // more loads than the separate kernel (tiles are one node thick in x)
        if (L.d.dim == 3 && l > 0 && mg->fuse_up && L.d.nnodes <= FUSE_MAX_NODES) {
            // the prolongation inside the first post-smoothing sweep
            const int ty = prolong_smooth_ty(L.d);
            const long long nb = (long long)div_up(L.d.nny, ty) * div_up(L.d.nnz, 32 / ty) * L.d.nnx;
            const dim3 blk(32, 9);
#define TOPO_PS(TYV)                                                                                   \
    launch_k(k_prolong_smooth3s<T, TYV>, (unsigned)nb, blk, 0, st, L.d, C.d, (const T*)zc, (const T*)cur, \
             (const T*)L.S, (const T*)L.R, rhs, (const T*)L.dinv, oth, (const uint8_t*)L.fixed, mg->omega_c, skip)
            if (ty == 8)
                TOPO_PS(8);
            else if (ty == 16)
                TOPO_PS(16);
            else
                TOPO_PS(32);
#undef TOPO_PS
            std::swap(cur, oth);
            s0 = 1;
        } else {
            if (L.d.dim == 3)
                launch_k(k_prolong_add<T, 3>, nbf, 256, 0, st, L.d, C.d, (const T*)zc, cur,
                         (const uint8_t*)L.fixed, skip);
            else
                launch_k(k_prolong_add<T, 2>, nbf, 256, 0, st, L.d, C.d, (const T*)zc, cur,
                         (const uint8_t*)L.fixed, skip);
        }
    }
    for (int s = s0; s < nu; ++s) {
        // the last fine-level sweep also forms r.z and the PCG beta when asked to
        const bool last = l == 0 && s == nu - 1 && fuse_rz;
        level_op<T>(g, mg, l, 1, E, cur, rhs, oth, skip, st, last ? fuse_rz : nullptr);
        if (last && fused) *fused = true;
        std::swap(cur, oth);
    }
    return cur;
}

template <typename T>
T* mg_vcycle(to_grid* g, MG<T>* mg, const T* r, const int* skip, cudaStream_t st, PcgScalars* fuse_rz,
             bool* fused, bool first_done) {
    if (fused) *fused = false;
    return vcycle_level<T>(g, mg, 0, mg->E, r, skip, st, fuse_rz, fused, first_done);
}

template MG<double>* mg_create<double>(to_grid*, int, int, double);
template MG<float>* mg_create<float>(to_grid*, int, int, double);
template void mg_destroy<double>(MG<double>*);
template void mg_destroy<float>(MG<float>*);
template void mg_wait_coarse<double>(MG<double>*, cudaStream_t);
template void mg_wait_coarse<float>(MG<float>*, cudaStream_t);
template void mg_setup<double>(to_grid*, MG<double>*, const double*, cudaStream_t);
template void mg_setup<float>(to_grid*, MG<float>*, const float*, cudaStream_t);
template double* mg_vcycle<double>(to_grid*, MG<double>*, const double*, const int*, cudaStream_t, PcgScalars*,
                                     bool*, bool);
template float* mg_vcycle<float>(to_grid*, MG<float>*, const float*, const int*, cudaStream_t, PcgScalars*,
                                   bool*, bool);

}  // namespace topo
