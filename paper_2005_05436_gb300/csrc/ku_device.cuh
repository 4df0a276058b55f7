// Per-element device helpers of the node-centric stiffness operator.
//
// The thread of node n visits the (up to) 2^dim elements around it; for each it
// accumulates E_e * Ke[rows of n's local DOFs, :] * u_e. EXO/EYO/EZO select the
// element (ex = ix - 1 + EXO, ...), so every Ke index is a compile-time constant.
// With REL, every gathered displacement is taken relative to u_n: the element
// rows annihilate rigid translations, so the product is unchanged in exact
// arithmetic, while FP32 rounding then acts on displacement differences instead
// of (possibly large) absolute displacements.
#pragma once

#include "common.cuh"

namespace topo {

// Local node index of the corner (ax, ay, az) of the unit element, ay = 1 for
// the top row (physical Y up): (0,0,0) (1,0,0) (1,1,0) (0,1,0), then z = 1.
__host__ __device__ constexpr int local_node(int ax, int ay, int az) {
    return 4 * az + (ay ? (ax ? 2 : 3) : (ax ? 1 : 0));
}
__host__ __device__ constexpr int lnx(int M) { return ((M & 3) == 1 || (M & 3) == 2) ? 1 : 0; }
__host__ __device__ constexpr int lny(int M) { return (M & 3) >= 2 ? 1 : 0; }
__host__ __device__ constexpr int lnz(int M) { return M >> 2; }

template <typename T, int EXO, int EYO, int EZO, bool REL = false>
__device__ __forceinline__ void ku3_elem(const KeP<T, 24>& ke, const T* __restrict__ E,
                                         const T* __restrict__ u, long long n, int ix, int iy, int iz,
                                         const Dims& d, long long sz, long long sx, T& a0, T& a1,
                                         T& a2, T c0 = T(0), T c1 = T(0), T c2 = T(0)) {
    const int ex = ix - 1 + EXO, ey = iy - 1 + EYO, ez = iz - 1 + EZO;
    if (ex < 0 || ex >= d.nelx || ey < 0 || ey >= d.nely || ez < 0 || ez >= d.nelz) return;
    const T Ee = E[ey + (long long)d.nely * (ez + (long long)d.nelz * ex)];
    constexpr int L = local_node(1 - EXO, EYO, 1 - EZO);
    T t0 = T(0), t1 = T(0), t2 = T(0);
#pragma unroll
    for (int M = 0; M < 8; ++M) {
        if (REL && M == local_node(1 - EXO, EYO, 1 - EZO)) continue;  // u_n - u_n = 0
        const long long m = n + (EYO - lny(M)) + sz * (EZO - 1 + lnz(M)) + sx * (EXO - 1 + lnx(M));
        T u0 = u[3 * m], u1 = u[3 * m + 1], u2 = u[3 * m + 2];
        if (REL) {
            u0 -= c0;
            u1 -= c1;
            u2 -= c2;
        }
        t0 += ke.k[(3 * L + 0) * 24 + 3 * M + 0] * u0 + ke.k[(3 * L + 0) * 24 + 3 * M + 1] * u1 +
              ke.k[(3 * L + 0) * 24 + 3 * M + 2] * u2;
        t1 += ke.k[(3 * L + 1) * 24 + 3 * M + 0] * u0 + ke.k[(3 * L + 1) * 24 + 3 * M + 1] * u1 +
              ke.k[(3 * L + 1) * 24 + 3 * M + 2] * u2;
        t2 += ke.k[(3 * L + 2) * 24 + 3 * M + 0] * u0 + ke.k[(3 * L + 2) * 24 + 3 * M + 1] * u1 +
              ke.k[(3 * L + 2) * 24 + 3 * M + 2] * u2;
    }
    a0 += Ee * t0;
    a1 += Ee * t1;
    a2 += Ee * t2;
}

template <typename T, int EXO, int EYO, bool REL = false>
__device__ __forceinline__ void ku2_elem(const KeP<T, 8>& ke, const T* __restrict__ E,
                                         const T* __restrict__ u, long long n, int ix, int iy,
                                         const Dims& d, long long sx, T& a0, T& a1, T c0 = T(0),
                                         T c1 = T(0)) {
    const int ex = ix - 1 + EXO, ey = iy - 1 + EYO;
    if (ex < 0 || ex >= d.nelx || ey < 0 || ey >= d.nely) return;
    const T Ee = E[ey + (long long)d.nely * ex];
    constexpr int L = local_node(1 - EXO, EYO, 0);
    T t0 = T(0), t1 = T(0);
#pragma unroll
    for (int M = 0; M < 4; ++M) {
        if (REL && M == local_node(1 - EXO, EYO, 0)) continue;
        const long long m = n + (EYO - lny(M)) + sx * (EXO - 1 + lnx(M));
        T u0 = u[2 * m], u1 = u[2 * m + 1];
        if (REL) {
            u0 -= c0;
            u1 -= c1;
        }
        t0 += ke.k[(2 * L + 0) * 8 + 2 * M] * u0 + ke.k[(2 * L + 0) * 8 + 2 * M + 1] * u1;
        t1 += ke.k[(2 * L + 1) * 8 + 2 * M] * u0 + ke.k[(2 * L + 1) * 8 + 2 * M + 1] * u1;
    }
    a0 += Ee * t0;
    a1 += Ee * t1;
}

// y_n = (K u)_n for one node (3D); REL as above.
template <typename T, bool REL>
__device__ __forceinline__ void ku3_node(const KeP<T, 24>& ke, const T* __restrict__ E,
                                         const T* __restrict__ u, long long n, const Dims& d, T& a0,
                                         T& a1, T& a2) {
    const long long sz = d.nny, sx = (long long)d.nny * d.nnz;
    const int iy = (int)(n % d.nny);
    const long long t = n / d.nny;
    const int iz = (int)(t % d.nnz);
    const int ix = (int)(t / d.nnz);
    T c0 = T(0), c1 = T(0), c2 = T(0);
    if (REL) {
        c0 = u[3 * n];
        c1 = u[3 * n + 1];
        c2 = u[3 * n + 2];
    }
    a0 = a1 = a2 = T(0);
    ku3_elem<T, 0, 0, 0, REL>(ke, E, u, n, ix, iy, iz, d, sz, sx, a0, a1, a2, c0, c1, c2);
    ku3_elem<T, 0, 1, 0, REL>(ke, E, u, n, ix, iy, iz, d, sz, sx, a0, a1, a2, c0, c1, c2);
    ku3_elem<T, 0, 0, 1, REL>(ke, E, u, n, ix, iy, iz, d, sz, sx, a0, a1, a2, c0, c1, c2);
    ku3_elem<T, 0, 1, 1, REL>(ke, E, u, n, ix, iy, iz, d, sz, sx, a0, a1, a2, c0, c1, c2);
    ku3_elem<T, 1, 0, 0, REL>(ke, E, u, n, ix, iy, iz, d, sz, sx, a0, a1, a2, c0, c1, c2);
    ku3_elem<T, 1, 1, 0, REL>(ke, E, u, n, ix, iy, iz, d, sz, sx, a0, a1, a2, c0, c1, c2);
    ku3_elem<T, 1, 0, 1, REL>(ke, E, u, n, ix, iy, iz, d, sz, sx, a0, a1, a2, c0, c1, c2);
    ku3_elem<T, 1, 1, 1, REL>(ke, E, u, n, ix, iy, iz, d, sz, sx, a0, a1, a2, c0, c1, c2);
}

// The same product with the 27-node neighbourhood of n loaded into registers
// once (relative to u_n) instead of once per element: 78 loads instead of 168.
template <typename T, int EXO, int EYO, int EZO>
__device__ __forceinline__ void ku3_elem_regs(const KeP<T, 24>& ke, const T* __restrict__ E, const T (&w)[27][3],
                                              int ix, int iy, int iz, const Dims& d, T& a0, T& a1, T& a2) {
    const int ex = ix - 1 + EXO, ey = iy - 1 + EYO, ez = iz - 1 + EZO;
    if (ex < 0 || ex >= d.nelx || ey < 0 || ey >= d.nely || ez < 0 || ez >= d.nelz) return;
    const T Ee = E[ey + (long long)d.nely * (ez + (long long)d.nelz * ex)];
    constexpr int L = local_node(1 - EXO, EYO, 1 - EZO);
    T t0 = T(0), t1 = T(0), t2 = T(0);
#pragma unroll
    for (int M = 0; M < 8; ++M) {
        if (M == L) continue;
        const int q = (EXO + lnx(M)) * 9 + (EZO + lnz(M)) * 3 + (EYO - lny(M) + 1);
        const T u0 = w[q][0], u1 = w[q][1], u2 = w[q][2];
        t0 += ke.k[(3 * L + 0) * 24 + 3 * M + 0] * u0 + ke.k[(3 * L + 0) * 24 + 3 * M + 1] * u1 +
              ke.k[(3 * L + 0) * 24 + 3 * M + 2] * u2;
        t1 += ke.k[(3 * L + 1) * 24 + 3 * M + 0] * u0 + ke.k[(3 * L + 1) * 24 + 3 * M + 1] * u1 +
              ke.k[(3 * L + 1) * 24 + 3 * M + 2] * u2;
        t2 += ke.k[(3 * L + 2) * 24 + 3 * M + 0] * u0 + ke.k[(3 * L + 2) * 24 + 3 * M + 1] * u1 +
              ke.k[(3 * L + 2) * 24 + 3 * M + 2] * u2;
    }
    a0 += Ee * t0;
    a1 += Ee * t1;
    a2 += Ee * t2;
}

template <typename T>
__device__ __forceinline__ void ku3_node_regs(const KeP<T, 24>& ke, const T* __restrict__ E,
                                              const T* __restrict__ u, long long n, const Dims& d, T& a0, T& a1,
                                              T& a2) {
    const long long sz = d.nny, sx = (long long)d.nny * d.nnz;
    const int iy = (int)(n % d.nny);
    const long long t = n / d.nny;
    const int iz = (int)(t % d.nnz);
    const int ix = (int)(t / d.nnz);
    const T c0 = u[3 * n], c1 = u[3 * n + 1], c2 = u[3 * n + 2];
    T w[27][3];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        const int dx = q / 9 - 1, dz = (q / 3) % 3 - 1, dy = q % 3 - 1;
        const bool ok = q != 13 && ix + dx >= 0 && ix + dx < d.nnx && iz + dz >= 0 && iz + dz < d.nnz &&
                        iy + dy >= 0 && iy + dy < d.nny;
        const long long m = n + dy + sz * dz + sx * dx;
        w[q][0] = ok ? u[3 * m] - c0 : T(0);
        w[q][1] = ok ? u[3 * m + 1] - c1 : T(0);
        w[q][2] = ok ? u[3 * m + 2] - c2 : T(0);
    }
    a0 = a1 = a2 = T(0);
    ku3_elem_regs<T, 0, 0, 0>(ke, E, w, ix, iy, iz, d, a0, a1, a2);
    ku3_elem_regs<T, 0, 1, 0>(ke, E, w, ix, iy, iz, d, a0, a1, a2);
    ku3_elem_regs<T, 0, 0, 1>(ke, E, w, ix, iy, iz, d, a0, a1, a2);
    ku3_elem_regs<T, 0, 1, 1>(ke, E, w, ix, iy, iz, d, a0, a1, a2);
    ku3_elem_regs<T, 1, 0, 0>(ke, E, w, ix, iy, iz, d, a0, a1, a2);
    ku3_elem_regs<T, 1, 1, 0>(ke, E, w, ix, iy, iz, d, a0, a1, a2);
    ku3_elem_regs<T, 1, 0, 1>(ke, E, w, ix, iy, iz, d, a0, a1, a2);
    ku3_elem_regs<T, 1, 1, 1>(ke, E, w, ix, iy, iz, d, a0, a1, a2);
}

template <typename T, bool REL>
__device__ __forceinline__ void ku2_node(const KeP<T, 8>& ke, const T* __restrict__ E,
                                         const T* __restrict__ u, long long n, const Dims& d, T& a0,
                                         T& a1) {
    const long long sx = d.nny;
    const int iy = (int)(n % d.nny);
    const int ix = (int)(n / d.nny);
    T c0 = T(0), c1 = T(0);
    if (REL) {
        c0 = u[2 * n];
        c1 = u[2 * n + 1];
    }
    a0 = a1 = T(0);
    ku2_elem<T, 0, 0, REL>(ke, E, u, n, ix, iy, d, sx, a0, a1, c0, c1);
    ku2_elem<T, 0, 1, REL>(ke, E, u, n, ix, iy, d, sx, a0, a1, c0, c1);
    ku2_elem<T, 1, 0, REL>(ke, E, u, n, ix, iy, d, sx, a0, a1, c0, c1);
    ku2_elem<T, 1, 1, REL>(ke, E, u, n, ix, iy, d, sx, a0, a1, c0, c1);
}

}  // namespace topo
