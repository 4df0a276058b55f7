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

// Element contribution with a modulus that is already 0 for elements outside
// the grid (no branch): every element around the node is evaluated.
template <typename T, int EXO, int EYO, int EZO>
__device__ __forceinline__ void ku3_elem_w(const KeP<T, 24>& ke, T Ee, const T (&w)[27][3], T& a0, T& a1,
                                           T& a2) {
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

// y_n = (K u)_n for one node (3D), relative to u_n (REL as above), with the
// 27-node neighbourhood loaded into registers once. Neighbour offsets are
// clamped once per axis, so a missing neighbour aliases an existing node, and the
// modulus of every element outside the grid is taken as exactly 0. A clamped
// neighbour only feeds elements outside the grid (its out-of-range coordinate
// is also theirs), whose zero modulus adds +-0 to the rows: the result equals
// skipping those elements. All offsets are 32-bit (grids below 2^31 / 3 nodes,
// checked at handle creation).
template <typename T>
__device__ __forceinline__ void ku3_node_clamped(const KeP<T, 24>& ke, const T* __restrict__ E,
                                                 const T* __restrict__ u, int n, const Dims& d, T& a0, T& a1,
                                                 T& a2) {
    const int nny = d.nny, nnz = d.nnz;
    const int iy = n % nny;
    const int t = n / nny;
    const int iz = t % nnz;
    const int ix = t / nnz;
    const int sz = 3 * nny, sx = 3 * nny * nnz;
    const int oy[3] = {iy > 0 ? -3 : 0, 0, iy < nny - 1 ? 3 : 0};
    const int oz[3] = {iz > 0 ? -sz : 0, 0, iz < nnz - 1 ? sz : 0};
    const int ox[3] = {ix > 0 ? -sx : 0, 0, ix < d.nnx - 1 ? sx : 0};
    const T* p = u + 3 * n;
    const T c0 = p[0], c1 = p[1], c2 = p[2];
    T w[27][3];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        if (q == 13) {
            w[q][0] = w[q][1] = w[q][2] = T(0);
            continue;
        }
        const T* pm = p + (ox[q / 9] + oz[(q / 3) % 3] + oy[q % 3]);
        w[q][0] = pm[0] - c0;
        w[q][1] = pm[1] - c1;
        w[q][2] = pm[2] - c2;
    }
    // Element moduli: element (ix-1+EXO, iy-1+EYO, iz-1+EZO), 0 outside the grid.
    const int nely = d.nely, nelz = d.nelz;
    const int eyc[2] = {iy > 0 ? iy - 1 : 0, iy < nely ? iy : nely - 1};
    const int ezc[2] = {iz > 0 ? iz - 1 : 0, iz < nelz ? iz : nelz - 1};
    const int exc[2] = {ix > 0 ? ix - 1 : 0, ix < d.nelx ? ix : d.nelx - 1};
    const bool vy[2] = {iy > 0, iy < nely}, vz[2] = {iz > 0, iz < nelz}, vx[2] = {ix > 0, ix < d.nelx};
    T Ev[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int bx = k >> 2, bz = (k >> 1) & 1, by = k & 1;
        const T e = E[eyc[by] + nely * (ezc[bz] + nelz * exc[bx])];
        Ev[k] = (vx[bx] && vy[by] && vz[bz]) ? e : T(0);
    }
    a0 = a1 = a2 = T(0);
    ku3_elem_w<T, 0, 0, 0>(ke, Ev[0], w, a0, a1, a2);
    ku3_elem_w<T, 0, 1, 0>(ke, Ev[1], w, a0, a1, a2);
    ku3_elem_w<T, 0, 0, 1>(ke, Ev[2], w, a0, a1, a2);
    ku3_elem_w<T, 0, 1, 1>(ke, Ev[3], w, a0, a1, a2);
    ku3_elem_w<T, 1, 0, 0>(ke, Ev[4], w, a0, a1, a2);
    ku3_elem_w<T, 1, 1, 0>(ke, Ev[5], w, a0, a1, a2);
    ku3_elem_w<T, 1, 0, 1>(ke, Ev[6], w, a0, a1, a2);
    ku3_elem_w<T, 1, 1, 1>(ke, Ev[7], w, a0, a1, a2);
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
