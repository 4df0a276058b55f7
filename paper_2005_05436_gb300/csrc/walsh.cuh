// The H8 element operator in the Walsh basis of the element's corners.
//
// The unit-cube element matrix Ke of an isotropic material (Sec. 4, App. C) is
// invariant under the three reflections of the cube (x -> 1 - x, ...), which
// act on the 24 DOFs by permuting corners and flipping the reflected
// displacement component. That group is (Z2)^3, its irreducible
// representations are the eight sign characters, and the 24-dimensional DOF
// space holds each of them three times (one per displacement component). By
// Schur's lemma Ke is therefore block diagonal in the symmetry-adapted basis
//   w[c][i] = sum_g (-1)^(c.g) u[g][i]      (c, g in {0,1}^3, i = x, y, z),
// i.e. the 8-point Walsh-Hadamard transform of each displacement component
// over the corners: eight 3x3 blocks, block k coupling the modes c = k xor e_i.
// With Ke = (1/64) H^T M H (H the unnormalised transform) the product is
//   Ke u = H^T (M (H u)),
// where M has eight distinct entries A, B, C, D, F, G, P, Q (the rigid
// translations and rotations are null modes, which zeroes whole rows), so one
// element product costs 27 + 33 + 22 additions / multiply-adds per component
// group instead of 24 x 24 multiply-adds.
//
// Corners are numbered in grid orientation: g = 4 gx + 2 gy + gz for the node
// (ex + gx, ey + gy, ez + gz); modes c = 4 cx + 2 cy + cz likewise. The signs
// below are those of that orientation (the element matrix's own local y axis
// runs against the grid's row index).
#pragma once

#include "common.cuh"

namespace topo {

// The distinct entries of M (A - B, B, C, D, F, G, P - Q, Q).
template <typename T>
struct WalshK {
    T amb, b, c, d, f, g, pmq, q;
};

// The seven non-constant Walsh modes of one component over the corners,
// formed from differences first (x-, y- and z-edges), so that rounding acts on
// displacement differences, never on absolute displacements. w[0] (the
// element mean, a rigid translation) is not formed.
template <typename T>
__host__ __device__ __forceinline__ void walsh_fwd(const T (&u)[8], T (&w)[8]) {
    const T dx00 = u[0] - u[4], dx01 = u[1] - u[5], dx10 = u[2] - u[6], dx11 = u[3] - u[7];
    const T p0 = dx00 + dx10, p1 = dx01 + dx11, q0 = dx00 - dx10, q1 = dx01 - dx11;
    w[4] = p0 + p1;
    w[5] = p0 - p1;
    w[6] = q0 + q1;
    w[7] = q0 - q1;
    const T a0 = (u[0] - u[2]) + (u[4] - u[6]), a1 = (u[1] - u[3]) + (u[5] - u[7]);
    w[2] = a0 + a1;
    w[3] = a0 - a1;
    w[1] = ((u[0] - u[1]) + (u[2] - u[3])) + ((u[4] - u[5]) + (u[6] - u[7]));
    w[0] = T(0);
}

// Inverse transform y[g] = sum_{c != 0} (-1)^(c.g) z[c] (z[0] is taken as 0).
template <typename T>
__host__ __device__ __forceinline__ void walsh_inv(const T (&z)[8], T (&y)[8]) {
    const T a01p = z[2] + z[3], a01m = z[2] - z[3];
    const T a10p = z[4] + z[5], a10m = z[4] - z[5];
    const T a11p = z[6] + z[7], a11m = z[6] - z[7];
    const T b000 = z[1] + a01p, b010 = z[1] - a01p;
    const T b001 = a01m - z[1], t = z[1] + a01m;
    const T b100 = a10p + a11p, b110 = a10p - a11p;
    const T b101 = a10m + a11m, b111 = a10m - a11m;
    y[0] = b000 + b100;
    y[4] = b000 - b100;
    y[1] = b001 + b101;
    y[5] = b001 - b101;
    y[2] = b010 + b110;
    y[6] = b010 - b110;
    y[3] = b111 - t;
    y[7] = (-t) - b111;
}

// Z = E * M * W for the three components' modes W[i][c] (W[i][0] unused).
template <typename T>
__host__ __device__ __forceinline__ void walsh_blocks(const WalshK<T>& k, T E, const T (&Wx)[8], const T (&Wy)[8],
                                                      const T (&Wz)[8], T (&Zx)[8], T (&Zy)[8], T (&Zz)[8]) {
    const T amb = E * k.amb, b = E * k.b, c = E * k.c, d = E * k.d;
    const T f = E * k.f, g = E * k.g, pmq = E * k.pmq, q = E * k.q;
    // character 000: modes (100,x) (010,y) (001,z); [[A,-B,B],[-B,A,-B],[B,-B,A]]
    {
        const T bt = b * (Wx[4] - Wy[2] + Wz[1]);
        Zx[4] = amb * Wx[4] + bt;
        Zy[2] = amb * Wy[2] - bt;
        Zz[1] = amb * Wz[1] + bt;
    }
    // 001: (101,x) (011,y); [[C,-D],[-D,C]]
    Zx[5] = c * Wx[5] - d * Wy[3];
    Zy[3] = c * Wy[3] - d * Wx[5];
    // 010: (110,x) (011,z); [[C,D],[D,C]]
    Zx[6] = c * Wx[6] + d * Wz[3];
    Zz[3] = c * Wz[3] + d * Wx[6];
    // 100: (110,y) (101,z); [[C,-D],[-D,C]]
    Zy[6] = c * Wy[6] - d * Wz[5];
    Zz[5] = c * Wz[5] - d * Wy[6];
    // 011: (111,x) alone; (001,y) (010,z) [[F,-F],[-F,F]]
    Zx[7] = g * Wx[7];
    {
        const T s = f * (Wy[1] - Wz[2]);
        Zy[1] = s;
        Zz[2] = -s;
    }
    // 101: (111,y) alone; (001,x) (100,z) [[F,F],[F,F]]
    Zy[7] = g * Wy[7];
    {
        const T s = f * (Wx[1] + Wz[4]);
        Zx[1] = s;
        Zz[4] = s;
    }
    // 110: (111,z) alone; (010,x) (100,y) [[F,-F],[-F,F]]
    Zz[7] = g * Wz[7];
    {
        const T s = f * (Wx[2] - Wy[4]);
        Zx[2] = s;
        Zy[4] = -s;
    }
    // 111: (011,x) (101,y) (110,z); [[P,-Q,Q],[-Q,P,-Q],[Q,-Q,P]]
    {
        const T qt = q * (Wx[3] - Wy[5] + Wz[6]);
        Zx[3] = pmq * Wx[3] + qt;
        Zy[5] = pmq * Wy[5] - qt;
        Zz[6] = pmq * Wz[6] + qt;
    }
    Zx[0] = Zy[0] = Zz[0] = T(0);
}

// y = E Ke u for one element: u[i][g], y[i][g] per component i, corners g.
template <typename T>
__host__ __device__ __forceinline__ void walsh_element(const WalshK<T>& k, T E, const T (&u)[3][8], T (&y)[3][8]) {
    T W[3][8], Z[3][8];
#pragma unroll
    for (int i = 0; i < 3; ++i) walsh_fwd<T>(u[i], W[i]);
    walsh_blocks<T>(k, E, W[0], W[1], W[2], Z[0], Z[1], Z[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) walsh_inv<T>(Z[i], y[i]);
}

// Host: the Walsh constants of a row-major 24 x 24 element matrix in the local
// node order of ku_device.cuh, and the largest deviation of M from the block
// pattern above (relative to max |M|). Returns false if the deviation exceeds
// 1e-12 (the element matrix lacks the cube's symmetry).
bool walsh_constants(const double* Ke, WalshK<double>& k, double* max_dev);

}  // namespace topo
