// FP32 matrix-free 3D K u with the Walsh-factored element product (walsh.cuh),
// two elements per thread in paired FP32 arithmetic (f32x2.cuh).
//
// Thread (ty, tz) of a block owns the element column pair (ey, A) and (ey, B),
// B = A + 1, in the (y, z) plane and marches along x; lane 0 of each F2
// register is element A, lane 1 element B, so every operation of the element
// product (forward Walsh transform, E-scaled blocks, inverse transform) is one
// paired instruction for both elements. A block covers TY element columns in y
// (all of them when nely <= 128, so no y halo) and TZ pairs in z, the first
// element row of every z tile but the first being a halo row; it owns the node
// rows whose contributing elements it computes. Node planes are staged into
// shared memory three deep with cp.async (zero outside the grid). The forward
// transform takes the differences within a node plane once per plane and
// reuses them for the two element layers that share the plane. Corner results
// are summed along x in registers (the +x corners carry to the next step),
// inside the pair along z, along y by warp shuffle (lane 0 of a warp through
// shared memory) and across pairs along z through shared memory: one barrier
// per plane. Each output is written once by one thread in a fixed summation
// order (deterministic, no atomics). Fused epilogues as in kernels_walsh.cu:
// K u, the damped Jacobi sweep, the residual, optionally with the PCG dot and
// its scalar update in the last block.
#include <algorithm>
#include <cmath>

#include "f32x2.cuh"
#include "kernels.h"
#include "walsh.cuh"

namespace topo {

namespace {

// Differences of one displacement component within a node plane, shared by
// the two element layers on either side of the plane: p[2 gy + gz] are the
// plane's four corners of the element pair (packed A, B).
struct PlaneDiff {
    F2 dy0, dy1, qz;  // p[0] - p[2], p[1] - p[3], (p[0] - p[1]) + (p[2] - p[3])
};

__device__ __forceinline__ PlaneDiff plane_diff(const F2 (&p)[4]) {
    PlaneDiff c;
    c.dy0 = p[0] - p[2];
    c.dy1 = p[1] - p[3];
    c.qz = (p[0] - p[1]) + (p[2] - p[3]);
    return c;
}

// The seven non-constant Walsh modes of one component (walsh_fwd's operations
// and association): a = plane ex (gx = 0), b = plane ex + 1 (gx = 1).
__device__ __forceinline__ void fwd_pair(const F2 (&a)[4], const PlaneDiff& ca, const F2 (&b)[4],
                                         const PlaneDiff& cb, F2 (&w)[8]) {
    const F2 dx00 = a[0] - b[0], dx01 = a[1] - b[1], dx10 = a[2] - b[2], dx11 = a[3] - b[3];
    const F2 p0 = dx00 + dx10, p1 = dx01 + dx11, q0 = dx00 - dx10, q1 = dx01 - dx11;
    w[4] = p0 + p1;
    w[5] = p0 - p1;
    w[6] = q0 + q1;
    w[7] = q0 - q1;
    const F2 a0 = ca.dy0 + cb.dy0, a1 = ca.dy1 + cb.dy1;
    w[2] = a0 + a1;
    w[3] = a0 - a1;
    w[1] = ca.qz + cb.qz;
}

// E-scaled Walsh blocks (walsh_blocks) with paired fused multiply-adds; kd is
// the block constants scaled by the pair's moduli, nd = -kd.d.
struct PairK {
    F2 amb, b, c, d, nd, f, g, pmq, q;
};

__device__ __forceinline__ PairK pair_constants(const WalshK<float>& k, F2 E) {
    PairK r;
    r.amb = E * F2(k.amb);
    r.b = E * F2(k.b);
    r.c = E * F2(k.c);
    r.d = E * F2(k.d);
    r.nd = -r.d;
    r.f = E * F2(k.f);
    r.g = E * F2(k.g);
    r.pmq = E * F2(k.pmq);
    r.q = E * F2(k.q);
    return r;
}

__device__ __forceinline__ void blocks_pair(const PairK& k, const F2 (&Wx)[8], const F2 (&Wy)[8], const F2 (&Wz)[8],
                                            F2 (&Zx)[8], F2 (&Zy)[8], F2 (&Zz)[8]) {
    {  // 000: (100,x) (010,y) (001,z)
        const F2 bt = k.b * ((Wx[4] - Wy[2]) + Wz[1]);
        Zx[4] = fma2(k.amb, Wx[4], bt);
        Zy[2] = fma2(k.amb, Wy[2], -bt);
        Zz[1] = fma2(k.amb, Wz[1], bt);
    }
    // 001: (101,x) (011,y)
    Zx[5] = fma2(k.c, Wx[5], k.nd * Wy[3]);
    Zy[3] = fma2(k.c, Wy[3], k.nd * Wx[5]);
    // 010: (110,x) (011,z)
    Zx[6] = fma2(k.c, Wx[6], k.d * Wz[3]);
    Zz[3] = fma2(k.c, Wz[3], k.d * Wx[6]);
    // 100: (110,y) (101,z)
    Zy[6] = fma2(k.c, Wy[6], k.nd * Wz[5]);
    Zz[5] = fma2(k.c, Wz[5], k.nd * Wy[6]);
    // 011, 101, 110
    Zx[7] = k.g * Wx[7];
    {
        const F2 s = k.f * (Wy[1] - Wz[2]);
        Zy[1] = s;
        Zz[2] = -s;
    }
    Zy[7] = k.g * Wy[7];
    {
        const F2 s = k.f * (Wx[1] + Wz[4]);
        Zx[1] = s;
        Zz[4] = s;
    }
    Zz[7] = k.g * Wz[7];
    {
        const F2 s = k.f * (Wx[2] - Wy[4]);
        Zx[2] = s;
        Zy[4] = -s;
    }
    {  // 111: (011,x) (101,y) (110,z)
        const F2 qt = k.q * ((Wx[3] - Wy[5]) + Wz[6]);
        Zx[3] = fma2(k.pmq, Wx[3], qt);
        Zy[5] = fma2(k.pmq, Wy[5], -qt);
        Zz[6] = fma2(k.pmq, Wz[6], qt);
    }
}

// Inverse transform (walsh_inv's operations): y[g] = sum_{c != 0} (-1)^(c.g) z[c].
__device__ __forceinline__ void inv_pair(const F2 (&z)[8], F2 (&y)[8]) {
    const F2 a01p = z[2] + z[3], a01m = z[2] - z[3];
    const F2 a10p = z[4] + z[5], a10m = z[4] - z[5];
    const F2 a11p = z[6] + z[7], a11m = z[6] - z[7];
    const F2 b000 = z[1] + a01p, b010 = z[1] - a01p;
    const F2 b001 = a01m - z[1], t = z[1] + a01m;
    const F2 b100 = a10p + a11p, b110 = a10p - a11p;
    const F2 b101 = a10m + a11m, b111 = a10m - a11m;
    y[0] = b000 + b100;
    y[4] = b000 - b100;
    y[1] = b001 + b101;
    y[5] = b001 - b101;
    y[2] = b010 + b110;
    y[6] = b010 - b110;
    y[3] = b111 - t;
    y[7] = -(t + b111);
}

}  // namespace

constexpr int WP_NODES = 4;  // staged nodes per thread and plane, at most (checked by the launcher)

// 4-byte asynchronous global -> shared copy, zero-filled when !pred.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool pred) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(pred ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Shared memory: four staged node planes, each component-major [3][2 TZ + 1][TY + 1],
// the z exchange [2][NT][6] and the y exchange across warps [2][NT / 32][9].
__host__ __device__ inline size_t walsh_pair_smem(int NT, int TY, int TZ) {
    return sizeof(float) * ((size_t)4 * 3 * (2 * TZ + 1) * (TY + 1) + 2 * NT * 6 + 2 * (NT / 32) * 9);
}

template <int NT, int MODE, bool PCG>
__global__ void __launch_bounds__(NT, 1)
    k_walsh3p(Dims d, WalshK<float> wk, int TY, int TZ, int LX, int ntY, int ntZ, unsigned yn_magic,
              const float* __restrict__ E, const float* __restrict__ u, const float* __restrict__ r,
              const float* __restrict__ dinv, float* __restrict__ out, const uint8_t* __restrict__ fixed,
              int mask_out, float omega, const int* skip, PcgScalars* pcg, double* partials, unsigned* counter) {
    extern __shared__ __align__(16) float smem[];
    if (skip && *skip) return;
    const int ZR = 2 * TZ + 1, YN = TY + 1, ZY = ZR * YN;
    const int PL = 3 * ZY;  // floats per staged plane
    float* sp = smem;
    float* zx = smem + 4 * PL;
    float* yx = zx + 2 * NT * 6;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool act = tid < TY * TZ;
    const int ty = act ? tid % TY : 0, tz = act ? tid / TY : 0;
    int bid = blockIdx.x;
    const int jY = bid % ntY;
    bid /= ntY;
    const int kZ = bid % ntZ;
    const int X0 = (bid / ntZ) * LX;
    const int ey0 = jY * (TY - 1), ez0 = kZ * (2 * TZ - 1);
    const int ey = ey0 + ty, A = ez0 + 2 * tz, B = A + 1;
    const int nny = d.nny, nnz = d.nnz, nnx = d.nnx, nely = d.nely, nelz = d.nelz;
    const long long plane = 3LL * nny * nnz;

    // The nodes this thread stages: staged node f = row * YN + col of the
    // block's (z, y) window, f = tid + k NT; goff: its first DOF within a
    // node plane (-1 outside the window or the grid).
    int goff[WP_NODES];
#pragma unroll
    for (int k = 0; k < WP_NODES; ++k) {
        const unsigned f = (unsigned)(tid + k * NT);
        const int row = (int)__umulhi(f, yn_magic);  // f / YN
        const int col = (int)f - row * YN;
        const int z = ez0 + row, y = ey0 + col;
        goff[k] = ((int)f < ZY && z < nnz && y < nny) ? 3 * (z * nny + y) : -1;
    }
    const int nsteps = min(LX, nnx - X0);  // output node planes X0 .. X0 + nsteps - 1
    auto stage = [&](int nx, int buf) {
        if (nx <= X0 + nsteps) {
            const bool pv = nx >= 0 && nx < nnx;
            float* P = sp + buf * PL;
#pragma unroll
            for (int k = 0; k < WP_NODES; ++k) {
                const int f = tid + k * NT;
                if (f < ZY) {
                    const bool ok = pv && goff[k] >= 0;
                    const float* g = ok ? u + (nx * plane + goff[k]) : u;
#pragma unroll
                    for (int c = 0; c < 3; ++c) cp_async4(P + c * ZY + f, g + (ok ? c : 0), ok);
                }
            }
        }
        cp_commit();
    };
    // c[2 gy + gz] = component i of node (ey + gy, A + gz) (lane A) and (ey + gy, B + gz) (lane B)
    auto corners = [&](const float* P, int i, F2 (&c)[4]) {
        const float* q = P + i * ZY + 2 * tz * YN + ty;
#pragma unroll
        for (int gy = 0; gy < 2; ++gy) {
            const float n0 = q[gy], n1 = q[YN + gy], n2 = q[2 * YN + gy];
            c[2 * gy] = F2::make(n0, n1);
            c[2 * gy + 1] = F2::make(n1, n2);
        }
    };
    const bool ey_in = act && ey < nely;
    const long long estride = (long long)nely * nelz;
    auto loadE = [&](int ex) {
        const bool xin = ey_in && ex >= 0 && ex < d.nelx;
        const long long e = (long long)ex * estride + ey;
        const float ea = (xin && A < nelz) ? E[e + (long long)nely * A] : 0.f;
        const float eb = (xin && B < nelz) ? E[e + (long long)nely * B] : 0.f;
        return F2::make(ea, eb);
    };
    // node ownership (see the header comment)
    const bool own_y = act && (ty >= 1 || jY == 0) && ey <= nely;
    const bool own_A = own_y && (tz >= 1 || kZ == 0) && A <= nelz;
    const bool own_B = own_y && B <= nelz;
    const bool extra_y = act && ty == TY - 1 && ey == nely - 1;
    const bool extra_z = own_y && tz == TZ - 1 && B == nelz - 1;
    DotAcc<float> dot;

    // The epilogue of one output value: component i of the node at DOF base gn
    // with K u = k, the node's u value uv and its operands rv, dv, fv.
    auto finish = [&](long long gn, int i, float k, float uv, float rv, float dv, bool fv) {
        float o = k;
        if (MODE == 1) o = uv + omega * dv * (rv - o);
        if (MODE == 2) o = rv - o;
        if (fv) o = 0.f;
        out[gn + i] = o;
        if (PCG) dot.add(MODE == 1 ? rv : uv, o);
    };
    auto finish_load = [&](long long gn, int i, float k) {
        const float uv = MODE != 2 ? u[gn + i] : 0.f;
        const float rv = MODE != 0 ? r[gn + i] : 0.f;
        const float dv = MODE == 1 ? dinv[gn + i] : 0.f;
        const bool fv = mask_out ? fixed[gn + i] != 0 : false;
        finish(gn, i, k, uv, rv, dv, fv);
    };

    // Step s: element plane ex = X0 - 1 + s between node planes ex (buffer
    // s % 4) and ex + 1 (buffer (s + 1) % 4); plane ex + 3 is staged into
    // buffer (s + 3) % 4 (which held plane ex - 1). cin: the +x corner sums of
    // element plane ex - 1; cout receives those of plane ex. Completes output
    // node plane ex (s > 0).
    auto step = [&](int s, F2 (&cin)[3][4], F2 (&cout)[3][4], F2 Ecur, F2& Enext) {
        const int ex = X0 - 1 + s;
        stage(ex + 3, (s + 3) & 3);
        Enext = loadE(ex + 1);
        const bool emit = s > 0;  // uniform over the block
        const long long gnA = 3LL * (ey + (long long)nny * (A + (long long)nnz * ex));
        const long long gnB = gnA + 3LL * nny;
        float rr[2][3], di[2][3], uo[2][3];
        bool fx[2][3];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const bool own = emit && (q ? own_B : own_A);
            const long long gn = q ? gnB : gnA;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                rr[q][i] = (MODE != 0 && own) ? r[gn + i] : 0.f;
                di[q][i] = (MODE == 1 && own) ? dinv[gn + i] : 0.f;
                fx[q][i] = (mask_out && own) ? fixed[gn + i] != 0 : false;
            }
        }
        const float* So = sp + (s & 3) * PL;
        const float* Sn = sp + ((s + 1) & 3) * PL;
        F2 W[3][8];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            F2 a[4], b[4];
            corners(So, i, a);
            corners(Sn, i, b);
            uo[0][i] = a[0].lo();  // u at the nodes (ey, A) and (ey, B) of plane ex
            uo[1][i] = a[0].hi();
            fwd_pair(a, plane_diff(a), b, plane_diff(b), W[i]);
        }
        {
            F2 Z[3][8];
            blocks_pair(pair_constants(wk, Ecur), W[0], W[1], W[2], Z[0], Z[1], Z[2]);
#pragma unroll
            for (int i = 0; i < 3; ++i) inv_pair(Z[i], W[i]);  // W: the corner results y[g]
        }
        const int par = s & 1;
        float ZA0[3], ZA1[3], ZB0[3], ZB1[3], ZT0[3], ZT1[3], uA[3], uB[3], uT[3];
        if (emit) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                F2 P[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) P[q] = W[i][q] + cin[i][q];  // x-complete sums of plane ex
                // inside the pair along z: node rows A, B = A + 1, B + 1
                ZA0[i] = P[0].lo();
                ZA1[i] = P[2].lo();
                ZB0[i] = P[1].lo() + P[0].hi();
                ZB1[i] = P[3].lo() + P[2].hi();
                ZT0[i] = P[1].hi();
                ZT1[i] = P[3].hi();
                // along y: the +y corners of the element column ey - 1
                uA[i] = __shfl_up_sync(0xffffffffu, ZA1[i], 1);
                uB[i] = __shfl_up_sync(0xffffffffu, ZB1[i], 1);
                uT[i] = __shfl_up_sync(0xffffffffu, ZT1[i], 1);
            }
            float* zo = zx + (size_t)(par * NT + tid) * 6;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                zo[i] = ZT0[i];
                zo[3 + i] = ZT1[i];
            }
            if (lane == 31) {
                float* yo = yx + (size_t)(par * (NT / 32) + warp) * 9;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    yo[i] = ZA1[i];
                    yo[3 + i] = ZB1[i];
                    yo[6 + i] = ZT1[i];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) cout[i][q] = W[i][4 + q];
        cp_wait_one();  // plane ex + 2 has landed (ex + 3 may still be in flight)
        __syncthreads();
        if (emit && act) {
            if (ty == 0) {
#pragma unroll
                for (int i = 0; i < 3; ++i) uA[i] = uB[i] = uT[i] = 0.f;
            } else if (lane == 0) {  // the column ey - 1 is lane 31 of the previous warp
                const float* yi = yx + (size_t)(par * (NT / 32) + warp - 1) * 9;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    uA[i] = yi[i];
                    uB[i] = yi[3 + i];
                    uT[i] = yi[6 + i];
                }
            }
            // along z: the +z corners of the pair below (tz - 1) at ey and at ey - 1
            float bl0[3] = {0.f, 0.f, 0.f}, bl1[3] = {0.f, 0.f, 0.f}, dl1[3] = {0.f, 0.f, 0.f};
            if (tz >= 1) {
                const float* zb = zx + (size_t)(par * NT + tid - TY) * 6;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    bl0[i] = zb[i];
                    bl1[i] = zb[3 + i];
                    dl1[i] = ty >= 1 ? zb[-6 + 3 + i] : 0.f;
                }
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (own_A)
                    finish(gnA, i, (ZA0[i] + uA[i]) + (bl0[i] + dl1[i]), uo[0][i], rr[0][i], di[0][i], fx[0][i]);
                if (own_B) finish(gnB, i, ZB0[i] + uB[i], uo[1][i], rr[1][i], di[1][i], fx[1][i]);
            }
            if (extra_z) {  // node row B + 1 = nelz: only the pair's element B reaches it
#pragma unroll
                for (int i = 0; i < 3; ++i) finish_load(gnB + 3LL * nny, i, ZT0[i] + uT[i]);
            }
            if (extra_y) {  // node column ey + 1 = nely: only the column ey reaches it
                const bool oA = (tz >= 1 || kZ == 0) && A <= nelz, oB = B <= nelz;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    if (oA) finish_load(gnA + 3, i, ZA1[i] + bl1[i]);
                    if (oB) finish_load(gnB + 3, i, ZB1[i]);
                    if (extra_z) finish_load(gnB + 3LL * nny + 3, i, ZT1[i]);
                }
            }
        }
    };

    // planes X0 - 1, X0, X0 + 1 into buffers 0, 1, 2
    stage(X0 - 1, 0);
    stage(X0, 1);
    stage(X0 + 1, 2);
    F2 Ea = loadE(X0 - 1), Eb;
    F2 Ka[3][4], Kb[3][4];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) Ka[i][q] = F2(0.f);
    cp_wait_one();  // planes X0 - 1 and X0 have landed
    __syncthreads();
    // two steps per trip so that the carried corner sums alternate without copies
    int s = 0;
    for (; s + 1 <= nsteps; s += 2) {
        step(s, Ka, Kb, Ea, Eb);
        step(s + 1, Kb, Ka, Eb, Ea);
    }
    if (s <= nsteps) step(s, Ka, Kb, Ea, Eb);
    cp_wait_all();

    if (PCG) {
        double v[1] = {dot.value()}, tot[1];
        if (last_block_totals<NT, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
            if (MODE == 1) {  // last V-cycle sweep: rz = r.z, beta = rz / rz_old
                pcg->beta = tot[0] / pcg->rz;
                pcg->rz = tot[0];
            } else {  // K p: alpha = rz / p.Ap
                pcg->pAp = tot[0];
                pcg->alpha = pcg->rz / tot[0];
            }
        }
    }
}

// ------------------------------------------------------------------ launch --

namespace {

struct PairTile {
    int NT = 0, TY = 0, TZ = 0, ntY = 0, ntZ = 0;
    double util = 0.0;  // owned nodes per element pair computed (per plane)
};

// Tiles of `first` columns, then `next` behind a halo column each; the last
// element column at a tile's last lane also gives that lane the grid's last
// node column: the number of tiles along one direction.
inline int tiles_along(int nel, int first, int next) { return nel <= first ? 1 : 1 + div_up(nel - first, next); }

// Tile shapes: TY element columns in y (all of them up to 128), TZ = NT / TY
// pairs in z (fewer on thin grids), NT threads; the shape whose launched
// threads own the most output nodes wins.
PairTile pick_pair_tile(const Dims& d) {
    PairTile best;
    const int nts[2] = {256, 384};  // 512 threads would leave 128 registers: the product spills there
    for (int NT : nts) {
        for (int TY = 1; TY <= 128; ++TY) {
            if (d.nely <= 128 && TY != d.nely) continue;  // one tile along y
            if (d.nely > 128 && TY < 2) continue;          // tiles after the first hold TY - 1 new columns
            // no more pairs than the grid's element rows need
            const int TZ = std::min(NT / TY, std::max(1, (d.nelz + 1) / 2));
            if (TZ < 1) continue;
            if ((2 * TZ + 1) * (TY + 1) > WP_NODES * NT) continue;
            if (walsh_pair_smem(NT, TY, TZ) > 200 * 1024) continue;
            const int ntY = tiles_along(d.nely, TY, TY - 1);
            const int ntZ = tiles_along(d.nelz, 2 * TZ, 2 * TZ - 1);
            const double lanes = (double)div_up(TY * TZ, 32) * 32;  // threads of the working warps
            const double util = (double)d.nny * d.nnz / ((double)ntY * ntZ * lanes * 2.0);
            if (util > best.util + 1e-9) best = PairTile{NT, TY, TZ, ntY, ntZ, util};
        }
    }
    return best;
}

template <int NT, int MODE, bool PCG>
void launch_pair_mode(const Dims& d, const WalshK<float>& wk, const PairTile& t, int LX, unsigned nb, size_t smem,
                      const float* E, const float* u, const float* r, const float* dinv, float* out,
                      const uint8_t* fixed, bool mask_out, float omega, const int* skip, PcgScalars* pcg,
                      double* partials, unsigned* counter, cudaStream_t st) {
    static bool attr = false;  // the same attribute value on every call
    if (!attr) {
        TOPO_CUDA(cudaFuncSetAttribute(k_walsh3p<NT, MODE, PCG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
        attr = true;
    }
    const unsigned magic = (unsigned)((((unsigned long long)1 << 32) + (t.TY + 1) - 1) / (t.TY + 1));
    k_walsh3p<NT, MODE, PCG><<<nb, NT, smem, st>>>(d, wk, t.TY, t.TZ, LX, t.ntY, t.ntZ, magic, E, u, r, dinv,
                                                   out, fixed, mask_out ? 1 : 0, omega, skip, pcg, partials,
                                                   counter);
    TOPO_CHECK_LAUNCH();
}

template <int NT>
void launch_pair_nt(const Dims& d, const WalshK<float>& wk, const PairTile& t, int LX, unsigned nb, size_t smem,
                    int mode, const float* E, const float* u, const float* r, const float* dinv, float* out,
                    const uint8_t* fixed, bool mask_out, float omega, const int* skip, PcgScalars* pcg,
                    double* partials, unsigned* counter, cudaStream_t st) {
#define TOPO_WP(MV, PV)                                                                                           \
    launch_pair_mode<NT, MV, PV>(d, wk, t, LX, nb, smem, E, u, r, dinv, out, fixed, mask_out, omega, skip, pcg, \
                                 partials, counter, st)
    if (mode == 0 && pcg)
        TOPO_WP(0, true);
    else if (mode == 1 && pcg)
        TOPO_WP(1, true);
    else if (mode == 0)
        TOPO_WP(0, false);
    else if (mode == 1)
        TOPO_WP(1, false);
    else
        TOPO_WP(2, false);
#undef TOPO_WP
}

}  // namespace

bool walsh_pair_supported(const Dims& d) { return d.dim == 3 && pick_pair_tile(d).NT > 0; }

void launch_walsh_pair3(const Dims& d, const WalshK<float>& wk, int mode, const float* E, const float* u,
                        const float* r, const float* dinv, float* out, const uint8_t* fixed, bool mask_out,
                        float omega, const int* skip, PcgScalars* pcg, double* partials, long long npartials,
                        unsigned* counter, int nsm, cudaStream_t st) {
    const PairTile t = pick_pair_tile(d);
    TOPO_REQUIRE(t.NT > 0, "no element-pair tile fits this grid");
    const long long tiles = (long long)t.ntY * t.ntZ;
    TOPO_REQUIRE(!pcg || tiles <= npartials, "more tiles than reduction partials");
    // about one block per SM over the launch, at least four node planes per
    // block (the first element plane of a block is a halo)
    const long long chunks = std::max<long long>(1, (long long)nsm / tiles);
    int LX = std::max(4, div_up(d.nnx, chunks));
    long long nb = tiles * div_up(d.nnx, LX);
    while (pcg && nb > npartials) {  // one partial per block
        LX *= 2;
        nb = tiles * div_up(d.nnx, LX);
    }
    const size_t smem = walsh_pair_smem(t.NT, t.TY, t.TZ);
    if (t.NT == 256)
        launch_pair_nt<256>(d, wk, t, LX, (unsigned)nb, smem, mode, E, u, r, dinv, out, fixed, mask_out, omega,
                            skip, pcg, partials, counter, st);
    else
        launch_pair_nt<384>(d, wk, t, LX, (unsigned)nb, smem, mode, E, u, r, dinv, out, fixed, mask_out, omega,
                            skip, pcg, partials, counter, st);
}

}  // namespace topo
