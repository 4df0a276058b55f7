// Matrix-free 3D K u with the Walsh-factored element product (walsh.cuh):
// element tiles marching along x.
//
// A block owns a (TY-1) x (TZ-1) column of nodes in (y, z) and a range of LX
// node planes along x. Its TY x TZ threads are the element columns of that
// node column plus a one-element halo in -y and -z, so every output node's
// eight elements are computed inside the block (no atomics: each output is
// written by one thread in a fixed summation order, bit-reproducible). Per x
// step the block stages the next node plane into shared memory (double
// buffered, loaded one step ahead), every thread forms E_e Ke u_e for its
// element and the eight corner results are summed: along x in registers (the
// +x corners carry to the next step), along y with one warp shuffle (a warp is
// a y-row of element columns), along z through shared memory — one barrier per
// step. The fused epilogues are those of the fine-level multigrid operator:
// K u, the damped Jacobi sweep and the residual, optionally with the PCG dot
// and its scalar update in the last block.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "kernels.h"
#include "ku_device.cuh"
#include "walsh.cuh"

namespace topo {

bool walsh_constants(const double* Ke, WalshK<double>& k, double* max_dev) {
    // H[(c,i), (L,i)] = (-1)^(c.g) for the corner g of local node L.
    int Lof[8];
    for (int g = 0; g < 8; ++g) Lof[g] = local_node(g >> 2, 1 - ((g >> 1) & 1), g & 1);
    auto sgn = [](int c, int g) { return (__builtin_popcount(c & g) & 1) ? -1.0 : 1.0; };
    static double M[24][24];
    double mmax = 0.0;
    for (int c = 0; c < 8; ++c)
        for (int i = 0; i < 3; ++i)
            for (int c2 = 0; c2 < 8; ++c2)
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0;
                    for (int a = 0; a < 8; ++a)
                        for (int b = 0; b < 8; ++b)
                            s += sgn(c, a) * sgn(c2, b) * Ke[(3 * Lof[a] + i) * 24 + 3 * Lof[b] + j];
                    M[3 * c + i][3 * c2 + j] = s / 64.0;
                    mmax = std::fmax(mmax, std::fabs(s / 64.0));
                }
    auto m = [&](int c, int i, int c2, int j) { return M[3 * c + i][3 * c2 + j]; };
    const double A = m(4, 0, 4, 0), B = m(4, 0, 1, 2), C = m(5, 0, 5, 0), D = -m(5, 0, 3, 1);
    const double F = m(1, 1, 1, 1), G = m(7, 0, 7, 0), P = m(3, 0, 3, 0), Q = m(3, 0, 6, 2);
    k = WalshK<double>{A - B, B, C, D, F, G, P - Q, Q};
    // Column (c2, j) of the pattern: the block product of the unit mode.
    double dev = 0.0;
    for (int c2 = 1; c2 < 8; ++c2)
        for (int j = 0; j < 3; ++j) {
            double W[3][8] = {}, Z[3][8];
            W[j][c2] = 1.0;
            walsh_blocks<double>(k, 1.0, W[0], W[1], W[2], Z[0], Z[1], Z[2]);
            for (int c = 0; c < 8; ++c)
                for (int i = 0; i < 3; ++i) dev = std::fmax(dev, std::fabs(Z[i][c] - m(c, i, c2, j)));
        }
    for (int r = 0; r < 24; ++r)  // the constant modes (rigid translations) are null
        for (int j = 0; j < 3; ++j) dev = std::fmax(dev, std::fabs(M[r][j]));
    *max_dev = mmax > 0.0 ? dev / mmax : dev;
    return *max_dev <= 1e-12;
}

// 4- or 8-byte asynchronous global -> shared copy; zero-filled when !pred.
template <typename T>
__device__ __forceinline__ void cp_async_val(T* smem, const T* gmem, bool pred) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(pred ? 4 : 0)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(pred ? 8 : 0)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

#ifndef TOPO_WALSH_MINB_F32
#define TOPO_WALSH_MINB_F32 2  // resident 256-thread blocks per SM the FP32 kernels are compiled for
#endif

// Minimum resident blocks per SM for the register budget of a TY x TZ block.
template <typename T, int NT>
struct WalshMinBlocks {
    static constexpr int v = sizeof(T) == 4 ? TOPO_WALSH_MINB_F32 * 256 / NT : 3 * 128 / NT;
};

template <typename T, int TY, int TZ, int MODE, bool PCG>
__global__ void __launch_bounds__(TY * TZ, (WalshMinBlocks<T, TY * TZ>::v))
    k_walsh3(Dims d, WalshK<T> wk, int LX, int ntY, int ntZ, const T* __restrict__ E, const T* __restrict__ u,
             const T* __restrict__ r, const T* __restrict__ dinv, T* __restrict__ out,
             const uint8_t* __restrict__ fixed, int mask_out, T omega, const int* skip, PcgScalars* pcg,
             double* partials, unsigned* counter) {
    constexpr int NT = TY * TZ;
    constexpr int PW = 3 * (TY + 1);         // values per staged row (3 components per node)
    constexpr int PN = PW * (TZ + 1);        // values per staged node plane
    constexpr int NPRE = (PN + NT - 1) / NT;  // staged values per thread
    __shared__ __align__(16) T sp[3][PN];     // node planes in flight (three-deep pipeline)
    __shared__ T sr[2][3][TZ][TY];
    pdl_begin();
    const int sk = skip ? *skip : 0;  // tested after the first planes are staged, so its load overlaps theirs

    const int tid = threadIdx.x, ty = tid % TY, tz = tid / TY;
    int bid = blockIdx.x;
    const int tY = bid % ntY;
    bid /= ntY;
    const int tZ = bid % ntZ;
    const int X0 = (bid / ntZ) * LX;
    const int Ye = tY * (TY - 1) - 1, Ze = tZ * (TZ - 1) - 1;
    const int ey = Ye + ty, ez = Ze + tz;  // this thread's element column
    const int nny = d.nny, nnz = d.nnz, nnx = d.nnx;
    const int plane = 3 * nny * nnz;

    // Plane-independent offsets of the values this thread stages (-1: outside).
    int goff[NPRE];
#pragma unroll
    for (int k = 0; k < NPRE; ++k) {
        const int f = tid + k * NT;
        const int row = f / PW, col = f - (f / PW) * PW;
        const int nz = Ze + row, v = 3 * Ye + col;
        goff[k] = (f < PN && nz >= 0 && nz < nnz && v >= 0 && v < 3 * nny) ? nz * 3 * nny + v : -1;
    }
    const int nsteps = min(LX, nnx - X0);  // output planes X0 .. X0 + nsteps - 1
    // Asynchronous copy of node plane nx into buffer buf (zeros outside the
    // grid); one commit group per call, empty past the block's last plane.
    auto stage = [&](int nx, int buf) {
        if (nx <= X0 + nsteps) {
            const bool pv = nx >= 0 && nx < nnx;
#pragma unroll
            for (int k = 0; k < NPRE; ++k) {
                const int f = tid + k * NT;
                if (f < PN) {
                    const bool ok = pv && goff[k] >= 0;
                    cp_async_val<T>(&sp[buf][f], ok ? u + (nx * plane + goff[k]) : u, ok);
                }
            }
        }
        cp_async_commit();
    };
    // c[i][2 gy + gz] = component i of node (ey + gy, ez + gz) of the staged plane.
    auto read_corners = [&](int buf, T (&c)[3][4]) {
#pragma unroll
        for (int gy = 0; gy < 2; ++gy)
#pragma unroll
            for (int gz = 0; gz < 2; ++gz)
#pragma unroll
                for (int i = 0; i < 3; ++i) c[i][2 * gy + gz] = sp[buf][(tz + gz) * PW + 3 * (ty + gy) + i];
    };
    const bool eyz = ey >= 0 && ey < d.nely && ez >= 0 && ez < d.nelz;
    const int eoff = ey + d.nely * ez, estride = d.nely * d.nelz;
    auto loadE = [&](int ex) { return (eyz && ex >= 0 && ex < d.nelx) ? E[eoff + ex * estride] : T(0); };
    const bool owner = ty >= 1 && tz >= 1 && ey < nny && ez < nnz;
    DotAcc<T> dot;

    // Step s: element plane ex = X0 - 1 + s; node plane ex is in uo, plane
    // ex + 1 is read from buffer bn into un, plane ex + 3 is staged into buffer
    // bs (which held plane ex). Completes output plane ex (s > 0). cin: the +x
    // corner sums of element plane ex - 1; cout receives those of plane ex.
    auto step = [&](int s, int bn, int bs, T (&uo)[3][4], T (&un)[3][4], T (&cin)[3][4], T (&cout)[3][4],
                    T Ecur, T& Enext) {
        const int ex = X0 - 1 + s;
        stage(ex + 3, bs);
        Enext = loadE(ex + 1);
        const bool emit = s > 0 && owner;
        const int gn = 3 * (ey + nny * (ez + nnz * ex));
        // epilogue operands, fetched before the element work
        T rr[3], di[3];
        bool fx[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            rr[i] = (MODE != 0 && emit) ? r[gn + i] : T(0);
            di[i] = (MODE == 1 && emit) ? dinv[gn + i] : T(0);
            fx[i] = (mask_out && emit) ? fixed[gn + i] != 0 : false;
        }
        read_corners(bn, un);
        T ue[3][8], ye[3][8];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ue[i][q] = uo[i][q];
                ue[i][4 + q] = un[i][q];
            }
        walsh_element<T>(wk, Ecur, ue, ye);
        T o00[3];
        if (s > 0) {
            // plane ex: x-complete sums at the four (gy, gz) corners
            T p[3][4];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) p[i][q] = ye[i][q] + cin[i][q];
            // y: add the +y corners of the element column below (lane ty - 1)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                p[i][0] += __shfl_up_sync(0xffffffffu, p[i][2], 1, TY);
                p[i][1] += __shfl_up_sync(0xffffffffu, p[i][3], 1, TY);
            }
            // z: publish the +z corner for the element column behind (tz + 1)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                sr[s & 1][i][tz][ty] = p[i][1];
                o00[i] = p[i][0];
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) cout[i][q] = ye[i][4 + q];
        cp_async_wait_one();  // plane ex + 2 has landed (ex + 3 may still be in flight)
        __syncthreads();
        if (emit) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T o = o00[i] + sr[s & 1][i][tz - 1][ty];
                if (MODE == 1) o = uo[i][0] + omega * di[i] * (rr[i] - o);
                if (MODE == 2) o = rr[i] - o;
                if (fx[i]) o = T(0);
                out[gn + i] = o;
                if (PCG) dot.add(MODE == 1 ? rr[i] : uo[i][0], o);
            }
        }
    };

    // planes X0 - 1, X0, X0 + 1 into buffers 0, 1, 2
    stage(X0 - 1, 0);
    stage(X0, 1);
    stage(X0 + 1, 2);
    T Ea = loadE(X0 - 1), Eb;
    cp_async_wait_one();
    __syncthreads();
    if (sk) {  // the same value in every thread; nothing written yet
        cp_async_wait_all();
        return;
    }
    T A[3][4], B[3][4], C0[3][4], C1[3][4];
    read_corners(0, A);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) C0[i][q] = T(0);
    __syncthreads();  // buffer 0 is restaged in the first step
    // Step s reads buffer (s + 1) % 3 and stages into s % 3.
    int s = 0, b0 = 0;  // b0 = s % 3
    for (; s + 1 <= nsteps; s += 2) {  // two steps per trip: the register roles alternate
        const int b1 = b0 == 2 ? 0 : b0 + 1, b2 = b1 == 2 ? 0 : b1 + 1;
        step(s, b1, b0, A, B, C0, C1, Ea, Eb);
        step(s + 1, b2, b1, B, A, C1, C0, Eb, Ea);
        b0 = b2;
    }
    if (s <= nsteps) step(s, b0 == 2 ? 0 : b0 + 1, b0, A, B, C0, C1, Ea, Eb);
    cp_async_wait_all();

    if (PCG) {
        double v[1] = {dot.value()}, tot[1];
        if (last_block_totals<NT, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
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

static int device_sms() {
    static const int v = [] {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 148;
        return n;
    }();
    return v;
}

// Fraction of the threads of a TY x TZ tiling that own an output node.
static double walsh_util(const Dims& d, int TY, int TZ) {
    const double ty = (double)div_up(d.nny, TY - 1) * TY, tz = (double)div_up(d.nnz, TZ - 1) * TZ;
    return (double)d.nny * d.nnz / (ty * tz);
}

template <typename T, int TY, int TZ>
static void walsh_launch_tile(const Dims& d, const WalshK<T>& wk, int mode, const T* E, const T* u, const T* r,
                              const T* dinv, T* out, const uint8_t* fixed, bool mask_out, T omega,
                              const int* skip, PcgScalars* pcg, double* partials, long long npartials,
                              unsigned* counter, int nsm, cudaStream_t st) {
    constexpr int NT = TY * TZ;
    const int ntY = div_up(d.nny, TY - 1), ntZ = div_up(d.nnz, TZ - 1);
    const long long tiles = (long long)ntY * ntZ;
    // About 1,536 threads per SM over the launch, at least four planes per
    // block (the first element plane of a block is a halo).
    const long long chunks = std::max<long long>(1, (long long)nsm * (1536 / NT) / tiles);
    int LX = std::max(4, div_up(d.nnx, chunks));
    long long nb = tiles * div_up(d.nnx, LX);
    while (pcg && nb > npartials) {  // one partial per block
        LX *= 2;
        nb = tiles * div_up(d.nnx, LX);
    }
#define TOPO_W(MV, PV)                                                                                  \
    launch_k(k_walsh3<T, TY, TZ, MV, PV>, (unsigned)nb, NT, 0, st, d, wk, LX, ntY, ntZ, E, u, r, dinv, out, \
             fixed, mask_out ? 1 : 0, omega, skip, pcg, partials, counter)
    if (mode == 0 && pcg)
        TOPO_W(0, true);
    else if (mode == 1 && pcg)
        TOPO_W(1, true);
    else if (mode == 0)
        TOPO_W(0, false);
    else if (mode == 1)
        TOPO_W(1, false);
    else
        TOPO_W(2, false);
#undef TOPO_W
}

template <typename T>
void launch_walsh_op3(const Dims& d, const WalshK<T>& wk, int mode, const T* E, const T* u, const T* r,
                      const T* dinv, T* out, const uint8_t* fixed, bool mask_out, T omega, const int* skip,
                      PcgScalars* pcg, double* partials, long long npartials, unsigned* counter, int nsm,
                      cudaStream_t st) {
    if (nsm <= 0) nsm = device_sms();
    // Tile shapes: 32 x 8 (a warp is one y-row), 8 x 8 and 16 x 16 (warps of
    // several rows); the one with the fewest threads per output node wins
    // (grids with nny = 16k + 1 fit 8 x 8 or 16 x 16 tiles better than 31-node rows).
    const double u1 = walsh_util(d, 32, 8), u2 = walsh_util(d, 8, 8), u3 = walsh_util(d, 16, 16);
    const int pick = (u1 >= u2 && u1 >= u3) ? 1 : (u2 >= u3 ? 2 : 3);
#define TOPO_WT(TYV, TZV)                                                                                     \
    walsh_launch_tile<T, TYV, TZV>(d, wk, mode, E, u, r, dinv, out, fixed, mask_out, omega, skip, pcg, partials, \
                                   npartials, counter, nsm, st)
    if (pick == 1)
        TOPO_WT(32, 8);
    else if (pick == 2)
        TOPO_WT(8, 8);
    else
        TOPO_WT(16, 16);
#undef TOPO_WT
}

template void launch_walsh_op3<double>(const Dims&, const WalshK<double>&, int, const double*, const double*,
                                       const double*, const double*, double*, const uint8_t*, bool, double,
                                       const int*, PcgScalars*, double*, long long, unsigned*, int,
                                       cudaStream_t);
template void launch_walsh_op3<float>(const Dims&, const WalshK<float>&, int, const float*, const float*,
                                      const float*, const float*, float*, const uint8_t*, bool, float,
                                      const int*, PcgScalars*, double*, long long, unsigned*, int,
                                      cudaStream_t);

}  // namespace topo
