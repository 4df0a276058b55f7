// Shared types and device helpers of the batched uneven-2D path (batch.cu,
// batch_mg.cu).
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include "grid.h"
#include "ku_device.cuh"

namespace topo {
namespace bt {

struct BInst {
    int nelx, nely, nnx, nny;
    long long el0, node0, nel;
    int tn0, tnn, te0, ten;  // node / element tile ranges in the tile tables
    int tap0, ntap;          // filter taps
    double volfrac, rmin, Hs, dv;
};

enum : int { ETA_NEWTON = 0, ETA_BISECT = 1 };
enum : int { OC_EXPAND = 0, OC_BISECT = 1, OC_DONE = 2, OC_SKIP = 3 };
enum : int { LOOP_ETA = 0, LOOP_REF = 1, LOOP_INNER = 2, LOOP_OC = 3 };

// Per-instance device state.
struct BS {
    double eta, lo, hi;                        // eta Newton / bisection (Sec. 3.2)
    int eta_mode, eta_it, eta_bis, eta_done;
    double rel_res;                            // FP64 relative residual of the last refinement test
    int ref_done, n_ref, inner_done, inner_it;
    int inner_total, stalled;                  // stalled: stopped by the stall rule (kb_resid)
    double rel_mark;                           // residual at the last stall-window mark
    double rz, alpha, beta_cg, irr0;           // inner PCG scalars
    double f_beta, f_alpha, f_pkp;             // FP64 outer flexible CG (previous p.Kp)
    int f_has_prev, pad2;
    double l1, l2, lm;                         // OC bracket and multiplier
    int oc_state, oc_steps, oc_grow, pad1;
    double c, V, ch;                           // compliance, volume, change
};

// Batch-wide device scalars.
struct BG {
    double penal, beta;
    int loop, status;
    int active[4];                    // instances still running each loop
    unsigned long long body_exec[4];  // body executions of each loop in this step
};

// Launch constants shared by the tiled kernels.
struct BK {
    const BInst* I;
    BS* S;
    BG* G;
    const int4* tiles;  // {instance, x0, y0, 0}
    int TY;
    double* partials;   // [2][pstride]
    long long pstride;
    unsigned* counters; // per instance, zero between reductions
};

// ------------------------------------------------------------- reductions

template <int NV>
__device__ __forceinline__ void block_sum_dyn(double (&v)[NV], double* sm /* [NV][32] */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[k * 32 + wid] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = warp_sum(lane < nw ? sm[k * 32 + lane] : 0.0);
    }
    __syncthreads();
}

// The tile's NV partial sums go to slot blockIdx.x; the last of the
// instance's nt tiles (t0 .. t0 + nt - 1) to arrive adds them in tile order and
// returns true with the totals valid in thread 0. All threads must call it.
template <int NV>
__device__ bool seg_reduce(const BK& k, int t0, int nt, unsigned* counter, double (&v)[NV], double (&tot)[NV]) {
    __shared__ double sm[NV * 32];
    __shared__ int am_last;
    block_sum_dyn<NV>(v, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) k.partials[q * k.pstride + blockIdx.x] = v[q];
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        am_last = (t == (unsigned)nt - 1u);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        s[q] = 0.0;
        for (int j = threadIdx.x; j < nt; j += blockDim.x) s[q] += __ldcg(&k.partials[q * k.pstride + t0 + j]);
    }
    block_sum_dyn<NV>(s, sm);
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = s[q];
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// (hi, lo) += (bh, bl) in float-float arithmetic (Knuth's TwoSum, then a
// renormalisation); symmetric in its two operands, so an xor butterfly leaves
// the same pair in every lane.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
    const float s = hi + bh;
    const float bb = s - hi;
    const float e = ((hi - (s - bb)) + (bh - bb)) + (lo + bl);
    hi = s + e;
    lo = e - (hi - s);
}

// seg_reduce for float-float per-thread sums (DotAcc<float>): the warp sums
// stay in FP32 pairs, FP64 enters once per warp (FP64 is 1/64 of the FP32 rate
// on this part, and these reductions run in every inner PCG pass).
template <int NV>
__device__ bool seg_reduce_ff(const BK& k, int t0, int nt, unsigned* counter, DotAcc<float> (&a)[NV],
                              double (&tot)[NV]) {
    __shared__ double sm[NV * 32];
    __shared__ int am_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        float hi = a[q].hi, lo = a[q].lo;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            ff_add(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
        if (lane == 0) sm[q * 32 + wid] = (double)hi + (double)lo;
    }
    __syncthreads();
    if (wid == 0) {
        double v[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = warp_sum(lane < nw ? sm[q * 32 + lane] : 0.0);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < NV; ++q) k.partials[q * k.pstride + blockIdx.x] = v[q];
            __threadfence();
            const unsigned t = atomicAdd(counter, 1u);
            am_last = (t == (unsigned)nt - 1u);
        }
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        s[q] = 0.0;
        for (int j = threadIdx.x; j < nt; j += blockDim.x) s[q] += __ldcg(&k.partials[q * k.pstride + t0 + j]);
    }
    block_sum_dyn<NV>(s, sm);
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = s[q];
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// ---------------------------------------------------------- element maths

// Relaxed Heaviside projection (Eq. 1), its x-derivative (Eq. 8) and its
// eta-derivative by the quotient rule of Eq. 1.
__device__ __forceinline__ double b_prj(double x, double eta, double beta) {
    const double te = tanh(beta * eta);
    return (te + tanh(beta * (x - eta))) / (te + tanh(beta * (1.0 - eta)));
}
__device__ __forceinline__ double b_dprj(double x, double eta, double beta) {
    const double t = tanh(beta * (x - eta));
    return beta * (1.0 - t * t) / (tanh(beta * eta) + tanh(beta * (1.0 - eta)));
}
__device__ __forceinline__ double b_deta(double x, double eta, double beta) {
    const double te = tanh(beta * eta), tx = tanh(beta * (x - eta)), t1 = tanh(beta * (1.0 - eta));
    const double num = te + tx, den = te + t1;
    const double dnum = beta * (1.0 - te * te) - beta * (1.0 - tx * tx);
    const double dden = beta * (1.0 - te * te) - beta * (1.0 - t1 * t1);
    return (dnum * den - num * dden) / (den * den);
}
// OC rule (Eq. 13) with move limits and box constraints.
__device__ __forceinline__ double b_oc(double x, double ocp, double lm, double move) {
    return fmax(0.0, fmax(x - move, fmin(1.0, fmin(x + move, ocp / lm))));
}

// Q4 node-centric K u at node (ix, iy) of one instance: E and u point at the
// instance's first element / DOF. Displacements are taken relative to the node
// (exact: the element rows annihilate translations); neighbour offsets are
// clamped per axis and elements outside the grid get modulus 0.
template <typename T>
__device__ __forceinline__ void bku2(const KeP<T, 8>& ke, const T* __restrict__ E, const T* __restrict__ u,
                                     int ix, int iy, int nelx, int nely, T& a0, T& a1) {
    const int nny = nely + 1;
    const T* p = u + 2 * (iy + nny * ix);
    const T c0 = p[0], c1 = p[1];
    const int oy[3] = {iy > 0 ? -2 : 0, 0, iy < nely ? 2 : 0};
    const int ox[3] = {ix > 0 ? -2 * nny : 0, 0, ix < nelx ? 2 * nny : 0};
    T w[9][2];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        if (q == 4) {
            w[q][0] = w[q][1] = T(0);
            continue;
        }
        const T* pm = p + (ox[q / 3] + oy[q % 3]);
        w[q][0] = pm[0] - c0;
        w[q][1] = pm[1] - c1;
    }
    const bool vx[2] = {ix > 0, ix < nelx}, vy[2] = {iy > 0, iy < nely};
    const int exc[2] = {ix > 0 ? ix - 1 : 0, ix < nelx ? ix : nelx - 1};
    const int eyc[2] = {iy > 0 ? iy - 1 : 0, iy < nely ? iy : nely - 1};
    a0 = a1 = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int EXO = k >> 1, EYO = k & 1;
        const T e = E[eyc[EYO] + nely * exc[EXO]];
        const T Ee = (vx[EXO] && vy[EYO]) ? e : T(0);
        const int L = local_node(1 - EXO, EYO, 0);
        T t0 = T(0), t1 = T(0);
#pragma unroll
        for (int M = 0; M < 4; ++M) {
            if (M == L) continue;
            const int q = (EXO + lnx(M)) * 3 + (EYO - lny(M) + 1);
            t0 += ke.k[(2 * L) * 8 + 2 * M] * w[q][0] + ke.k[(2 * L) * 8 + 2 * M + 1] * w[q][1];
            t1 += ke.k[(2 * L + 1) * 8 + 2 * M] * w[q][0] + ke.k[(2 * L + 1) * 8 + 2 * M + 1] * w[q][1];
        }
        a0 += Ee * t0;
        a1 += Ee * t1;
    }
}

__device__ __forceinline__ double b_cont(double par, const to_continuation& c, int loop) {
    if (loop >= c.istart && par < c.maxpar && c.isteps > 0 && loop % c.isteps == 0)
        par = c.kind == TO_CNT_ADD ? par + c.delta : fmin(c.maxpar, par * c.delta);
    return par;
}

// Tile position of this thread: (x, y) = (column, row) of a node or element.
#define B_TILE(k)                                          \
    const int4 tl = (k).tiles[blockIdx.x];                 \
    const int inst = tl.x;                                 \
    const BInst& I = (k).I[inst];                          \
    BS& S = (k).S[inst];                                   \
    const int tx_ = tl.y + (int)threadIdx.x / (k).TY;      \
    const int ty_ = tl.z + (int)threadIdx.x % (k).TY;

// ------------------------------------------------------------ multigrid

// One instance at one level of the batched geometric multigrid (level 0 is the
// design grid). Coarse grids have ceil(n / 2) elements per axis; children that
// fall outside an odd grid are dropped from the Galerkin sums.
struct LInst {
    int nelx, nely, nnx, nny;
    long long el0, node0;  // offsets into this level's element / node arrays
    int tn0, tnn;          // this level's node tiles
    int depth, pad;        // number of levels of the instance
};

// Coarsest level of one instance: dense inverse of its nc x nc operator.
struct CInst {
    int level, nc, nnx, nny;
    long long node0, a0;   // node offset within the level; offset of the inverse in the pool
    const float* S;        // the level's stencils (SoA, stride nnode)
    const uint8_t* fixed;  // the level's Dirichlet mask
    const float* rhs;      // the level's right-hand side
    float* z;              // the level's V-cycle output buffer
    long long nnode;       // SoA stride of S
};

struct BMGLevel {
    std::vector<LInst> hL;
    LInst* dL = nullptr;
    std::vector<long long> hstart;  // element offsets per instance [count + 1]
    long long* dstart = nullptr;
    int4* tiles = nullptr;
    int ntiles = 0;
    long long tile_cap = 0;
    long long nel = 0, nnode = 0;
    float *Kel = nullptr, *S = nullptr, *R = nullptr, *dinv = nullptr;
    float *z = nullptr, *t = nullptr, *w = nullptr, *r = nullptr;
    uint8_t* fixed = nullptr;
    uint8_t* touched = nullptr;  // [nel] coarse levels: a fine Dirichlet DOF lies under the element
};

struct BMG {
    int nlev = 0;
    int nu = 1;
    float omega = 1.f;
    std::vector<BMGLevel> lev;
    std::vector<CInst> hC;
    CInst* dC = nullptr;
    int max_nc = 0;
    double* Aw = nullptr;  // FP64 factor / triangular inverse pool
    float* Ainv = nullptr; // FP32 inverses
    float* Cj = nullptr;   // level-1 constants P_j^T Ke P_j [4][64]
    float arow[8] = {};    // row sums of |Ke| (fine-level l1 diagonal)
};

// Kernel view of one level.
struct BKL {
    const LInst* L;
    BS* S;
    const int4* tiles;
    int TY;
    int level;
};

}  // namespace bt
}  // namespace topo

struct to_batch;
namespace topo {
namespace bt {
// batch_mg.cu
void bmg_create(to_batch* b);
void bmg_tiles(to_batch* b);
void bmg_setup(to_batch* b, cudaStream_t st);
// Enqueues one V-cycle on r0 (level-0 residual) for the running instances
// (skip_inner: also skip instances whose inner solve has stopped); returns the
// level-0 buffer that holds the result.
float* bmg_vcycle(to_batch* b, cudaStream_t st, const float* r0, int skip_inner);
}  // namespace bt
}  // namespace topo

// The opaque handle behind the to_batch_* entry points.
struct to_batch {
    to_params p{};
    int count = 0;
    cudaStream_t ust = nullptr, st = nullptr, sb[2] = {};
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev0 = nullptr, ev1 = nullptr;
    std::vector<void*> allocs;
    std::vector<topo::bt::BInst> hI;
    long long nel = 0, nnode = 0;
    topo::bt::BInst* dI = nullptr;
    topo::bt::BS* dS = nullptr;
    topo::bt::BG* dG = nullptr;
    int2* toff = nullptr;
    float2* tw = nullptr;      // filter weights as float pairs
    float2 *fs1 = nullptr, *fs2 = nullptr;  // filter inputs as float pairs
    int4* ntiles = nullptr;
    int4* etiles = nullptr;
    int n_nt = 0, n_et = 0;
    int nty = 32, ntx = 4, ety = 32, etx = 4;
    long long tile_cap = 0;
    double* partials = nullptr;
    unsigned* counters = nullptr;
    const double* F = nullptr;
    const uint8_t* fixed = nullptr;
    double *xt = nullptr, *dprj = nullptr, *dc = nullptr, *dcf = nullptr, *dV0 = nullptr, *ocP = nullptr,
           *E64 = nullptr;
    float *E32 = nullptr, *dinv = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *Ap32 = nullptr;
    // inner solution of the FP32 PCG, accumulated in FP64: rounded to FP32 at
    // every step it would limit the inner solve's true residual to about
    // eps_32 || |K| |x| || (the recursion for r32 never sees that rounding)
    double* xin = nullptr;
    double *r64 = nullptr, *p64 = nullptr, *Kp64 = nullptr;  // outer flexible CG
    topo::KeP<double, 8> ke64{};
    topo::KeP<float, 8> ke32{};
    cudaGraphExec_t exec = nullptr;
    const void* cap[4] = {};
    long long k_static = 0, k_body[4] = {};
    topo::bt::BG hG{};
    std::vector<topo::bt::BS> hS;
    topo::bt::BMG* mg = nullptr;  // batched multigrid (precond = TO_PC_GMG)
    float *z0 = nullptr, *t0 = nullptr, *w0 = nullptr;  // level-0 V-cycle buffers
};
