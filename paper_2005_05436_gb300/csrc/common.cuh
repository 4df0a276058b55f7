// Shared device infrastructure of the topopt CUDA path (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>

#include "topopt.h"

namespace topo {

// ---------------------------------------------------------------- errors --

struct Error : std::runtime_error {
    to_status code;
    Error(to_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define TOPO_CUDA(expr)                                                              \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess)                                                       \
            throw ::topo::Error(_e == cudaErrorMemoryAllocation ? TO_ENOMEM : TO_ECUDA, \
                                std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// Kernel-launch accounting: every launch site adds its kernel count; kernels
// enqueued during a graph capture are counted when the graph is launched.
void count_launches(long long n);
long long launches_total();
void set_capturing(bool on);
long long captured_launches_reset();  // kernels enqueued during captures since the last call

#define TOPO_CHECK_LAUNCH()             \
    do {                                \
        TOPO_CUDA(cudaGetLastError());  \
        ::topo::count_launches(1);      \
    } while (0)

// Programmatic dependent launch. Launches made through launch_k while
// set_pdl(true) is in effect on the calling thread carry the programmatic
// stream-serialisation attribute: the grid may be scheduled as soon as every
// block of the preceding grid has passed pdl_begin(), and its own pdl_begin()
// blocks until that grid has completed and its memory is visible. Every kernel
// launched through launch_k calls pdl_begin() before it touches global memory;
// for a grid launched without the attribute both instructions are no-ops.
bool pdl_on();
void set_pdl(bool on);
struct PdlScope {  // set_pdl(on) for the lifetime of the scope
    bool prev;
    explicit PdlScope(bool on) : prev(pdl_on()) { set_pdl(on); }
    ~PdlScope() { set_pdl(prev); }
};

__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args&&... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = pdl_on() ? 1 : 0;
    TOPO_CUDA(cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...));
    count_launches(1);
}

#define TOPO_REQUIRE(cond, msg)                                                      \
    do {                                                                             \
        if (!(cond)) throw ::topo::Error(TO_EINVAL, msg);                            \
    } while (0)

// ------------------------------------------------------------ grid sizes --

// Structured-grid dimensions in the paper's numbering (Sec. 3, PRE.2). A 2D grid
// is stored as nelz = 1, nnz = 1 so that the 3D index formulas reduce to 2D.
struct Dims {
    int dim;
    int nelx, nely, nelz;
    int nnx, nny, nnz;
    long long nel, nnodes, ndof;
};

inline Dims make_dims(int dim, int nelx, int nely, int nelz) {
    Dims d;
    d.dim = dim;
    d.nelx = nelx;
    d.nely = nely;
    d.nelz = dim == 3 ? nelz : 1;
    d.nnx = nelx + 1;
    d.nny = nely + 1;
    d.nnz = dim == 3 ? nelz + 1 : 1;
    d.nel = (long long)d.nelx * d.nely * d.nelz;
    d.nnodes = (long long)d.nnx * d.nny * d.nnz;
    d.ndof = d.nnodes * dim;
    return d;
}

// Element stiffness matrix as a kernel parameter (constant bank, warp-uniform
// reads); all indices into it are compile-time constants in the kernels.
template <typename T, int D>
struct KeP {
    T k[D * D];
};

// Filter window (Eq. 2): nw taps with offsets (ox, oy, oz) and cone weights.
struct FilterTaps {
    int nw;
    const int* off;   // [nw * 3] (ox, oy, oz)
    const double* w;  // [nw]
    const float* wf;  // [nw]
    // The same window as rows along x for the tiled filter (kernels_filter.cu):
    // row k has offsets (oy, oz) = rows[4k], rows[4k + 1], and its x offsets
    // run from rows[4k + 2] in rows[4k + 3] chunks of FILTER_K; its weights are
    // rw[rowbase(k) + i] (zero where the cone weight is 0), rowbase(k) = the sum
    // of FILTER_K * chunks of the rows before; rwh / rwl split them into two
    // floats (hi = (float) w, lo = (float) (w - hi)).
    int R, Rz, nrows;
    const int* rows;
    const double* rw;
    const float* rwh;
    const float* rwl;
};

constexpr int FILTER_K = 8;  // outputs per thread along x in the tiled filter

__host__ __device__ inline int mirror_index(int j, int n) {
    // Repeated border-duplicating reflection ('N' padding).
    int p = 2 * n;
    int r = j % p;
    if (r < 0) r += p;
    return r < n ? r : p - 1 - r;
}

// ------------------------------------------------------------ reductions --

// x^p for the penalisation exponent: small integer exponents (the usual
// p = 3 and its p - 1 = 2) by repeated multiplication, since the FP64 pow is a
// long instruction sequence at the FP64 rate; other exponents by pow.
__device__ __forceinline__ double powp(double x, double p) {
    if (p == 1.0) return x;
    if (p == 2.0) return x * x;
    if (p == 3.0) return x * x * x;
    if (p == 4.0) {
        const double x2 = x * x;
        return x2 * x2;
    }
    return pow(x, p);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-thread dot-product accumulator. For double it is a plain FMA chain. For
// float it keeps the sum as an unevaluated pair (hi, lo): each product a*b is
// split exactly into p + e (e = fma(a, b, -p)), p is added to hi by Knuth's
// TwoSum and all rounding errors collect in lo, giving about 48 significant
// bits. FP64 enters only when the thread's pair is handed to the block
// reduction, which keeps FP64 instructions (slow on this part) out of the
// per-element work of the FP32 solver.
template <typename T>
struct DotAcc {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};

template <>
struct DotAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);  // never contracted into an FMA
        const float e = fmaf(a, b, -p);
        const float s = hi + p;
        const float bb = s - hi;
        const float err = (hi - (s - bb)) + (p - bb);
        hi = s;
        lo += err + e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Deterministic block sum of NV values per thread; result valid in thread 0.
template <int NT, int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm /* NV*NT/32 */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[k * (NT / 32) + wid] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < NT / 32 ? sm[k * (NT / 32) + lane] : 0.0;
            v[k] = warp_sum(t);
        }
    }
    __syncthreads();
}

// This thread's share of sum_i p[i] (i = threadIdx.x + k NT): sixteen loads
// per trip, all issued before the first is added (so a thread waits for memory
// once per sixteen values, not once per value), into eight chains; the order is
// fixed by n and NT, so the result is deterministic.
template <int NT>
__device__ __forceinline__ double partial_sum(const double* p, int n) {
    constexpr int M = 16;
    double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += M * NT) {
        double v[M];
#pragma unroll
        for (int k = 0; k < M; ++k) v[k] = i + k * NT < n ? __ldcg(&p[i + k * NT]) : 0.0;
#pragma unroll
        for (int k = 0; k < M; ++k) a[k & 7] += v[k];
    }
    return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

// Two-level deterministic reduction inside one launch: every block stores its
// NV partials, the last block to arrive sums them in block order and returns
// true with the totals in tot (thread 0 valid). partials: [NV * gridDim.x].
// Blocks are numbered x-fastest over a 1D, 2D or 3D grid.
template <int NT, int NV>
__device__ bool last_block_totals(double (&v)[NV], double* partials, unsigned* counter,
                                  double (&tot)[NV]) {
    __shared__ double sm[NV * NT / 32];
    __shared__ bool am_last;
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_sum<NT, NV>(v, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partials[k * nb + bid] = v[k];
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        am_last = (t == nb - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] = partial_sum<NT>(partials + (size_t)k * nb, (int)nb);
    block_sum<NT, NV>(s, sm);
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = s[k];
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// --------------------------------------------------------- grid barrier --

// Sense-free generation barrier for cooperative launches. Every wait is bounded
// by a clock64 deadline; on timeout (or when another block already failed) the
// error word is set and all blocks return false so the kernel can exit.
struct GridBarrier {
    unsigned count;
    unsigned gen;
    int error;  // 0 ok, TO_ETIMEOUT
    int pad;
};

__device__ __forceinline__ bool grid_sync(GridBarrier* b, long long deadline) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {  // one thread per block arrives
        volatile unsigned* vgen = &b->gen;
        volatile int* verr = &b->error;
        unsigned my_gen = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(&b->count, 1u);
        ok = 1;
        if (arrived == gridDim.x - 1) {
            b->count = 0u;
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            long long t0 = clock64();
            while (*vgen == my_gen) {
                if (*verr != 0 || clock64() - t0 > deadline) {
                    atomicExch(&b->error, (int)TO_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Reduction across a cooperative grid: every block ends with the same totals,
// summed in block order. Uses ping-pong partial buffers (parity) so that the
// next reduction cannot overwrite partials that a slow block still reads.
template <int NT, int NV>
__device__ bool grid_totals(double (&v)[NV], double* partials /* [2][NV][gridDim] */, int parity,
                            GridBarrier* bar, long long deadline, double (&tot)[NV]) {
    __shared__ double sm[NV * NT / 32];
    __shared__ double res[NV];
    double* P = partials + (size_t)parity * NV * gridDim.x;
    block_sum<NT, NV>(v, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) P[k * gridDim.x + blockIdx.x] = v[k];
    }
    if (!grid_sync(bar, deadline)) return false;
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        s[k] = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) s[k] += __ldcg(&P[k * gridDim.x + i]);
    }
    block_sum<NT, NV>(s, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) res[k] = s[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = res[k];
    __syncthreads();
    return true;
}

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace topo
