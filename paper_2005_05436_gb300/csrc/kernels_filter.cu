// Density filter (Eq. 2) and its chain rule (Eq. 7) by shared-memory tiles.
//
// A block stages its element tile plus a halo of R = ceil(rmin) - 1 elements on
// every side into shared memory, resolving the mirror ('N') or zero ('D')
// padding once per staged value, and, for the chain rule, the product
// in * dprj / Hs there as well. Each thread then forms FILTER_K outputs along
// x: the window is walked as rows along x (fixed y and z offsets, FilterTaps
// rows), and each row in chunks of FILTER_K x offsets, so that 2 FILTER_K - 1
// staged values and FILTER_K weights serve FILTER_K^2 multiply-adds.
//
// Two arithmetics: FP64 (one FP64 FMA per tap), and float-float for the mixed
// path (values and weights split into two floats each, products formed with
// the error-free FMA product and summed with TwoSum, about 2^-47 relative
// per product; the FP64 pipe runs at 1/64 of the FP32 rate on this GPU).
#include "kernels.h"

namespace topo {

namespace {

constexpr int FTY = 32;  // lanes along y

struct FF {
    float hi, lo;
};

// s + p * q for p = ph + pl, q = qh + ql, s kept as (hi, lo) by TwoSum.
__device__ __forceinline__ void ff_mac(FF& s, float ph, float pl, float qh, float ql) {
    const float p = __fmul_rn(ph, qh);
    const float e = fmaf(ph, qh, -p);                 // exact error of the leading product
    const float t = fmaf(ph, ql, fmaf(pl, qh, e));    // small terms (pl * ql dropped)
    const float sh = __fadd_rn(s.hi, p);
    const float bb = __fsub_rn(sh, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(sh, bb)), __fsub_rn(p, bb));
    s.hi = sh;
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, t));
}

// Staged value of element j (x, y, z indices before padding): in[j] (forward)
// or in[j] dprj[j] / Hs[j] (chain rule); 0 outside the grid under 'D'.
__device__ __forceinline__ double staged_value(const Dims& d, int bcN, int jx, int jy, int jz,
                                               const double* __restrict__ in, const double* __restrict__ dprj,
                                               const double* __restrict__ rHs, double rHs_const) {
    if (bcN) {
        jx = mirror_index(jx, d.nelx);
        jy = mirror_index(jy, d.nely);
        jz = mirror_index(jz, d.nelz);
    } else if (jx < 0 || jx >= d.nelx || jy < 0 || jy >= d.nely || jz < 0 || jz >= d.nelz) {
        return 0.0;
    }
    const long long j = jy + (long long)d.nely * (jz + (long long)d.nelz * jx);
    double v = in[j];
    if (dprj) v = v * dprj[j] * (rHs ? rHs[j] : rHs_const);
    return v;
}

// Tile: FTY elements along y, BZ along z, BX * FILTER_K along x; shared
// memory [SX][SZ][SY] with the halo (FP64 values, or hi / lo float planes).
template <int BZ, int BX, bool FFA>
__global__ void __launch_bounds__(FTY * BZ * BX) k_filter_tile(Dims d, FilterTaps t, int bcN,
                                                             const double* __restrict__ rHs, double rHs_const,
                                                             const double* __restrict__ in,
                                                             const double* __restrict__ dprj, double* __restrict__ out,
                                                             const int8_t* __restrict__ passive,
                                                             const double* __restrict__ keep) {
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    constexpr int NT = FTY * BZ * BX;
    const int R = t.R, Rz = t.Rz;
    const int SY = FTY + 2 * R, SZ = BZ + 2 * Rz, SX = BX * FILTER_K + 2 * R;
    const int XS = SZ * SY;  // stride of one x plane in the tile
    const int total = SX * XS;
    const int y0 = blockIdx.x * FTY, z0 = blockIdx.y * BZ, x0 = blockIdx.z * (BX * FILTER_K);
    double* sv = reinterpret_cast<double*>(fsm_raw);
    float* sh = reinterpret_cast<float*>(fsm_raw);
    float* sl = sh + total;
    for (int i = threadIdx.x; i < total; i += NT) {
        const int xs = i / XS, rem = i - xs * XS;
        const int zs = rem / SY, ys = rem - zs * SY;
        const double v = staged_value(d, bcN, x0 - R + xs, y0 - R + ys, z0 - Rz + zs, in, dprj, rHs, rHs_const);
        if (FFA) {
            const float h = (float)v;
            sh[i] = h;
            sl[i] = (float)(v - (double)h);
        } else {
            sv[i] = v;
        }
    }
    __syncthreads();
    const int ty = threadIdx.x % FTY, tz = (threadIdx.x / FTY) % BZ, tx = threadIdx.x / (FTY * BZ);
    const int ey = y0 + ty, ez = z0 + tz, exb = x0 + tx * FILTER_K;
    double acc[FILTER_K];
    FF facc[FILTER_K];
#pragma unroll
    for (int k = 0; k < FILTER_K; ++k) {
        acc[k] = 0.0;
        facc[k] = FF{0.f, 0.f};
    }
    int wbase = 0;
    for (int r = 0; r < t.nrows; ++r) {
        const int oy = __ldg(&t.rows[4 * r]), oz = __ldg(&t.rows[4 * r + 1]);
        const int dx0 = __ldg(&t.rows[4 * r + 2]), nch = __ldg(&t.rows[4 * r + 3]);
        // staged index of (x = exb + dx0, y = ey + oy, z = ez + oz)
        int base = (tx * FILTER_K + R + dx0) * XS + (tz + Rz + oz) * SY + (ty + R + oy);
        for (int c = 0; c < nch; ++c, base += FILTER_K * XS, wbase += FILTER_K) {
            if (FFA) {
                float vh[2 * FILTER_K - 1], vl[2 * FILTER_K - 1];
#pragma unroll
                for (int j = 0; j < 2 * FILTER_K - 1; ++j) {
                    // the last chunk may reach past the staged window only with zero weights
                    const int idx = min(base + j * XS, total - 1);
                    vh[j] = sh[idx];
                    vl[j] = sl[idx];
                }
#pragma unroll
                for (int j = 0; j < FILTER_K; ++j) {
                    const float wh = __ldg(&t.rwh[wbase + j]), wl = __ldg(&t.rwl[wbase + j]);
#pragma unroll
                    for (int k = 0; k < FILTER_K; ++k) ff_mac(facc[k], wh, wl, vh[k + j], vl[k + j]);
                }
                // renormalise (hi, lo) so that lo stays within one ulp of hi (Fast2Sum, |hi| >= |lo|)
#pragma unroll
                for (int k = 0; k < FILTER_K; ++k) {
                    const float s2 = __fadd_rn(facc[k].hi, facc[k].lo);
                    facc[k].lo = __fsub_rn(facc[k].lo, __fsub_rn(s2, facc[k].hi));
                    facc[k].hi = s2;
                }
            } else {
                double v[2 * FILTER_K - 1];
#pragma unroll
                for (int j = 0; j < 2 * FILTER_K - 1; ++j) v[j] = sv[min(base + j * XS, total - 1)];
#pragma unroll
                for (int j = 0; j < FILTER_K; ++j) {
                    const double w = __ldg(&t.rw[wbase + j]);
#pragma unroll
                    for (int k = 0; k < FILTER_K; ++k) acc[k] = fma(w, v[k + j], acc[k]);
                }
            }
        }
    }
    if (ey >= d.nely || ez >= d.nelz) return;
#pragma unroll
    for (int k = 0; k < FILTER_K; ++k) {
        const int ex = exb + k;
        if (ex >= d.nelx) break;
        const long long e = ey + (long long)d.nely * (ez + (long long)d.nelz * ex);
        double s = FFA ? (double)facc[k].hi + (double)facc[k].lo : acc[k];
        if (!dprj) s = s * (rHs ? rHs[e] : rHs_const);
        if (passive && passive[e] != 0) s = keep[e];
        out[e] = s;
    }
}

}  // namespace

size_t filter_tile_smem(const Dims& d, const FilterTaps& t) {
    const int BZ = d.dim == 3 ? 8 : 1, BX = d.dim == 3 ? 1 : 8;
    return (size_t)8 * (BX * FILTER_K + 2 * t.R) * (BZ + 2 * t.Rz) * (FTY + 2 * t.R);
}

bool launch_filter_tiled(const Dims& d, const FilterTaps& t, char bc, const double* rHs, double rHs_const,
                         const double* in, const double* dprj, double* out, const int8_t* passive,
                         const double* keep, bool float_float, cudaStream_t st) {
    const size_t smem = filter_tile_smem(d, t);
    if (!t.rows || smem > 200 * 1024) return false;
    const int bcN = bc == 'N';
#define TOPO_FT(BZV, BXV, FFV)                                                                                  \
    do {                                                                                                        \
        static bool attr = false; /* the same attribute value on every call */                                 \
        if (!attr) {                                                                                            \
            TOPO_CUDA(cudaFuncSetAttribute(k_filter_tile<BZV, BXV, FFV>,                                        \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));            \
            attr = true;                                                                                        \
        }                                                                                                       \
        const dim3 grid(div_up(d.nely, FTY), div_up(d.nelz, BZV), div_up(d.nelx, BXV * FILTER_K));             \
        k_filter_tile<BZV, BXV, FFV><<<grid, FTY * BZV * BXV, smem, st>>>(d, t, bcN, rHs, rHs_const, in, dprj, \
                                                                         out, passive, keep);                  \
    } while (0)
    if (d.dim == 3) {
        if (float_float)
            TOPO_FT(8, 1, true);
        else
            TOPO_FT(8, 1, false);
    } else {
        if (float_float)
            TOPO_FT(1, 8, true);
        else
            TOPO_FT(1, 8, false);
    }
#undef TOPO_FT
    TOPO_CHECK_LAUNCH();
    return true;
}

}  // namespace topo
