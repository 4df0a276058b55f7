// Batched geometric multigrid for the uneven 2D instances of batch.cu: the
// preconditioner of the FP32 inner PCG (the multigrid-preconditioned CG that the
// paper cites for its 3D code, Sec. 4, applied to every instance at once).
//
// Every instance has its own hierarchy: a level halves each axis (ceil(n / 2),
// so odd grids coarsen too) until the level has at most COARSE_NDOF DOFs.
// Coarse element matrices are Galerkin sums sum_j P_j^T K_j P_j over the four
// children (children outside an odd grid contribute nothing; on the first
// coarse level K_j = E_j Ke with the fine Dirichlet DOFs masked, or the
// constant-matrix sum sum_j E_j C_j when no child DOF is fixed). Coarse levels
// are stored as 9-point block stencils acting on displacements relative to the
// centre node (row sums R), smoothed by l1-Jacobi; the coarsest level of each
// instance is solved by its dense FP32 inverse (FP64 Cholesky). A V-cycle runs
// level-synchronously over the whole batch: the downward sweep of every level,
// one dense kernel for every instance's coarsest level, then the upward sweep.
#include "batch.cuh"

namespace topo {
namespace bt {
namespace {

constexpr long long COARSE_NDOF = 256;  // stop coarsening at or below this many DOFs
constexpr int MAX_LEVELS = 14;
constexpr int DENSE_MAX = 1024;

__host__ __device__ inline float pn_w(int j, int b, int B) {
    // weight of coarse corner B at the position of child j's corner b
    // (bilinear; positions in half-element units 0, 1, 2 along each axis)
    const int px = lnx(j) + lnx(b), py = lny(j) + lny(b);
    const float wx = lnx(B) ? 0.5f * px : 0.5f * (2 - px);
    const float wy = lny(B) ? 0.5f * py : 0.5f * (2 - py);
    return wx * wy;
}

__device__ __forceinline__ bool bskip(const BS& S, int skip_inner) {
    return S.ref_done || (skip_inner && S.inner_done);
}

// Tile position over one level's node tiles.
#define BL_TILE(k)                                         \
    const int4 tl = (k).tiles[blockIdx.x];                 \
    const int inst = tl.x;                                 \
    const LInst& L = (k).L[inst];                          \
    BS& S = (k).S[inst];                                   \
    const int ix = tl.y + (int)threadIdx.x / (k).TY;       \
    const int iy = tl.z + (int)threadIdx.x % (k).TY;

struct RowAbs8 {
    float a[8];
};

// ------------------------------------------------------------------ set-up

// Level 0 l1-Jacobi weights: 1 / sum_e E_e sum_j |Ke[row, j]|; 0 at fixed DOFs.
__global__ void kbm_l1_fine(BKL k, const RowAbs8 ra, const float* __restrict__ E32,
                            const uint8_t* __restrict__ fixed, float* __restrict__ dinv) {
    BL_TILE(k)
    (void)S;
    if (ix >= L.nnx || iy >= L.nny) return;
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int EXO = q >> 1, EYO = q & 1;
        const int ex = ix - 1 + EXO, ey = iy - 1 + EYO;
        if (ex < 0 || ex >= L.nelx || ey < 0 || ey >= L.nely) continue;
        const float Ee = E32[L.el0 + ey + (long long)L.nely * ex];
        const int Ln = local_node(1 - EXO, EYO, 0);
        a0 += Ee * ra.a[2 * Ln];
        a1 += Ee * ra.a[2 * Ln + 1];
    }
    const long long i = 2 * (L.node0 + iy + (long long)L.nny * ix);
    dinv[i] = fixed[i] ? 0.f : 1.f / a0;
    dinv[i + 1] = fixed[i + 1] ? 0.f : 1.f / a1;
}

// One warp per coarse element: Kc = sum_j P_j^T K_j P_j (8 x 8, row-major, local
// node order of local_node()). touched_c[ec] = 1 if a fine Dirichlet DOF lies
// under the element (level 1: among its 3 x 3 fine nodes; deeper: under one of
// its children); an untouched element matrix annihilates the rigid
// translations exactly (K_j does, and P_j maps a coarse translation to the same
// fine one).
template <bool FROM_FINE>
__global__ void __launch_bounds__(256) kbm_galerkin(const LInst* __restrict__ Lc, const long long* __restrict__ cstart,
                                                    int count, long long nelc, const LInst* __restrict__ Lf,
                                                    const float* __restrict__ Ef, const uint8_t* __restrict__ fixed_f,
                                                    const KeP<float, 8> ke, const float* __restrict__ Cj,
                                                    const float* __restrict__ Kf, float* __restrict__ Kc,
                                                    const uint8_t* __restrict__ touched_f,
                                                    uint8_t* __restrict__ touched_c) {
    __shared__ float pw[64];  // [j][b][B]
    __shared__ float Ks[8][256];
    __shared__ float Ts[8][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) pw[i] = pn_w(i >> 4, (i >> 2) & 3, i & 3);
    __syncthreads();
    const long long ec = (long long)blockIdx.x * 8 + warp;
    if (ec >= nelc) return;  // whole warps; only warp-level syncs below
    int lo = 0, hi = count - 1;  // the instance whose element range holds ec
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cstart[mid] <= ec)
            lo = mid;
        else
            hi = mid - 1;
    }
    const LInst& C = Lc[lo];
    const LInst& F = Lf[lo];
    const long long le = ec - C.el0;
    const int ey = (int)(le % C.nely), ex = (int)(le / C.nely);
    float* K = Ks[warp];
    float* T = Ts[warp];
    if (FROM_FINE) {
        const bool inside = 2 * ex + 1 < F.nelx && 2 * ey + 1 < F.nely;
        bool fx = false;
        if (lane < 18) {
            const int q = lane >> 1, c = lane & 1, fy = 2 * ey + q % 3, fxn = 2 * ex + q / 3;
            if (fy < F.nny && fxn < F.nnx) fx = fixed_f[2 * (F.node0 + fy + (long long)F.nny * fxn) + c] != 0;
        }
        const bool any_fixed = __any_sync(0xffffffffu, fx);
        if (lane == 0) touched_c[ec] = any_fixed ? 1 : 0;
        if (inside && !any_fixed) {
            float Ej[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int exf = 2 * ex + lnx(j), eyf = 2 * ey + (1 - lny(j));
                Ej[j] = Ef[F.el0 + eyf + (long long)F.nely * exf];
            }
            for (int idx = lane; idx < 64; idx += 32) {
                float s = 0.f;
#pragma unroll
                for (int j = 0; j < 4; ++j) s += Ej[j] * Cj[j * 64 + idx];
                Kc[ec * 64 + idx] = s;
            }
            return;
        }
    } else if (lane == 0) {
        int tch = 0;
        for (int j = 0; j < 4; ++j) {
            const int exf = 2 * ex + lnx(j), eyf = 2 * ey + (1 - lny(j));
            if (exf < F.nelx && eyf < F.nely) tch |= touched_f[F.el0 + eyf + (long long)F.nely * exf];
        }
        touched_c[ec] = (uint8_t)tch;
    }
    for (int idx = lane; idx < 256; idx += 32) {
        const int j = idx >> 6, rem = idx & 63, row = rem >> 3, col = rem & 7;
        const int exf = 2 * ex + lnx(j), eyf = 2 * ey + (1 - lny(j));
        float v = 0.f;
        if (exf < F.nelx && eyf < F.nely) {
            const long long ef = F.el0 + eyf + (long long)F.nely * exf;
            if (FROM_FINE) {
                const int a = row >> 1, c = row & 1, bb = col >> 1, kk = col & 1;
                const long long na = F.node0 + (eyf + 1 - lny(a)) + (long long)F.nny * (exf + lnx(a));
                const long long nb = F.node0 + (eyf + 1 - lny(bb)) + (long long)F.nny * (exf + lnx(bb));
                const bool masked = fixed_f[2 * na + c] || fixed_f[2 * nb + kk];
                v = masked ? 0.f : Ef[ef] * ke.k[rem];
            } else {
                v = Kf[ef * 64 + rem];
            }
        }
        K[idx] = v;
    }
    __syncwarp();
    // T[j][a][c][B][k] = sum_b K_j[(a,c),(b,k)] w_j[b][B]
    for (int idx = lane; idx < 256; idx += 32) {
        const int k = idx & 1, B = (idx >> 1) & 3, c = (idx >> 3) & 1, a = (idx >> 4) & 3, j = idx >> 6;
        float s = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) s += K[j * 64 + (a * 2 + c) * 8 + b * 2 + k] * pw[j * 16 + b * 4 + B];
        T[idx] = s;
    }
    __syncwarp();
    // Kc[(A,c),(B,k)] = sum_j sum_a w_j[a][A] T[j][a][c][B][k]
    for (int idx = lane; idx < 64; idx += 32) {
        const int row = idx >> 3, col = idx & 7, A = row >> 1, c = row & 1, B = col >> 1, k = col & 1;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int a = 0; a < 4; ++a) s += pw[j * 16 + a * 4 + A] * T[j * 64 + a * 16 + c * 8 + B * 2 + k];
        Kc[ec * 64 + idx] = s;
    }
}

// Node stencils of a coarse level from its element matrices: S[s][c][k] is the
// (n, n + s) block summed over the elements containing both nodes, R the row
// sums (the operator applied to the unit translations), stored as exactly 0 at
// a node none of whose elements is touched by a Dirichlet DOF (summed in FP32
// they would hold the rounding of cancelling blocks, which the relative form
// R_n u_n applies to absolute displacements); l1-Jacobi weights; DOFs with a
// zero diagonal become Dirichlet.
__global__ void kbm_stencil(BKL k, const float* __restrict__ Kel, const uint8_t* __restrict__ touched,
                            float* __restrict__ Sst, float* __restrict__ R, float* __restrict__ dinv,
                            uint8_t* __restrict__ fixed, long long nn) {
    BL_TILE(k)
    (void)S;
    if (ix >= L.nnx || iy >= L.nny) return;
    const long long n = L.node0 + iy + (long long)L.nny * ix;
    float rs[4] = {0.f, 0.f, 0.f, 0.f}, l1[2] = {0.f, 0.f}, dg[2] = {0.f, 0.f};
    for (int s = 0; s < 9; ++s) {
        const int mx = ix + s / 3 - 1, my = iy + s % 3 - 1;
        float blk[4] = {0.f, 0.f, 0.f, 0.f};
        if (mx >= 0 && mx < L.nnx && my >= 0 && my < L.nny) {
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int exo = o >> 1, eyo = o & 1;
                const int ex = ix - 1 + exo, ey = iy - 1 + eyo;
                if (ex < 0 || ex >= L.nelx || ey < 0 || ey >= L.nely) continue;
                const int bx = mx - ex, brow = my - ey;
                if (bx < 0 || bx > 1 || brow < 0 || brow > 1) continue;
                const int Ln = local_node(1 - exo, eyo, 0), Lm = local_node(bx, 1 - brow, 0);
                const float* Ke = Kel + (L.el0 + ey + (long long)L.nely * ex) * 64;
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int q = 0; q < 2; ++q) blk[c * 2 + q] += Ke[(Ln * 2 + c) * 8 + Lm * 2 + q];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            Sst[((long long)s * 4 + q) * nn + n] = blk[q];
            rs[q] += blk[q];
        }
        l1[0] += fabsf(blk[0]) + fabsf(blk[1]);
        l1[1] += fabsf(blk[2]) + fabsf(blk[3]);
        if (s == 4) {
            dg[0] = blk[0];
            dg[1] = blk[3];
        }
    }
    bool tch = false;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int ex = ix - 1 + (o >> 1), ey = iy - 1 + (o & 1);
        if (ex >= 0 && ex < L.nelx && ey >= 0 && ey < L.nely) tch |= touched[L.el0 + ey + (long long)L.nely * ex] != 0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) R[(long long)q * nn + n] = tch ? rs[q] : 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const bool f = !(dg[c] > 0.f);
        fixed[2 * n + c] = f;
        dinv[2 * n + c] = f ? 0.f : 1.f / l1[c];
    }
}

// One CTA per instance: assemble the coarsest operator (FP64), Cholesky
// A = L L^T, X = L^-1, and the inverse A^-1 = X^T X stored in FP32. Dirichlet
// DOFs get identity rows and columns.
__global__ void __launch_bounds__(256) kbm_dense_factor(const CInst* __restrict__ Cs, double* __restrict__ Aw,
                                                        float* __restrict__ Ainv) {
    const CInst& c = Cs[blockIdx.x];
    const int n = c.nc, tid = threadIdx.x, nt = blockDim.x;
    double* A = Aw + 2 * c.a0;
    double* X = A + (long long)n * n;
    for (long long i = tid; i < (long long)n * n; i += nt) {
        A[i] = 0.0;
        X[i] = 0.0;
    }
    __syncthreads();
    const int nnodes = c.nnx * c.nny;
    for (int q = tid; q < nnodes; q += nt) {
        const int ix = q / c.nny, iy = q % c.nny;
        const long long gn = c.node0 + q;
        for (int cc = 0; cc < 2; ++cc) {
            const int row = 2 * q + cc;
            if (c.fixed[2 * gn + cc]) {
                A[(long long)row * n + row] = 1.0;
                continue;
            }
            for (int s = 0; s < 9; ++s) {
                const int mx = ix + s / 3 - 1, my = iy + s % 3 - 1;
                if (mx < 0 || mx >= c.nnx || my < 0 || my >= c.nny) continue;
                const int m = my + c.nny * mx;
                for (int kk = 0; kk < 2; ++kk) {
                    if (c.fixed[2 * (c.node0 + m) + kk]) continue;
                    A[(long long)row * n + 2 * m + kk] = (double)c.S[((long long)s * 4 + cc * 2 + kk) * c.nnode + gn];
                }
            }
        }
    }
    __syncthreads();
    __shared__ double piv;
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            const double d = A[(long long)k * n + k];
            piv = d > 0.0 ? sqrt(d) : 1.0;
            A[(long long)k * n + k] = piv;
        }
        __syncthreads();
        const double pk = piv;
        for (int i = k + 1 + tid; i < n; i += nt) A[(long long)i * n + k] /= pk;
        __syncthreads();
        for (int i = k + 1 + tid; i < n; i += nt) {
            const double lik = A[(long long)i * n + k];
            double* Ai = A + (long long)i * n;
            for (int j = k + 1; j <= i; ++j) Ai[j] -= lik * A[(long long)j * n + k];
        }
        __syncthreads();
    }
    for (int j = tid; j < n; j += nt) {  // column j of X = L^-1
        X[(long long)j * n + j] = 1.0 / A[(long long)j * n + j];
        for (int i = j + 1; i < n; ++i) {
            double s = 0.0;
            const double* Ai = A + (long long)i * n;
            for (int m = j; m < i; ++m) s += Ai[m] * X[(long long)m * n + j];
            X[(long long)i * n + j] = -s / Ai[i];
        }
    }
    __syncthreads();
    for (long long idx = tid; idx < (long long)n * n; idx += nt) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        if (j > i) continue;
        double s = 0.0;
        for (int m = i; m < n; ++m) s += X[(long long)m * n + i] * X[(long long)m * n + j];
        Ainv[c.a0 + (long long)i * n + j] = (float)s;
        Ainv[c.a0 + (long long)j * n + i] = (float)s;
    }
}

// ----------------------------------------------------------------- V-cycle

__global__ void kbm_jacobi_first(BKL k, const float* __restrict__ dinv, const float* __restrict__ rhs,
                                 float* __restrict__ z, float omega, int skip_inner) {
    BL_TILE(k)
    if (bskip(S, skip_inner) || L.depth <= k.level + 1) return;
    if (ix >= L.nnx || iy >= L.nny) return;
    const long long i = 2 * (L.node0 + iy + (long long)L.nny * ix);
    z[i] = omega * dinv[i] * rhs[i];
    z[i + 1] = omega * dinv[i + 1] * rhs[i + 1];
}

// Level 0, matrix-free: MODE 1 out = u + omega D^-1 (rhs - K u); MODE 2
// out = rhs - K u; Dirichlet DOFs 0.
template <int MODE>
__global__ void kbm_fine_op(BKL k, const KeP<float, 8> ke, const float* __restrict__ E32, const float* __restrict__ u,
                            const float* __restrict__ rhs, const float* __restrict__ dinv, float* __restrict__ out,
                            const uint8_t* __restrict__ fixed, float omega, int skip_inner) {
    BL_TILE(k)
    if (bskip(S, skip_inner)) return;
    if (ix >= L.nnx || iy >= L.nny) return;
    float a[2];
    bku2<float>(ke, E32 + L.el0, u + 2 * L.node0, ix, iy, L.nelx, L.nely, a[0], a[1]);
    const long long i = 2 * (L.node0 + iy + (long long)L.nny * ix);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float o = MODE == 1 ? u[i + c] + omega * dinv[i + c] * (rhs[i + c] - a[c]) : rhs[i + c] - a[c];
        if (fixed[i + c]) o = 0.f;
        out[i + c] = o;
    }
}

// Coarse levels: the same modes with the stencils, in the relative form
// sum_{m != n} S_nm (u_m - u_n) + R_n u_n.
template <int MODE>
__global__ void kbm_stencil_op(BKL k, const float* __restrict__ Sst, const float* __restrict__ R,
                               const float* __restrict__ u, const float* __restrict__ rhs,
                               const float* __restrict__ dinv, float* __restrict__ out,
                               const uint8_t* __restrict__ fixed, float omega, long long nn, int skip_inner) {
    BL_TILE(k)
    if (bskip(S, skip_inner) || L.depth <= k.level + 1) return;
    if (ix >= L.nnx || iy >= L.nny) return;
    const long long n = L.node0 + iy + (long long)L.nny * ix;
    const float u0 = u[2 * n], u1 = u[2 * n + 1];
    float a0 = R[0 * nn + n] * u0 + R[1 * nn + n] * u1;
    float a1 = R[2 * nn + n] * u0 + R[3 * nn + n] * u1;
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        if (s == 4) continue;
        const int mx = ix + s / 3 - 1, my = iy + s % 3 - 1;
        if (mx < 0 || mx >= L.nnx || my < 0 || my >= L.nny) continue;
        const long long m = L.node0 + my + (long long)L.nny * mx;
        const float d0 = u[2 * m] - u0, d1 = u[2 * m + 1] - u1;
        a0 += Sst[((long long)s * 4 + 0) * nn + n] * d0 + Sst[((long long)s * 4 + 1) * nn + n] * d1;
        a1 += Sst[((long long)s * 4 + 2) * nn + n] * d0 + Sst[((long long)s * 4 + 3) * nn + n] * d1;
    }
    const long long i = 2 * n;
    const float a[2] = {a0, a1};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float o = MODE == 1 ? u[i + c] + omega * dinv[i + c] * (rhs[i + c] - a[c]) : rhs[i + c] - a[c];
        if (fixed[i + c]) o = 0.f;
        out[i + c] = o;
    }
}

// r_c = P^T w_f over the coarse nodes of level l + 1 (weights 1, 1/2, 1/4).
__global__ void kbm_restrict(BKL kc, const LInst* __restrict__ Lf, const float* __restrict__ wf,
                             float* __restrict__ rc, const uint8_t* __restrict__ fixed_c, int skip_inner) {
    BL_TILE(kc)
    if (bskip(S, skip_inner)) return;
    if (ix >= L.nnx || iy >= L.nny) return;
    const LInst& F = Lf[inst];
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int ox = -1; ox <= 1; ++ox)
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy) {
            const int fx = 2 * ix + ox, fy = 2 * iy + oy;
            if (fx < 0 || fx >= F.nnx || fy < 0 || fy >= F.nny) continue;
            const float w = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f);
            const long long f = F.node0 + fy + (long long)F.nny * fx;
            a0 += w * wf[2 * f];
            a1 += w * wf[2 * f + 1];
        }
    const long long i = 2 * (L.node0 + iy + (long long)L.nny * ix);
    rc[i] = fixed_c[i] ? 0.f : a0;
    rc[i + 1] = fixed_c[i + 1] ? 0.f : a1;
}

// z_f += P z_c over the nodes of level l.
__global__ void kbm_prolong(BKL kf, const LInst* __restrict__ Lc, const float* __restrict__ zc,
                            float* __restrict__ zf, const uint8_t* __restrict__ fixed_f, int skip_inner) {
    BL_TILE(kf)
    if (bskip(S, skip_inner) || L.depth <= kf.level + 1) return;
    if (ix >= L.nnx || iy >= L.nny) return;
    const LInst& C = Lc[inst];
    const int x0 = ix >> 1, y0 = iy >> 1;
    const int nxs = (ix & 1) ? 2 : 1, nys = (iy & 1) ? 2 : 1;
    const float wx = (ix & 1) ? 0.5f : 1.f, wy = (iy & 1) ? 0.5f : 1.f;
    float a0 = 0.f, a1 = 0.f;
    for (int a = 0; a < nxs; ++a)
        for (int bq = 0; bq < nys; ++bq) {
            const long long m = C.node0 + (y0 + bq) + (long long)C.nny * (x0 + a);
            a0 += wx * wy * zc[2 * m];
            a1 += wx * wy * zc[2 * m + 1];
        }
    const long long i = 2 * (L.node0 + iy + (long long)L.nny * ix);
    if (!fixed_f[i]) zf[i] += a0;
    if (!fixed_f[i + 1]) zf[i + 1] += a1;
}

// z = A_c^-1 rhs on every instance's coarsest level (one CTA per instance).
__global__ void __launch_bounds__(256) kbm_dense_apply(const CInst* __restrict__ Cs, const BS* __restrict__ Sarr,
                                                       const float* __restrict__ Ainv, int skip_inner) {
    __shared__ float rs[DENSE_MAX];
    const CInst& c = Cs[blockIdx.x];
    if (bskip(Sarr[blockIdx.x], skip_inner)) return;
    const int n = c.nc;
    const float* rhs = c.rhs + 2 * c.node0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) rs[q] = rhs[q];
    __syncthreads();
    const float* Ai = Ainv + c.a0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < n; ++r) s += Ai[(long long)r * n + q] * rs[r];
        c.z[2 * c.node0 + q] = s;
    }
}

template <typename T>
T* mg_alloc(to_batch* b, size_t count) {
    void* p = nullptr;
    TOPO_CUDA(cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)));
    b->allocs.push_back(p);
    return (T*)p;
}

BKL level_k(const to_batch* b, int l) {
    const BMGLevel& V = b->mg->lev[l];
    return BKL{V.dL, b->dS, V.tiles, b->nty, l};
}

}  // namespace

// Hierarchy of every instance, level arrays and the coarsest dense pools.
void bmg_create(to_batch* b) {
    BMG* mg = new BMG();
    b->mg = mg;
    mg->nu = std::max(1, b->p.mg_nu);
    mg->omega = (float)b->p.mg_omega;
    const int count = b->count;
    std::vector<std::vector<std::pair<int, int>>> dims(count);
    int nlev = 0;
    for (int i = 0; i < count; ++i) {
        auto& d = dims[i];
        d.push_back({b->hI[i].nelx, b->hI[i].nely});
        for (;;) {
            const int x = d.back().first, y = d.back().second;
            const long long ndof = 2LL * (x + 1) * (y + 1);
            if ((d.size() >= 2 && ndof <= COARSE_NDOF) || (int)d.size() >= MAX_LEVELS) break;
            d.push_back({(x + 1) / 2, (y + 1) / 2});
        }
        nlev = std::max(nlev, (int)d.size());
    }
    mg->nlev = nlev;
    mg->lev.resize(nlev);
    for (int l = 0; l < nlev; ++l) {
        BMGLevel& V = mg->lev[l];
        V.hL.assign(count, LInst{});
        V.hstart.assign(count + 1, 0);
        long long el = 0, nd = 0;
        for (int i = 0; i < count; ++i) {
            LInst& Li = V.hL[i];
            Li.depth = (int)dims[i].size();
            V.hstart[i] = el;
            if (l >= Li.depth) {
                Li.el0 = el;
                Li.node0 = nd;
                continue;
            }
            Li.nelx = dims[i][l].first;
            Li.nely = dims[i][l].second;
            Li.nnx = Li.nelx + 1;
            Li.nny = Li.nely + 1;
            if (l == 0) {
                Li.el0 = b->hI[i].el0;
                Li.node0 = b->hI[i].node0;
            } else {
                Li.el0 = el;
                Li.node0 = nd;
            }
            el += (long long)Li.nelx * Li.nely;
            nd += (long long)Li.nnx * Li.nny;
        }
        V.hstart[count] = el;
        V.nel = el;
        V.nnode = nd;
        long long cap = 0;
        for (int ty : {32, 64, 16, 128, 256})
            for (int tx : {1, 2, 4, 8, 16}) {
                long long t = 0;
                for (const LInst& Li : V.hL)
                    if (Li.nnx > 0) t += (long long)((Li.nnx + tx - 1) / tx) * ((Li.nny + ty - 1) / ty);
                cap = std::max(cap, t);
            }
        V.tile_cap = cap;
        V.tiles = mg_alloc<int4>(b, cap);
        V.dL = mg_alloc<LInst>(b, count);
        V.dstart = mg_alloc<long long>(b, count + 1);
        TOPO_CUDA(cudaMemcpyAsync(V.dstart, V.hstart.data(), (count + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                                  b->st));
        if (l == 0) {
            V.dinv = b->dinv;
            V.fixed = const_cast<uint8_t*>(b->fixed);
            V.z = b->z0 = mg_alloc<float>(b, 2 * nd);
            V.t = b->t0 = mg_alloc<float>(b, 2 * nd);
            V.w = b->w0 = mg_alloc<float>(b, 2 * nd);
        } else {
            V.Kel = mg_alloc<float>(b, V.nel * 64);
            V.touched = mg_alloc<uint8_t>(b, V.nel);
            V.S = mg_alloc<float>(b, 36 * nd);
            V.R = mg_alloc<float>(b, 4 * nd);
            V.dinv = mg_alloc<float>(b, 2 * nd);
            V.fixed = mg_alloc<uint8_t>(b, 2 * nd);
            V.z = mg_alloc<float>(b, 2 * nd);
            V.t = mg_alloc<float>(b, 2 * nd);
            V.w = mg_alloc<float>(b, 2 * nd);
            V.r = mg_alloc<float>(b, 2 * nd);
        }
    }
    // coarsest level of each instance
    mg->hC.resize(count);
    long long pool = 0;
    for (int i = 0; i < count; ++i) {
        const int c = (int)dims[i].size() - 1;
        const LInst& Li = mg->lev[c].hL[i];
        CInst& C = mg->hC[i];
        C.level = c;
        C.nnx = Li.nnx;
        C.nny = Li.nny;
        C.nc = 2 * Li.nnx * Li.nny;
        TOPO_REQUIRE(c >= 1 && C.nc <= DENSE_MAX, "batched multigrid: coarsest level too large");
        C.node0 = Li.node0;
        C.a0 = pool;
        C.S = mg->lev[c].S;
        C.fixed = mg->lev[c].fixed;
        C.rhs = mg->lev[c].r;
        C.z = mg->lev[c].t;  // the buffer that holds every level's result after the up-sweep
        C.nnode = mg->lev[c].nnode;
        pool += (long long)C.nc * C.nc;
        mg->max_nc = std::max(mg->max_nc, C.nc);
    }
    mg->dC = mg_alloc<CInst>(b, count);
    mg->Aw = mg_alloc<double>(b, 2 * pool);
    mg->Ainv = mg_alloc<float>(b, pool);
    TOPO_CUDA(cudaMemcpyAsync(mg->dC, mg->hC.data(), count * sizeof(CInst), cudaMemcpyHostToDevice, b->st));
    // level-1 constants C_j = P_j^T Ke P_j and the l1 row sums of Ke
    std::vector<double> K;
    element_matrix(2, b->p.nu, K);
    std::vector<float> cj(4 * 64);
    for (int j = 0; j < 4; ++j)
        for (int row = 0; row < 8; ++row)
            for (int col = 0; col < 8; ++col) {
                const int A = row >> 1, c = row & 1, B = col >> 1, k = col & 1;
                double s = 0.0;
                for (int a = 0; a < 4; ++a)
                    for (int bb = 0; bb < 4; ++bb)
                        s += (double)pn_w(j, a, A) * K[(a * 2 + c) * 8 + bb * 2 + k] * (double)pn_w(j, bb, B);
                cj[j * 64 + row * 8 + col] = (float)s;
            }
    mg->Cj = mg_alloc<float>(b, cj.size());
    TOPO_CUDA(cudaMemcpyAsync(mg->Cj, cj.data(), cj.size() * sizeof(float), cudaMemcpyHostToDevice, b->st));
    for (int r = 0; r < 8; ++r) {
        double s = 0.0;
        for (int c = 0; c < 8; ++c) s += std::fabs(K[r * 8 + c]);
        mg->arow[r] = (float)s;
    }
    TOPO_CUDA(cudaStreamSynchronize(b->st));
}

// Node tile tables of every level with the batch's node-tile shape.
void bmg_tiles(to_batch* b) {
    BMG* mg = b->mg;
    if (!mg) return;
    for (int l = 0; l < mg->nlev; ++l) {
        BMGLevel& V = mg->lev[l];
        std::vector<int4> t;
        for (int i = 0; i < b->count; ++i) {
            LInst& Li = V.hL[i];
            Li.tn0 = (int)t.size();
            if (Li.nnx > 0)
                for (int x0 = 0; x0 < Li.nnx; x0 += b->ntx)
                    for (int y0 = 0; y0 < Li.nny; y0 += b->nty) t.push_back(make_int4(i, x0, y0, 0));
            Li.tnn = (int)t.size() - Li.tn0;
        }
        TOPO_REQUIRE((long long)t.size() <= V.tile_cap, "multigrid tile table overflow");
        V.ntiles = (int)t.size();
        TOPO_CUDA(cudaMemcpyAsync(V.tiles, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, b->st));
        TOPO_CUDA(cudaMemcpyAsync(V.dL, V.hL.data(), V.hL.size() * sizeof(LInst), cudaMemcpyHostToDevice, b->st));
    }
    TOPO_CUDA(cudaStreamSynchronize(b->st));
}

// Per design iteration: fine l1 weights, Galerkin products, stencils, coarsest
// inverses.
void bmg_setup(to_batch* b, cudaStream_t st) {
    BMG* mg = b->mg;
    const int th = b->nty * b->ntx;
    RowAbs8 ra;
    for (int r = 0; r < 8; ++r) ra.a[r] = mg->arow[r];
    {
        const BKL k0 = level_k(b, 0);
        kbm_l1_fine<<<mg->lev[0].ntiles, th, 0, st>>>(k0, ra, b->E32, b->fixed, b->dinv);
        TOPO_CHECK_LAUNCH();
    }
    for (int l = 1; l < mg->nlev; ++l) {
        BMGLevel& V = mg->lev[l];
        const BMGLevel& Fv = mg->lev[l - 1];
        const int blocks = div_up(V.nel, 8);
        if (l == 1)
            kbm_galerkin<true><<<blocks, 256, 0, st>>>(V.dL, V.dstart, b->count, V.nel, Fv.dL, b->E32, b->fixed,
                                                       b->ke32, mg->Cj, nullptr, V.Kel, nullptr, V.touched);
        else
            kbm_galerkin<false><<<blocks, 256, 0, st>>>(V.dL, V.dstart, b->count, V.nel, Fv.dL, nullptr, nullptr,
                                                        b->ke32, nullptr, Fv.Kel, V.Kel, Fv.touched, V.touched);
        TOPO_CHECK_LAUNCH();
        kbm_stencil<<<V.ntiles, th, 0, st>>>(level_k(b, l), V.Kel, V.touched, V.S, V.R, V.dinv, V.fixed, V.nnode);
        TOPO_CHECK_LAUNCH();
    }
    kbm_dense_factor<<<b->count, 256, 0, st>>>(mg->dC, mg->Aw, mg->Ainv);
    TOPO_CHECK_LAUNCH();
}

float* bmg_vcycle(to_batch* b, cudaStream_t st, const float* r0, int skip_inner) {
    BMG* mg = b->mg;
    const int th = b->nty * b->ntx, L = mg->nlev, nu = mg->nu;
    const float om = mg->omega;
    std::vector<float*> cur(L);
    for (int l = 0; l + 1 < L; ++l) {
        BMGLevel& V = mg->lev[l];
        const BKL k = level_k(b, l);
        const float* rhs = l == 0 ? r0 : V.r;
        kbm_jacobi_first<<<V.ntiles, th, 0, st>>>(k, V.dinv, rhs, V.z, om, skip_inner);
        TOPO_CHECK_LAUNCH();
        float* c = V.z;
        float* o = V.t;
        for (int s = 1; s < nu; ++s) {
            if (l == 0)
                kbm_fine_op<1><<<V.ntiles, th, 0, st>>>(k, b->ke32, b->E32, c, rhs, V.dinv, o, V.fixed, om, skip_inner);
            else
                kbm_stencil_op<1><<<V.ntiles, th, 0, st>>>(k, V.S, V.R, c, rhs, V.dinv, o, V.fixed, om, V.nnode,
                                                            skip_inner);
            TOPO_CHECK_LAUNCH();
            std::swap(c, o);
        }
        if (l == 0)
            kbm_fine_op<2><<<V.ntiles, th, 0, st>>>(k, b->ke32, b->E32, c, rhs, V.dinv, V.w, V.fixed, om, skip_inner);
        else
            kbm_stencil_op<2><<<V.ntiles, th, 0, st>>>(k, V.S, V.R, c, rhs, V.dinv, V.w, V.fixed, om, V.nnode,
                                                        skip_inner);
        TOPO_CHECK_LAUNCH();
        BMGLevel& Cv = mg->lev[l + 1];
        kbm_restrict<<<Cv.ntiles, th, 0, st>>>(level_k(b, l + 1), V.dL, V.w, Cv.r, Cv.fixed, skip_inner);
        TOPO_CHECK_LAUNCH();
        cur[l] = c;
    }
    kbm_dense_apply<<<b->count, 256, 0, st>>>(mg->dC, b->dS, mg->Ainv, skip_inner);
    TOPO_CHECK_LAUNCH();
    for (int l = L - 2; l >= 0; --l) {
        BMGLevel& V = mg->lev[l];
        const BKL k = level_k(b, l);
        const float* rhs = l == 0 ? r0 : V.r;
        kbm_prolong<<<V.ntiles, th, 0, st>>>(k, mg->lev[l + 1].dL, mg->lev[l + 1].t, cur[l], V.fixed, skip_inner);
        TOPO_CHECK_LAUNCH();
        float* c = cur[l];
        float* o = c == V.z ? V.t : V.z;
        for (int s = 0; s < nu; ++s) {
            if (l == 0)
                kbm_fine_op<1><<<V.ntiles, th, 0, st>>>(k, b->ke32, b->E32, c, rhs, V.dinv, o, V.fixed, om, skip_inner);
            else
                kbm_stencil_op<1><<<V.ntiles, th, 0, st>>>(k, V.S, V.R, c, rhs, V.dinv, o, V.fixed, om, V.nnode,
                                                            skip_inner);
            TOPO_CHECK_LAUNCH();
            std::swap(c, o);
        }
        TOPO_REQUIRE(c == V.t, "V-cycle buffer parity");
    }
    return mg->lev[0].t;
}

}  // namespace bt
}  // namespace topo
