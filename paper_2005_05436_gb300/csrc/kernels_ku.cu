// Stiffness-operator kernels: matrix-free K(xPhys) u, Jacobi diagonal, element
// strain energies / compliance sensitivities and the lower-triangle CSR
// assembly K^(s) (Ferrari & Sigmund 2020, Eqs. 4-6 and 10-11).
//
// 3D K u runs on the Walsh-factored element tiles of kernels_walsh.cu; the
// node-centric kernels here (2D, and 3D with ku_impl 1) gather, for each of the
// (up to) 2^dim elements around node n, E_e times the Ke rows of n's local DOFs
// against the element's displacement vector u_e. Every output is written by
// exactly one thread (no atomics, deterministic), and all Ke indices are
// compile-time constants so Ke is read from the constant bank.
#include "kernels.h"
#include "ku_device.cuh"

namespace topo {

template <typename T, bool PCG>
__global__ void __launch_bounds__(256) k_apply_K3(Dims d, const KeP<T, 24> ke, const T* __restrict__ E,
                                                  const T* __restrict__ u, T* __restrict__ y,
                                                  const uint8_t* __restrict__ fixed, int mask_out,
                                                  PcgScalars* pcg, double* partials, unsigned* counter) {
    if (PCG && pcg->done) return;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double dot = 0.0;
    if (n < d.nnodes) {
        T a0, a1, a2;
        ku3_node_clamped<T>(ke, E, u, (int)n, d, a0, a1, a2);
        if (mask_out) {
            if (fixed[3 * n + 0]) a0 = T(0);
            if (fixed[3 * n + 1]) a1 = T(0);
            if (fixed[3 * n + 2]) a2 = T(0);
        }
        y[3 * n + 0] = a0;
        y[3 * n + 1] = a1;
        y[3 * n + 2] = a2;
        if (PCG) dot = (double)u[3 * n] * a0 + (double)u[3 * n + 1] * a1 + (double)u[3 * n + 2] * a2;
    }
    if (PCG) {
        double v[1] = {dot}, tot[1];
        if (last_block_totals<256, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
            pcg->pAp = tot[0];
            pcg->alpha = pcg->rz / tot[0];
        }
    }
}

// ------------------------------------------------------------ 2D (Q4) K u --

template <typename T, bool PCG>
__global__ void __launch_bounds__(256) k_apply_K2(Dims d, const KeP<T, 8> ke, const T* __restrict__ E,
                                                  const T* __restrict__ u, T* __restrict__ y,
                                                  const uint8_t* __restrict__ fixed, int mask_out,
                                                  PcgScalars* pcg, double* partials, unsigned* counter) {
    if (PCG && pcg->done) return;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double dot = 0.0;
    if (n < d.nnodes) {
        T a0, a1;
        ku2_node<T, true>(ke, E, u, n, d, a0, a1);
        if (mask_out) {
            if (fixed[2 * n + 0]) a0 = T(0);
            if (fixed[2 * n + 1]) a1 = T(0);
        }
        y[2 * n + 0] = a0;
        y[2 * n + 1] = a1;
        if (PCG) dot = (double)u[2 * n] * a0 + (double)u[2 * n + 1] * a1;
    }
    if (PCG) {
        double v[1] = {dot}, tot[1];
        if (last_block_totals<256, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
            pcg->pAp = tot[0];
            pcg->alpha = pcg->rz / tot[0];
        }
    }
}

template <typename T>
void launch_apply_K(const Dims& d, const KeP<T, 24>& ke3, const KeP<T, 8>& ke2, const WalshK<T>& wk,
                    bool node_centric, const T* E, const T* u, T* y, const uint8_t* fixed, bool mask_out,
                    cudaStream_t st) {
    const int nb = div_up(d.nnodes, 256);
    if (d.dim == 3 && !node_centric) {
        launch_walsh_op3<T>(d, wk, 0, E, u, nullptr, nullptr, y, fixed, mask_out, T(0), nullptr, nullptr,
                            nullptr, 0, nullptr, 0, st);
        return;
    }
    if (d.dim == 3)
        k_apply_K3<T, false><<<nb, 256, 0, st>>>(d, ke3, E, u, y, fixed, mask_out, nullptr, nullptr, nullptr);
    else
        k_apply_K2<T, false><<<nb, 256, 0, st>>>(d, ke2, E, u, y, fixed, mask_out, nullptr, nullptr, nullptr);
    TOPO_CHECK_LAUNCH();
}

template void launch_apply_K<double>(const Dims&, const KeP<double, 24>&, const KeP<double, 8>&,
                                     const WalshK<double>&, bool, const double*, const double*, double*,
                                     const uint8_t*, bool, cudaStream_t);
template void launch_apply_K<float>(const Dims&, const KeP<float, 24>&, const KeP<float, 8>&,
                                    const WalshK<float>&, bool, const float*, const float*, float*,
                                    const uint8_t*, bool, cudaStream_t);

// ------------------------------------------------------------- diagonal --

template <typename T, int D>
__global__ void k_diag_inv(Dims d, const KeP<T, D> ke, const T* __restrict__ E,
                           const uint8_t* __restrict__ fixed, T* __restrict__ dinv) {
    constexpr int dim = D == 24 ? 3 : 2;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.nnodes) return;
    const int iy = (int)(n % d.nny);
    const long long t = n / d.nny;
    const int iz = (int)(t % d.nnz);
    const int ix = (int)(t / d.nnz);
    T acc[dim];
#pragma unroll
    for (int c = 0; c < dim; ++c) acc[c] = T(0);
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int exo = (o >> 2) & 1, ezo = (o >> 1) & 1, eyo = o & 1;
        if (dim == 2 && ezo) continue;
        const int ex = ix - 1 + exo, ey = iy - 1 + eyo, ez = dim == 3 ? iz - 1 + ezo : 0;
        if (ex < 0 || ex >= d.nelx || ey < 0 || ey >= d.nely || ez < 0 || ez >= d.nelz) continue;
        const T Ee = E[ey + (long long)d.nely * (ez + (long long)d.nelz * ex)];
        const int L = local_node(1 - exo, eyo, dim == 3 ? 1 - ezo : 0);
#pragma unroll
        for (int c = 0; c < dim; ++c) acc[c] += Ee * ke.k[(dim * L + c) * D + dim * L + c];
    }
#pragma unroll
    for (int c = 0; c < dim; ++c) dinv[dim * n + c] = fixed[dim * n + c] ? T(0) : T(1) / acc[c];
}

template <typename T>
void launch_diag_inv(const Dims& d, const KeP<T, 24>& ke3, const KeP<T, 8>& ke2, const T* E,
                     const uint8_t* fixed, T* dinv, cudaStream_t st) {
    const int nb = div_up(d.nnodes, 256);
    if (d.dim == 3)
        k_diag_inv<T, 24><<<nb, 256, 0, st>>>(d, ke3, E, fixed, dinv);
    else
        k_diag_inv<T, 8><<<nb, 256, 0, st>>>(d, ke2, E, fixed, dinv);
    TOPO_CHECK_LAUNCH();
}
template void launch_diag_inv<double>(const Dims&, const KeP<double, 24>&, const KeP<double, 8>&,
                                      const double*, const uint8_t*, double*, cudaStream_t);
template void launch_diag_inv<float>(const Dims&, const KeP<float, 24>&, const KeP<float, 8>&,
                                     const float*, const uint8_t*, float*, cudaStream_t);

// --------------------------------------------------------- sensitivities --

template <int D>
__global__ void __launch_bounds__(256) k_sensitivity(Dims d, const KeP<double, D> ke,
                                                     const double* __restrict__ xphys,
                                                     const double* __restrict__ U,
                                                     const int8_t* __restrict__ passive, double penal,
                                                     double E0, double Emin, double* __restrict__ dc,
                                                     double* energy_sum, double* partials,
                                                     unsigned* counter) {
    constexpr int dim = D == 24 ? 3 : 2;
    constexpr int NN = D / dim;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double esum = 0.0;
    if (e < d.nel) {
        const int ey = (int)(e % d.nely);
        const long long t = e / d.nely;
        const int ez = (int)(t % d.nelz);
        const int ex = (int)(t / d.nelz);
        double ue[D];
#pragma unroll
        for (int M = 0; M < NN; ++M) {
            const long long m = (ey + 1 - lny(M)) + (long long)d.nny * ((ez + lnz(M)) + (long long)d.nnz * (ex + lnx(M)));
#pragma unroll
            for (int c = 0; c < dim; ++c) ue[dim * M + c] = U[dim * m + c];
        }
        // u^T Ke u = sum_i Ke_ii u_i^2 + 2 sum_{i>j} Ke_ij u_i u_j
        double ce = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double r = 0.5 * ke.k[i * D + i] * ue[i];
#pragma unroll
            for (int j = 0; j < i; ++j) r += ke.k[i * D + j] * ue[j];
            ce += 2.0 * r * ue[i];
        }
        const double x = xphys[e];
        const double Ee = Emin + powp(x, penal) * (E0 - Emin);
        esum = Ee * ce;
        dc[e] = (passive && passive[e] != 0) ? 0.0 : -penal * (E0 - Emin) * powp(x, penal - 1.0) * ce;
    }
    double v[1] = {esum}, tot[1];
    if (last_block_totals<256, 1>(v, partials, counter, tot) && threadIdx.x == 0) *energy_sum = tot[0];
}

// 3D: ce_e = u_e^T Ke u_e = w^T M w with w the Walsh modes of u_e over the
// corners and M the block-diagonal form of Ke (walsh.cuh): about 170 FP64
// operations per element instead of the dense quadratic form's 324.
__global__ void __launch_bounds__(256) k_sensitivity3_walsh(Dims d, const WalshK<double> wk,
                                                            const double* __restrict__ xphys,
                                                            const double* __restrict__ U,
                                                            const int8_t* __restrict__ passive, double penal,
                                                            double E0, double Emin, double* __restrict__ dc,
                                                            double* energy_sum, double* partials,
                                                            unsigned* counter) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double esum = 0.0;
    if (e < d.nel) {
        const int ey = (int)(e % d.nely);
        const long long t = e / d.nely;
        const int ez = (int)(t % d.nelz);
        const int ex = (int)(t / d.nelz);
        double u[3][8];
#pragma unroll
        for (int g = 0; g < 8; ++g) {  // corner g = 4 gx + 2 gy + gz: node (ex + gx, ey + gy, ez + gz)
            const long long m = (ey + ((g >> 1) & 1)) + (long long)d.nny * ((ez + (g & 1)) + (long long)d.nnz * (ex + (g >> 2)));
#pragma unroll
            for (int c = 0; c < 3; ++c) u[c][g] = U[3 * m + c];
        }
        double W[3][8], Z[3][8];
#pragma unroll
        for (int c = 0; c < 3; ++c) walsh_fwd<double>(u[c], W[c]);
        walsh_blocks<double>(wk, 1.0, W[0], W[1], W[2], Z[0], Z[1], Z[2]);
        double ce = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 1; q < 8; ++q) ce = fma(W[c][q], Z[c][q], ce);
        const double x = xphys[e];
        const double xp1 = powp(x, penal - 1.0);
        const double Ee = Emin + xp1 * x * (E0 - Emin);
        esum = Ee * ce;
        dc[e] = (passive && passive[e] != 0) ? 0.0 : -penal * (E0 - Emin) * xp1 * ce;
    }
    double v[1] = {esum}, tot[1];
    if (last_block_totals<256, 1>(v, partials, counter, tot) && threadIdx.x == 0) *energy_sum = tot[0];
}

void launch_sensitivity(const Dims& d, const KeP<double, 24>& ke3, const KeP<double, 8>& ke2,
                        const WalshK<double>& wk, bool node_centric, const double* xphys, const double* U,
                        const int8_t* passive, double penal, double E0, double Emin, double* dc,
                        double* energy_sum, double* partials, unsigned* counter, cudaStream_t st) {
    const int nb = div_up(d.nel, 256);
    if (d.dim == 3 && !node_centric)
        k_sensitivity3_walsh<<<nb, 256, 0, st>>>(d, wk, xphys, U, passive, penal, E0, Emin, dc, energy_sum,
                                                 partials, counter);
    else if (d.dim == 3)
        k_sensitivity<24><<<nb, 256, 0, st>>>(d, ke3, xphys, U, passive, penal, E0, Emin, dc,
                                              energy_sum, partials, counter);
    else
        k_sensitivity<8><<<nb, 256, 0, st>>>(d, ke2, xphys, U, passive, penal, E0, Emin, dc,
                                             energy_sum, partials, counter);
    TOPO_CHECK_LAUNCH();
}

// ------------------------------------------------------- CSR assembly --

// Lower-triangle row lengths: a DOF row couples to every DOF of the (existing)
// 3^dim neighbour nodes; the columns <= row are those of lower-numbered nodes
// plus components <= c of its own node.
__global__ void k_lower_counts(Dims d, int32_t* counts) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.ndof) return;
    const long long n = r / d.dim;
    const int c = (int)(r % d.dim);
    const int iy = (int)(n % d.nny);
    const long long t = n / d.nny;
    const int iz = (int)(t % d.nnz);
    const int ix = (int)(t / d.nnz);
    int cnt = 0;
    const int zlo = d.dim == 3 ? -1 : 0, zhi = d.dim == 3 ? 1 : 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dz = zlo; dz <= zhi; ++dz)
            for (int dy = -1; dy <= 1; ++dy) {
                const int mx = ix + dx, mz = iz + dz, my = iy + dy;
                if (mx < 0 || mx >= d.nnx || mz < 0 || mz >= d.nnz || my < 0 || my >= d.nny) continue;
                if (dx == 0 && dz == 0 && dy == 0) {
                    cnt += c + 1;
                    goto done;
                }
                cnt += d.dim;
            }
done:
    counts[r] = cnt;
}

__global__ void k_lower_fill(Dims d, const double* __restrict__ Ke /* [D*D] */, const double* __restrict__ E,
                             const int32_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                             double* __restrict__ val) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.ndof) return;
    const int dim = d.dim, D = dim == 3 ? 24 : 8;
    const long long n = r / dim;
    const int c = (int)(r % dim);
    const int iy = (int)(n % d.nny);
    const long long t = n / d.nny;
    const int iz = (int)(t % d.nnz);
    const int ix = (int)(t / d.nnz);
    long long k = row_ptr[r];
    const int zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dz = zlo; dz <= zhi; ++dz)
            for (int dy = -1; dy <= 1; ++dy) {
                const int mx = ix + dx, mz = iz + dz, my = iy + dy;
                if (mx < 0 || mx >= d.nnx || mz < 0 || mz >= d.nnz || my < 0 || my >= d.nny) continue;
                const long long m = my + (long long)d.nny * (mz + (long long)d.nnz * mx);
                const bool self = (dx == 0 && dz == 0 && dy == 0);
                const int kmax = self ? c : dim - 1;
                for (int kc = 0; kc <= kmax; ++kc) {
                    double s = 0.0;
                    // elements containing both n and m
                    for (int exo = 0; exo < 2; ++exo)
                        for (int ezo = 0; ezo < (dim == 3 ? 2 : 1); ++ezo)
                            for (int eyo = 0; eyo < 2; ++eyo) {
                                const int ex = ix - 1 + exo, ey = iy - 1 + eyo, ez = dim == 3 ? iz - 1 + ezo : 0;
                                if (ex < 0 || ex >= d.nelx || ey < 0 || ey >= d.nely || ez < 0 || ez >= d.nelz) continue;
                                const int bx = mx - ex, bz = mz - ez;
                                const int byrow = my - ey;  // 0: top row (Y-up 1), 1: bottom row (Y-up 0)
                                if (bx < 0 || bx > 1 || bz < 0 || bz > 1 || byrow < 0 || byrow > 1) continue;
                                const int Ln = local_node(1 - exo, eyo, dim == 3 ? 1 - ezo : 0);
                                const int Lm = local_node(bx, 1 - byrow, bz);
                                s += E[ey + (long long)d.nely * (ez + (long long)d.nelz * ex)] *
                                     Ke[(dim * Ln + c) * D + dim * Lm + kc];
                            }
                    col[k] = (int32_t)(dim * m + kc);
                    val[k] = s;
                    ++k;
                }
                if (self) return;
            }
}

void launch_lower_row_counts(const Dims& d, int32_t* counts, cudaStream_t st) {
    k_lower_counts<<<div_up(d.ndof, 256), 256, 0, st>>>(d, counts);
    TOPO_CHECK_LAUNCH();
}

void launch_lower_fill_dev(const Dims& d, const double* Ke_dev, const double* E, const int32_t* row_ptr,
                           int32_t* col, double* val, cudaStream_t st) {
    k_lower_fill<<<div_up(d.ndof, 128), 128, 0, st>>>(d, Ke_dev, E, row_ptr, col, val);
    TOPO_CHECK_LAUNCH();
}

// ---------------------------------------------------------------- scan --

constexpr int SCAN_NT = 1024;

__global__ void k_scan_blocks(const int32_t* __restrict__ in, long long n, long long* __restrict__ out,
                              long long* __restrict__ block_sums) {
    __shared__ long long ws[SCAN_NT / 32];
    const long long i = (long long)blockIdx.x * SCAN_NT + threadIdx.x;
    long long v = i < n ? in[i] : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < SCAN_NT / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_NT / 32) ws[lane] = w;
    }
    __syncthreads();
    const long long incl = x + (wid > 0 ? ws[wid - 1] : 0);
    if (i < n) out[i] = incl - v;  // exclusive within the block
    if (threadIdx.x == SCAN_NT - 1) block_sums[blockIdx.x] = incl;
}

__global__ void k_scan_sums(long long* block_sums, int nb, long long* total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long acc = 0;
    for (int b = 0; b < nb; ++b) {
        long long s = block_sums[b];
        block_sums[b] = acc;
        acc += s;
    }
    *total = acc;
}

__global__ void k_scan_add(const long long* __restrict__ part, long long n,
                           const long long* __restrict__ block_sums, const long long* total,
                           int32_t* __restrict__ out) {
    const long long i = (long long)blockIdx.x * SCAN_NT + threadIdx.x;
    if (i < n) out[i] = (int32_t)(part[i] + block_sums[blockIdx.x]);
    if (i == n) out[n] = (int32_t)(*total);
}

size_t scan_tmp_size(long long n) {
    const long long nb = (n + SCAN_NT - 1) / SCAN_NT;
    return sizeof(long long) * (size_t)(n + nb + 1);
}

void launch_exclusive_scan(const int32_t* counts, int32_t* out, long long n, void* tmp,
                           long long* total_dev, cudaStream_t st) {
    const int nb = div_up(n, SCAN_NT);
    long long* part = (long long*)tmp;
    long long* bs = part + n;
    k_scan_blocks<<<nb, SCAN_NT, 0, st>>>(counts, n, part, bs);
    k_scan_sums<<<1, 32, 0, st>>>(bs, nb, total_dev);
    k_scan_add<<<div_up(n + 1, SCAN_NT), SCAN_NT, 0, st>>>(part, n, bs, total_dev, out);
    TOPO_CHECK_LAUNCH();
    count_launches(2);
}

}  // namespace topo
