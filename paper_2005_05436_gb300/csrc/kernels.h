// Host-side launchers of the topopt kernels. All launch on `st`.
#pragma once

#include "common.cuh"
#include "walsh.cuh"

namespace topo {

// Device-resident scalars of one PCG solve (Jacobi or multigrid preconditioned).
struct PcgScalars {
    double rz, rz_new, pAp, alpha, beta;
    double rr, bb, rtol2;
    int done;     // 0 running, 1 converged, 2 cap reached, 3 NaN
    int iters;
    int maxit;
    int pad;
};

// ---- stiffness operator (kernels_ku.cu) ----
// y = K(E) u over all nodes (node-centric gather). mask_out zeroes fixed rows.
// If pcg != nullptr: y = K p with the PCG dot p.Ap fused; the last block sets
// alpha = rz / pAp; the launch is a no-op once pcg->done != 0.
// 3D: the Walsh-factored element tiles (kernels_walsh.cu) unless node_centric.
template <typename T>
void launch_apply_K(const Dims& d, const KeP<T, 24>& ke3, const KeP<T, 8>& ke2, const WalshK<T>& wk,
                    bool node_centric, const T* E, const T* u, T* y, const uint8_t* fixed, bool mask_out,
                    cudaStream_t st);

// 3D K u by Walsh-factored element tiles (kernels_walsh.cu), with the fused
// epilogues of the fine multigrid operator: mode 0 out = K u; 1 out = u +
// omega dinv (r - K u); 2 out = r - K u; fixed rows zeroed if mask_out. With
// pcg (modes 0 and 1): the FP64 dot u.out (mode 0) or r.out (mode 1) over the
// grid and, in the last block, alpha = rz / pAp (mode 0) or beta = rz_new / rz,
// rz = rz_new (mode 1); partials needs one value per block (npartials).
// Reads of u cover the node planes around out's: out must not alias u.
template <typename T>
void launch_walsh_op3(const Dims& d, const WalshK<T>& wk, int mode, const T* E, const T* u, const T* r,
                      const T* dinv, T* out, const uint8_t* fixed, bool mask_out, T omega, const int* skip,
                      PcgScalars* pcg, double* partials, long long npartials, unsigned* counter, int nsm,
                      cudaStream_t st);

// The same FP32 operator and epilogues with two elements per thread in paired
// FP32 arithmetic (kernels_walsh_pair.cu); walsh_pair_supported: a tile shape
// fits the grid (3D).
bool walsh_pair_supported(const Dims& d);
void launch_walsh_pair3(const Dims& d, const WalshK<float>& wk, int mode, const float* E, const float* u,
                        const float* r, const float* dinv, float* out, const uint8_t* fixed, bool mask_out,
                        float omega, const int* skip, PcgScalars* pcg, double* partials, long long npartials,
                        unsigned* counter, int nsm, cudaStream_t st);

// Jacobi inverse diagonal: dinv[i] = 1 / K_ii (0 at fixed DOFs).
template <typename T>
void launch_diag_inv(const Dims& d, const KeP<T, 24>& ke3, const KeP<T, 8>& ke2, const T* E,
                     const uint8_t* fixed, T* dinv, cudaStream_t st);

// Element strain energies ce_e = u_e^T Ke u_e; dc_e = -p (E0-Emin) x^(p-1) ce_e on
// active elements (0 on passive ones). Fused deterministic sum of E_e ce_e
// written to *energy_sum.
// 3D: the Walsh form of Ke (wk) unless node_centric.
void launch_sensitivity(const Dims& d, const KeP<double, 24>& ke3, const KeP<double, 8>& ke2,
                        const WalshK<double>& wk, bool node_centric, const double* xphys, const double* U,
                        const int8_t* passive, double penal, double E0, double Emin, double* dc,
                        double* energy_sum, double* partials, unsigned* counter, cudaStream_t st);

// CSR lower triangle K^(s): row counts, then fill (row_ptr from a scan).
void launch_lower_row_counts(const Dims& d, int32_t* counts, cudaStream_t st);
// Ke_dev: the element matrix [D*D] in device memory (dynamic indices).
void launch_lower_fill_dev(const Dims& d, const double* Ke_dev, const double* E,
                           const int32_t* row_ptr, int32_t* col, double* val, cudaStream_t st);
// Exclusive scan of n int32 counts into out[n+1] (out[n] = total), int64 total
// to *total_dev. Uses tmp of at least scan_tmp_size(n) bytes.
size_t scan_tmp_size(long long n);
void launch_exclusive_scan(const int32_t* counts, int32_t* out, long long n, void* tmp,
                           long long* total_dev, cudaStream_t st);

// ---- design kernels (kernels_design.cu) ----
template <typename T>
void launch_modulus(long long n, const double* x, double penal, double E0, double Emin, T* E,
                    cudaStream_t st);

// Forward filter out = (A in) / Hs (dprj == nullptr) or chain rule
// out = A (dprj * in / Hs), with the division as a product with rHs = 1/Hs
// (the array, or rHs_const where it is nullptr). If passive_keep != nullptr
// (forward only), passive elements take the value of `keep` instead
// (xPhys(act) = xTilde(act)).
// The shared-memory tile kernel (kernels_filter.cu) does it when its tile fits
// shared memory, in FP64 or (float_float) in float-float arithmetic; otherwise
// one thread per element gathers its taps from global memory in FP64.
void launch_filter(const Dims& d, const FilterTaps& taps, char bc, const double* rHs, double rHs_const,
                   const double* in, const double* dprj, double* out, const int8_t* passive,
                   const double* keep, cudaStream_t st, bool float_float = false);
// The tile kernel alone; false (nothing launched) when its tile does not fit.
bool launch_filter_tiled(const Dims& d, const FilterTaps& t, char bc, const double* rHs, double rHs_const,
                         const double* in, const double* dprj, double* out, const int8_t* passive,
                         const double* keep, bool float_float, cudaStream_t st);

struct ProjectOut {
    double eta;
    int newton;
    int status;
};
// Cooperative: eta Newton/bisection (if vp) then xphys = prj, dprj.
void launch_project(long long n, const double* xt, double* xphys, double* dprj, double beta,
                    double eta0, double volfrac, int vp, double tol, int maxit, long long deadline,
                    double* partials, GridBarrier* bar, ProjectOut* out, int nblocks, cudaStream_t st);
int project_max_blocks();

struct OcOut {
    double lm;
    int steps;
    int status;
};

// Device state of the OC search with the volume taken on the physical field of
// each candidate (launch_oc_filtered): bracket, the candidate's lm and phase
// (0 growing the bracket, 1 bisecting, 2 done, 3 nothing to do).
struct OcfState {
    double l1, l2, lmid;
    int phase, grows, steps, status;
};

// OC update whose bisection tests mean(prj(filter(x(lm)))) > volfrac (Sec. 3.2,
// the general variant for a fixed threshold eta; projection only when ft > 1;
// passive elements 1 / 0 after filtering; eta from eta_dev when non-null, e.g.
// the eta* of the same design iteration). Each step is three launches
// (candidate, forward filter, projected volume with the bracket update in the
// last block); the host checks the phase every four steps. xc, xf: [nEl]
// scratch; on return x holds the last candidate and out the last lm.
void launch_oc_filtered(const Dims& d, const FilterTaps& taps, char bc, const double* rHs, double rHs_const,
                        double* x, const double* dc, const double* dV0, const int8_t* passive, long long nact,
                        double move, double volfrac, int ft, double eta, const double* eta_dev, double beta,
                        double tol, int maxit, double* ocp, double* xc, double* xf, OcfState* sdev,
                        OcfState* shost, double* partials, unsigned* counter, OcOut* out, cudaStream_t st);
// Cooperative OC update: bisection with 15 candidates per pass (TO_OC_BISECTION)
// or the explicit primal-dual iteration of Appendix A (TO_OC_PRIMAL_DUAL).
void launch_oc(long long n, double* x, const double* dc, const double* dV0, const int8_t* passive,
               long long nact, double move, double volfrac, double tol, int maxit, long long deadline,
               double* ocp, double* partials, GridBarrier* bar, OcOut* out, int nblocks,
               cudaStream_t st, int method = TO_OC_BISECTION);
int oc_max_blocks();

// Deterministic dot products / norms: out[0] = sum a*b (b == nullptr: sum a*a).
void launch_dot(long long n, const double* a, const double* b, double* out, double* partials,
                unsigned* counter, cudaStream_t st);
// out[0] = sum (a-b)^2, out[1] = sum a; also copies a into b when copy != 0.
void launch_change(long long n, const double* a, double* b, double* out, int copy,
                   double* partials, unsigned* counter, cudaStream_t st);
void launch_fill(long long n, double* a, double v, cudaStream_t st);
// out = 1 / in
void launch_recip(long long n, const double* in, double* out, cudaStream_t st);
void launch_dv(long long n, const int8_t* passive, double v, double* dV, cudaStream_t st);

// ---- PCG vector kernels (kernels_design.cu) ----
// r = mask ? 0 : b - Ax ; z = dinv r ; p = z ; rz, rr, bb. x masked to 0 at fixed DOFs.
void launch_pcg_init(long long n, const double* b, const double* Ax, double* x, double* r,
                     double* z, double* p, const double* dinv, const uint8_t* fixed,
                     PcgScalars* s, double* partials, unsigned* counter, cudaStream_t st);
void launch_pcg_update(long long n, double* x, double* r, double* z, const double* p,
                       const double* Ap, const double* dinv, PcgScalars* s, double* partials,
                       unsigned* counter, cudaStream_t st);
void launch_pcg_dir(long long n, const double* z, double* p, const PcgScalars* s, cudaStream_t st);
void launch_mask_copy(long long n, const double* in, double* out, const uint8_t* fixed,
                      cudaStream_t st);

}  // namespace topo
