// Geometric multigrid preconditioner for K(xPhys)(free, free) on the
// structured grid (the multigrid-preconditioned CG that the paper uses for its
// 3D timings, Sec. 4 and Table 4, designed here from the textbook method).
//
// Level 0 is the design grid, applied matrix-free from E and Ke. Each coarser
// level halves every axis; its operator is the Galerkin product P^T K P with
// trilinear (bilinear) prolongation P masked at the fine Dirichlet DOFs, formed
// element by element (Kc = sum over the 8 (4) children of P_j^T K_j P_j, which
// equals P^T K P exactly) and stored as a node stencil for application. The
// coarsest level is solved with a dense inverse (factored in FP64, stored in the solve's
// precision) when small enough, else smoothed. Smoother: damped Jacobi, nu pre and nu post sweeps, so
// the V-cycle is a symmetric positive definite operator usable inside CG.
#pragma once

#include <vector>

#include "kernels.h"

struct to_grid;

namespace topo {

template <typename T>
struct MGLevel {
    Dims d{};
    T* S = nullptr;         // stencil, SoA [NS * dim * dim][nnodes] (coarse levels)
    T* R = nullptr;         // row sums of the stencil blocks [dim * dim][nnodes] (coarse levels)
    T* Kel = nullptr;       // element matrices [nel][D * D] (coarse levels)
    uint8_t* touched = nullptr;  // [nel] (coarse levels): a fine Dirichlet DOF lies under the element
    T* dinv = nullptr;      // Jacobi inverse diagonal [ndof]
    uint8_t* fixed = nullptr;  // [ndof]; level 0: the problem's; coarse: zero-diagonal DOFs
    T *r = nullptr, *z = nullptr, *t = nullptr, *w = nullptr;  // [ndof] work vectors
};

template <typename T>
struct MG {
    int nlev = 0;
    int nu = 2;
    int nu_fine = 0;        // sweeps on level 0 when > 0 (else nu)
    T omega = T(0.6);       // l1-Jacobi weight on the finest level
    T omega_c = T(0.6);     // and on the coarser ones
    int nc = 0;             // coarsest DOFs (dense inverse) or 0 (smoothing only)
    std::vector<MGLevel<T>> lev;
    double* A = nullptr;    // coarsest dense matrix and its Cholesky factor [nc * nc], FP64
    T* Ainv = nullptr;      // its inverse [nc * nc], in the solve's precision
    double* A_work = nullptr;  // column workspace of the inverse [nc * nc]
    double* Dblk = nullptr;    // inverses of the factor's diagonal blocks
    // FP32 hierarchy: the same matrix factored in FP32 first (the FP64 branch runs
    // only where that factorization lost four digits at a pivot)
    float *A32 = nullptr, *A32_work = nullptr, *Dblk32 = nullptr;
    T* Cj = nullptr;        // P_j^T Ke P_j of the 2^dim children of a coarse element
    int* status = nullptr;  // device [2]: the FP32 factorization lost four digits at a pivot (FP64
                            // branch taken); the FP64 factorization floored a pivot
    const T* E = nullptr;   // fine modulus of the current set-up
    int coarse_every = 1;   // rebuild the coarsest inverse at every k-th set-up
    long long setups = 0;
    // the coarsest factorization runs on a stream of its own (one CTA for most
    // of it), so that other work on the set-up stream overlaps it
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, ready = nullptr;
    bool pending = false;   // ready has not been waited on yet
    bool fuse_up = true;    // 3D coarse levels: prolongation fused into the first post-sweep
    std::vector<void*> allocs;
};

// Allocate the hierarchy for the handle's grid (no numerical content yet).
template <typename T>
MG<T>* mg_create(to_grid* g, int max_levels, int nu, double omega);
template <typename T>
void mg_destroy(MG<T>* mg);
// Rebuild every level from the fine modulus E (type T) of the current design.
template <typename T>
void mg_setup(to_grid* g, MG<T>* mg, const T* E, cudaStream_t st);
// Make st wait for the coarsest factorization of the last set-up (before the
// first V-cycle after a set-up).
template <typename T>
void mg_wait_coarse(MG<T>* mg, cudaStream_t st);
// Enqueue one V-cycle z = M r on level 0; returns the buffer holding z. All
// launches are skipped while *skip != 0 (skip may be nullptr).
template <typename T>
// fuse_rz (optional): the last fine-level sweep also computes r.z and the PCG
// beta into it (*fused reports whether it could).
// first_done: the caller has already formed level 0's first damped Jacobi
// iterate lev[0].z = omega lev[0].dinv r.
T* mg_vcycle(to_grid* g, MG<T>* mg, const T* r, const int* skip, cudaStream_t st, PcgScalars* fuse_rz = nullptr,
             bool* fused = nullptr, bool first_done = false);

// Fine-level operator kernels (matrix-free), shared with the Krylov solvers:
// mode 0: out = K u (masked); 1: out = u + omega dinv (r - K u); 2: out = r - K u.
// If pcg != nullptr (mode 0): fused p.Ap in FP64 and alpha = rz / pAp.
template <typename T>
void launch_fine_op(const to_grid* g, int mode, const T* E, const T* u, const T* r, const T* dinv,
                    T* out, T omega, const int* skip, PcgScalars* pcg, cudaStream_t st);

}  // namespace topo
