/*
 * topopt.h - C ABI of the GB300 (sm_103a) SIMP topology-optimisation hot path.
 *
 * The library computes one design iteration of minimum-compliance topology
 * optimisation on structured 2D Q4 / 3D H8 grids as defined by Ferrari &
 * Sigmund (2020), "A new generation 99 line Matlab code for compliance
 * topology optimization and its extension to 3D": density filter (Eq. 2),
 * Heaviside projection with volume-preserving threshold (Eq. 1, Sec. 3.2),
 * state solve K(xPhys) U = F (Eqs. 4-5) by preconditioned CG with a
 * matrix-free stiffness operator, compliance sensitivities (Eq. 6) and their
 * chain rule (Eq. 7), and the OC update with the lambda# bracket (Eqs. 13-14,
 * 17).
 *
 * Conventions (all entry points):
 *  - Every function returns a to_status; TO_OK is 0. On failure,
 *    to_last_error() returns a thread-local message. Nothing throws or aborts
 *    across the ABI.
 *  - Array arguments are caller-owned DEVICE pointers (e.g. torch CUDA tensors)
 *    unless the comment says "host". The library never frees caller memory.
 *  - Work is enqueued on the stream given to to_init_grid (NULL = the legacy
 *    default stream). Entry points that return host scalars (pointers marked
 *    "host out") synchronise that stream before returning; the others are
 *    asynchronous. Inside to_step and to_solve the handle also uses private
 *    streams: the learned warm start forks from that stream and is joined
 *    back before the call's later work; the coarsest multigrid factorization
 *    touches only buffers of the handle and is joined before the first
 *    V-cycle (or the next set-up) that uses it, and by to_destroy.
 *  - Layouts follow the paper's column-major numbering (Sec. 3, PRE.2),
 *    0-based: node n = iy + (nely+1)(iz + (nelz+1) ix), element
 *    e = iy + nely (iz + nelz ix), DOF = dim*n + c with c = 0 (X, along ix),
 *    1 (Y, up = -iy), 2 (Z, along iz). 2D grids use nelz = 0.
 *  - FP64 arrays are float64 (double), masks uint8 / int8.
 *  - Caller arrays must not overlap unless a comment allows in-place use.
 */
#ifndef TOPOPT_H
#define TOPOPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum to_status {
    TO_OK = 0,
    TO_EINVAL = 1,    /* bad argument (sizes, NULL pointer, parameter range) */
    TO_ENOMEM = 2,    /* device allocation failed */
    TO_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    TO_ENOTCONV = 4,  /* an iteration hit its cap before its tolerance */
    TO_ENAN = 5,      /* a NaN or Inf appeared in a residual or a reduction */
    TO_ETIMEOUT = 6   /* a device-side wait passed its clock deadline */
} to_status;

enum { TO_FP64 = 0, TO_MIXED = 1 };                        /* to_params.precision */
enum { TO_PC_JACOBI = 0, TO_PC_GMG = 1 };                  /* to_params.precond */
enum { TO_CNT_ADD = 0, TO_CNT_MUL = 1 };                   /* to_continuation.kind */
enum { TO_OC_BISECTION = 0, TO_OC_PRIMAL_DUAL = 1, TO_OC_PHYSICAL_VOLUME = 2 };  /* to_params.oc_method */
enum { TO_REFINE_RELIABLE = 0, TO_REFINE_FLEXIBLE = 1 };   /* to_params.refine */

/* Continuation parCont = {istart, maxPar, isteps, deltaPar} (Sec. 3): after the
 * OC update of iteration `loop` (1-based), if loop >= istart, par < maxpar and
 * loop % isteps == 0, then par += delta (TO_CNT_ADD, the paper) or
 * par = min(maxpar, par * delta) (TO_CNT_MUL). */
typedef struct to_continuation {
    int32_t istart;
    int32_t isteps;
    double maxpar;
    double delta;
    int32_t kind;
    int32_t _pad;
} to_continuation;

/* Problem and solver parameters (the arguments of top99neo / top3D125, Sec. 3,
 * plus the solver controls of the GPU path). Fill with to_params_init. */
typedef struct to_params {
    int32_t dim;            /* 2 or 3 */
    int32_t nelx, nely, nelz;  /* elements per axis; nelz = 0 for 2D */
    double E0, Emin, nu;    /* Eq. (5) moduli and Poisson ratio (1, 1e-9, 0.3) */
    double volfrac;         /* volume fraction f of Eq. (3) */
    double penal;           /* SIMP exponent p of Eq. (5), initial value */
    double rmin;            /* filter radius of Eq. (2) */
    int32_t ft;             /* 1: filter; 2: + projection, fixed eta; 3: + volume-preserving eta */
    int32_t ftBC;           /* 'N' mirror (zero-Neumann) or 'D' zero padding */
    double eta, beta;       /* projection threshold (initial) and sharpness (initial) */
    double move;            /* OC move limit mu */
    to_continuation penal_cnt, beta_cnt;
    double newton_tol;      /* |mean(prj) - volfrac| stop of the eta Newton (paper: 1e-6) */
    int32_t newton_maxit;   /* Newton cap before the bisection fallback (50) */
    int32_t oc_maxit;       /* lambda bisection cap (200) */
    double oc_tol;          /* (l2-l1)/(l1+l2) stop of the bisection (paper: 1e-4) */
    double cg_rtol;         /* ||F - K U|| / ||F|| stop of the state solve (1e-8) */
    int32_t cg_maxit;       /* PCG iteration cap */
    int32_t precision;      /* TO_FP64 or TO_MIXED */
    int32_t precond;        /* TO_PC_JACOBI or TO_PC_GMG */
    int32_t mg_levels;      /* GMG levels incl. the fine grid, 0 = automatic */
    int64_t deadline_cycles;/* clock64 limit of every device-side wait (2e9) */
    double inner_rtol;      /* TO_MIXED: relative tolerance of each FP32 inner solve (1e-3); with
                               TO_REFINE_RELIABLE the drop of each PCG segment, or the smaller
                               drop 0.3 cg_rtol / (current FP64 residual) that still reaches
                               cg_rtol, when that is larger */
    double mg_omega;        /* GMG l1-Jacobi smoother weight (1.8): every level smooths with the l1
                               row sums, which bound the spectrum of D_l1^-1 K by 1, so the V-cycle
                               stays symmetric positive definite for any weight in (0, 2); 1.8 took
                               18 % fewer PCG iterations than 1.0 on the 96x48x48 cantilever */
    int32_t mg_nu;          /* GMG pre- and post-smoothing sweeps per level (2) */
    int32_t ku_impl;        /* 3D stiffness operator: 0 auto (= 3);
                               1 node-centric gather with the dense 24x24 Ke (CUDA cores, FP32 and
                               FP64); 2 tensor cores for the FP32 fine operator of TO_MIXED (tcgen05
                               TF32 MMAs with split operands, element slabs streamed along x, A
                               operands read in place from the staged node planes; FP64
                               products as 3); 3 element tiles with
                               Ke factored in the Walsh basis of the element corners (CUDA cores,
                               FP32 and FP64); 4 as 3, with the FP32 products computed for two
                               elements per thread in paired FP32 instructions (FP64 products as 3;
                               TO_EINVAL if no tile shape fits the grid) */
    int32_t loop_mode;      /* PCG loop: 0 one CUDA-graph launch with a conditional WHILE node
                               (default); 1 the same kernels launched from a host loop, polled
                               every 8 iterations (for profilers that do not follow
                               device-side graph iterations) */
    int32_t mg_coarse_every;/* GMG: rebuild the coarsest dense inverse at every k-th set-up (1: every
                               set-up); an older inverse keeps the V-cycle symmetric positive
                               definite, so only the iteration count can change */
    int32_t oc_method;      /* OC multiplier search: TO_OC_BISECTION (Sec. 3, Eq. 17 bracket, oc_tol,
                               oc_maxit) or TO_OC_PRIMAL_DUAL (Appendix A: closed-form dual map
                               iterated from lambda# until two iterates of sqrt(lambda) differ by
                               at most 1e-10; oc_maxit caps it), both solving mean(x_new) = volfrac;
                               or TO_OC_PHYSICAL_VOLUME (Sec. 3.2, the general variant for a fixed
                               threshold: each bisection candidate is filtered, its passive
                               elements set to 1 / 0 and, for ft > 1, projected with the current
                               eta and beta, and the bisection solves mean of that field =
                               volfrac; oc_tol, oc_maxit). */
    int32_t pae_q0;         /* periodic Anderson extrapolation of the OC iteration (Sec. 3.6) from
                               loop pae_q0 on; 0: off */
    int32_t pae_q;          /* extrapolate when (loop - pae_q0 + 1) is a multiple of pae_q (4) */
    int32_t pae_m;          /* history columns m_r, 1..4 (4) */
    double pae_alpha;       /* damping of the other steps, x += alpha r (0.9) */
    double pae_zeta;        /* damping of the extrapolated step (1) */
    int32_t inner_maxit;    /* TO_MIXED (to_step, to_solve and the batched solve): iteration cap of
                               each FP32 inner solve (2000; the batched solve caps at 1000 with
                               Jacobi and 200 with GMG as well); a stalled inner solve hands its
                               iterate to the FP64 flexible-CG step, whose exact line search still
                               lowers the energy. >= 1, else TO_EINVAL */
    int32_t refine;         /* TO_MIXED, single grid: how the FP64 residual corrects the FP32 solve.
                               In both schemes the FP32 PCG (vectors, operator, preconditioner in
                               FP32) accumulates its iterate in FP64.
                               TO_REFINE_RELIABLE (default): one FP32 PCG whose residual is
                               replaced by the true FP64 residual b - K U (FP64 U += FP32
                               correction) each time it has fallen by inner_rtol; the search
                               direction is kept across the replacement (the Krylov space is not
                               restarted) while the true residual fell at least a quarter as far
                               as the recursive one, else the next segment restarts from the true
                               residual; if a segment reaches min(inner_maxit, 400) iterations,
                               or 16 + 4 times the first segment's iterations per decade of drop,
                               or a replacement does not halve the FP64 residual, the solve
                               continues as TO_REFINE_FLEXIBLE. TO_REFINE_FLEXIBLE: FP32 inner
                               solves to inner_rtol from scratch, each followed by one FP64
                               flexible-CG step (exact line search). If either ends in a
                               non-finite value, or at 60 refinements with cg_maxit not reached,
                               the FP64 PCG finishes the solve (to_solve_info.fallback). */
    int32_t mg_unfused;     /* GMG, 3D coarse levels of at most 16,384 nodes: 0 prolongation fused
                               into the first post-smoothing sweep (default); 1 separate kernels
                               (same arithmetic and order, for comparison) */
    int32_t pdl_off;        /* 0 (default): the kernels of a PCG iteration are launched with
                               programmatic dependent launch, so that each grid is scheduled while
                               its predecessor runs and waits for it before reading memory (same
                               arithmetic and order); 1: plain stream-ordered launches */
    int32_t mg_nu_fine;     /* GMG: pre- and post-smoothing sweeps on the finest level; 0 (default):
                               mg_nu, like the coarser levels; 1..16 otherwise, else TO_EINVAL */
    int32_t _pad5;
    double mg_omega_coarse; /* GMG: l1-Jacobi weight on the levels below the finest; 0 (default):
                               mg_omega; else in (0, 2), else TO_EINVAL */
} to_params;

typedef struct to_grid to_grid;  /* opaque handle: workspaces, filter weights, graphs */

/* Result of one state solve. */
typedef struct to_solve_info {
    int32_t iters;          /* PCG iterations (inner iterations in TO_MIXED) */
    int32_t refinements;    /* outer FP64 refinement steps (TO_MIXED), else 0 */
    double rel_res;         /* ||F - K U||_2 / ||F||_2 in FP64 at exit */
    int32_t status;         /* to_status of the solve */
    int32_t fallback;       /* TO_MIXED: 1 if the FP32 iteration failed (a non-finite value, or
                               the refinement cap with cg_maxit not reached) and the FP64 PCG
                               finished the solve (iters counts both), else 0 */
    double t_setup_ms;      /* preconditioner set-up (CUDA events) */
    double t_krylov_ms;     /* PCG iterations (the inner FP32 solves in TO_MIXED) */
    double t_resid_ms;      /* FP64 true residuals and refinement updates */
} to_solve_info;

/* Design state advanced by to_step. Device pointers are caller-owned, FP64:
 * x[nEl] design variables, xPhys[nEl] physical densities, xOld[nEl] previous
 * xPhys (ch measure), U[nDof] displacements (warm start in, solution out).
 * Host scalars eta, penal, beta and loop are read and updated. */
typedef struct to_state {
    double* x;
    double* xPhys;
    double* xOld;
    double* U;
    double eta, penal, beta;
    int32_t loop;
    int32_t _pad;
} to_state;

/* Per-iteration record (the listing's log line: It, C, V, ch, penal, beta,
 * eta, lm) plus solver and timing counters. */
typedef struct to_iter_info {
    int32_t loop;
    int32_t n_cg;           /* PCG iterations of the state solve */
    int32_t n_refine;       /* FP64 refinement steps (TO_MIXED) */
    int32_t n_newton;       /* eta Newton steps */
    int32_t n_bisect;       /* lambda bisection steps */
    int32_t status;
    double c;               /* compliance F^T U (Eq. 3) */
    double V;               /* mean(xPhys) */
    double ch;              /* ||xPhys - xOld||_2 / sqrt(nEl) */
    double penal, beta, eta, lm;
    double rel_res;         /* final FP64 relative residual of the solve */
    double t_filter_ms, t_solve_ms, t_sens_ms, t_oc_ms;  /* CUDA-event phase times */
    double t_setup_ms, t_krylov_ms, t_resid_ms;          /* split of t_solve_ms */
    double t_warm_ms;       /* learned warm start (inside t_solve_ms), 0 without a network */
    double warm_a, warm_b;  /* its starting point: warm_a U_prev + warm_b U_net */
    double warm_err_prev;   /* energy-norm error of U_prev relative to that of U = 0: ||U_prev - U||_K^2 / ||U||_K^2 */
    double warm_err;        /* the same for the warm start actually used (<= warm_err_prev under
                               TO_WARM_ENERGY) */
    int32_t pae;            /* Anderson extrapolation of this step: 0 off, 1 damped step, 2 extrapolated */
    int32_t fallback;       /* to_solve_info.fallback of the state solve */
    double warm_res_prev;   /* ||F - K U_prev|| / ||F|| over the free DOFs (operator products in the
                               warm start's precision), 0 without a network */
    double warm_res;        /* the same for the warm start actually used (<= warm_res_prev under
                               TO_WARM_RESIDUAL) */
} to_iter_info;

/* Thread-local message of the last failing call ("" if none). */
const char* to_last_error(void);

/* sizeof(to_params), sizeof(to_state), sizeof(to_iter_info) for binding checks. */
size_t to_sizeof_params(void);
size_t to_sizeof_state(void);
size_t to_sizeof_iter_info(void);

/* Defaults of the paper (Appendix B/C, PRE.1): E0 = 1, Emin = 1e-9, nu = 0.3,
 * volfrac 0.5, penal 3, rmin 1.5 (2D) / sqrt(3) (3D), ft = 3, 'N', eta 0.5,
 * beta 2, move 0.2, continuation penal {1, 25, 3, +0.25}, beta {1, 25, 2, +2};
 * Newton tol 1e-6, bisection tol 1e-4, PCG rtol 1e-8, FP64, Jacobi. p (host out). */
to_status to_params_init(to_params* p, int32_t dim, int32_t nelx, int32_t nely, int32_t nelz);

/* Create a grid handle (Sec. 3 PRE.1-PRE.6): validates p, copies the load F[nDof],
 * the fixed-DOF mask fixed[nDof] (1 = restrained, Appendix B/C PRE.3) and the
 * optional passive mask passive[nEl] (0 active, 1 solid P1, -1 void P0; NULL =
 * all active) into handle-owned device memory, builds Ke (Gauss quadrature of
 * the Q4 / H8 element, Appendix B/C), the filter window (Eq. 2) and the
 * normalisation Hs, and allocates the workspaces. `stream` is a cudaStream_t
 * (NULL = default stream). *out (host out) receives the handle. */
to_status to_init_grid(const to_params* p, const double* F, const uint8_t* fixed,
                       const int8_t* passive, void* stream, to_grid** out);

/* Free the handle and its device memory (NULL is a no-op). */
void to_destroy(to_grid* g);

/* Current continuation scalars (p of Eq. 5, beta of Eq. 1, eta) used by the
 * stand-alone entry points below. to_step keeps them in step. */
to_status to_set_scalars(to_grid* g, double penal, double beta, double eta);

/* Lower triangle K^(s) of the assembled K(xPhys) (Sec. 3.1, Eqs. 10-11) in CSR
 * with sorted column indices, duplicates summed, fixed DOFs kept.
 * nnz (host in/out): capacity of col/val in, number of entries out.
 * row_ptr[nDof+1], col[nnz] int32, val[nnz] FP64 device arrays. With val == NULL
 * only *nnz is computed. TO_EINVAL if the capacity is too small. */
to_status to_assemble_lower(to_grid* g, const double* xPhys, int64_t* nnz,
                            int32_t* row_ptr, int32_t* col, double* val);

/* Matrix-free y = K(xPhys) u (Eqs. 4-5): y = sum_e E_e Ke u_e with
 * E_e = Emin + xPhys_e^p (E0 - Emin). masked != 0: u at fixed DOFs is treated
 * as 0 and y at fixed DOFs is 0 (the operator K(free, free) padded with zeros).
 * u[nDof], y[nDof]; y must not alias u. */
to_status to_apply_K(to_grid* g, const double* xPhys, const double* u, double* y, int32_t masked);

/* State solve K(xPhys)(free, free) U = F (Eq. 4) by PCG (Jacobi or geometric
 * multigrid; TO_MIXED: FP32 inner solves with FP64 iterative refinement) to
 * ||F - K U|| <= cg_rtol ||F|| in FP64. F[nDof] (NULL = the handle's load),
 * U[nDof]: warm start in, solution out (0 at fixed DOFs). info (host out, may
 * be NULL). TO_ENOTCONV if cg_maxit is reached (U holds the last iterate). */
to_status to_solve(to_grid* g, const double* xPhys, const double* F, double* U,
                   to_solve_info* info);

/* Density filter (Eq. 2, reading: xTilde = (A x) / Hs with A the cone-weight
 * correlation under 'N' mirror or 'D' zero padding, Hs = A 1).
 * dprj == NULL: forward out = (A in) / Hs.
 * dprj != NULL: chain rule out = A^T (dprj * in / Hs) = H^T (dprj * in) (Eq. 7
 * in the exact order). in[nEl], out[nEl], dprj[nEl]; out must not alias in. */
to_status to_filter(to_grid* g, const double* in, double* out, const double* dprj);

/* Heaviside projection (Eq. 1) with its derivative (Eq. 8) at the handle's beta:
 * xPhys = prj(xTilde, eta), dprj = d prj / d xTilde. volume_preserving != 0:
 * first solve mean(prj(xTilde, eta)) = volfrac for eta by Newton from
 * *eta_inout (Sec. 3.2, Eq. 15), falling back to bisection on [0, 1].
 * eta_inout (host in/out). xTilde, xPhys, dprj [nEl]. */
to_status to_project(to_grid* g, const double* xTilde, double* xPhys, double* dprj,
                     double* eta_inout, int32_t volume_preserving);

/* Sensitivities (Eq. 6): dc_e = -p (E0 - Emin) xPhys_e^(p-1) u_e^T Ke u_e on
 * active elements, 0 on passive ones; c_out (host out, may be NULL) = F^T U
 * with the handle's F. xPhys[nEl], U[nDof], dc[nEl]. */
to_status to_sensitivity(to_grid* g, const double* xPhys, const double* U, double* dc,
                         double* c_out);

/* OC update (Eqs. 13-14) of the active design variables in place:
 * x <- clamp(x sqrt(max(0, -dc/dV0)) / lm, max(0, x - move), min(1, x + move)),
 * with lm = sqrt(lambda) found by bisection on [0, lambda#] (Eq. 17) until
 * (l2 - l1)/(l1 + l2) <= oc_tol, testing mean(x) > volfrac. The upper bracket
 * is doubled while it is still feasible-violating. x[nEl] in/out, dc, dV0 [nEl];
 * lm_out (host out, may be NULL). Returns TO_ENOTCONV, with x and lm_out
 * holding the last candidate, when the search stops at oc_maxit steps before
 * the bracket meets oc_tol. */
to_status to_oc_update(to_grid* g, double* x, const double* dc, const double* dV0,
                       double* lm_out);

/* One full design iteration (Sec. 3, RL.1-RL.4): filter, projection with
 * volume-preserving eta (ft = 3), ch, state solve (warm-started from s->U),
 * sensitivities, chain rule, OC update and continuation. s (host in/out,
 * device arrays inside), info (host out, may be NULL). The iteration is
 * completed in every case below and info->status repeats the return value:
 * TO_ENAN when the compliance is not finite, the solve's TO_ENOTCONV when it
 * stopped above cg_rtol, TO_ENOTCONV when the OC multiplier search stopped at
 * oc_maxit before meeting oc_tol, TO_ETIMEOUT when a grid-barrier wait passed
 * deadline_cycles (then s and info are not updated). */
to_status to_step(to_grid* g, to_state* s, to_iter_info* info);

/* OC update that allocates no device memory. The paper has no counterpart: this
 * entry exists for callers that cannot call cudaMalloc, for example a process
 * whose device memory is already reserved by another allocator (a framework's
 * caching pool, so cudaMalloc would fail), or a latency-critical loop that must
 * not take the implicit device synchronisation of cudaMalloc / cudaFree.
 * It computes exactly what to_oc_update computes, without a grid handle:
 * x[nel] (device, in/out) is updated from dc[nel], dV0[nel] and the optional
 * passive[nel] mask (device; NULL = all active) with the given volfrac, move,
 * oc_tol, oc_maxit and deadline_cycles, on `stream` (a cudaStream_t, NULL =
 * default stream); lm_out (host out, may be NULL) receives lm = sqrt(lambda).
 * Scratch: one file-scope device array of 8,651,520 bytes; it bounds nel to
 * 1,048,576 elements (larger nel returns TO_EINVAL). CUDA loads the module
 * that holds the array lazily, so the array is reserved on a device by the
 * first call there (or when the context is created, under
 * CUDA_MODULE_LOADING=EAGER) and held until the process exits; that first call
 * may also synchronise the device. Make one call early on each device, before
 * handing its free memory to another allocator and before any stream capture:
 * the first call also resolves the array's device address with that device
 * current and caches it. A cudaDeviceReset makes the cached address stale: do
 * not use this entry on a device after resetting it in the same process. The
 * array keeps the last call's contents; the call clears what must start at
 * zero. All calls share the array, so calls that overlap on the GPU (other
 * streams, other host threads) race: serialise them. The call synchronises
 * `stream` before returning. Apart from that first module load it calls no
 * cudaMalloc, cudaFree or allocating library routine. Errors: TO_EINVAL for
 * a NULL array, nel out of range, bad scalars or no active element;
 * TO_ETIMEOUT when a grid-barrier wait passed deadline_cycles; TO_ENOTCONV
 * as to_oc_update; each with a message in to_last_error(). */
to_status to_oc_update_noalloc(int64_t nel, double* x, const double* dc, const double* dV0,
                               const int8_t* passive, double volfrac, double move, double oc_tol,
                               int32_t oc_maxit, int64_t deadline_cycles, void* stream,
                               double* lm_out);

/* The FP32 stiffness operator of the TO_MIXED inner solve, y = K(xPhys) u
 * (masked as to_apply_K with masked = 1), for checking it against the FP64
 * one: u is rounded to FP32, the product runs as the node-centric dense-Ke
 * gather on CUDA cores (impl = 1), on tensor cores (impl = 2, tcgen05 TF32
 * with split operands, 3D only) or as Walsh-factored element tiles on CUDA
 * cores (impl = 3, 3D only) and y is returned widened to FP64. Needs a handle
 * created with TO_MIXED. u[nDof], y[nDof] device FP64. */
to_status to_apply_K_fp32(to_grid* g, const double* xPhys, const double* u, double* y, int32_t impl);

/* Instrumentation (no counterpart in the paper): number of kernels this library
 * has launched in this process; a CUDA-graph launch counts its kernel nodes. */
int64_t to_kernel_launches(void);

/* Instrumentation (no counterpart in the paper): average device time in
 * microseconds (us, host out) of one launch of the matrix-free K u kernel of
 * `precision` (TO_FP64 or TO_MIXED) at E(xPhys), measured with CUDA events
 * around `reps` back-to-back launches on the handle's stream, in the launch
 * configuration the solver uses. */
to_status to_time_apply_K(to_grid* g, const double* xPhys, int32_t precision, int32_t reps, double* us);

/* Instrumentation (no counterpart in the paper): cost of the tensor-core
 * instruction the FP32 operator of ku_impl 2 is built from. On every SM,
 * blocks_per_sm (1, 2 or 4) blocks each run `issuers` (1..8) threads that
 * issue `reps` tcgen05.mma kind::tf32 of shape m x n x 8 (m 64 or 128; n 8..256,
 * a multiple of 16 for m = 128; issuers x n <= 512 / blocks_per_sm) into
 * their own tensor-memory accumulators from zero-filled shared memory.
 * cycles (host out): clock64 cycles per MMA seen by one issuing thread, from
 * its first issue to the completion of its last; mac_per_cycle (host out):
 * multiply-adds per cycle of one SM. Runs on the current device's default
 * stream and waits for it; allocates and frees its own scratch. TO_EINVAL on other arguments, TO_ETIMEOUT if a
 * completion wait passes its limit. */
to_status to_time_tf32_mma(int32_t m, int32_t n, int32_t issuers, int32_t blocks_per_sm, int32_t reps,
                           double* cycles, double* mac_per_cycle);

/* ------------------------------------------------------------------------
 * Batched uneven 2D instances (no counterpart in the paper, which solves one
 * problem at a time). Each instance is an independent 2D Q4 problem of Sec. 3
 * with its own grid, volume fraction, filter radius, loads and supports; all
 * share the material, the projection/continuation settings and the solver
 * controls of a base to_params. One to_batch_step advances every instance by
 * one design iteration (RL.1-RL.4: filter, eta Newton and projection, state
 * solve, sensitivities, back-filter, OC, continuation) with ONE CUDA-graph
 * launch. Inside it each kernel covers all instances through a table of
 * element or node tiles (a tile never straddles two instances); per-instance
 * sums are reduced by the last tile of the instance in tile order, so results
 * do not depend on scheduling; the eta Newton, the FP64 refinement with its
 * FP32 inner Jacobi-PCG, and the lambda bisection run as conditional WHILE
 * nodes until every instance has met its own stopping test.
 *
 * Layout: instance k's elements occupy [el_off[k], el_off[k+1]) of every
 * element array, in the paper's column-major order (e = iy + nely ix); its DOFs
 * occupy [dof_off[k], dof_off[k+1]) of every DOF array (DOF 2 n + c,
 * n = iy + (nely + 1) ix). Offsets: to_batch_offsets.
 * ------------------------------------------------------------------------ */

typedef struct to_instance {
    int32_t nelx, nely;     /* Q4 elements per axis (>= 1) */
    double volfrac;         /* volume fraction of this instance, in (0, 1) */
    double rmin;            /* filter radius of this instance (> 0), 'N' padding */
} to_instance;

typedef struct to_batch to_batch;  /* opaque: instance table, tiles, workspaces, graph */

/* Element-tile shape search (to_batch_autotune): candidate k is a tile of
 * cand_ty[k] rows (along y, the fast index) x cand_tx[k] columns, one thread
 * per node (node kernels) or element (element kernels). */
typedef struct to_tile_info {
    int32_t node_ty, node_tx;   /* chosen node-tile shape */
    int32_t elem_ty, elem_tx;   /* chosen element-tile shape */
    int32_t n_candidates;
    int32_t cand_ty[8], cand_tx[8];
    double node_us[8];          /* batched FP32 K u, microseconds per launch */
    double elem_us[8];          /* batched forward filter, microseconds per launch */
} to_tile_info;

/* Record of one batched design iteration. */
typedef struct to_batch_info {
    int32_t loop;               /* design iteration counter after the step (1-based) */
    int32_t status;             /* TO_OK, or TO_ENOTCONV when an instance stopped above cg_rtol
                                   (refinement cap, or stalled) */
    int32_t max_refinements;    /* max over instances of the FP64 refinement steps */
    int32_t max_inner_iters;    /* max over instances of the inner PCG iterations (all refinements) */
    int32_t newton_passes;      /* lockstep passes of the eta loop (all instances) */
    int32_t inner_passes;       /* lockstep passes of the inner PCG loop */
    int32_t oc_passes;          /* lockstep passes of the lambda loop */
    int32_t stalled;            /* instances whose FP64 residual did not halve over 10 refinements
                                   and stopped there above cg_rtol (status TO_ENOTCONV; their
                                   rel_res in to_batch_results) */
    double max_rel_res;         /* max over instances of ||F - K U|| / ||F|| (FP64) at exit */
    double penal, beta;         /* after the continuation of this iteration */
    double ms;                  /* device time of the graph launch (CUDA events) */
    int64_t kernels;            /* kernels executed by the graph launch */
} to_batch_info;

/* Creates the batch. base: dim 2, precision TO_MIXED, ftBC 'N'; its nelx,
 * nely, volfrac and rmin are ignored (per instance instead). inst: host array
 * [count]. F, fixed: device arrays over the concatenated DOFs (F FP64, fixed
 * 1 = Dirichlet DOF), read at every step (caller-owned, must stay valid).
 * stream: cudaStream_t or NULL. Initial state: eta = base eta, penal and beta
 * the base values, loop 0; tile shapes 32 x 4 until to_batch_autotune.
 * TO_EINVAL on bad arguments; TO_ENOMEM. */
to_status to_batch_init(const to_params* base, int32_t count, const to_instance* inst, const double* F,
                        const uint8_t* fixed, void* stream, to_batch** out);

/* Host arrays [count + 1] of element and DOF offsets (either may be NULL). */
to_status to_batch_offsets(const to_batch* b, int64_t* el_off, int64_t* dof_off);

/* Times every candidate tile shape on the batch (reps launches each of the
 * batched FP32 K u and forward filter at a uniform design), keeps the fastest
 * node and element shapes, and reports the timings in info (may be NULL). */
to_status to_batch_autotune(to_batch* b, int32_t reps, to_tile_info* info);

/* One design iteration of every instance. Device FP64 arrays over the
 * concatenated layout, caller-owned: x (in/out design variables), xPhys
 * (out), xOld (in/out previous xPhys, all ones before the first step), U
 * (in warm start / out displacements). The graph is captured on the first
 * call and re-captured when a pointer or the tile shapes change. */
to_status to_batch_step(to_batch* b, double* x, double* xPhys, double* xOld, double* U, to_batch_info* info);

/* Per-instance results of the last step into host arrays [count] (any may be
 * NULL): compliance c = F^T U, V = mean(xPhys), ch, eta, lm (the OC
 * multiplier sqrt(lambda)), inner PCG iterations, refinements, FP64 relative
 * residual. */
to_status to_batch_results(const to_batch* b, double* c, double* V, double* ch, double* eta, double* lm,
                           int32_t* inner_iters, int32_t* refinements, double* rel_res);

void to_batch_destroy(to_batch* b);

/* ------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper): a small 3D convolutional
 * encoder-decoder, trained on (xPhys, F, U) triples that the method itself
 * produces, predicts a displacement direction from the node density and the
 * load; the state solve then starts from its energy-optimal multiple (see
 * to_learned_warm_start). The converged relative residual is unchanged: only
 * the starting point, and so the iteration count, can differ.
 *
 * Network (levels 3, base channels c, 3x3x3 convolutions with zero padding,
 * 2x2x2 mean pooling, nearest 2x upsampling, additive skips):
 *   e0 = relu(conv(relu(conv(x, 4->c)), c->c))
 *   e1 = relu(conv(relu(conv(pool(e0), c->2c)), 2c->2c))
 *   e2 = relu(conv(relu(conv(pool(e1), 2c->4c)), 4c->4c))
 *   d1 = relu(conv(relu(conv(up(e2), 4c->2c)) + e1, 2c->2c))
 *   d0 = relu(conv(relu(conv(up(d1), 2c->c)) + e0, c->c))
 *   y  = conv(d0, c->3)
 * Tensors are device FP32 arrays [N][D][H][W][C] (channels last) with D, H, W
 * multiples of 4. Parameters: one flat FP32 vector, layer by layer
 * W[27][cin][cout] then b[cout], tap t = (dx+1)*9 + (dy+1)*3 + (dz+1).
 * ------------------------------------------------------------------------ */

typedef struct to_net to_net;

typedef struct to_net_cfg {
    int32_t base;   /* channels of the first level (16): a multiple of 4, at most 64 */
    int32_t bf16;   /* 1: activations and convolution weights in BF16 (products
                       accumulated in FP32); 0: FP32 throughout */
    int32_t in_ch;  /* 4: node density and the three load components */
    int32_t out_ch; /* 3: the displacement direction */
    int32_t cuda_cores_only; /* 0: tcgen05 tensor cores for the BF16 layers with 16, 32 or 64 input
                                and output channels (default); 1: every layer on CUDA cores */
    int32_t _pad;
} to_net_cfg;

/* Creates a network with all parameters 0 (set them with to_net_set_params). */
to_status to_net_create(const to_net_cfg* cfg, void* stream, to_net** out);
int64_t to_net_param_count(const to_net* net);
/* theta: device FP32 [to_net_param_count]; resets the Adam moments. */
to_status to_net_set_params(to_net* net, const float* theta);
to_status to_net_get_params(const to_net* net, float* theta);
/* y[N][D][H][W][3] = network(x[N][D][H][W][4]). */
to_status to_net_forward(to_net* net, const float* x, int32_t N, int32_t D, int32_t H, int32_t W, float* y);
/* Adds the gradient of L = mean over valid entries of (y - target)^2 (mask:
 * uint8 [N][D][H][W], 1 = valid voxel) to the internal gradient; loss (host
 * out, may be NULL) receives L. */
to_status to_net_accumulate(to_net* net, const float* x, const float* target, const uint8_t* mask, int32_t N,
                            int32_t D, int32_t H, int32_t W, double* loss);
/* Adds the gradient for an output gradient gy[N][D][H][W][3] (dL/dy), using
 * the activations of the last to_net_forward, which must have had this shape. */
to_status to_net_backward(to_net* net, const float* gy, int32_t N, int32_t D, int32_t H, int32_t W);
to_status to_net_get_grad(const to_net* net, float* grad);
to_status to_net_zero_grad(to_net* net);
/* One Adam step (bias-corrected) with gradient grad_scale * internal gradient;
 * the internal gradient is zeroed. */
to_status to_net_adam(to_net* net, double lr, double beta1, double beta2, double eps, double grad_scale);
void to_net_destroy(to_net* net);

/* Attaches a network to a 3D grid (NULL detaches; the grid does not own it):
 * every to_step then starts its state solve from the minimiser of the
 * potential energy 1/2 U^T K U - F^T U over span{U, U_net}, U the previous
 * solution and U_net the network's output on the step's xPhys (a 2 x 2
 * Rayleigh-Ritz step with operator products in the handle's precision; U is
 * kept when the network adds nothing). The solve still runs to cg_rtol.
 * stride (1 or 2): the network works on the node grid coarsened by stride
 * (coarse node I on fine node stride*I; loads restricted by full weighting,
 * the output prolongated trilinearly); fixed at the first use of the grid. */
to_status to_set_warm_start(to_grid* g, to_net* net, int32_t stride);

/* How the warm start combines U (the previous solution) and U_net:
 * TO_WARM_ENERGY (default): the minimiser of the potential energy over
 * span{U, U_net}, as above. TO_WARM_RESIDUAL: the minimiser of the residual
 * norm ||F - K (a U + b U_net)||_2 over the free DOFs, the norm of the solve's
 * stopping test, so the start's residual never exceeds that of U (five more
 * dot products). TO_EINVAL for other values. */
enum { TO_WARM_ENERGY = 0, TO_WARM_RESIDUAL = 1 };
to_status to_set_warm_start_rule(to_grid* g, int32_t rule);
/* Network input of the grid at xPhys: x[D][H][W][4] on the (coarsened) node
 * grid padded to multiples of 4 (D, H, W along x, z, y): the mean density of
 * the elements around each node (-1 at nodes with a Dirichlet DOF) and the
 * restricted load / max|F|; zero in the padding.
 * dims (host out [3], may be NULL) = D, H, W; x = NULL only queries dims. */
to_status to_learned_features(to_grid* g, const double* xPhys, float* x, int32_t* dims);
/* Training target for displacements U: t[D][H][W][3] = U / rms(U) at the
 * (coarse) nodes, 0 in the padding; mask[D][H][W] = 1 on nodes. */
to_status to_learned_target(to_grid* g, const double* U, float* t, uint8_t* mask);
/* Energy objective of one network output y[D][H][W][3] (the grid's padded node
 * layout) for the design xPhys whose converged compliance is c_star:
 * L = 1 - (F^T U_h)^2 / (U_h^T K U_h c_star), the relative energy-norm error
 * of the best multiple of U_h (U_h = y on the free DOFs; K at the grid's
 * current penal). loss (host out) = L, gy = dL/dy (FP32, same layout). */
to_status to_learned_energy_grad(to_grid* g, const double* xPhys, const float* y, double c_star, float* gy,
                                 double* loss);

/* Struct sizes, for bindings that mirror these layouts. */
size_t to_sizeof_net_cfg(void);
size_t to_sizeof_instance(void);
size_t to_sizeof_tile_info(void);
size_t to_sizeof_batch_info(void);

#ifdef __cplusplus
}
#endif

#endif /* TOPOPT_H */
