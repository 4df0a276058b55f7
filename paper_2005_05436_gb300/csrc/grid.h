// The opaque grid handle behind the C ABI.
#pragma once

#include <vector>

#include "kernels.h"

namespace topo {

// Device-resident scalars read back once per call.
struct DevScalars {
    ProjectOut po;
    OcOut oo;
    double change[2];  // sum (xPhys - xOld)^2, sum xPhys
    double c;          // F^T U
    double esum;       // sum E_e u_e^T Ke u_e
    long long nnz;
    PcgScalars pcg;
    double res[4];     // refinement norms
    OcfState ocf;      // OC search on the physical field
    int pae_ok;        // the Anderson least-squares system was regular
    int pad_;
};

struct Solver;  // solver.cu

// Unit-element stiffness by 2x2(x2) Gauss quadrature, row-major D x D (api.cu).
void element_matrix(int dim, double nu, std::vector<double>& K);
// Records msg as the thread's last error and returns s (api.cu).
to_status api_fail(to_status s, const std::string& msg);

}  // namespace topo

struct to_grid {
    to_params p;
    topo::Dims d;
    int dev = 0, nsm = 0;
    cudaStream_t ust = nullptr;  // caller's stream
    cudaStream_t st = nullptr;   // work stream: the caller's, or a private one for NULL
    bool own_stream = false;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t[5] = {};
    std::vector<void*> allocs;

    double penal = 3.0, beta = 2.0, eta = 0.5;

    // Ke in the constant bank (kernel parameters) and in device memory
    topo::KeP<double, 24> ke3{};
    topo::KeP<double, 8> ke2{};
    topo::KeP<float, 24> ke3f{};
    topo::KeP<float, 8> ke2f{};
    topo::WalshK<double> wk{};   // Ke in the Walsh basis (3D, walsh.cuh)
    topo::WalshK<float> wkf{};
    std::vector<double> Ke_host;
    double* Ke_dev = nullptr;

    // problem data
    double* F = nullptr;
    uint8_t* fixed = nullptr;
    int8_t* passive = nullptr;
    long long nact = 0, nsolid = 0, nvoid = 0;

    // filter
    topo::FilterTaps taps{};
    double Hs_const = 1.0;
    double* Hs = nullptr;  // 'D' only
    // 1/Hs, which the filters multiply by (an FP64 divide is a long sequence at the FP64 rate)
    double rHs_const = 1.0;
    double* rHs = nullptr;  // 'D' only

    // workspaces
    double *E = nullptr, *xt = nullptr, *dprj = nullptr, *dc = nullptr, *dcf = nullptr;
    double *dV = nullptr, *dV0 = nullptr, *ocp = nullptr;
    float* Ef = nullptr;
    double* v[7] = {};  // nDof vectors
    double* partials = nullptr;
    long long npartials = 0;
    unsigned* counter = nullptr;
    topo::GridBarrier* bar = nullptr;
    topo::GridBarrier hbar{};
    topo::DevScalars* ds = nullptr;
    topo::DevScalars* hs = nullptr;  // pinned mirror
    int proj_blocks = 0, oc_blocks = 0;
    void* scan_tmp = nullptr;  // CSR assembly scan workspace (lazy)
    float* ke_tc = nullptr;    // Ke packed as the tensor-core B operand (TO_MIXED, 3D)
    int* tc_err = nullptr;     // device error word of the tensor-core operator
    bool use_tc = false;       // the FP32 fine operator runs on tensor cores
    bool node_centric = false; // 3D K u by the node-centric dense-Ke kernels (ku_impl 1)
    bool walsh_pair = false;   // FP32 3D K u by the element-pair kernel (kernels_walsh_pair.cu)

    topo::Solver* solver = nullptr;
    to_net* net = nullptr;     // learned warm start (to_set_warm_start), not owned
    void* warm = nullptr;      // its workspace (warm.cu)
    int warm_stride = 1;       // the network's node-grid coarsening (1 or 2)
    int warm_rule = TO_WARM_ENERGY;  // how the warm start combines U_prev and U_net
    void* pae = nullptr;       // Anderson extrapolation history (pae.cu)
};

namespace topo {
// Ke kernel parameters of the handle in the arithmetic type T.
template <typename T>
inline const KeP<T, 24>& grid_ke3(const to_grid* g);
template <>
inline const KeP<double, 24>& grid_ke3<double>(const to_grid* g) { return g->ke3; }
template <>
inline const KeP<float, 24>& grid_ke3<float>(const to_grid* g) { return g->ke3f; }
template <typename T>
inline const WalshK<T>& grid_wk(const to_grid* g);
template <>
inline const WalshK<double>& grid_wk<double>(const to_grid* g) { return g->wk; }
template <>
inline const WalshK<float>& grid_wk<float>(const to_grid* g) { return g->wkf; }
template <typename T>
inline const KeP<T, 8>& grid_ke2(const to_grid* g);
template <>
inline const KeP<double, 8>& grid_ke2<double>(const to_grid* g) { return g->ke2; }
template <>
inline const KeP<float, 8>& grid_ke2<float>(const to_grid* g) { return g->ke2f; }

void grid_sync_in(to_grid* g);
void warm_free(to_grid* g);
// Periodic Anderson extrapolation (pae.cu): keep x before the OC step, then
// replace the OC output by the damped or extrapolated step (it = loop - q0);
// returns 1 (damped) or 2 (extrapolation attempted; DevScalars::pae_ok says
// whether it was taken). pae_free releases the history.
void pae_before_oc(to_grid* g, const double* x, cudaStream_t st);
int pae_after_oc(to_grid* g, double* x, int it, cudaStream_t st);
void pae_free(to_grid* g);
void learned_warm_start(to_grid* g, const double* xPhys, double* U, double* coef, double* ms, double* energy,
                        double* resid);
void grid_sync_out(to_grid* g);
void solver_init(to_grid* g);
void solver_free(to_grid* g);
// Solve K(E)(free, free) U = b with g->E already set; U: warm start in, solution out.
// Preconditioner set-up for the modulus in g->E on the grid stream; the next solve_state skips it.
void solver_setup(to_grid* g);
// Forget a set-up that no solve consumed (an entry point that failed after solver_setup).
void solver_discard_setup(to_grid* g);
to_status solve_state(to_grid* g, const double* b, double* U, to_solve_info* info);
// Tensor-core FP32 fine operator (ku_tc.cu); modes as launch_fine_op.
void launch_fine_op_tc(const to_grid* g, int mode, const float* E, const float* u, const float* r, const float* dinv,
                       float* out, float omega, const int* skip, PcgScalars* pcg, cudaStream_t st);
void tc_pack_ke(const std::vector<double>& Ke, std::vector<float>& pack);
// y = K(xPhys) u by the FP32 operator of the mixed path (impl 1 CUDA cores, 2 tensor cores).
void apply_K_fp32(to_grid* g, const double* xPhys, const double* u, double* y, int impl);
// Enqueue `reps` launches of the mixed-precision K u kernel between events e0, e1.
void time_apply_K_mixed(to_grid* g, const double* xPhys, int reps, cudaEvent_t e0, cudaEvent_t e1);
}  // namespace topo
