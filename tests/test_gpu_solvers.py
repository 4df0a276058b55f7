"""State solves of every precision x preconditioner pair against the oracle.

FP64 Jacobi / GMG PCG and the mixed FP32-inner / FP64-refinement solves must
reach ||F - K U|| <= cg_rtol ||F|| measured in FP64, and agree with the
oracle's banded-Cholesky solution to the accuracy that residual implies.
"""
import math

import numpy as np
import pytest

from oracle import topopt_oracle as O
from paper_2005_05436_gb300 import inputs as I
from tests._util import design_field, make_grid, rel, to_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COMBOS = [("fp64", "jacobi"), ("fp64", "gmg"), ("mixed", "jacobi"), ("mixed", "gmg")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


def _kw(precision, precond, **kw):
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED, TO_PC_GMG, TO_PC_JACOBI
    kw["precision"] = TO_MIXED if precision == "mixed" else TO_FP64
    kw["precond"] = TO_PC_GMG if precond == "gmg" else TO_PC_JACOBI
    return kw


@pytest.mark.parametrize("precision,precond", COMBOS)
@pytest.mark.parametrize("shape", [(60, 20, 0), (64, 32, 0), (24, 12, 12), (16, 8, 8), (13, 7, 5), (67, 23, 0)])
def test_solve_matches_direct(shape, precision, precond):
    # 1e-8 (the state-solve bar): on some designs even the oracle's Cholesky
    # solution only attains an FP64 residual of ~5e-9
    rtol = 1e-8
    g, F, fixed = make_grid(shape, **_kw(precision, precond, penal=3.0, cg_rtol=rtol, cg_maxit=100000))
    og = O.Grid(*shape)
    Ke = O.element_stiffness(og.dim)
    xp = design_field(shape, 12, lo=0.02)
    Ud = O.solve_direct(og, Ke, O.simp_modulus(xp, 3.0), F, fixed)
    U = torch.zeros(g.ndof, dtype=torch.float64, device="cuda")
    info = g.solve(to_cuda(xp), U)
    assert info.rel_res <= rtol, (info.rel_res, info.iters, info.refinements)
    Ug = U.cpu().numpy()
    assert rel(Ug, Ud) <= 1e-5
    assert abs(F @ Ug - F @ Ud) <= 1e-6 * abs(F @ Ud)
    if precision == "mixed":
        assert info.refinements >= 1


@pytest.mark.parametrize("precond", ["jacobi", "gmg"])
@pytest.mark.parametrize("shape", [(24, 12, 12), (16, 8, 8), (13, 7, 5), (31, 17, 46)])
def test_mixed_solve_on_tensor_cores_matches_direct(shape, precond):
    """The mixed solve with its FP32 fine operator on tensor cores (ku_impl 2:
    K p with p.Ap, the last smoothing sweep with r.z and the residual, all as
    TF32 MMAs) reaches the FP64 residual and the oracle's direct solution as the
    CUDA-core operator does."""
    rtol = 1e-8
    g, F, fixed = make_grid(shape, **_kw("mixed", precond, penal=3.0, cg_rtol=rtol, cg_maxit=100000, ku_impl=2))
    og = O.Grid(*shape)
    Ke = O.element_stiffness(og.dim)
    xp = design_field(shape, 12, lo=0.02)
    Ud = O.solve_direct(og, Ke, O.simp_modulus(xp, 3.0), F, fixed)
    U = torch.zeros(g.ndof, dtype=torch.float64, device="cuda")
    info = g.solve(to_cuda(xp), U)
    assert info.rel_res <= rtol, (info.rel_res, info.iters, info.refinements)
    Ug = U.cpu().numpy()
    assert rel(Ug, Ud) <= 1e-5
    assert abs(F @ Ug - F @ Ud) <= 1e-6 * abs(F @ Ud)
    assert info.refinements >= 1


@pytest.mark.parametrize("precision,precond", COMBOS)
def test_solve_full_size_cantilever(precision, precond):
    """96x48x48 cantilever at rtol 1e-8 (FP64 residual); all four solvers agree on c."""
    shape = (96, 48, 48)
    g, F, fixed = make_grid(shape, **_kw(precision, precond, penal=3.0, cg_rtol=1e-8, cg_maxit=50000))
    x = design_field(shape, 4, lo=0.02)
    U = torch.zeros(g.ndof, dtype=torch.float64, device="cuda")
    info = g.solve(to_cuda(x), U)
    assert info.rel_res <= 1e-8
    c = float(np.dot(F, U.cpu().numpy()))
    _full_c.setdefault("c", []).append((precision, precond, c, info.iters))
    ref = _full_c["c"][0][2]
    assert abs(c - ref) <= 1e-6 * abs(ref), _full_c["c"]
    if precond == "gmg":
        # homogeneous initial design (x = 0.12): multigrid needs few iterations
        U.zero_()
        info = g.solve(to_cuda(np.full(g.nel, 0.12)), U)
        assert info.rel_res <= 1e-8 and info.iters < 80, (info.iters, info.refinements)


_full_c = {}


@pytest.mark.parametrize("precond", ["gmg"])
def test_design_iterations_parity_gmg(precond):
    """20 design iterations of the 12x6x6 cantilever with FP64 GMG-PCG vs the oracle."""
    from tests.test_gpu_parity import _run_parity
    _run_parity((12, 6, 6), 20, **_kw("fp64", precond, volfrac=0.12, penal=3.0, rmin=math.sqrt(3),
                                      beta=2.0, newton_tol=1e-14, oc_tol=1e-15, cg_rtol=1e-12,
                                      cg_maxit=100000))


def test_mixed_design_loop_tracks_fp64():
    """20 iterations of the 48x24x24 cantilever: mixed+GMG compliance within 1e-6 of FP64+GMG."""
    from paper_2005_05436_gb300.topopt import Design
    shape = (48, 24, 24)
    runs = {}
    for precision in ("fp64", "mixed"):
        g, F, fixed = make_grid(shape, **_kw(precision, "gmg", volfrac=0.12, penal=3.0, rmin=math.sqrt(3),
                                             beta=2.0, cg_rtol=1e-10, cg_maxit=50000, newton_tol=1e-12,
                                             oc_tol=1e-12))
        d = Design(g, to_cuda(I.initial_design(g.nel, 0.12)))
        runs[precision] = [d.step() for _ in range(20)]
    for a, b in zip(runs["fp64"], runs["mixed"]):
        assert abs(a["c"] - b["c"]) <= 1e-6 * abs(a["c"]), (a["loop"], a["c"], b["c"])
        assert b["rel_res"] <= 1e-10
