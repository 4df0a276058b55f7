"""Solver options that change how, not what, the state solve computes.

pdl_off: the PCG iteration's kernels launched with or without programmatic
dependent launch give bitwise the same solve (same arithmetic, same order, the
reductions deterministic). mg_omega, mg_omega_coarse, mg_nu_fine: other
smoothing schedules of the multigrid preconditioner reach the FP64 residual and
the oracle's banded-Cholesky solution as the defaults do; only the iteration
counts move.
"""
import numpy as np
import pytest

from oracle import topopt_oracle as O
from tests._util import design_field, make_grid, rel, to_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


def _solve(shape, precision, **opts):
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED, TO_PC_GMG
    g, F, fixed = make_grid(shape, precision=TO_MIXED if precision == "mixed" else TO_FP64, precond=TO_PC_GMG,
                            penal=3.0, cg_rtol=1e-8, cg_maxit=100000, **opts)
    xp = design_field(shape, 12, lo=0.02)
    U = torch.zeros(g.ndof, dtype=torch.float64, device="cuda")
    info = g.solve(to_cuda(xp), U)
    g.close()
    return info, U.cpu().numpy(), xp, F, fixed


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(24, 12, 12), (60, 20, 0)])
def test_pdl_on_and_off_give_the_same_solve(shape, precision):
    on, U_on, _, _, _ = _solve(shape, precision, pdl_off=0)
    off, U_off, _, _, _ = _solve(shape, precision, pdl_off=1)
    assert on.iters == off.iters and on.refinements == off.refinements
    np.testing.assert_array_equal(U_on, U_off)


@pytest.mark.parametrize("opts", [dict(mg_nu_fine=2), dict(mg_omega=1.0), dict(mg_omega_coarse=1.5),
                                  dict(mg_omega=1.95, mg_omega_coarse=1.95), dict(mg_nu=2, mg_nu_fine=1)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_smoothing_schedules_reach_the_direct_solution(opts, precision):
    shape = (16, 8, 8)
    info, U, xp, F, fixed = _solve(shape, precision, **opts)
    assert info.rel_res <= 1e-8, (info.rel_res, info.iters)
    og = O.Grid(*shape)
    Ud = O.solve_direct(og, O.element_stiffness(3), O.simp_modulus(xp, 3.0), F, fixed)
    assert rel(U, Ud) <= 1e-5
    assert abs(F @ U - F @ Ud) <= 1e-6 * abs(F @ Ud)
