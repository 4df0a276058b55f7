"""The 3D coarse-level V-cycle with the prolongation fused into the first
post-smoothing sweep (k_prolong_smooth3s) against the separate prolongation
and smoothing kernels (to_params.mg_unfused = 1): both compute u = cur + P z_c
and the sweep in the same order, so the design iterations must agree (iteration counts equal,
compliances to rounding). The grids' coarse levels take every tile height
(8, 16 and 32 nodes along y; odd node counts) in both precisions."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


def _run(shape, mixed, unfused):
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED, TO_PC_GMG, inputs as I
    from paper_2005_05436_gb300.topopt import Design
    from tests._util import make_grid, to_cuda
    g, F, fixed = make_grid(shape, precision=TO_MIXED if mixed else TO_FP64, precond=TO_PC_GMG, volfrac=0.15,
                            penal=3.0, rmin=math.sqrt(3), beta=2.0, cg_rtol=1e-9, cg_maxit=20000,
                            mg_unfused=unfused)
    d = Design(g, to_cuda(I.initial_design(g.nel, 0.15)))
    out = [d.step() for _ in range(4)]
    g.close()
    return [(s["n_cg"], s["c"]) for s in out]


@pytest.mark.parametrize("shape,mixed", [((48, 24, 24), True), ((64, 48, 16), True), ((40, 26, 12), True),
                                         ((33, 13, 11), False), ((24, 12, 12), False)])
def test_fused_prolongation_matches_separate_kernels(shape, mixed):
    fused, separate = _run(shape, mixed, 0), _run(shape, mixed, 1)
    for (n1, c1), (n0, c0) in zip(fused, separate):
        assert abs(n1 - n0) <= 1, (fused, separate)
        assert abs(c1 - c0) <= 1e-8 * abs(c0), (c1, c0)
