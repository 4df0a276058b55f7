"""The mixed-precision state solve on a design where plain iterative
refinement fails.

Instance 91 of the batched workload (a 379 x 102 Q4 grid, rmin 7.58,
volfrac 0.47): at its 4th and 6th design iterations the plain refinement
x += d of the FP32 inner solutions diverged (FP64 residual 2e2 at the cap,
compliance 218 against 58.03). The FP64 flexible-CG outer loop must reach the
FP64 residual 1e-8 at every iteration and track the FP64 path's compliance.
"""
import pytest

from paper_2005_05436_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


def _design(precision):
    from paper_2005_05436_gb300 import TO_PC_GMG, default_params
    from paper_2005_05436_gb300.topopt import Design, Grid
    q = I.batched_instances(256, seed=20050543)[91]
    p = default_params(2, q.nelx, q.nely, 0, precision=precision, precond=TO_PC_GMG, mg_nu=1, volfrac=q.volfrac,
                       rmin=q.rmin, penal=3.0, beta=2.0, cg_rtol=1e-8, cg_maxit=100000,
                       penal_cnt=(1, 3.0, 25, 0.25), beta_cnt=(1, 16.0, 25, 2.0, 1))
    g = Grid(p, torch.from_numpy(q.F).cuda(), torch.from_numpy(q.fixed).cuda())
    return g, Design(g, torch.full((g.nel,), q.volfrac, dtype=torch.float64, device="cuda"))


def test_mixed_flexible_refinement_converges_where_plain_refinement_diverged():
    """Every solve ends at an FP64 residual <= 1e-8. On this design a relative
    residual of 1e-8 bounds the energy error only through the smallest
    eigenvalue of K (void elements at Emin = 1e-9), so two paths that both meet
    it (mixed and FP64) agree on the compliance to about 1e-3 here, not to the
    1e-6 they reach on the cantilever benchmark."""
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED
    g1, d1 = _design(TO_MIXED)
    g2, d2 = _design(TO_FP64)
    for _ in range(6):
        a = d1.step()
        b = d2.step()
        assert a["status"] == 0 and a["rel_res"] <= 1e-8, a
        assert b["rel_res"] <= 1e-8
        assert abs(a["c"] - b["c"]) <= 2e-3 * abs(b["c"]), (a["loop"], a["c"], b["c"])
    g1.close()
    g2.close()
