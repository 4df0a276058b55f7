"""The mixed-precision state solve on a design where plain iterative
refinement fails.

Instance 91 of the batched workload (a 379 x 102 Q4 grid, rmin 7.58,
volfrac 0.47): at its 4th and 6th design iterations the plain refinement
x += d of the FP32 inner solutions diverged (FP64 residual 2e2 at the cap,
compliance 218 against 58.03). Both mixed schemes must reach the FP64 residual
1e-8 at every iteration and track the FP64 path's compliance.
"""
import pytest

from paper_2005_05436_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


def _design(precision, refine=0):
    from paper_2005_05436_gb300 import TO_PC_GMG, default_params
    from paper_2005_05436_gb300.topopt import Design, Grid
    q = I.batched_instances(256, seed=20050543)[91]
    p = default_params(2, q.nelx, q.nely, 0, precision=precision, precond=TO_PC_GMG, mg_nu=1, volfrac=q.volfrac,
                       rmin=q.rmin, penal=3.0, beta=2.0, cg_rtol=1e-8, cg_maxit=100000, refine=refine,
                       penal_cnt=(1, 3.0, 25, 0.25), beta_cnt=(1, 16.0, 25, 2.0, 1))
    g = Grid(p, torch.from_numpy(q.F).cuda(), torch.from_numpy(q.fixed).cuda())
    return g, Design(g, torch.full((g.nel,), q.volfrac, dtype=torch.float64, device="cuda"))


def test_mixed_solves_converge_where_plain_refinement_diverged():
    """Every solve of both mixed schemes (reliable updates, which on this design
    stall in FP32 and hand over to the flexible-CG steps, and flexible CG alone)
    ends at an FP64 residual <= 1e-8, with no more than twice the inner
    iterations of flexible CG. The compliances agree with the FP64 path to 5e-3:
    on this design a relative residual bounds the energy error only through the
    smallest eigenvalue of K (void elements at Emin = 1e-9); measured, the FP64
    path and flexible CG, both solved to 1e-10, still differ by 3.5e-3 at the
    third design iteration (76.409 against 76.680), so 1e-8 residuals cannot
    fix c more closely here than they do on the cantilever benchmark (1e-6)."""
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED, TO_REFINE_FLEXIBLE, TO_REFINE_RELIABLE
    runs = {"fp64": _design(TO_FP64), "reliable": _design(TO_MIXED, TO_REFINE_RELIABLE),
            "flexible": _design(TO_MIXED, TO_REFINE_FLEXIBLE)}
    n_cg = {k: 0 for k in runs}
    for _ in range(6):
        out = {k: d.step(check=False) for k, (g, d) in runs.items()}
        for k, a in out.items():
            assert a["status"] == 0 and a["rel_res"] <= 1e-8, (k, a)
            n_cg[k] += a["n_cg"]
        for k in ("reliable", "flexible"):
            assert abs(out[k]["c"] - out["fp64"]["c"]) <= 5e-3 * abs(out["fp64"]["c"]), (k, out[k]["c"], out["fp64"]["c"])
    assert n_cg["reliable"] <= 2 * n_cg["flexible"], n_cg
    for g, _ in runs.values():
        g.close()
