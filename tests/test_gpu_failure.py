"""Failure detection through the C ABI, without faulting the GPU.

Every failure is made on the host or by a bounded wait running out:
- a PCG iteration cap of 1 (the solve cannot reach cg_rtol): TO_ENOTCONV;
- a NaN placed in the load on the host: TO_ENAN from the solve and the step;
- a grid-barrier deadline of one clock cycle in the cooperative projection and
  OC kernels: every waiting block gives up, sets the barrier's error word and
  returns, and the call reports TO_ETIMEOUT; a handle created afterwards with
  the default deadline still computes the oracle's result (the context is
  intact);
- an OC bisection cap of one step: TO_ENOTCONV with the last candidate kept.

Also the resume property of the design loop: 10 iterations, state copied to
the host, handle destroyed, a new handle restored from the copy and run for 10
more gives bitwise the design of 20 uninterrupted iterations (the state of a
design iteration is x, xPhys, xOld, U and the host scalars eta, penal, beta,
loop; every reduction has a fixed summation order).
"""
import math

import numpy as np
import pytest

from oracle import topopt_oracle as O
from paper_2005_05436_gb300 import inputs as I
from tests._util import make_grid, rel, to_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


def _status_of(fn):
    from paper_2005_05436_gb300._lib import TopoptError
    with pytest.raises(TopoptError) as e:
        fn()
    return e.value.status


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(60, 20, 0), (12, 6, 6)])
def test_iteration_cap_gives_enotconv(shape, precision):
    """Jacobi preconditioning: one PCG iteration cannot reach 1e-10 (a multigrid
    whose coarsest level is the whole grid would solve these grids exactly)."""
    from paper_2005_05436_gb300 import TO_ENOTCONV, TO_FP64, TO_MIXED, TO_PC_JACOBI
    from paper_2005_05436_gb300.topopt import Design
    prec = TO_FP64 if precision == "fp64" else TO_MIXED
    g, F, fixed = make_grid(shape, cg_rtol=1e-10, cg_maxit=1, precision=prec, precond=TO_PC_JACOBI)
    xp = to_cuda(np.full(g.nel, 0.5))
    U = torch.zeros(g.ndof, dtype=torch.float64, device="cuda")
    assert _status_of(lambda: g.solve(xp, U)) == TO_ENOTCONV
    info = g.solve(xp, U, check=False)
    assert info.status == TO_ENOTCONV and info.rel_res > 1e-10
    d = Design(g, to_cuda(I.initial_design(g.nel, g.params.volfrac)))
    assert _status_of(d.step) == TO_ENOTCONV
    got = d.step(check=False)
    assert got["status"] == TO_ENOTCONV and got["loop"] == 2  # the iteration still completes
    g.close()


@pytest.mark.parametrize("shape", [(30, 10, 0), (8, 4, 4)])
def test_nan_load_gives_enan(shape):
    from paper_2005_05436_gb300 import TO_ENAN
    from paper_2005_05436_gb300.topopt import Design
    F, fixed = (I.cantilever_3d(*shape) if shape[2] else I.mbb_half_beam(shape[0], shape[1]))
    F = F.copy()
    F[np.flatnonzero(fixed == 0)[3]] = np.nan
    g, _, _ = make_grid(shape, F=F, fixed=fixed, cg_rtol=1e-10, cg_maxit=5000)
    U = torch.zeros(g.ndof, dtype=torch.float64, device="cuda")
    assert _status_of(lambda: g.solve(to_cuda(np.full(g.nel, 0.5)), U)) == TO_ENAN
    d = Design(g, to_cuda(I.initial_design(g.nel, g.params.volfrac)))
    got = d.step(check=False)
    assert got["status"] == TO_ENAN
    g.close()


def test_barrier_deadline_gives_etimeout_and_context_survives():
    from paper_2005_05436_gb300 import TO_ETIMEOUT
    shape = (120, 40, 0)  # enough elements for a multi-block cooperative grid
    g, F, fixed = make_grid(shape, volfrac=0.4, beta=8.0, deadline_cycles=1, newton_tol=1e-14, oc_tol=1e-15)
    g.set_scalars(3.0, 8.0, 0.3)
    og = O.Grid(*shape)
    xt = np.clip(O.filter_forward(og, I.random_design(g.nel, 9), 1.5, "N"), 0, 1)
    xphys = torch.empty(g.nel, dtype=torch.float64, device="cuda")
    dprj = torch.empty_like(xphys)
    assert _status_of(lambda: g.project(to_cuda(xt), xphys, dprj, 0.3, True)) == TO_ETIMEOUT
    rng = np.random.default_rng(3)
    x = np.clip(0.4 + 0.3 * rng.standard_normal(g.nel), 0.0, 1.0)
    dc = -np.abs(rng.standard_normal(g.nel))
    dV0 = np.full(g.nel, 1.0 / (g.nel * 0.4))
    assert _status_of(lambda: g.oc_update(to_cuda(x), to_cuda(dc), to_cuda(dV0))) == TO_ETIMEOUT
    g.close()
    # the context is still usable: a handle with the default deadline matches the oracle
    g2, _, _ = make_grid(shape, volfrac=0.4, beta=8.0, newton_tol=1e-14, oc_tol=1e-15)
    g2.set_scalars(3.0, 8.0, 0.3)
    eta = g2.project(to_cuda(xt), xphys, dprj, 0.3, True)
    eta_ref, _ = O.eta_newton(xt, 0.3, 8.0, 0.4, tol=1e-14)
    assert abs(eta - eta_ref) <= 1e-11
    assert rel(xphys.cpu().numpy(), O.prj(xt, eta_ref, 8.0)) <= 1e-11
    xg = to_cuda(x)
    lm = g2.oc_update(xg, to_cuda(dc), to_cuda(dV0))
    xr, lm_ref, _ = O.oc_update(x, dc, dV0, np.ones(g2.nel, bool), 0.2, 0.4, tol=1e-15)
    assert abs(lm - lm_ref) <= 1e-12 * lm_ref
    g2.close()


def test_oc_iteration_cap_gives_enotconv():
    from paper_2005_05436_gb300 import TO_ENOTCONV
    g, _, _ = make_grid((60, 20, 0), volfrac=0.4, oc_tol=1e-15, oc_maxit=1)
    rng = np.random.default_rng(4)
    x = np.clip(0.4 + 0.3 * rng.standard_normal(g.nel), 0.0, 1.0)
    dc = -np.abs(rng.standard_normal(g.nel))
    dV0 = np.full(g.nel, 1.0 / (g.nel * 0.4))
    xg = to_cuda(x)
    assert _status_of(lambda: g.oc_update(xg, to_cuda(dc), to_cuda(dV0))) == TO_ENOTCONV
    # one bisection step from [0, lambda#]: the midpoint, applied to x
    xr, lm_ref, steps = O.oc_update(x, dc, dV0, np.ones(g.nel, bool), 0.2, 0.4, tol=1e-15, maxit=1)
    assert steps == 1
    assert np.abs(xg.cpu().numpy() - xr).max() <= 1e-12
    g.close()


def _snapshot(d):
    return {"t": [t.cpu().numpy().copy() for t in (d.x, d.xPhys, d.xOld, d.U)],
            "s": (d.st.eta, d.st.penal, d.st.beta, d.st.loop)}


@pytest.mark.parametrize("arm", ["fp64_gmg", "mixed_gmg"])
def test_resume_is_bitwise(arm):
    """10 + save + 10 iterations equal 20 uninterrupted ones, bit for bit."""
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED, TO_PC_GMG
    from paper_2005_05436_gb300.topopt import Design
    shape = (16, 8, 8)
    kw = dict(volfrac=0.12, penal=3.0, rmin=math.sqrt(3), beta=2.0, cg_rtol=1e-8, cg_maxit=100000,
              precision=TO_FP64 if arm.startswith("fp64") else TO_MIXED, precond=TO_PC_GMG,
              penal_cnt=(1, 3.0, 25, 0.25), beta_cnt=(5, 16.0, 5, 2.0, 1))
    g, F, fixed = make_grid(shape, **kw)
    x0 = to_cuda(I.initial_design(g.nel, 0.12))
    d = Design(g, x0)
    for _ in range(20):
        d.step()
    whole = _snapshot(d)
    g.close()

    g1, _, _ = make_grid(shape, **kw)
    d1 = Design(g1, x0)
    for _ in range(10):
        d1.step()
    saved = _snapshot(d1)
    g1.close()

    g2, _, _ = make_grid(shape, **kw)
    d2 = Design(g2, to_cuda(saved["t"][0]))
    for t, a in zip((d2.x, d2.xPhys, d2.xOld, d2.U), saved["t"]):
        t.copy_(torch.from_numpy(a))
    d2.st.eta, d2.st.penal, d2.st.beta, d2.st.loop = saved["s"]
    for _ in range(10):
        d2.step()
    resumed = _snapshot(d2)
    g2.close()
    assert resumed["s"] == whole["s"]
    for a, b in zip(resumed["t"], whole["t"]):
        np.testing.assert_array_equal(a, b)
