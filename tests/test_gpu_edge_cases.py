"""Degenerate and boundary cases of the design iteration against the oracle:
zero load, filter-only (ft = 1) and fixed-threshold (ft = 2) projection,
extreme volume fractions (the lambda# bracket must grow, reading R6), and a
zero-load instance inside a batch."""
import dataclasses

import numpy as np
import pytest

from oracle import topopt_oracle as O
from paper_2005_05436_gb300 import inputs as I
from tests._util import assert_design_matches, make_grid, max_abs, rel, to_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


def _parity(shape, n_iter, F=None, fixed=None, tol_x=1e-8, **kw):
    from paper_2005_05436_gb300.topopt import Design
    g, F, fixed = make_grid(shape, F=F, fixed=fixed, **kw)
    p = g.params
    op = O.Params.parity(nelx=shape[0], nely=shape[1], nelz=shape[2], volfrac=p.volfrac, penal=p.penal,
                         rmin=p.rmin, beta=p.beta, eta=p.eta, move=p.move, ft=p.ft, ftBC=chr(p.ftBC))
    s = O.initial_state(op)
    Ke = O.element_stiffness(3 if shape[2] else 2)
    d = Design(g, to_cuda(I.initial_design(g.nel, p.volfrac)))
    infos = []
    for k in range(n_iter):
        ref = O.design_step(op, s, F, fixed, None, Ke)
        got = d.step()
        assert_design_matches(k, got, ref, d.xPhys.cpu().numpy(), s.xphys, d.x.cpu().numpy(), s.x, tol=tol_x)
        assert abs(got["c"] - ref["c"]) <= 1e-8 * max(abs(ref["c"]), 1e-300), (k, got["c"], ref["c"])
        assert abs(got["V"] - ref["V"]) <= 1e-10
        infos.append((got, ref))
    g.close()
    return infos


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(20, 10, 0), (6, 3, 3)])
def test_zero_load(precision, shape):
    """F = 0: U = 0, c = 0, dc = 0, so the OC bracket is empty and x stays."""
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED, TO_PC_GMG
    F, fixed = (I.cantilever_3d(*shape) if shape[2] else I.mbb_half_beam(shape[0], shape[1]))
    infos = _parity(shape, 3, F=np.zeros_like(F), fixed=fixed, volfrac=0.4, rmin=1.5,
                    precision=TO_FP64 if precision == "fp64" else TO_MIXED, precond=TO_PC_GMG,
                    newton_tol=1e-14, oc_tol=1e-15, cg_rtol=1e-12)
    for got, ref in infos:
        assert got["c"] == 0.0 and ref["c"] == 0.0
        assert got["lm"] == 0.0 and got["n_bisect"] == 0


@pytest.mark.parametrize("ft", [1, 2])
def test_filter_only_and_fixed_threshold(ft):
    # the FP64 Jacobi-PCG floor of these void-region designs sits near 1e-12
    _parity((30, 10, 0), 8, ft=ft, volfrac=0.4, rmin=2.0, beta=4.0, eta=0.45, newton_tol=1e-14, oc_tol=1e-15,
            cg_rtol=1e-11, cg_maxit=100000)


@pytest.mark.parametrize("volfrac", [0.05, 0.95])
def test_extreme_volume_fractions(volfrac):
    """A nearly void design (volfrac 0.05) is the hard case for the solve: FP64
    Jacobi-PCG stalls short of 1e-12 there, so the multigrid PCG runs it."""
    from paper_2005_05436_gb300 import TO_PC_GMG
    _parity((24, 8, 0), 6, volfrac=volfrac, rmin=1.5, newton_tol=1e-14, oc_tol=1e-15, cg_rtol=1e-11,
            cg_maxit=100000, precond=TO_PC_GMG)


def test_zero_load_instance_in_a_batch():
    """One instance without load rides along: its compliance is 0 and its design
    does not move; the others match the oracle."""
    from paper_2005_05436_gb300 import TO_MIXED, TO_PC_GMG, default_params
    from paper_2005_05436_gb300.topopt import Batch
    insts = I.batched_instances(3, seed=4, nelx_range=(12, 24))
    insts = [dataclasses.replace(q, rmin=1.5) for q in insts]
    insts[1] = dataclasses.replace(insts[1], F=np.zeros_like(insts[1].F))
    p = default_params(2, 8, 4, precision=TO_MIXED, precond=TO_PC_GMG, newton_tol=1e-14, oc_tol=1e-15,
                       cg_rtol=1e-11, cg_maxit=20000)
    F = np.concatenate([q.F for q in insts])
    fixed = np.concatenate([q.fixed for q in insts])
    x0 = np.concatenate([I.initial_design(q.nelx * q.nely, q.volfrac) for q in insts])
    b = Batch(p, [(q.nelx, q.nely, q.volfrac, q.rmin) for q in insts], to_cuda(F), to_cuda(fixed), to_cuda(x0))
    Ke = O.element_stiffness(2)
    ops = [O.Params.parity(nelx=q.nelx, nely=q.nely, nelz=0, volfrac=q.volfrac, penal=p.penal, rmin=q.rmin,
                           beta=p.beta, eta=p.eta, move=p.move, ft=p.ft, ftBC="N") for q in insts]
    states = [O.initial_state(op) for op in ops]
    x_first = None
    for it in range(3):
        b.step()
        res = b.results()
        x = b.x.cpu().numpy()
        for k, q in enumerate(insts):
            ref = O.design_step(ops[k], states[k], q.F, q.fixed, None, Ke)
            sl = slice(b.el_off[k], b.el_off[k + 1])
            assert rel(x[sl], states[k].x) <= 1e-8, (it, k)
            assert max_abs(x[sl], states[k].x) <= 1e-8, (it, k)
            assert abs(res["lm"][k] - ref["lm"]) <= 1e-7 * abs(ref["lm"]), (it, k)
            assert abs(res["c"][k] - ref["c"]) <= 1e-8 * max(abs(ref["c"]), 1e-300), (it, k)
        assert res["c"][1] == 0.0 and res["lm"][1] == 0.0
        sl1 = slice(b.el_off[1], b.el_off[2])
        if x_first is None:
            x_first = x[sl1].copy()
        np.testing.assert_array_equal(x[sl1], x_first)
