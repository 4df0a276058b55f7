"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (normwise, ||gpu - oracle|| / ||oracle||): 1e-10 on K u, c and dc,
1e-12 on filter and projection outputs (same operations, different summation
order), bit-exact on CSR structure and OC move-limit/box decisions up to
rounding, 1e-8 on xPhys over 20 design iterations.
"""
import math

import numpy as np
import pytest

from oracle import topopt_oracle as O
from paper_2005_05436_gb300 import inputs as I
from tests._util import assert_design_matches, make_grid, max_abs, problem, rel, simp_field, to_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(60, 20, 0), (67, 23, 0), (1, 1, 0), (9, 1, 0), (24, 12, 12), (13, 7, 5), (1, 1, 1), (5, 1, 3)]
# 3D grids spanning several element tiles of the Walsh operator (31 x 7 node columns in
# FP32, 31 x 3 in FP64) with ragged ends in every direction
TILE_SHAPES = [(40, 70, 17), (9, 31, 7), (3, 62, 2), (33, 1, 15)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _xphys(g, seed):
    return simp_field(g.nel, seed)


@pytest.mark.parametrize("ku_impl", [0, 1])
@pytest.mark.parametrize("shape", SHAPES + TILE_SHAPES)
@pytest.mark.parametrize("masked", [0, 1])
def test_apply_K_fp64(shape, masked, ku_impl):
    """ku_impl 0: Walsh-factored element tiles (3D); 1: node-centric dense-Ke gather."""
    g, F, fixed = make_grid(shape, penal=3.0, ku_impl=ku_impl)
    og = O.Grid(*shape)
    Ke = O.element_stiffness(og.dim)
    xp = _xphys(g, 1)
    u = I.random_vector(g.ndof, 2)
    y = torch.empty(g.ndof, dtype=torch.float64, device="cuda")
    g.apply_K(to_cuda(xp), to_cuda(u), y, masked=bool(masked))
    ref = O.apply_K(og, Ke, O.simp_modulus(xp, 3.0), u, fixed if masked else None)
    assert rel(y.cpu().numpy(), ref) <= 1e-12


def test_apply_K_full_size_sampled_rows():
    """96x48x48 cantilever: sampled rows against element-by-element oracle sums."""
    shape = (96, 48, 48)
    g, F, fixed = make_grid(shape, penal=3.0)
    og = O.Grid(*shape)
    Ke = O.element_stiffness(3)
    xp = _xphys(g, 3)
    u = I.random_vector(g.ndof, 4)
    y = torch.empty(g.ndof, dtype=torch.float64, device="cuda")
    g.apply_K(to_cuda(xp), to_cuda(u), y, masked=True)
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([rng.integers(0, g.ndof, 200), [0, 1, 2, g.ndof - 1, g.ndof - 3]]))
    ref = O.apply_K_rows(og, Ke, O.simp_modulus(xp, 3.0), u, rows, fixed)
    got = y.cpu().numpy()[rows]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-12 * scale


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,rmin,bc", [((60, 20, 0), 2.4, "N"), ((67, 23, 0), 3.3, "D"),
                                           ((30, 10, 0), 9.0, "N"), ((9, 1, 0), 2.5, "N"),
                                           ((6, 4, 0), 0.8, "N"), ((24, 12, 12), math.sqrt(3), "N"),
                                           ((13, 7, 5), 2.2, "D"), ((3, 2, 2), 4.0, "N"),
                                           ((300, 100, 0), 9.0, "N"), ((131, 47, 0), 36.0, "N"),
                                           ((97, 45, 0), 18.0, "D"), ((41, 19, 13), 3.5, "N")])
def test_filter_forward_backward(shape, rmin, bc, precision):
    """FP64 handles filter in FP64 (within 1e-13 of the oracle), mixed handles in
    float-float arithmetic (within 1e-12: every product of the split value and
    weight keeps about 2^-47 of relative error, so a sum of n taps is off by up
    to n 2^-47 in the worst case, 3e-11 at the 4,049 taps of rmin 36, and by
    about sqrt(n) 2^-47 typically); tile kernel with halos of up to 35
    elements, ragged tiles, repeated mirror reflections."""
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED
    g, F, fixed = make_grid(shape, rmin=rmin, ftBC=bc, precision=TO_MIXED if precision == "mixed" else TO_FP64)
    og = O.Grid(*shape)
    x = I.random_design(g.nel, 6)
    gr = I.random_vector(g.nel, 7)
    dp = 0.5 + I.random_design(g.nel, 8)
    out = torch.empty(g.nel, dtype=torch.float64, device="cuda")
    tol = 1e-12 if precision == "mixed" else 1e-13
    g.filter(to_cuda(x), out)
    assert rel(out.cpu().numpy(), O.filter_forward(og, x, rmin, bc)) <= tol
    g.filter(to_cuda(gr), out, to_cuda(dp))
    assert rel(out.cpu().numpy(), O.filter_backward(og, gr, rmin, bc, dp)) <= tol


@pytest.mark.parametrize("shape", [(60, 20, 0), (13, 7, 5), (96, 48, 48)])
@pytest.mark.parametrize("beta,eta0", [(2.0, 0.5), (8.0, 0.3), (16.0, 0.6)])
def test_project_volume_preserving(shape, beta, eta0):
    g, F, fixed = make_grid(shape, beta=beta, volfrac=0.4, newton_tol=1e-14)
    g.set_scalars(3.0, beta, eta0)
    og = O.Grid(*shape)
    xt = np.clip(O.filter_forward(og, simp_field(g.nel, 9), 1.5, "N"), 0, 1) if g.nel < 5e4 else \
        I.random_design(g.nel, 9)
    xphys = torch.empty(g.nel, dtype=torch.float64, device="cuda")
    dprj = torch.empty_like(xphys)
    eta = g.project(to_cuda(xt), xphys, dprj, eta0, True)
    eta_ref, _ = O.eta_newton(xt, eta0, beta, 0.4, tol=1e-14)
    assert abs(eta - eta_ref) <= 1e-11
    assert rel(xphys.cpu().numpy(), O.prj(xt, eta_ref, beta)) <= 1e-11
    assert rel(dprj.cpu().numpy(), O.dprj(xt, eta_ref, beta)) <= 1e-10
    assert abs(xphys.mean().item() - 0.4) <= 1e-13


def test_project_fixed_eta_and_uniform_field():
    g, F, fixed = make_grid((20, 10, 0), beta=8.0, volfrac=0.5, newton_tol=1e-14)
    g.set_scalars(3.0, 8.0, 0.3)
    xt = np.full(g.nel, 0.5)
    xphys = torch.empty(g.nel, dtype=torch.float64, device="cuda")
    dprj = torch.empty_like(xphys)
    # uniform 0.5 with target 0.5: eta* = 0.5 exactly (Newton leaves [0,1], bisection finds it)
    eta = g.project(to_cuda(xt), xphys, dprj, 0.3, True)
    assert abs(eta - 0.5) <= 1e-12
    x2 = I.random_design(g.nel, 3)
    eta2 = g.project(to_cuda(x2), xphys, dprj, 0.3, False)
    assert eta2 == 0.3
    assert rel(xphys.cpu().numpy(), O.prj(x2, 0.3, 8.0)) <= 1e-14


@pytest.mark.parametrize("shape", [(60, 20, 0), (67, 23, 0), (13, 7, 5), (24, 12, 12)])
def test_sensitivity_and_compliance_at_oracle_U(shape):
    g, F, fixed = make_grid(shape, penal=3.0)
    og = O.Grid(*shape)
    Ke = O.element_stiffness(og.dim)
    # a well-conditioned design: with isolated void elements (mechanisms) u_e^T Ke u_e
    # is dominated by cancellation noise in any FP64 implementation
    xp = 0.1 + 0.9 * I.random_design(g.nel, 10)
    U = O.solve_direct(og, Ke, O.simp_modulus(xp, 3.0), F, fixed)
    dc_ref, c_ref, _ = O.sensitivity(og, Ke, xp, U, F, 3.0)
    dc = torch.empty(g.nel, dtype=torch.float64, device="cuda")
    c = g.sensitivity(to_cuda(xp), to_cuda(U), dc)
    assert rel(dc.cpu().numpy(), dc_ref) <= 1e-10
    assert abs(c - c_ref) <= 1e-10 * abs(c_ref)


@pytest.mark.parametrize("shape", [(60, 20, 0), (24, 12, 12), (200, 100, 0)])
@pytest.mark.parametrize("tol", [1e-4, 1e-15])
def test_oc_update(shape, tol):
    g, F, fixed = make_grid(shape, volfrac=0.4, oc_tol=tol, move=0.2)
    n = g.nel
    rng = np.random.default_rng(11)
    x = np.clip(0.4 + 0.3 * rng.standard_normal(n), 0.0, 1.0)
    dc = -np.abs(rng.standard_normal(n)) * 10 ** rng.uniform(-6, 2, n)
    dV0 = np.full(n, 1.0 / (n * 0.4)) * (1 + 0.1 * rng.random(n))
    xr, lm_ref, steps = O.oc_update(x, dc, dV0, np.ones(n, bool), 0.2, 0.4, tol=tol)
    xt = to_cuda(x)
    lm = g.oc_update(xt, to_cuda(dc), to_cuda(dV0))
    assert abs(lm - lm_ref) <= max(tol, 1e-14) * 4 * lm_ref
    # the same bisection decisions give the same midpoints up to the rounding of the initial
    # bracket; one different decision (e.g. a wrongly trusted FP32 screen) moves lm by at least
    # half the bracket width at that step
    assert abs(lm - lm_ref) <= 1e-12 * lm_ref, (lm, lm_ref)
    assert rel(xt.cpu().numpy(), xr) <= (1e-12 if tol < 1e-10 else 1e-3)
    if tol < 1e-10:
        assert abs(xt.mean().item() - 0.4) <= 1e-10


@pytest.mark.parametrize("precond", ["jacobi", "gmg"])
@pytest.mark.parametrize("shape", [(60, 20, 0), (30, 7, 0), (12, 6, 6), (7, 5, 3)])
def test_solve_against_direct(shape, precond):
    """FP64 PCG against the oracle's banded Cholesky solve: U within 1e-8
    normwise, c = F^T U within 1e-8, at a relative residual of 1e-12 or, where
    the design's FP64 residual floor is higher, 4 times that floor. The floor is
    the relative residual ||F - K U_direct|| / ||F|| of the oracle's own direct
    solution: no FP64 method gets far below it (measured on these designs:
    1.0e-9 at 60x20 and 1.7e-9 at 30x7 in 2D, where void elements at E = 1.2e-4
    make plane-stress K very ill-conditioned; 2e-13 and 3e-13 in 3D)."""
    from paper_2005_05436_gb300 import TO_PC_GMG, TO_PC_JACOBI
    og = O.Grid(*shape)
    Ke = O.element_stiffness(og.dim)
    F, fixed = problem(shape)
    xp = np.clip(simp_field(og.nel, 12), 0.05, 1)
    E = O.simp_modulus(xp, 3.0)
    Ud = O.solve_direct(og, Ke, E, F, fixed)
    res = O.full_from_lower(O.assemble_lower(og, Ke, E)) @ Ud - F
    res[fixed.astype(bool)] = 0.0
    floor = np.linalg.norm(res) / np.linalg.norm(F)
    rtol = max(1e-12, 4.0 * floor)
    if og.dim == 3:
        assert rtol <= 1.2e-12, floor  # the 3D designs keep (about) the original target
    g, _, _ = make_grid(shape, penal=3.0, cg_rtol=rtol, cg_maxit=200000,
                        precond=TO_PC_GMG if precond == "gmg" else TO_PC_JACOBI)
    U = torch.zeros(g.ndof, dtype=torch.float64, device="cuda")
    info = g.solve(to_cuda(xp), U)
    assert info.rel_res <= rtol, (info.rel_res, rtol)
    assert rel(U.cpu().numpy(), Ud) <= 1e-8, rel(U.cpu().numpy(), Ud)
    c_gpu = float(np.dot(F, U.cpu().numpy()))
    assert abs(c_gpu - F @ Ud) <= 1e-8 * abs(F @ Ud)


@pytest.mark.parametrize("shape", [(6, 4, 0), (13, 7, 0), (3, 2, 2), (5, 4, 3)])
def test_assemble_lower_csr(shape):
    g, F, fixed = make_grid(shape, penal=3.0)
    og = O.Grid(*shape)
    Ke = O.element_stiffness(og.dim)
    xp = _xphys(g, 13)
    ref = O.assemble_lower(og, Ke, O.simp_modulus(xp, 3.0))
    rp, col, val = g.assemble_lower(to_cuda(xp))
    np.testing.assert_array_equal(rp.cpu().numpy(), ref.indptr)
    np.testing.assert_array_equal(col.cpu().numpy(), ref.indices)
    np.testing.assert_allclose(val.cpu().numpy(), ref.data, rtol=0, atol=1e-14 * np.abs(ref.data).max())


def _run_parity(shape, n_iter, **kw):
    from paper_2005_05436_gb300.topopt import Design
    g, F, fixed = make_grid(shape, **kw)
    p = g.params
    op = O.Params.parity(nelx=shape[0], nely=shape[1], nelz=shape[2], volfrac=p.volfrac,
                         penal=p.penal, rmin=p.rmin, beta=p.beta, eta=p.eta, move=p.move,
                         ft=p.ft, ftBC=chr(p.ftBC),
                         penal_cnt=(p.penal_cnt.istart, p.penal_cnt.maxpar, p.penal_cnt.isteps,
                                    p.penal_cnt.delta),
                         beta_cnt=(p.beta_cnt.istart, p.beta_cnt.maxpar, p.beta_cnt.isteps,
                                   p.beta_cnt.delta),
                         penal_kind="add" if p.penal_cnt.kind == 0 else "mul",
                         beta_kind="add" if p.beta_cnt.kind == 0 else "mul",
                         oc_method={0: "bisection", 1: "primal_dual", 2: "filtered"}[p.oc_method],
                         pae_q0=p.pae_q0, pae_q=p.pae_q, pae_m=p.pae_m, pae_alpha=p.pae_alpha,
                         pae_zeta=p.pae_zeta)
    s = O.initial_state(op)
    Ke = O.element_stiffness(3 if shape[2] else 2)
    d = Design(g, to_cuda(I.initial_design(g.nel, p.volfrac)))
    worst = 0.0
    for k in range(n_iter):
        ref = O.design_step(op, s, F, fixed, None, Ke)
        got = d.step()
        assert got["loop"] == ref["loop"]
        worst = max(worst, assert_design_matches(k, got, ref, d.xPhys.cpu().numpy(), s.xphys,
                                                 d.x.cpu().numpy(), s.x))
        assert abs(got["c"] - ref["c"]) <= 1e-8 * abs(ref["c"]), (k, got["c"], ref["c"])
        assert abs(got["eta"] - ref["eta"]) <= 1e-9
        assert got["penal"] == ref["penal"] and got["beta"] == ref["beta"]
        assert got["pae"] == ref["pae"], (k, got["pae"], ref["pae"])
    return worst


@pytest.mark.parametrize("shape", [(60, 20, 0), (24, 12, 12), (200, 100, 0)])
@pytest.mark.parametrize("with_passive", [False, True])
def test_oc_update_primal_dual(shape, with_passive):
    """Appendix A's explicit primal-dual OC against the oracle's, and against the
    GPU bisection run to 1e-15 (the same volume equation)."""
    from paper_2005_05436_gb300 import TO_OC_PRIMAL_DUAL
    n = int(np.prod([v for v in shape if v]))
    rng = np.random.default_rng(12)
    passive = None
    act = np.ones(n, bool)
    if with_passive:
        passive = np.zeros(n, np.int8)
        idx = rng.choice(n, n // 20, replace=False)
        passive[idx[: n // 40]] = 1
        passive[idx[n // 40:]] = -1
        act = passive == 0
    x = np.clip(0.4 + 0.3 * rng.standard_normal(n), 0.0, 1.0)
    if with_passive:
        x[passive == 1], x[passive == -1] = 1.0, 0.0
    dc = -np.abs(rng.standard_normal(n)) * 10 ** rng.uniform(-6, 2, n)
    dV0 = np.full(n, 1.0 / (n * 0.4)) * (1 + 0.1 * rng.random(n))
    xr, lm_ref, it = O.oc_update_primal_dual(x, dc, dV0, act, 0.2, 0.4)
    assert it <= 50
    g, _, _ = make_grid(shape, volfrac=0.4, move=0.2, oc_method=TO_OC_PRIMAL_DUAL, passive=passive)
    xt = to_cuda(x)
    lm = g.oc_update(xt, to_cuda(dc), to_cuda(dV0))
    assert abs(lm - lm_ref) <= 1e-12 * lm_ref, (lm, lm_ref)
    assert np.abs(xt.cpu().numpy() - xr).max() <= 1e-12
    gb, _, _ = make_grid(shape, volfrac=0.4, move=0.2, oc_tol=1e-15, passive=passive)
    xb = to_cuda(x)
    lmb = gb.oc_update(xb, to_cuda(dc), to_cuda(dV0))
    assert abs(lm - lmb) <= 1e-9 * lmb
    assert np.abs(xt.cpu().numpy() - xb.cpu().numpy()).max() <= 1e-9


@pytest.mark.parametrize("ft", [1, 3])
def test_design_iterations_primal_dual_parity(ft):
    from paper_2005_05436_gb300 import TO_OC_PRIMAL_DUAL
    _run_parity((60, 20, 0), 12, volfrac=0.5, penal=3.0, rmin=2.4, beta=2.0, ft=ft, newton_tol=1e-14,
                oc_method=TO_OC_PRIMAL_DUAL, cg_rtol=1e-12, cg_maxit=200000)
    _run_parity((12, 6, 6), 8, volfrac=0.12, penal=3.0, rmin=math.sqrt(3), beta=2.0, ft=ft, newton_tol=1e-14,
                oc_method=TO_OC_PRIMAL_DUAL, cg_rtol=1e-12, cg_maxit=200000)


@pytest.mark.parametrize("shape", [(60, 20, 0), (12, 6, 6)])
@pytest.mark.parametrize("with_passive", [False, True])
def test_oc_update_physical_volume(shape, with_passive):
    """The general OC variant of Sec. 3.2 (volume of the filtered, projected
    candidate, fixed threshold) against the oracle at a 1e-15 bracket."""
    from paper_2005_05436_gb300 import TO_OC_PHYSICAL_VOLUME
    n = int(np.prod([v for v in shape if v]))
    rng = np.random.default_rng(13)
    passive = None
    act = np.ones(n, bool)
    if with_passive:
        passive = np.zeros(n, np.int8)
        idx = rng.choice(n, n // 10, replace=False)
        passive[idx[: n // 20]] = 1
        passive[idx[n // 20:]] = -1
        act = passive == 0
    x = np.clip(0.35 + 0.25 * rng.standard_normal(n), 0.0, 1.0)
    if with_passive:
        x[passive == 1], x[passive == -1] = 1.0, 0.0
    dc = -np.abs(rng.standard_normal(n)) * 10 ** rng.uniform(-4, 1, n)
    dV0 = np.full(n, 1.0 / (n * 0.35)) * (1 + 0.1 * rng.random(n))
    og = O.Grid(*shape)
    xr, lm_ref, steps = O.oc_update_filtered(og, x, dc, dV0, act, 0.2, 0.35, 2.0, "N", 2, 0.4, 4.0, passive,
                                             tol=1e-15)
    g, _, _ = make_grid(shape, volfrac=0.35, move=0.2, rmin=2.0, ft=2, oc_tol=1e-15,
                        oc_method=TO_OC_PHYSICAL_VOLUME, passive=passive)
    g.set_scalars(3.0, 4.0, 0.4)
    xt = to_cuda(x)
    lm = g.oc_update(xt, to_cuda(dc), to_cuda(dV0))
    assert abs(lm - lm_ref) <= 1e-13 * lm_ref, (lm, lm_ref)
    assert np.abs(xt.cpu().numpy() - xr).max() <= 1e-12


@pytest.mark.parametrize("ft", [2, 3])
def test_design_iterations_physical_volume_parity(ft):
    from paper_2005_05436_gb300 import TO_OC_PHYSICAL_VOLUME
    _run_parity((60, 20, 0), 10, volfrac=0.5, penal=3.0, rmin=2.4, beta=4.0, eta=0.4, ft=ft, newton_tol=1e-14,
                oc_tol=1e-15, oc_method=TO_OC_PHYSICAL_VOLUME, cg_rtol=1e-12, cg_maxit=200000)
    _run_parity((12, 6, 6), 6, volfrac=0.12, penal=3.0, rmin=math.sqrt(3), beta=4.0, eta=0.4, ft=ft,
                newton_tol=1e-14, oc_tol=1e-15, oc_method=TO_OC_PHYSICAL_VOLUME, cg_rtol=1e-12,
                cg_maxit=200000)


def test_design_iterations_anderson_extrapolation_parity():
    """Periodic Anderson extrapolation of the OC iteration (Sec. 3.6): damped steps
    and, every q = 4th step from q0, the least-squares extrapolation over m_r = 4
    history columns, against the oracle over the design iterations (ft 1, 2D;
    ft 3, 3D), including which steps were extrapolated."""
    _run_parity((60, 20, 0), 18, volfrac=0.5, penal=3.0, rmin=2.4, ft=1, newton_tol=1e-14, oc_tol=1e-15,
                cg_rtol=1e-12, cg_maxit=200000, pae_q0=3, pae_q=4, pae_m=4, pae_alpha=0.9, pae_zeta=1.0)
    _run_parity((12, 6, 6), 12, volfrac=0.12, penal=3.0, rmin=math.sqrt(3), beta=2.0, ft=3, newton_tol=1e-14,
                oc_tol=1e-15, cg_rtol=1e-12, cg_maxit=200000, pae_q0=2, pae_q=4, pae_m=3, pae_alpha=0.9,
                pae_zeta=1.0)


def test_design_iterations_mbb_60x20_parity():
    """Config 1 shape (60x20 MBB, rmin 2.4, ft = 3, beta 2) for 20 iterations."""
    _run_parity((60, 20, 0), 20, volfrac=0.5, penal=3.0, rmin=2.4, beta=2.0, newton_tol=1e-14,
                oc_tol=1e-15, cg_rtol=1e-12, cg_maxit=200000)


def test_design_iterations_cantilever_parity():
    _run_parity((12, 6, 6), 20, volfrac=0.12, penal=3.0, rmin=math.sqrt(3), beta=2.0,
                newton_tol=1e-14, oc_tol=1e-15, cg_rtol=1e-12, cg_maxit=200000)


_TRAJECTORIES = {}


def _oracle_trajectory(shape, n_iter):
    """The oracle's first n_iter design iterations of the 3D cantilever in parity
    mode (volfrac 0.12, penal 3, rmin sqrt(3), ft 3, beta 2), computed once per
    module and shared by the GPU arms below."""
    key = (shape, n_iter)
    if key not in _TRAJECTORIES:
        op = O.Params.parity(nelx=shape[0], nely=shape[1], nelz=shape[2], volfrac=0.12, penal=3.0,
                             rmin=math.sqrt(3), beta=2.0, penal_cnt=(1, 3.0, 25, 0.0),
                             beta_cnt=(1, 2.0, 25, 0.0))
        F, fixed = problem(shape)
        s = O.initial_state(op)
        Ke = O.element_stiffness(3)
        traj = []
        for _ in range(n_iter):
            ref = O.design_step(op, s, F, fixed, None, Ke)
            traj.append((dict(ref), s.xphys.copy(), s.x.copy()))
        _TRAJECTORIES[key] = traj
    return _TRAJECTORIES[key]


@pytest.mark.parametrize("arm", ["fp64_jacobi", "fp64_gmg", "mixed_gmg"])
def test_design_iterations_cantilever_24x12x12_parity(arm):
    """20 design iterations of the 24x12x12 cantilever (several Walsh tiles along
    y and z, four multigrid levels) against the oracle's banded-Cholesky run:
    xPhys and x elementwise within 1e-8, c within 1e-8, ch, V, eta and the OC
    multiplier. The mixed arm (FP32 inner PCG, FP64 flexible-CG refinement) is
    held to the same bounds: its FP64 residual is driven to the same 1e-12."""
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED, TO_PC_GMG, TO_PC_JACOBI
    from paper_2005_05436_gb300.topopt import Design
    shape, n_iter = (24, 12, 12), 20
    traj = _oracle_trajectory(shape, n_iter)
    prec = TO_MIXED if arm.startswith("mixed") else TO_FP64
    pc = TO_PC_JACOBI if arm.endswith("jacobi") else TO_PC_GMG
    g, F, fixed = make_grid(shape, volfrac=0.12, penal=3.0, rmin=math.sqrt(3), beta=2.0, newton_tol=1e-14,
                            oc_tol=1e-15, cg_rtol=1e-12, cg_maxit=200000, precision=prec, precond=pc,
                            penal_cnt=(1, 3.0, 25, 0.0), beta_cnt=(1, 2.0, 25, 0.0))
    d = Design(g, to_cuda(I.initial_design(g.nel, 0.12)))
    for k, (ref, xphys_ref, x_ref) in enumerate(traj):
        got = d.step()
        assert got["loop"] == ref["loop"]
        assert got["rel_res"] <= 1e-12, (k, got["rel_res"])
        assert_design_matches(k, got, ref, d.xPhys.cpu().numpy(), xphys_ref, d.x.cpu().numpy(), x_ref)
        assert abs(got["c"] - ref["c"]) <= 1e-8 * abs(ref["c"]), (k, got["c"], ref["c"])
        assert abs(got["eta"] - ref["eta"]) <= 1e-9, (k, got["eta"], ref["eta"])
    g.close()


def test_design_iterations_with_continuation_and_dirichlet_filter():
    _run_parity((30, 10, 0), 12, volfrac=0.3, penal=1.0, rmin=1.8, beta=2.0, ftBC="D",
                penal_cnt=(1, 3.0, 4, 0.25), beta_cnt=(1, 16.0, 5, 2.0, 1), newton_tol=1e-14,
                oc_tol=1e-15, cg_rtol=1e-12, cg_maxit=200000)


@pytest.mark.parametrize("sign", [-1.0, 1.0])
def test_frame_reinforcement_parity(sign):
    """The frame-reinforcement workload of Sec. 3.5 (passive solid frame and void
    opening, distributed vertical and height-proportional horizontal loads, ft = 3,
    no continuation), scaled to 100 x 100 with rmin 2: design iterations against
    the oracle, passive densities kept exactly."""
    from paper_2005_05436_gb300.topopt import Design
    from paper_2005_05436_gb300 import TO_PC_GMG
    F, fixed, pas = I.frame_reinforcement(100, 100, sign)
    # the void opening (E = Emin) puts the FP64 PCG floor near 1e-11: multigrid PCG to 1e-10
    g, _, _ = make_grid((100, 100, 0), F=F, fixed=fixed, passive=pas, volfrac=0.2, penal=3.0, rmin=2.0,
                        ft=3, eta=0.5, beta=2.0, newton_tol=1e-14, oc_tol=1e-15, cg_rtol=1e-10,
                        cg_maxit=200000, precond=TO_PC_GMG, penal_cnt=(1, 3.0, 1000, 0.0),
                        beta_cnt=(1, 2.0, 1000, 0.0))
    op = O.Params.parity(nelx=100, nely=100, volfrac=0.2, penal=3.0, rmin=2.0, ft=3, eta=0.5, beta=2.0,
                         penal_cnt=(1, 3.0, 1000, 0.0), beta_cnt=(1, 2.0, 1000, 0.0))
    s = O.initial_state(op, pas)
    Ke = O.element_stiffness(2)
    d = Design(g, to_cuda(s.x.copy()))
    for k in range(6):
        ref = O.design_step(op, s, F, fixed, pas, Ke)
        got = d.step()
        assert rel(d.xPhys.cpu().numpy(), s.xphys) <= 1e-8, (k, rel(d.xPhys.cpu().numpy(), s.xphys))
        assert abs(got["c"] - ref["c"]) <= 1e-8 * abs(ref["c"]), (k, got["c"], ref["c"])
    x = d.x.cpu().numpy()
    assert np.all(x[pas == 1] == 1.0) and np.all(x[pas == -1] == 0.0)


def test_passive_elements_step():
    """Passive solid/void sets (frame reinforcement, scaled down)."""
    from paper_2005_05436_gb300.topopt import Design
    F, fixed, pas = I.frame_reinforcement(100, 100)
    g, _, _ = make_grid((100, 100, 0), F=F, fixed=fixed, passive=pas, volfrac=0.2, rmin=4.0,
                        cg_rtol=1e-10, cg_maxit=200000)
    x0 = I.initial_design(g.nel, 0.2, pas)
    d = Design(g, to_cuda(x0))
    for _ in range(3):
        info = d.step()
    x = d.x.cpu().numpy()
    assert np.all(x[pas == 1] == 1.0) and np.all(x[pas == -1] == 0.0)
    assert abs(info["V"] - 0.2) < 1e-3
