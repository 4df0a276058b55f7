"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: values the
paper prints, closed forms, library routines implementing the same definition,
invariants, or brute force on tiny inputs.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import topopt_oracle as O
from paper_2005_05436_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
NU = 0.3


def _golden():
    with open(os.path.join(GOLD, "ke_paper.json")) as f:
        return json.load(f)


# --------------------------------------------------------------------- Ke --

def test_q4_ke_equals_paper_coefficients():
    """Appendix B prints Ke = (c1 + nu c2) / (1 - nu^2) / 24 (lower triangle)."""
    g = _golden()
    ref = (np.array(g["q4_c1"]) + NU * np.array(g["q4_c2"])) / (1 - NU ** 2) / 24
    Ke = O.element_stiffness(2, NU)
    np.testing.assert_allclose(O.lower_vector(Ke), ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.from_lower_vector(ref, 8), Ke, rtol=0, atol=1e-15)


def test_h8_ke_equals_paper_coefficients():
    """Appendix C prints all 300 lower-triangle coefficients,
    Ke = (a + nu b) / ((1 + nu)(2 nu - 1) 144): the oracle's quadrature Ke must
    reproduce every one of them (an off-diagonal sign or index error that kept
    symmetry and the rigid modes would still fail here)."""
    g = _golden()
    assert len(g["h8_a"]) == len(g["h8_b"]) == 24 * 25 // 2
    s = 1.0 / ((1 + NU) * (2 * NU - 1) * 144)
    ref = s * (np.array(g["h8_a"], float) + NU * np.array(g["h8_b"], float))
    Ke = O.element_stiffness(3, NU)
    np.testing.assert_allclose(O.lower_vector(Ke), ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.from_lower_vector(ref, 24), Ke, rtol=0, atol=1e-15)
    # the printed matrix also holds for another Poisson ratio (a and b separately)
    for nu in (0.0, 0.45):
        s2 = 1.0 / ((1 + nu) * (2 * nu - 1) * 144)
        ref2 = s2 * (np.array(g["h8_a"], float) + nu * np.array(g["h8_b"], float))
        np.testing.assert_allclose(O.lower_vector(O.element_stiffness(3, nu)), ref2, rtol=0, atol=1e-14)


def _rigid_modes(dim):
    X = O._local_node_coords(dim)
    modes = []
    for c in range(dim):
        m = np.zeros((X.shape[0], dim))
        m[:, c] = 1.0
        modes.append(m.ravel())
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (0, 2)]
    for a, b in pairs:
        m = np.zeros((X.shape[0], dim))
        m[:, a] = -X[:, b]
        m[:, b] = X[:, a]
        modes.append(m.ravel())
    return np.array(modes).T


@pytest.mark.parametrize("dim,nnull", [(2, 3), (3, 6)])
def test_ke_symmetric_psd_rigid_null_space(dim, nnull):
    Ke = O.element_stiffness(dim, NU)
    assert np.array_equal(Ke, Ke.T) or np.abs(Ke - Ke.T).max() < 1e-16
    ev = np.linalg.eigvalsh(Ke)
    assert ev.min() > -1e-14
    assert int(np.sum(np.abs(ev) < 1e-12)) == nnull
    R = _rigid_modes(dim)
    assert np.abs(Ke @ R).max() < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_ke_uniform_strain_energy(dim):
    """A linear displacement field u = G X is reproduced exactly by the element,
    so u^T Ke u = eps : C : eps times the unit volume (plane stress in 2D)."""
    rng = np.random.default_rng(1)
    Gm = rng.standard_normal((dim, dim))
    X = O._local_node_coords(dim)
    u = (X @ Gm.T).ravel()
    eps = 0.5 * (Gm + Gm.T)
    if dim == 2:
        E = 1.0
        sxx = E / (1 - NU ** 2) * (eps[0, 0] + NU * eps[1, 1])
        syy = E / (1 - NU ** 2) * (eps[1, 1] + NU * eps[0, 0])
        sxy = E / (2 * (1 + NU)) * 2 * eps[0, 1]
        energy = sxx * eps[0, 0] + syy * eps[1, 1] + 2 * sxy * eps[0, 1]
    else:
        lam = NU / ((1 + NU) * (1 - 2 * NU))
        mu = 1 / (2 * (1 + NU))
        sig = lam * np.trace(eps) * np.eye(3) + 2 * mu * eps
        energy = float(np.sum(sig * eps))
    Ke = O.element_stiffness(dim, NU)
    assert abs(u @ Ke @ u - energy) < 1e-13 * max(1.0, abs(energy))


@pytest.mark.parametrize("nu", [0.1, 0.3, 0.45])
def test_h8_ke_reflection_symmetry_and_walsh_blocks(nu):
    """An isotropic cube element is unchanged by the reflections x -> 1 - x (and
    y, z), which permute the corners and flip the reflected displacement
    component. Consequently Ke is block diagonal in the Walsh basis of the
    corners: mode c of component i only couples to modes c' of components j with
    c xor e_i = c' xor e_j (eight 3x3 blocks), and the constant modes are null."""
    Ke = O.element_stiffness(3, nu)
    X = O._local_node_coords(3).astype(int)
    key = {tuple(p): a for a, p in enumerate(X)}
    for axis in range(3):
        P = np.zeros((24, 24))
        for a, p in enumerate(X):
            q = p.copy()
            q[axis] = 1 - q[axis]
            b = key[tuple(q)]
            for i in range(3):
                P[3 * b + i, 3 * a + i] = -1.0 if i == axis else 1.0
        assert np.abs(P @ Ke @ P.T - Ke).max() < 1e-15
    H = np.zeros((24, 24))
    for c in range(8):
        cv = np.array([c >> 2, (c >> 1) & 1, c & 1])
        for a, p in enumerate(X):
            for i in range(3):
                H[3 * c + i, 3 * a + i] = (-1.0) ** int(cv @ p)
    M = H @ Ke @ H.T / 64
    np.testing.assert_allclose(H.T @ M @ H, Ke, atol=1e-15)
    char = [(c ^ (4 >> i)) for c in range(8) for i in range(3)]
    off = max(abs(M[r, s]) for r in range(24) for s in range(24) if char[r] != char[s])
    assert off < 1e-15 * np.abs(M).max()
    assert np.abs(M[:3, :]).max() < 1e-15 and np.abs(M[:, :3]).max() < 1e-15


# --------------------------------------------------------------- assembly --

@pytest.mark.parametrize("shape", [(4, 3, 0), (3, 2, 2)])
def test_lower_assembly_recovers_bruteforce_full_matrix(shape):
    """Eq. (11): K = K^(s) + K^(s)^T - diag K^(s) equals element-by-element dense
    assembly; K^(s) is lower triangular; I_r has m d(d+1)/2 entries (Table 1)."""
    g = O.Grid(*shape)
    Ke = O.element_stiffness(g.dim, NU)
    E = I.random_design(g.nel, 3) + 0.1
    iK, jK, _, _ = O.reduced_index_set(g)
    assert len(iK) == g.nel * g.d * (g.d + 1) // 2
    assert np.all(iK >= jK)
    Ks = O.assemble_lower(g, Ke, E)
    assert sp_is_lower(Ks)
    K = O.full_from_lower(Ks).toarray()
    Kb = np.zeros((g.ndof, g.ndof))
    C = O.element_dofs(g)
    for e in range(g.nel):
        for a in range(g.d):
            for b in range(g.d):
                Kb[C[e, a], C[e, b]] += E[e] * Ke[a, b]
    np.testing.assert_allclose(K, Kb, rtol=0, atol=1e-14)


def sp_is_lower(Ks):
    c = Ks.tocoo()
    return bool(np.all(c.row >= c.col))


def test_table1_index_counts():
    """Table 1 (H strategy): |I_r| = m d(d+1)/2; 2D 100^2 -> 360,000 and 3D 16^3 ->
    1,228,800 pairs (the paper's 3D 16^3 entry counts both index columns)."""
    assert 100 * 100 * 8 * 9 // 2 == 360000
    assert 16 ** 3 * 24 * 25 // 2 * 2 == 2457600


def test_connectivity_matches_paper_offsets():
    """Appendix B: cMat = cVec + [0, 1, 2nely+2, 2nely+3, 2nely, 2nely+1, -2, -1]
    with cVec = 2 nodeNrs + 1 (1-based); Appendix C similarly for 3D."""
    nelx, nely = 5, 3
    g = O.Grid(nelx, nely)
    C = O.element_dofs(g) + 1  # to 1-based
    for ix in range(nelx):
        for iy in range(nely):
            n1 = iy + (nely + 1) * ix + 1  # 1-based node number of the top-left node
            cvec = 2 * n1 + 1
            off = [0, 1, 2 * nely + 2, 2 * nely + 3, 2 * nely, 2 * nely + 1, -2, -1]
            assert list(C[iy + nely * ix]) == [cvec + o for o in off]
    nelx, nely, nelz = 3, 2, 2
    g = O.Grid(nelx, nely, nelz)
    C = O.element_dofs(g) + 1
    a = 3 * (nely + 1) * (nelz + 1)
    b = 3 * (nely + 1)
    c = 3 * (nely + 1) * (nelz + 2)
    off = [0, 1, 2, a, a + 1, a + 2, a - 3, a - 2, a - 1, -3, -2, -1,
           b, b + 1, b + 2, c, c + 1, c + 2, c - 3, c - 2, c - 1, b - 3, b - 2, b - 1]
    for ix in range(nelx):
        for iz in range(nelz):
            for iy in range(nely):
                n1 = iy + (nely + 1) * (iz + (nelz + 1) * ix) + 1
                e = iy + nely * (iz + nelz * ix)
                assert list(C[e]) == [3 * n1 + 1 + o for o in off]


@pytest.mark.parametrize("shape", [(6, 4, 0), (3, 3, 2)])
def test_patch_test_linear_field(shape):
    """Homogeneous grid, linear displacement field: interior nodal forces vanish."""
    g = O.Grid(*shape)
    Ke = O.element_stiffness(g.dim, NU)
    rng = np.random.default_rng(5)
    Gm = rng.standard_normal((g.dim, g.dim))
    coords = []
    for n in range(g.nnodes):
        if g.dim == 2:
            ix, iy = divmod(n, g.nely + 1)
            coords.append((ix, -iy))
        else:
            ix, rem = divmod(n, (g.nely + 1) * (g.nelz + 1))
            iz, iy = divmod(rem, g.nely + 1)
            coords.append((ix, -iy, iz))
    Xn = np.array(coords, float)
    u = (Xn @ Gm.T).ravel()
    y = O.apply_K(g, Ke, np.ones(g.nel), u)
    interior = []
    for n, X in enumerate(coords):
        lim = [g.nelx, g.nely] + ([g.nelz] if g.dim == 3 else [])
        absX = [abs(v) for v in X]
        if all(0 < a < l for a, l in zip(absX, lim)):
            interior.extend(range(g.dim * n, g.dim * n + g.dim))
    assert len(interior) > 0
    assert np.abs(y[interior]).max() < 1e-13


def test_rigid_modes_in_null_space_of_assembled_K():
    g = O.Grid(4, 3, 2)
    Ke = O.element_stiffness(3, NU)
    E = I.random_design(g.nel, 7) + 0.01
    K = O.full_from_lower(O.assemble_lower(g, Ke, E))
    for c in range(3):
        t = np.zeros(g.ndof)
        t[c::3] = 1.0
        assert np.abs(K @ t).max() < 1e-13


def test_apply_K_rows_matches_assembled_product():
    g = O.Grid(5, 4, 3)
    Ke = O.element_stiffness(3, NU)
    E = I.random_design(g.nel, 11)
    u = I.random_vector(g.ndof, 12)
    _, fixed = I.cantilever_3d(5, 4, 3)
    y = O.apply_K(g, Ke, E, u, fixed)
    rows = np.arange(0, g.ndof, 7)
    np.testing.assert_allclose(O.apply_K_rows(g, Ke, E, u, rows, fixed), y[rows],
                               rtol=0, atol=1e-13)


# ------------------------------------------------------------------ solve --

def test_uniaxial_bar_exact_solution():
    """Plane-stress block under uniform tension: the exact displacement field is
    linear, so the Q4 solution equals it to rounding."""
    nelx, nely = 8, 4
    g = O.Grid(nelx, nely)
    Ke = O.element_stiffness(2, NU)
    F = np.zeros(g.ndof)
    fixed = np.zeros(g.ndof, np.uint8)
    sigma = 1.0
    for iy in range(nely + 1):
        fixed[2 * g.node(iy, 0)] = 1
        w = 0.5 if iy in (0, nely) else 1.0
        F[2 * g.node(iy, nelx)] = sigma * w
    fixed[2 * g.node(nely, 0) + 1] = 1  # bottom-left node: no vertical motion
    U = O.solve_direct(g, Ke, np.ones(g.nel), F, fixed)
    for ix in range(nelx + 1):
        for iy in range(nely + 1):
            n = g.node(iy, ix)
            X, Y = ix, nely - iy  # height above the bottom edge
            assert abs(U[2 * n] - sigma * X) < 1e-11
            assert abs(U[2 * n + 1] + NU * sigma * Y) < 1e-11


@pytest.mark.parametrize("shape", [(12, 6, 0), (4, 3, 3)])
def test_direct_solve_residual_and_compliance_identities(shape):
    g = O.Grid(*shape)
    Ke = O.element_stiffness(g.dim, NU)
    F, fixed = I.mbb_half_beam(g.nelx, g.nely) if g.dim == 2 else \
        I.cantilever_3d(g.nelx, g.nely, g.nelz)
    E = O.simp_modulus(I.random_design(g.nel, 2), 3.0)
    U = O.solve_direct(g, Ke, E, F, fixed)
    K = O.full_from_lower(O.assemble_lower(g, Ke, E))
    free = ~fixed.astype(bool)
    r = (K @ U - F)[free]
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(F)
    assert np.all(U[~free] == 0)
    c1 = F @ U
    c2 = U @ (K @ U)
    c3 = np.sum(E * O.element_energy(g, Ke, U))
    assert abs(c1 - c2) <= 1e-9 * abs(c1)
    assert abs(c1 - c3) <= 1e-9 * abs(c1)
    # homogeneous scaling: K(s E) U = F  ->  c scales as 1/s
    U2 = O.solve_direct(g, Ke, 4.0 * E, F, fixed)
    assert abs(4.0 * (F @ U2) - c1) <= 1e-9 * abs(c1)


def test_pcg_matches_direct():
    g = O.Grid(16, 8)
    Ke = O.element_stiffness(2, NU)
    F, fixed = I.mbb_half_beam(16, 8)
    E = O.simp_modulus(I.random_design(g.nel, 9), 3.0)
    Ud = O.solve_direct(g, Ke, E, F, fixed)
    Up, it, rel = O.solve_pcg(g, Ke, E, F, fixed, rtol=1e-13)
    assert rel <= 1e-13
    assert np.linalg.norm(Up - Ud) <= 1e-7 * np.linalg.norm(Ud)


def test_pcg_threaded_products_are_bitwise_the_same():
    """The row-block threaded matrix product changes only the execution: the
    iterates, iteration count and residual equal the one-thread run bit for bit."""
    g = O.Grid(10, 5, 5)
    Ke = O.element_stiffness(3, NU)
    F, fixed = I.cantilever_3d(10, 5, 5)
    E = O.simp_modulus(I.random_design(g.nel, 4), 3.0)
    U1, it1, rel1 = O.solve_pcg(g, Ke, E, F, fixed, rtol=1e-10)
    U4, it4, rel4 = O.solve_pcg(g, Ke, E, F, fixed, rtol=1e-10, threads=4)
    assert it1 == it4 and rel1 == rel4
    np.testing.assert_array_equal(U1, U4)


# ----------------------------------------------------------------- filter --

def _dense(op, n):
    return np.column_stack([op(np.eye(n)[:, k]) for k in range(n)])


@pytest.mark.parametrize("shape,rmin,bc", [((7, 5, 0), 2.4, "N"), ((7, 5, 0), 2.4, "D"),
                                           ((4, 3, 3), math.sqrt(3), "N"),
                                           ((3, 2, 0), 3.5, "N")])
def test_filter_symmetric_and_row_sums(shape, rmin, bc):
    """V2: with mirror padding A is symmetric with constant row sums; with zero
    padding A is symmetric and its row sums vary. A^T is the explicit scatter."""
    g = O.Grid(*shape)
    A = _dense(lambda v: O.filter_A(g, v, rmin, bc), g.nel)
    AT = _dense(lambda v: O.filter_AT(g, v, rmin, bc), g.nel)
    np.testing.assert_allclose(AT, A.T, rtol=0, atol=1e-13)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-13)
    offs, w = O.filter_offsets(rmin, g.dim)
    rs = A.sum(axis=1)
    if bc == "N":
        np.testing.assert_allclose(rs, w.sum(), rtol=1e-14)
    else:
        assert rs.max() - rs.min() > 1e-3


@pytest.mark.parametrize("shape,rmin,bc", [((9, 6, 0), 2.4, "N"), ((9, 6, 0), 3.0, "D"),
                                           ((5, 4, 3), math.sqrt(3), "N"),
                                           ((5, 4, 3), 2.2, "D"), ((3, 2, 0), 4.5, "N")])
def test_filter_equals_scipy_ndimage_correlate(shape, rmin, bc):
    """A x equals scipy.ndimage.correlate with the cone kernel: mode 'reflect'
    (border-duplicating mirror, repeated) for 'N', zero 'constant' for 'D'."""
    g = O.Grid(*shape)
    x = I.random_design(g.nel, 4)
    offs, w = O.filter_offsets(rmin, g.dim)
    R = int(math.ceil(rmin)) - 1
    k = np.zeros((2 * R + 1,) * g.dim)
    for o, wo in zip(offs, w):
        k[tuple(oo + R for oo in o)] = wo
    mode = "reflect" if bc == "N" else "constant"
    ref = ndi.correlate(x.reshape(g.shape), k, mode=mode, cval=0.0).ravel()
    np.testing.assert_allclose(O.filter_A(g, x, rmin, bc), ref, rtol=0, atol=1e-12)


def test_filter_invariants():
    g = O.Grid(12, 7)
    c = np.full(g.nel, 0.37)
    np.testing.assert_allclose(O.filter_forward(g, c, 2.4, "N"), c, rtol=1e-14)
    np.testing.assert_allclose(O.filter_forward(g, c, 2.4, "D"), c, rtol=1e-14)
    x = I.random_design(g.nel, 8)
    assert abs(O.filter_forward(g, x, 2.4, "N").mean() - x.mean()) < 1e-14
    # rmin <= 1: window of one element -> identity
    np.testing.assert_array_equal(O.filter_forward(g, x, 1.0, "N"), x)
    np.testing.assert_allclose(O.filter_forward(g, x, 0.7, "D"), x, rtol=2e-16, atol=0)


def test_window_weights_3d_corners_zero():
    """rmin = sqrt(3): the 27-point window has 19 nonzero weights; the 8 corners
    sit exactly at distance rmin."""
    offs, w = O.filter_offsets(math.sqrt(3), 3)
    assert len(offs) == 27 and int(np.sum(w > 0)) == 19


# ------------------------------------------------------------- projection --

def test_projection_identities_and_derivatives():
    x = np.linspace(0.0, 1.0, 41)
    for beta in (1.0, 2.0, 8.0, 16.0):
        for eta in (0.3, 0.5, 0.62):
            assert abs(O.prj(np.array(0.0), eta, beta)) < 1e-15
            assert abs(O.prj(np.array(1.0), eta, beta) - 1.0) < 1e-15
            h = 1e-6
            fd = (O.prj(x + h, eta, beta) - O.prj(x - h, eta, beta)) / (2 * h)
            np.testing.assert_allclose(O.dprj(x, eta, beta), fd, rtol=1e-6, atol=1e-7)
            fde = (O.prj(x, eta + h, beta) - O.prj(x, eta - h, beta)) / (2 * h)
            np.testing.assert_allclose(O.deta(x, eta, beta), fde, rtol=1e-6, atol=1e-7)
            # closed form of the eta-derivative: -beta sech^2(beta(x-eta))
            # sinh(beta x) sinh(beta(1-x)) / sinh(beta)
            cf = -beta / np.cosh(beta * (x - eta)) ** 2 * np.sinh(beta * x) * \
                np.sinh(beta * (1 - x)) / np.sinh(beta)
            np.testing.assert_allclose(O.deta(x, eta, beta), cf, rtol=1e-11, atol=1e-13)


def test_eta_newton_special_cases():
    xt = np.full(100, 0.5)
    eta, _ = O.eta_newton(xt, 0.3, 8.0, 0.5, tol=1e-14)
    assert abs(eta - 0.5) < 1e-12
    xt = I.random_design(500, 3)
    vf = xt.mean()
    eta, it = O.eta_newton(xt, 0.5, 4.0, vf, tol=1e-14)
    assert abs(np.mean(O.prj(xt, eta, 4.0)) - vf) <= 1e-14
    # g(eta) is decreasing (Sec. 3.2): root unique
    etas = np.linspace(0.01, 0.99, 50)
    g = [np.mean(O.prj(xt, e, 4.0)) for e in etas]
    assert np.all(np.diff(g) < 0)


# ---------------------------------------------------------- sensitivities --

@pytest.mark.parametrize("shape", [(6, 3, 0), (3, 2, 2)])
def test_compliance_gradient_wrt_xphys_central_fd(shape):
    g = O.Grid(*shape)
    Ke = O.element_stiffness(g.dim, NU)
    F, fixed = I.mbb_half_beam(g.nelx, g.nely) if g.dim == 2 else \
        I.cantilever_3d(g.nelx, g.nely, g.nelz)
    xp = 0.2 + 0.7 * I.random_design(g.nel, 21)
    penal = 3.0

    def c_of(xv):
        U = O.solve_direct(g, Ke, O.simp_modulus(xv, penal), F, fixed)
        return F @ U

    U = O.solve_direct(g, Ke, O.simp_modulus(xp, penal), F, fixed)
    dc, c, _ = O.sensitivity(g, Ke, xp, U, F, penal)
    h = 1e-6
    fd = np.array([(c_of(xp + h * np.eye(g.nel)[e]) - c_of(xp - h * np.eye(g.nel)[e])) / (2 * h)
                   for e in range(g.nel)])
    assert np.linalg.norm(dc - fd) <= 1e-6 * np.linalg.norm(fd)


@pytest.mark.parametrize("shape,rmin", [((8, 4, 0), 1.6), ((3, 2, 2), 1.5)])
def test_design_gradient_through_filter_and_projection(shape, rmin):
    """Reading R1: H^T(dprj * dc/dxhat) is the exact gradient (eta frozen)."""
    g = O.Grid(*shape)
    Ke = O.element_stiffness(g.dim, NU)
    F, fixed = I.mbb_half_beam(g.nelx, g.nely) if g.dim == 2 else \
        I.cantilever_3d(g.nelx, g.nely, g.nelz)
    x = 0.2 + 0.6 * I.random_design(g.nel, 31)
    eta, beta, penal = 0.45, 4.0, 3.0

    def c_of(xv):
        xp = O.prj(O.filter_forward(g, xv, rmin, "N"), eta, beta)
        U = O.solve_direct(g, Ke, O.simp_modulus(xp, penal), F, fixed)
        return F @ U

    xt = O.filter_forward(g, x, rmin, "N")
    xp = O.prj(xt, eta, beta)
    U = O.solve_direct(g, Ke, O.simp_modulus(xp, penal), F, fixed)
    dc, _, _ = O.sensitivity(g, Ke, xp, U, F, penal)
    grad = O.filter_backward(g, dc, rmin, "N", O.dprj(xt, eta, beta))
    h = 1e-6
    fd = np.array([(c_of(x + h * np.eye(g.nel)[e]) - c_of(x - h * np.eye(g.nel)[e])) / (2 * h)
                   for e in range(g.nel)])
    assert np.linalg.norm(grad - fd) <= 1e-6 * np.linalg.norm(fd)
    # the order printed in Eq. (7) is not the gradient
    wrong = O.dprj(xt, eta, beta) * O.filter_backward(g, dc, rmin, "N")
    assert np.linalg.norm(wrong - fd) > 1e-3 * np.linalg.norm(fd)


# --------------------------------------------------------------------- OC --

def test_oc_volume_limits_and_lambda_bracket():
    n = 400
    rng = np.random.default_rng(2)
    x = 0.5 * np.ones(n)
    dc = -rng.random(n) * 10
    dV0 = np.full(n, 1.0 / (n * 0.5))
    act = np.ones(n, bool)
    xn, lm, steps = O.oc_update(x, dc, dV0, act, 0.2, 0.5, tol=1e-15)
    assert abs(xn.mean() - 0.5) <= 1e-12
    assert np.all(xn >= np.maximum(0, x - 0.2) - 1e-15)
    assert np.all(xn <= np.minimum(1, x + 0.2) + 1e-15)
    assert steps <= 200
    # lambda# (Eq. 17): without active bounds the unclamped mean equals volfrac
    ocP = x * np.sqrt(-dc / dV0)
    lam_sharp = np.mean(ocP) / 0.5
    assert abs(np.mean(ocP / lam_sharp) - 0.5) < 1e-15


@pytest.mark.parametrize("seed,with_passive", [(0, False), (1, False), (2, True), (3, True)])
def test_oc_primal_dual_equals_bisection(seed, with_passive):
    """The explicit primal-dual OC (Appendix A) solves the volume equation the
    bisection solves: same lm and design as a bisection run to 1e-15, the volume
    met exactly, the move and box limits kept, and few iterations."""
    r = np.random.default_rng(seed)
    n = 500
    x = np.clip(r.uniform(0.0, 1.0, n), 0.0, 1.0)
    dc = -np.exp(r.normal(0.0, 2.0, n))          # compliance sensitivities are negative
    dV0 = np.full(n, 1.0 / (n * 0.4)) * r.uniform(0.5, 1.5, n)
    act = np.ones(n, bool)
    if with_passive:
        act[r.choice(n, 40, replace=False)] = False
    xb, lmb, _ = O.oc_update(x, dc, dV0, act, 0.2, 0.4, tol=1e-15, maxit=400)
    xp, lmp, it = O.oc_update_primal_dual(x, dc, dV0, act, 0.2, 0.4)
    assert it <= 30
    assert abs(lmp - lmb) <= 1e-9 * lmb
    assert np.abs(xp - xb).max() <= 1e-9
    assert abs(np.mean(xp) - 0.4) <= 1e-12
    assert np.all(xp[act] >= np.maximum(x[act] - 0.2, 0.0) - 1e-15)
    assert np.all(xp[act] <= np.minimum(x[act] + 0.2, 1.0) + 1e-15)
    np.testing.assert_array_equal(xp[~act], x[~act])


def test_oc_primal_dual_special_cases():
    """No sensitivity: the design stays. Every element free of its limits: one
    closed-form step gives x_e = ocP_e / lm with mean exactly the volume fraction."""
    n = 64
    x = np.full(n, 0.5)
    xn, lm, it = O.oc_update_primal_dual(x, np.zeros(n), np.full(n, 1.0), np.ones(n, bool), 0.2, 0.5)
    assert lm == 0.0 and it == 0
    np.testing.assert_array_equal(xn, x)
    r = np.random.default_rng(9)
    dc = -r.uniform(0.9, 1.1, n)   # sensitivities close to each other: no element reaches a limit
    xn, lm, it = O.oc_update_primal_dual(x, dc, np.full(n, 1.0), np.ones(n, bool), 0.2, 0.5)
    ocP = x * np.sqrt(-dc)
    np.testing.assert_allclose(xn, ocP / lm, rtol=1e-15)
    assert abs(np.mean(xn) - 0.5) <= 1e-15
    assert abs(lm - np.sum(ocP) / (0.5 * n)) <= 1e-15 * lm


def test_oc_filtered_reduces_to_bisection_and_meets_physical_volume():
    """The general OC variant (volume on the filtered/projected candidate): with
    an identity filter (rmin <= 1) and no projection it is the plain bisection,
    value for value; with a real filter and a fixed-threshold projection the
    physical volume meets volfrac to the bracket tolerance, the move limits hold
    and passive elements keep their densities."""
    g = O.Grid(30, 20)
    r = np.random.default_rng(4)
    n = g.nel
    x = np.clip(0.3 + 0.2 * r.standard_normal(n), 0.0, 1.0)
    dc = -np.abs(r.standard_normal(n)) * 10 ** r.uniform(-3, 1, n)
    dV0 = np.full(n, 1.0 / (n * 0.3))
    act = np.ones(n, bool)
    xa, la, sa = O.oc_update(x, dc, dV0, act, 0.2, 0.3, tol=1e-12)
    xb, lb, sb = O.oc_update_filtered(g, x, dc, dV0, act, 0.2, 0.3, 0.9, "N", 1, 0.5, 2.0, tol=1e-12)
    np.testing.assert_array_equal(xa, xb)
    assert la == lb and sa == sb
    pas = np.zeros(n, np.int8)
    pas[:20], pas[20:40] = 1, -1
    x[pas == 1], x[pas == -1] = 1.0, 0.0
    act = pas == 0
    xn, lm, steps = O.oc_update_filtered(g, x, dc, dV0, act, 0.2, 0.3, 2.5, "N", 2, 0.4, 4.0, pas, tol=1e-15)
    xf = O.filter_forward(g, xn, 2.5, "N")
    xf[pas == 1], xf[pas == -1] = 1.0, 0.0
    assert abs(np.mean(O.prj(xf, 0.4, 4.0)) - 0.3) <= 1e-12
    assert np.all(xn[act] >= np.maximum(x[act] - 0.2, 0.0) - 1e-15)
    assert np.all(xn[act] <= np.minimum(x[act] + 0.2, 1.0) + 1e-15)
    np.testing.assert_array_equal(xn[~act], x[~act])


def test_pae_extrapolation_reaches_the_fixed_point_of_an_affine_map():
    """On an affine contraction U(x) = A x + c the extrapolation step is a
    GMRES-like minimal-residual step: with as many history columns as
    dimensions it lands on the fixed point (I - A)^-1 c exactly (up to
    rounding); the damped steps are x + alpha r."""
    r = np.random.default_rng(5)
    n = 3
    A = 0.3 * r.standard_normal((n, n)) / n
    c = 0.2 + 0.1 * r.random(n)
    xstar = np.linalg.solve(np.eye(n) - A, c)
    assert np.all((xstar > 0) & (xstar < 1))
    h = {}
    x = np.full(n, 0.5)
    for it in range(4):  # q = 4, m = 3: steps 0..2 damped, step 3 extrapolated
        res = A @ x + c - x
        xn, kind = O.pae_update(h, x, res, it, 3, 4, 0.9, 1.0)
        if it < 3:
            assert kind == 1
            np.testing.assert_allclose(xn, np.clip(x + 0.9 * res, 0, 1), rtol=0, atol=1e-15)
        else:
            assert kind == 2
            np.testing.assert_allclose(xn, xstar, rtol=0, atol=1e-12)
        x = xn


def test_solve_small_matches_numpy_and_flags_singular():
    r = np.random.default_rng(6)
    B = r.standard_normal((4, 4))
    G = B.T @ B + 0.1 * np.eye(4)
    b = r.standard_normal(4)
    np.testing.assert_allclose(O.solve_small(G, b), np.linalg.solve(G, b), rtol=1e-12)
    S = np.outer([1.0, 2.0, 3.0], [1.0, 2.0, 3.0])
    assert O.solve_small(S, np.ones(3)) is None


def test_oc_paper_mode_step_count():
    """Sec. 3.3: with the lambda# bracket ~14 bisection steps at tol 1e-4."""
    n = 1200
    rng = np.random.default_rng(4)
    x = rng.uniform(0.2, 0.8, n)
    x *= 0.5 / x.mean()
    dc = -rng.random(n)
    dV0 = np.full(n, 1.0 / (n * 0.5))
    _, _, steps = O.oc_update(x, dc, dV0, np.ones(n, bool), 0.2, 0.5, tol=1e-4)
    assert 10 <= steps <= 16


def test_continuation_schedules():
    p = 1.0
    seq = []
    for loop in range(1, 201):
        p = O.continuation(p, (1, 3.0, 25, 0.25), loop, "add")
        seq.append(p)
    assert seq[23] == 1.0 and seq[24] == 1.25 and seq[199] == 3.0
    b = 2.0
    for loop in range(1, 101):
        b = O.continuation(b, (1, 16.0, 25, 2.0), loop, "mul")
    assert b == 16.0


# ------------------------------------------------------ end-to-end (soft) --

def test_mbb_60x20_behaviour():
    """Sec. 3.2/3.3 soft checks on the paper's MBB: 1-2 Newton steps, eta* in
    [0.4, 0.52], about 14 bisections, volume held at volfrac."""
    p = O.Params(60, 20, volfrac=0.5, penal=3.0, rmin=2.4, beta=2.0)
    F, fixed = I.mbb_half_beam(60, 20)
    s = O.run(p, F, fixed, maxit=20)
    for h in s.history[1:]:
        assert 1 <= h["n_newton"] <= 3
        assert 0.4 <= h["eta"] <= 0.52
        assert 11 <= h["n_bisect"] <= 16
        assert abs(h["V"] - 0.5) < 1e-5
    c = [h["c"] for h in s.history]
    assert c[-1] < 0.5 * c[0]


def test_parity_mode_is_deterministic():
    p = O.Params.parity(nelx=20, nely=10, volfrac=0.4, rmin=1.8)
    F, fixed = I.mbb_half_beam(20, 10)
    a = O.run(p, F, fixed, maxit=5)
    b = O.run(p, F, fixed, maxit=5)
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.xphys, b.xphys)
