"""Plain, slow FP64 CPU oracle of the SIMP design iteration (Ferrari & Sigmund 2020).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. It
shares no code with the CUDA path; its only input-side dependency is the seeded
problem-data module ``paper_2005_05436_gb300.inputs``, which holds no arithmetic
of the method.

Each function follows one passage of the paper (section / equation / appendix);
library primitives (scipy sparse assembly, LAPACK banded Cholesky) serve as
single steps. There is no blocking, fusion or reordering beyond what the
definitions state. Floating point is IEEE FP64 throughout.

Readings of silent, ambiguous or garbled passages (each one is listed in the
design notes of the repository as well):

R1  chain rule: dc/dx = H^T (dprj * dc/dxhat) in 2D and 3D (the 2D listing's
    order, which is the exact gradient; Eq. 7 and the 3D listing apply dprj
    after H^T).
R2  filter: xtilde = (A x) / Hs (Eq. 2 and the 2D listing), A the unnormalised
    cone-weight correlation, Hs = A 1.
R3  the sensitivities treat the volume-preserving eta as a constant (Sec. 3.2).
R4  eta* solves mean(prj(xtilde, eta)) = volfrac (the listings' target).
R5  tolerances: "paper" mode keeps Newton |g| <= 1e-6 and bisection
    (l2-l1)/(l1+l2) <= 1e-4; "parity" mode uses 1e-14 / 1e-15 so that
    summation-order differences cannot flip a branch by more than rounding.
    Newton is capped (50 steps) and falls back to bisection on eta in [0, 1];
    lambda bisection is capped at 200 steps.
R6  if the volume at the lambda# upper bracket still exceeds volfrac (move
    limits clamp), the bracket is doubled until it does not (cap 60).
R7  real(sqrt(.)) of the OC rule is sqrt(max(0, .)).
R8  a tie mean(x) == volfrac moves the upper end (strict ">" as the listing).
R9  continuation is additive (paper) or multiplicative (doubling), applied
    after the OC update with the post-increment loop counter.
R13 mirror padding wider than the grid repeats the reflection.
R14 ch = ||xPhys - xOld||_2 / sqrt(nEl) in 2D and 3D.
R19 "masked" K u: fixed DOFs of u are treated as 0 and fixed rows of y are 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

# ----------------------------------------------------------------------------
# Grid numbering (Sec. 3, PRE.2; Appendix B/C connectivity)
# ----------------------------------------------------------------------------


@dataclass
class Grid:
    nelx: int
    nely: int
    nelz: int = 0  # 0 = 2D

    @property
    def dim(self):
        return 3 if self.nelz else 2

    @property
    def nel(self):
        return self.nelx * self.nely * (self.nelz if self.nelz else 1)

    @property
    def nnodes(self):
        return (self.nelx + 1) * (self.nely + 1) * ((self.nelz + 1) if self.nelz else 1)

    @property
    def ndof(self):
        return self.dim * self.nnodes

    @property
    def d(self):
        """Local DOFs per element: 8 (Q4) or 24 (H8)."""
        return 8 if self.dim == 2 else 24

    @property
    def shape(self):
        """Element array shape in numpy C order: (nelx, nely) or (nelx, nelz, nely)."""
        if self.dim == 2:
            return (self.nelx, self.nely)
        return (self.nelx, self.nelz, self.nely)

    def node(self, iy, ix, iz=0):
        return iy + (self.nely + 1) * (iz + ((self.nelz + 1) if self.nelz else 1) * ix)


def element_nodes(g: Grid):
    """Local-to-global node table [nEl, 2^dim] (Appendix B/C, cMat).

    Local node order (physical X = ix, Y = -iy, Z = iz):
    2D: (0,0) (1,0) (1,1) (0,1) -> rows/cols (iy+1,ix) (iy+1,ix+1) (iy,ix+1) (iy,ix);
    3D: the same four at iz, then the same four at iz+1.
    """
    if g.dim == 2:
        ix, iy = np.meshgrid(np.arange(g.nelx), np.arange(g.nely), indexing="ij")
        ix, iy = ix.ravel(), iy.ravel()  # element e = iy + nely*ix (C order of (nelx, nely))
        cols = [(iy + 1, ix), (iy + 1, ix + 1), (iy, ix + 1), (iy, ix)]
        return np.stack([g.node(a, b) for a, b in cols], axis=1)
    ix, iz, iy = np.meshgrid(np.arange(g.nelx), np.arange(g.nelz), np.arange(g.nely),
                             indexing="ij")
    ix, iz, iy = ix.ravel(), iz.ravel(), iy.ravel()
    quad = [(1, 0), (1, 1), (0, 1), (0, 0)]  # (dy, dx) of the four nodes of one z-face
    cols = []
    for dz in (0, 1):
        for dy, dx in quad:
            cols.append(g.node(iy + dy, ix + dx, iz + dz))
    return np.stack(cols, axis=1)


def element_dofs(g: Grid):
    """Connectivity matrix C [nEl, d] of global DOFs (0-based), Eq. (9)."""
    nodes = element_nodes(g)
    dofs = nodes[:, :, None] * g.dim + np.arange(g.dim)[None, None, :]
    return dofs.reshape(g.nel, g.d)


# ----------------------------------------------------------------------------
# Element stiffness (Appendix B/C element matrices): 2x2 / 2x2x2 Gauss rule
# ----------------------------------------------------------------------------


def _local_node_coords(dim):
    if dim == 2:
        return np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    q = [[0, 0], [1, 0], [1, 1], [0, 1]]
    return np.array([[a, b, c] for c in (0, 1) for a, b in q], float)


def _shape_grad(xi, nodes):
    """Gradients of the multilinear shape functions on the unit cell at xi."""
    nn, dim = nodes.shape
    G = np.zeros((nn, dim))
    for a in range(nn):
        for k in range(dim):
            v = 1.0
            for m in range(dim):
                lin = xi[m] if nodes[a, m] == 1 else 1.0 - xi[m]
                if m == k:
                    v *= 1.0 if nodes[a, m] == 1 else -1.0
                else:
                    v *= lin
            G[a, k] = v
    return G


def element_stiffness(dim, nu=0.3, E=1.0):
    """Unit-element stiffness matrix Ke [d, d] by Gauss quadrature.

    2D: bilinear Q4, plane stress, unit thickness; 3D: trilinear H8, isotropic
    linear elasticity. Both on the unit square/cube with the local node order
    of ``element_nodes``, DOFs interleaved per node (X, Y[, Z]).
    """
    nodes = _local_node_coords(dim)
    nn = nodes.shape[0]
    d = dim * nn
    if dim == 2:
        D = E / (1 - nu ** 2) * np.array([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]])
    else:
        lam = E * nu / ((1 + nu) * (1 - 2 * nu))
        mu = E / (2 * (1 + nu))
        D = np.zeros((6, 6))
        D[:3, :3] = lam
        D[np.arange(3), np.arange(3)] += 2 * mu
        D[3:, 3:] = mu * np.eye(3)
    gp = [0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)]
    w = 1.0 / (2 ** dim)
    Ke = np.zeros((d, d))
    pts = [(a, b) for a in gp for b in gp] if dim == 2 else \
        [(a, b, c) for a in gp for b in gp for c in gp]
    for xi in pts:
        G = _shape_grad(np.array(xi), nodes)
        if dim == 2:
            B = np.zeros((3, d))
            for a in range(nn):
                B[0, 2 * a] = G[a, 0]
                B[1, 2 * a + 1] = G[a, 1]
                B[2, 2 * a] = G[a, 1]
                B[2, 2 * a + 1] = G[a, 0]
        else:
            B = np.zeros((6, d))
            for a in range(nn):
                gx, gy, gz = G[a]
                B[0, 3 * a] = gx
                B[1, 3 * a + 1] = gy
                B[2, 3 * a + 2] = gz
                B[3, 3 * a] = gy          # gamma_xy
                B[3, 3 * a + 1] = gx
                B[4, 3 * a + 1] = gz      # gamma_yz
                B[4, 3 * a + 2] = gy
                B[5, 3 * a] = gz          # gamma_xz
                B[5, 3 * a + 2] = gx
        Ke += w * B.T @ D @ B
    return Ke


def lower_vector(Ke):
    """Column-major lower triangle of Ke (the paper's storage V(K^(s)_e), Sec. 3.1)."""
    d = Ke.shape[0]
    return np.array([Ke[i, j] for j in range(d) for i in range(j, d)])


def from_lower_vector(v, d):
    """Full symmetric matrix from its column-major lower triangle (Appendix B, Ke0)."""
    L = np.zeros((d, d))
    k = 0
    for j in range(d):
        for i in range(j, d):
            L[i, j] = v[k]
            k += 1
    return L + L.T - np.diag(np.diag(L))


# ----------------------------------------------------------------------------
# SIMP interpolation (Eq. 5) and assembly of the lower triangle (Sec. 3.1)
# ----------------------------------------------------------------------------


def simp_modulus(xphys, penal, E0=1.0, Emin=1e-9):
    """E(xhat) = Emin + xhat^p (E0 - Emin), Eq. (5)."""
    return Emin + xphys ** penal * (E0 - Emin)


def reduced_index_set(g: Grid):
    """I_r of Eq. (10): pairs (iK >= jK) of the element lower triangles, plus the
    local (i, j) pair of each entry, in column-major lower order."""
    C = element_dofs(g)
    d = g.d
    sI = np.array([i for j in range(d) for i in range(j, d)])
    sII = np.array([j for j in range(d) for i in range(j, d)])
    iK = C[:, sI]
    jK = C[:, sII]
    hi = np.maximum(iK, jK)
    lo = np.minimum(iK, jK)
    return hi.ravel(), lo.ravel(), sI, sII


def assemble_lower(g: Grid, Ke, E):
    """K^(s): lower triangle of K(xhat) assembled from I_r (Eq. 10), CSR, duplicates
    summed, sorted column indices. Fixed DOFs are kept."""
    iK, jK, _, _ = reduced_index_set(g)
    sK = (lower_vector(Ke)[None, :] * E[:, None]).ravel()
    Ks = sp.coo_matrix((sK, (iK, jK)), shape=(g.ndof, g.ndof)).tocsr()
    Ks.sum_duplicates()
    Ks.sort_indices()
    return Ks


def full_from_lower(Ks):
    """K = K^(s) + K^(s)^T - diag K^(s), Eq. (11)."""
    return (Ks + Ks.T - sp.diags(Ks.diagonal())).tocsr()


def apply_K(g: Grid, Ke, E, u, fixed=None):
    """y = K(xhat) u through the assembled matrix; with ``fixed``, the masked
    product of reading R19 (u_fixed treated as 0, y_fixed = 0)."""
    K = full_from_lower(assemble_lower(g, Ke, E))
    u = np.array(u, float)
    if fixed is not None:
        u[fixed.astype(bool)] = 0.0
    y = K @ u
    if fixed is not None:
        y[fixed.astype(bool)] = 0.0
    return y


def apply_K_rows(g: Grid, Ke, E, u, rows, fixed=None):
    """Selected rows of K u summed element by element (for grids too large to
    assemble in a test): y_r = sum_{e containing r} E_e Ke[loc(r), :] u_e."""
    C = element_dofs(g)
    u = np.array(u, float)
    if fixed is not None:
        u[fixed.astype(bool)] = 0.0
    out = np.zeros(len(rows))
    dim = g.dim
    for k, r in enumerate(rows):
        node = r // dim
        # the elements around a node: brute-force over the node's coordinates
        if dim == 2:
            ix, iy = divmod(node, g.nely + 1)
            cand = [(ey, ex) for ex in (ix - 1, ix) for ey in (iy - 1, iy)
                    if 0 <= ex < g.nelx and 0 <= ey < g.nely]
            els = [ey + g.nely * ex for ey, ex in cand]
        else:
            nny, nnz = g.nely + 1, g.nelz + 1
            ix, rem = divmod(node, nny * nnz)
            iz, iy = divmod(rem, nny)
            els = [ey + g.nely * (ez + g.nelz * ex)
                   for ex in (ix - 1, ix) for ez in (iz - 1, iz) for ey in (iy - 1, iy)
                   if 0 <= ex < g.nelx and 0 <= ez < g.nelz and 0 <= ey < g.nely]
        s = 0.0
        for e in els:
            loc = int(np.nonzero(C[e] == r)[0][0])
            s += E[e] * float(Ke[loc] @ u[C[e]])
        out[k] = 0.0 if (fixed is not None and fixed[r]) else s
    return out


# ----------------------------------------------------------------------------
# State solve K(free, free) U = F (Eq. 4; Appendix B/C direct Cholesky)
# ----------------------------------------------------------------------------


def solve_direct(g: Grid, Ke, E, F, fixed):
    """Banded Cholesky of the lower triangle of K(free, free), then forward and
    backward substitution (LAPACK pbtrf / pbtrs). U[fixed] = 0."""
    Ks = assemble_lower(g, Ke, E)
    free = np.nonzero(~fixed.astype(bool))[0]
    Kff = Ks[free][:, free].tocoo()
    n = len(free)
    bw = int(np.max(Kff.row - Kff.col)) if Kff.nnz else 0
    ab = np.zeros((bw + 1, n))
    ab[Kff.row - Kff.col, Kff.col] = Kff.data
    cb = sla.cholesky_banded(ab, lower=True)
    U = np.zeros(g.ndof)
    U[free] = sla.cho_solve_banded((cb, True), F[free])
    return U


def _row_blocks_matvec(A, threads):
    """y = A x with the rows of the CSR matrix A split into `threads` blocks, one
    thread each (scipy's CSR product releases the GIL). Every row is summed by
    the same routine in the same order as the one-block product, so the result
    is bitwise that of A @ x; only the execution is parallel."""
    if threads <= 1:
        return lambda x: A @ x
    from concurrent.futures import ThreadPoolExecutor
    n = A.shape[0]
    cuts = [n * k // threads for k in range(threads + 1)]
    blocks = [A[cuts[k]:cuts[k + 1]] for k in range(threads)]
    pool = ThreadPoolExecutor(threads)

    def mv(x):
        out = np.empty(n)
        for k, y in enumerate(pool.map(lambda B: B @ x, blocks)):
            out[cuts[k]:cuts[k + 1]] = y
        return out
    return mv


def solve_pcg(g: Grid, Ke, E, F, fixed, rtol=1e-8, maxit=100000, U0=None, threads=1):
    """Jacobi-preconditioned CG on K(free, free) (used where a direct solve does
    not fit). threads > 1 runs the matrix products on that many host threads
    (bitwise the same iterates). Returns (U, iterations, relative residual)."""
    K = full_from_lower(assemble_lower(g, Ke, E))
    free = np.nonzero(~fixed.astype(bool))[0]
    Kff = K[free][:, free].tocsr()
    Kmv = _row_blocks_matvec(Kff, threads)
    b = F[free]
    x = np.zeros(len(free)) if U0 is None else np.array(U0[free], float)
    dinv = 1.0 / Kff.diagonal()
    r = b - Kmv(x)
    bn = np.linalg.norm(b)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    it = 0
    rel = np.linalg.norm(r) / bn if bn > 0 else 0.0
    while rel > rtol and it < maxit:
        Ap = Kmv(p)
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        it += 1
        rel = np.linalg.norm(r) / bn
        if rel <= rtol:
            break
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    U = np.zeros(g.ndof)
    U[free] = x
    return U, it, rel


# ----------------------------------------------------------------------------
# Density filter (Eq. 2; Sec. 3 PRE.5 and RL.1) with 'N' mirror or 'D' zero padding
# ----------------------------------------------------------------------------


def filter_offsets(rmin, dim):
    """Window offsets -ceil(rmin)+1 .. ceil(rmin)-1 per axis and cone weights
    h = max(0, rmin - |o|) (Eq. 2, element-centre distance). Offsets are in the
    axis order (x, y) or (x, z, y) of ``Grid.shape``."""
    R = int(math.ceil(rmin)) - 1
    rng = range(-R, R + 1)
    offs, w = [], []
    if dim == 2:
        for ox in rng:
            for oy in rng:
                offs.append((ox, oy))
                w.append(max(0.0, rmin - math.sqrt(ox * ox + oy * oy)))
    else:
        for ox in rng:
            for oz in rng:
                for oy in rng:
                    offs.append((ox, oz, oy))
                    w.append(max(0.0, rmin - math.sqrt(ox * ox + oy * oy + oz * oz)))
    return offs, np.array(w)


def _mirror(j, n):
    """Repeated mirror reflection with border duplication (R13)."""
    r = np.mod(j, 2 * n)
    return np.where(r < n, r, 2 * n - 1 - r)


def filter_A(g: Grid, x, rmin, bc="N"):
    """Unnormalised correlation A x: (A x)_e = sum_o h(o) x[e + o] with the
    padding rule of ``bc``."""
    X = np.asarray(x, float).reshape(g.shape)
    out = np.zeros_like(X)
    offs, w = filter_offsets(rmin, g.dim)
    n = X.shape
    for o, wo in zip(offs, w):
        if wo == 0.0:
            continue
        idx = []
        valid = []
        for a in range(len(n)):
            j = np.arange(n[a]) + o[a]
            if bc == "N":
                idx.append(_mirror(j, n[a]))
                valid.append(np.ones(n[a], bool))
            else:
                valid.append((j >= 0) & (j < n[a]))
                idx.append(np.clip(j, 0, n[a] - 1))
        vals = X[np.ix_(*idx)]
        if len(n) == 2:
            mask = valid[0][:, None] & valid[1][None, :]
        else:
            mask = valid[0][:, None, None] & valid[1][None, :, None] & valid[2][None, None, :]
        out += wo * np.where(mask, vals, 0.0)
    return out.ravel()


def filter_AT(g: Grid, y, rmin, bc="N"):
    """Transpose A^T y written as the explicit scatter of A (no symmetry assumed)."""
    Y = np.asarray(y, float).reshape(g.shape)
    out = np.zeros_like(Y)
    offs, w = filter_offsets(rmin, g.dim)
    n = Y.shape
    for o, wo in zip(offs, w):
        if wo == 0.0:
            continue
        idx = []
        valid = []
        for a in range(len(n)):
            j = np.arange(n[a]) + o[a]
            if bc == "N":
                idx.append(_mirror(j, n[a]))
                valid.append(np.ones(n[a], bool))
            else:
                valid.append((j >= 0) & (j < n[a]))
                idx.append(np.clip(j, 0, n[a] - 1))
        grids = np.meshgrid(*idx, indexing="ij")
        vgrid = np.meshgrid(*valid, indexing="ij")
        mask = np.logical_and.reduce(vgrid)
        np.add.at(out, tuple(gr[mask] for gr in grids), wo * Y[mask])
    return out.ravel()


def filter_Hs(g: Grid, rmin, bc="N"):
    """Hs = A 1, the normalising weights (Sec. 3 PRE.5)."""
    return filter_A(g, np.ones(g.nel), rmin, bc)


def filter_forward(g: Grid, x, rmin, bc="N"):
    """xtilde = (A x) / Hs, Eq. (2) (reading R2)."""
    return filter_A(g, x, rmin, bc) / filter_Hs(g, rmin, bc)


def filter_backward(g: Grid, grad, rmin, bc="N", dprj=None):
    """H^T (dprj * grad) = A^T (dprj * grad / Hs), the chain rule of Eq. (7) in
    the exact order (reading R1)."""
    s = np.asarray(grad, float)
    if dprj is not None:
        s = s * dprj
    return filter_AT(g, s / filter_Hs(g, rmin, bc), rmin, bc)


# ----------------------------------------------------------------------------
# Heaviside projection (Eq. 1, Eq. 8) and volume-preserving eta (Sec. 3.2)
# ----------------------------------------------------------------------------


def prj(x, eta, beta):
    """Relaxed Heaviside projection, Eq. (1)."""
    return (np.tanh(beta * eta) + np.tanh(beta * (x - eta))) / \
        (np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta)))


def dprj(x, eta, beta):
    """d prj / d xtilde, Eq. (8)."""
    return beta * (1.0 - np.tanh(beta * (x - eta)) ** 2) / \
        (np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta)))


def deta(x, eta, beta):
    """d prj / d eta by the quotient rule of Eq. (1) (the printed Eq. 16 is garbled)."""
    num = np.tanh(beta * eta) + np.tanh(beta * (x - eta))
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    sech2 = lambda a: 1.0 - np.tanh(a) ** 2
    dnum = beta * sech2(beta * eta) - beta * sech2(beta * (x - eta))
    dden = beta * sech2(beta * eta) - beta * sech2(beta * (1.0 - eta))
    return (dnum * den - num * dden) / den ** 2


def eta_newton(xt, eta, beta, volfrac, tol=1e-6, maxit=50):
    """Volume-preserving threshold (Eq. 15, Sec. 3.2): Newton on
    g(eta) = mean(prj(xt, eta)) - volfrac from the previous eta, with the
    derivative mean(deta); capped, and a step that leaves [0, 1] (or a
    non-finite g) hands over to bisection on [0, 1] (reading R5).
    Returns (eta, newton steps)."""
    f = np.mean(prj(xt, eta, beta)) - volfrac
    it = 0
    while abs(f) > tol and it < maxit:
        eta = eta - f / np.mean(deta(xt, eta, beta))
        it += 1
        if not 0.0 <= eta <= 1.0:  # a step out of [0, 1]: hand over to bisection
            break
        f = np.mean(prj(xt, eta, beta)) - volfrac
    if not (abs(f) <= tol and 0.0 <= eta <= 1.0):
        lo, hi = 0.0, 1.0  # g is decreasing in eta (Sec. 3.2)
        for _ in range(200):
            eta = 0.5 * (lo + hi)
            f = np.mean(prj(xt, eta, beta)) - volfrac
            if abs(f) <= tol or hi - lo <= 1e-16:
                break
            if f > 0:
                lo = eta
            else:
                hi = eta
            it += 1
    return eta, it


# ----------------------------------------------------------------------------
# Sensitivities (Eq. 6) and OC update (Eqs. 13-14, 17)
# ----------------------------------------------------------------------------


def element_energy(g: Grid, Ke, U):
    """ce_e = u_e^T Ke u_e (Appendix B, RL.3)."""
    Ue = U[element_dofs(g)]
    return np.sum((Ue @ Ke) * Ue, axis=1)


def sensitivity(g: Grid, Ke, xphys, U, F, penal, E0=1.0, Emin=1e-9, active=None):
    """dc/dxhat = -p (E0 - Emin) xhat^(p-1) u_e^T Ke u_e on active elements,
    0 on passive ones (Eq. 6); compliance c = F^T U (Eq. 3).
    Returns (dc, c, ce)."""
    ce = element_energy(g, Ke, U)
    dc = -penal * (E0 - Emin) * xphys ** (penal - 1.0) * ce
    if active is not None:
        dc = np.where(active, dc, 0.0)
    return dc, float(F @ U), ce


def oc_update(x, dc, dV0, active, move, volfrac, tol=1e-4, maxit=200):
    """OC rule (Eqs. 13-14) with lm = sqrt(lambda) found by bisection on the
    bracket [0, lambda#] of Eq. (17) (readings R6-R8).
    Returns (x_new, lm, bisection steps)."""
    x = np.array(x, float)
    act = np.asarray(active, bool)
    xT = x[act]
    xU, xL = xT + move, xT - move
    ocP = xT * np.sqrt(np.maximum(0.0, -dc[act] / dV0[act]))
    l1, l2 = 0.0, np.mean(ocP) / volfrac

    def update(lm):
        xn = x.copy()
        xn[act] = np.maximum(np.maximum(np.minimum(np.minimum(ocP / lm, xU), 1.0), xL), 0.0)
        return xn

    if not l2 > 0.0:
        return x, 0.0, 0
    # reading R6: grow the bracket while its upper end is still too small
    grow = 0
    while np.mean(update(l2)) > volfrac and grow < 60:
        l1, l2 = l2, 2.0 * l2
        grow += 1
    steps = 0
    lmid = l2
    xn = update(l2)
    while (l2 - l1) / (l1 + l2) > tol and steps < maxit:
        lmid = 0.5 * (l1 + l2)
        xn = update(lmid)
        if np.mean(xn) > volfrac:
            l1 = lmid
        else:
            l2 = lmid
        steps += 1
    return xn, lmid, steps


def oc_update_primal_dual(x, dc, dV0, active, move, volfrac, tol=1e-10, maxit=200):
    """Explicit primal-dual form of the same OC step (Appendix A: the primal map
    puts each active element at its move/box limit or at ocP / lm, the dual map
    solves the volume equation for lm = sqrt(lambda) in closed form over the
    resulting sets), started from the estimate lambda# of Eq. (17) and iterated
    until two iterates of lm differ by at most tol (reading R21: elements at a
    limit belong to that limit's set; passive elements keep their densities and
    their volume). Returns (x_new, lm, iterations)."""
    x = np.array(x, float)
    act = np.asarray(active, bool)
    xT = x[act]
    up = np.minimum(xT + move, 1.0)
    lo = np.maximum(xT - move, 0.0)
    ocP = xT * np.sqrt(np.maximum(0.0, -dc[act] / dV0[act]))
    n = x.size
    fixed_volume = float(np.sum(x[~act]))
    lm = np.mean(ocP) / volfrac
    if not lm > 0.0:
        return x, 0.0, 0
    it = 0
    while it < maxit:
        t = ocP / lm
        at_up = t >= up
        at_lo = (t <= lo) & ~at_up
        mid = ~(at_up | at_lo)
        num = float(np.sum(ocP[mid]))
        den = volfrac * n - float(np.sum(up[at_up])) - float(np.sum(lo[at_lo])) - fixed_volume
        it += 1
        if not (num > 0.0 and den > 0.0):
            break
        lm_new = num / den
        converged = abs(lm_new - lm) <= tol
        lm = lm_new
        if converged:
            break
    xn = x.copy()
    xn[act] = np.minimum(np.maximum(ocP / lm, lo), up)
    return xn, lm, it


def oc_update_filtered(g, x, dc, dV0, active, move, volfrac, rmin, bc, ft, eta, beta, passive=None,
                       tol=1e-4, maxit=200):
    """OC step whose volume test is taken on the physical field of each candidate
    (Sec. 3.2, the general variant for a fixed threshold): every bisection
    candidate x(lm) of Eq. (14) is filtered (Eq. 2), its passive elements are set
    to 1 (solid) and 0 (void), and it is projected (Eq. 1, threshold eta fixed)
    when ft > 1; lm moves up while the mean of that field exceeds volfrac. The
    bracket starts from lambda# (Eq. 17) and grows while its upper end still gives
    too much volume (reading R6). Returns (x_new, lm, bisection steps)."""
    x = np.array(x, float)
    act = np.asarray(active, bool)
    pas = np.zeros(x.size, np.int8) if passive is None else np.asarray(passive, np.int8)
    xT = x[act]
    xU, xL = xT + move, xT - move
    ocP = xT * np.sqrt(np.maximum(0.0, -dc[act] / dV0[act]))
    l1, l2 = 0.0, np.mean(ocP) / volfrac

    def update(lm):
        xn = x.copy()
        xn[act] = np.maximum(np.maximum(np.minimum(np.minimum(ocP / lm, xU), 1.0), xL), 0.0)
        return xn

    def physical_volume(xn):
        xf = filter_forward(g, xn, rmin, bc)
        xf[pas == 1] = 1.0
        xf[pas == -1] = 0.0
        if ft > 1:
            xf = prj(xf, eta, beta)
        return float(np.mean(xf))

    if not l2 > 0.0:
        return x, 0.0, 0
    grow = 0
    xn = update(l2)
    while physical_volume(xn) > volfrac and grow < 60:
        l1, l2 = l2, 2.0 * l2
        xn = update(l2)
        grow += 1
    steps = 0
    lmid = l2
    while (l2 - l1) / (l1 + l2) > tol and steps < maxit:
        lmid = 0.5 * (l1 + l2)
        xn = update(lmid)
        if physical_volume(xn) > volfrac:
            l1 = lmid
        else:
            l2 = lmid
        steps += 1
    return xn, lmid, steps


def solve_small(G, b, rel=1e-14):
    """Gaussian elimination with partial pivoting for the m x m normal equations
    of the extrapolation (m <= 8); None when a pivot falls below rel times the
    largest diagonal entry (the extrapolation step is then skipped)."""
    G = np.array(G, float)
    b = np.array(b, float)
    m = b.size
    scale = max(float(np.max(np.abs(np.diag(G)))) if m else 0.0, 1e-300)
    for k in range(m):
        piv = k + int(np.argmax(np.abs(G[k:, k])))
        if not abs(G[piv, k]) > rel * scale:
            return None
        if piv != k:
            G[[k, piv]] = G[[piv, k]]
            b[[k, piv]] = b[[piv, k]]
        for i in range(k + 1, m):
            f = G[i, k] / G[k, k]
            G[i, k:] -= f * G[k, k:]
            b[i] -= f * b[k]
    y = np.zeros(m)
    for i in range(m - 1, -1, -1):
        y[i] = (b[i] - G[i, i + 1:] @ y[i + 1:]) / G[i, i]
    return y


def pae_update(h, x, r, it, m, q, alpha, zeta):
    """Periodic Anderson extrapolation of the OC fixed-point iteration (Sec. 3.6):
    r = U(x) - x is the OC step's residual on the active elements and it the step
    counted from q0. The differences of x and r between consecutive steps go to
    cyclic slots (slot (it - 1) mod m, the last m of them kept); when (it + 1) is
    a multiple of q (reading R23) gamma minimises ||r - R gamma|| (normal
    equations) and x + zeta r - (X + zeta R) gamma is taken, otherwise the damped
    step x + alpha r; the result is clipped to [0, 1]. h holds the slots and the
    previous x and r. Returns (x_new, kind) with kind 1 damped, 2 extrapolated."""
    if it == 0 or "X" not in h:
        h["X"] = np.zeros((m, x.size))
        h["R"] = np.zeros((m, x.size))
        h["filled"] = 0
    if it >= 1:
        k = (it - 1) % m
        h["X"][k] = x - h["xold"]
        h["R"][k] = r - h["rold"]
        h["filled"] = min(h["filled"] + 1, m)
    kind, xn = 1, None
    if it >= 1 and (it + 1) % q == 0:
        f = h["filled"]
        Rm, Xm = h["R"][:f].T, h["X"][:f].T
        gamma = solve_small(Rm.T @ Rm, Rm.T @ r)
        if gamma is not None:
            xn = x + zeta * r - (Xm + zeta * Rm) @ gamma
            kind = 2
    if xn is None:
        xn = x + alpha * r
    h["xold"], h["rold"] = x.copy(), r.copy()
    return np.clip(xn, 0.0, 1.0), kind


def continuation(par, cnt, loop, kind="add"):
    """Continuation of Sec. 3 (parCont = {istart, maxPar, isteps, deltaPar});
    kind "add" (paper) or "mul" (doubling, clamped to maxPar) (reading R9)."""
    istart, maxpar, isteps, delta = cnt
    if loop >= istart and par < maxpar and loop % isteps == 0:
        par = par + delta if kind == "add" else min(maxpar, par * delta)
    return par


# ----------------------------------------------------------------------------
# One design iteration and the redesign loop (Sec. 3 RL.1-RL.4)
# ----------------------------------------------------------------------------


@dataclass
class Params:
    nelx: int
    nely: int
    nelz: int = 0
    volfrac: float = 0.5
    penal: float = 3.0
    rmin: float = 2.4
    ft: int = 3
    ftBC: str = "N"
    eta: float = 0.5
    beta: float = 2.0
    move: float = 0.2
    E0: float = 1.0
    Emin: float = 1e-9
    nu: float = 0.3
    penal_cnt: tuple = (1, 3.0, 25, 0.25)
    beta_cnt: tuple = (1, 2.0, 25, 2.0)
    penal_kind: str = "add"
    beta_kind: str = "add"
    newton_tol: float = 1e-6
    oc_tol: float = 1e-4
    oc_method: str = "bisection"  # or "primal_dual" (Appendix A), "filtered" (Sec. 3.2, general variant)
    pae_q0: int = 0               # first loop of the periodic Anderson extrapolation (0: off)
    pae_q: int = 4
    pae_m: int = 4
    pae_alpha: float = 0.9
    pae_zeta: float = 1.0
    solver: str = "direct"
    cg_rtol: float = 1e-10
    threads: int = 1              # host threads of the PCG matrix products (same iterates for any count)

    @classmethod
    def parity(cls, **kw):
        """Tight tolerances of reading R5."""
        kw.setdefault("newton_tol", 1e-14)
        kw.setdefault("oc_tol", 1e-15)
        return cls(**kw)


@dataclass
class State:
    x: np.ndarray
    xphys: np.ndarray
    xold: np.ndarray
    U: np.ndarray
    eta: float
    penal: float
    beta: float
    loop: int = 0
    history: list = field(default_factory=list)
    pae: dict = field(default_factory=dict)


def initial_state(p: Params, passive=None):
    """Initial design accounting for passive sets (Appendix B, PRE.6)."""
    g = Grid(p.nelx, p.nely, p.nelz)
    pas = np.zeros(g.nel, np.int8) if passive is None else np.asarray(passive, np.int8)
    act = pas == 0
    nS, nV = int(np.sum(pas == 1)), int(np.sum(pas == -1))
    x = np.zeros(g.nel)
    x[act] = (p.volfrac * (g.nel - nV) - nS) / max(1, int(act.sum()))
    x[pas == 1] = 1.0
    return State(x=x, xphys=x.copy(), xold=np.ones(g.nel), U=np.zeros(g.ndof),
                 eta=p.eta, penal=p.penal, beta=p.beta)


def design_step(p: Params, s: State, F, fixed, passive=None, Ke=None):
    """One redesign iteration RL.1-RL.4 in the listing's order. Mutates s."""
    g = Grid(p.nelx, p.nely, p.nelz)
    Ke = element_stiffness(g.dim, p.nu) if Ke is None else Ke
    pas = np.zeros(g.nel, np.int8) if passive is None else np.asarray(passive, np.int8)
    act = pas == 0
    s.loop += 1
    # RL.1 physical density
    xtilde = filter_forward(g, s.x, p.rmin, p.ftBC)
    xphys = s.x.copy()
    xphys[act] = xtilde[act]
    dp = np.ones(g.nel)
    n_newton = 0
    if p.ft > 1:
        if p.ft == 3:
            s.eta, n_newton = eta_newton(xphys, s.eta, s.beta, p.volfrac, p.newton_tol)
        dp = dprj(xtilde, s.eta, s.beta)
        xphys = prj(xphys, s.eta, s.beta)
    ch = float(np.linalg.norm(xphys - s.xold) / math.sqrt(g.nel))
    s.xold = xphys.copy()
    s.xphys = xphys
    # RL.2 modulus, assembly, solve
    E = simp_modulus(xphys, s.penal, p.E0, p.Emin)
    n_cg = 0
    if p.solver == "direct":
        U = solve_direct(g, Ke, E, F, fixed)
    else:
        U, n_cg, _ = solve_pcg(g, Ke, E, F, fixed, rtol=p.cg_rtol, U0=s.U, threads=p.threads)
    s.U = U
    # RL.3 sensitivities and back-filter
    dc, c, _ = sensitivity(g, Ke, xphys, U, F, s.penal, p.E0, p.Emin, act)
    dV = np.where(act, 1.0 / (g.nel * p.volfrac), 0.0)
    dc = filter_backward(g, dc, p.rmin, p.ftBC, dp)
    dV0 = filter_backward(g, dV, p.rmin, p.ftBC, dp)
    # RL.4 OC and continuation
    x_prev = s.x.copy()
    if p.oc_method == "primal_dual":
        s.x, lm, n_bis = oc_update_primal_dual(s.x, dc, dV0, act, p.move, p.volfrac)
    elif p.oc_method == "filtered":
        s.x, lm, n_bis = oc_update_filtered(g, s.x, dc, dV0, act, p.move, p.volfrac, p.rmin, p.ftBC, p.ft,
                                            s.eta, s.beta, pas, p.oc_tol)
    else:
        s.x, lm, n_bis = oc_update(s.x, dc, dV0, act, p.move, p.volfrac, p.oc_tol)
    pae_kind = 0
    if p.pae_q0 > 0 and s.loop >= p.pae_q0:
        xa, pae_kind = pae_update(s.pae, x_prev[act], s.x[act] - x_prev[act], s.loop - p.pae_q0, p.pae_m,
                                  p.pae_q, p.pae_alpha, p.pae_zeta)
        s.x[act] = xa
    s.penal = continuation(s.penal, p.penal_cnt, s.loop, p.penal_kind)
    s.beta = continuation(s.beta, p.beta_cnt, s.loop, p.beta_kind)
    info = dict(loop=s.loop, c=c, V=float(np.mean(xphys)), ch=ch, penal=s.penal,
                beta=s.beta, eta=s.eta, lm=lm, n_newton=n_newton, n_bisect=n_bis,
                n_cg=n_cg, pae=pae_kind)
    s.history.append(info)
    return info


def run(p: Params, F, fixed, passive=None, maxit=100, stop_ch=1e-6):
    """Redesign loop until ch <= stop_ch or maxit iterations (Sec. 3)."""
    s = initial_state(p, passive)
    Ke = element_stiffness(3 if p.nelz else 2, p.nu)
    ch = 1.0
    while ch > stop_ch and s.loop < maxit:
        ch = design_step(p, s, F, fixed, passive, Ke)["ch"]
    return s
