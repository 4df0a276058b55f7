"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import math

import numpy as np

from paper_2005_05436_gb300 import inputs as I


def rel(a, b):
    """Normwise relative difference ||a - b|| / ||b||."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def problem(shape):
    """(F, fixed) of the MBB beam (2D) or the cantilever (3D)."""
    nelx, nely, nelz = shape
    if nelz:
        return I.cantilever_3d(nelx, nely, nelz)
    return I.mbb_half_beam(nelx, nely)


def to_cuda(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def make_grid(shape, **kw):
    """A CUDA Grid handle with the problem of ``problem(shape)``."""
    import torch
    from paper_2005_05436_gb300 import default_params
    from paper_2005_05436_gb300.topopt import Grid
    nelx, nely, nelz = shape
    dim = 3 if nelz else 2
    passive = kw.pop("passive", None)
    F = kw.pop("F", None)
    fixed = kw.pop("fixed", None)
    if F is None:
        F, fixed = problem(shape)
    p = default_params(dim, nelx, nely, nelz, **kw)
    g = Grid(p, to_cuda(F), to_cuda(fixed, torch.uint8),
             None if passive is None else to_cuda(passive, torch.int8))
    return g, F, fixed


def simp_field(nel, seed, lo=0.001):
    """A design field with the value mix of a SIMP iterate (mostly near 0 or 1)."""
    return np.clip(I.random_design(nel, seed, "binary"), lo, 1.0)


def design_field(shape, seed, rmin=2.5, beta=8.0, lo=0.0):
    """A coherent design like a SIMP iterate: a random field filtered with the
    oracle's cone filter and projected (solid and void regions with smooth
    transitions), values in [lo, 1]."""
    from oracle import topopt_oracle as O
    g = O.Grid(*shape)
    x = O.filter_forward(g, I.random_design(g.nel, seed), rmin, "N")
    z = (x - np.median(x)) / max(np.std(x), 1e-12)   # unit-variance coherent field
    x = O.prj(0.5 + 0.25 * z, 0.5, beta)              # mostly solid or void, smooth edges
    return np.clip(x, lo, 1.0)


def max_abs(a, b):
    """Largest elementwise |a - b| (0 for empty arrays)."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.max(np.abs(a - b))) if b.size else 0.0


def assert_design_matches(tag, got, ref, xphys, xphys_ref, x, x_ref, tol=1e-8, lm_rtol=1e-7):
    """One design iteration of the CUDA path against the oracle's.

    x and xPhys lie in [0, 1], so besides the normwise difference every element
    must lie within ``tol`` of the oracle's (an error confined to a boundary tile
    or a ragged edge cannot hide under the norm). ch and V are bounded by the
    elementwise error (|d ch| <= 2 max|d xPhys|, |d V| <= max|d xPhys|); the OC
    multiplier follows dc, which tracks c, so it gets a relative bound."""
    e_p, e_x = max_abs(xphys, xphys_ref), max_abs(x, x_ref)
    assert rel(xphys, xphys_ref) <= tol and e_p <= tol, (tag, "xPhys", rel(xphys, xphys_ref), e_p)
    assert rel(x, x_ref) <= tol and e_x <= tol, (tag, "x", rel(x, x_ref), e_x)
    assert abs(got["ch"] - ref["ch"]) <= 2 * tol, (tag, "ch", got["ch"], ref["ch"])
    assert abs(got["V"] - ref["V"]) <= tol, (tag, "V", got["V"], ref["V"])
    assert abs(got["lm"] - ref["lm"]) <= lm_rtol * abs(ref["lm"]), (tag, "lm", got["lm"], ref["lm"])
    return max(e_p, e_x)
