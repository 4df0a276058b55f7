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
