"""Seeded synthetic inputs shared by the CUDA path, its tests, the bench and the oracle.

This module holds no arithmetic of the topology-optimisation method: only the
problem data (load vectors, supports, passive masks) of the paper's benchmark
problems and seeded random fields. It imports nothing from the rest of the
package, so the oracle may use it without touching the CUDA path.

Numbering (Ferrari & Sigmund 2020, Sec. 3, PRE.2; the 2D and 3D listings of
Appendices B and C): nodes and elements are numbered column-major with the row
index ``iy`` running fastest (downwards), then ``iz`` (3D), then the column
``ix``. 0-based:

* node    n = iy + (nely+1) * (iz + (nelz+1) * ix)
* element e = iy + nely * (iz + nelz * ix)
* DOF     dim * n + c, c = 0 (X, along ix), 1 (Y, up = -iy), 2 (Z, along iz)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def node_id(iy, ix, iz=0, *, nely, nelz=0):
    """0-based node number of the grid node at (iy, iz, ix)."""
    nny = nely + 1
    nnz = nelz + 1
    return iy + nny * (iz + nnz * ix)


def counts(nelx, nely, nelz=0):
    """(dim, nEl, nNodes, nDof) of a structured grid; nelz = 0 means 2D."""
    dim = 3 if nelz else 2
    nel = nelx * nely * (nelz if nelz else 1)
    nnodes = (nelx + 1) * (nely + 1) * ((nelz + 1) if nelz else 1)
    return dim, nel, nnodes, dim * nnodes


def mbb_half_beam(nelx, nely):
    """Half MBB beam (Sec. 3, the 2D example; Appendix B, PRE.3).

    Unit downward load on the Y DOF of the top-left node; X DOFs of the left
    edge fixed (symmetry); Y DOF of the bottom-right node fixed (roller).
    Returns (F[nDof] float64, fixed[nDof] uint8).
    """
    _, _, _, ndof = counts(nelx, nely)
    F = np.zeros(ndof)
    fixed = np.zeros(ndof, np.uint8)
    F[2 * node_id(0, 0, nely=nely) + 1] = -1.0
    for iy in range(nely + 1):
        fixed[2 * node_id(iy, 0, nely=nely) + 0] = 1
    fixed[2 * node_id(nely, nelx, nely=nely) + 1] = 1
    return F, fixed


def cantilever_3d(nelx, nely, nelz):
    """3D cantilever (Sec. 4 and Appendix C, PRE.3).

    All DOFs of the x = 0 face clamped; a line load along the edge
    (ix = nelx, iz = 0), acting on the Z DOF with magnitude
    -sin(pi * iy / nely), iy = 0..nely (peak 1 at mid-height).
    Returns (F[nDof] float64, fixed[nDof] uint8).
    """
    _, _, _, ndof = counts(nelx, nely, nelz)
    F = np.zeros(ndof)
    fixed = np.zeros(ndof, np.uint8)
    for iy in range(nely + 1):
        n = node_id(iy, nelx, 0, nely=nely, nelz=nelz)
        F[3 * n + 2] = -math.sin(math.pi * iy / nely)
    for iz in range(nelz + 1):
        for iy in range(nely + 1):
            n = node_id(iy, 0, iz, nely=nely, nelz=nelz)
            fixed[3 * n:3 * n + 3] = 1
    return F, fixed


def cantilever_family(nelx, nely, nelz, seed):
    """Seeded member of the 3D cantilever family used to generate training data
    for the learned warm start: the x = 0 face clamped, and on the x = nelx face
    either a line load (along y or z, sine or uniform profile, random unit
    direction) or 1-3 unit point loads of random direction, plus a volume
    fraction ~ U[0.1, 0.3]. Returns (F, fixed, volfrac)."""
    rng = np.random.default_rng(seed)
    _, _, _, ndof = counts(nelx, nely, nelz)
    F = np.zeros(ndof)
    fixed = np.zeros(ndof, np.uint8)
    for iz in range(nelz + 1):
        for iy in range(nely + 1):
            n = node_id(iy, 0, iz, nely=nely, nelz=nelz)
            fixed[3 * n:3 * n + 3] = 1

    def unit():
        v = rng.standard_normal(3)
        return v / np.linalg.norm(v)

    if rng.random() < 0.5:
        d = unit()
        sine = rng.random() < 0.5
        if rng.random() < 0.5:  # along y at a random z
            iz = int(rng.integers(0, nelz + 1))
            for iy in range(nely + 1):
                w = math.sin(math.pi * iy / nely) if sine else 1.0 / (nely + 1)
                F[3 * node_id(iy, nelx, iz, nely=nely, nelz=nelz):][:3] += w * d
        else:  # along z at a random y
            iy = int(rng.integers(0, nely + 1))
            for iz in range(nelz + 1):
                w = math.sin(math.pi * iz / nelz) if sine else 1.0 / (nelz + 1)
                F[3 * node_id(iy, nelx, iz, nely=nely, nelz=nelz):][:3] += w * d
    else:
        for _ in range(int(rng.integers(1, 4))):
            iy, iz = int(rng.integers(0, nely + 1)), int(rng.integers(0, nelz + 1))
            F[3 * node_id(iy, nelx, iz, nely=nely, nelz=nelz):][:3] += unit()
    return F, fixed, float(rng.uniform(0.1, 0.3))


def frame_reinforcement(nelx, nely, sign=-1.0):
    """Frame-reinforcement example of Sec. 3.5 (passive frame and opening).

    sign = -1: the height-proportional horizontal load points left (the paper's
    listing), +1: right (the second design of its figure).
    Returns (F, fixed, passive) with passive[e] = 1 (solid), -1 (void), 0.
    nelx and nely must be multiples of 50.
    """
    _, nel, _, ndof = counts(nelx, nely)
    F = np.zeros(ndof)
    fixed = np.zeros(ndof, np.uint8)
    # vertical distributed load of total -2 on the top row of nodes
    for ix in range(nelx + 1):
        F[2 * node_id(0, ix, nely=nely) + 1] += -2.0 / (nelx + 1)
    # horizontal height-proportional load on the right column of nodes
    for iy in range(nely + 1):
        F[2 * node_id(iy, nelx, nely=nely) + 0] += sign * iy / float(nely) ** 2
    fixed[[0, 1, ndof - 1]] = 1
    passive = np.zeros(nel, np.int8)
    E = np.arange(nel).reshape(nelx, nely)  # E[ix, iy] = element number
    t_y, t_x = nely // 50, nelx // 50
    solid = np.zeros((nelx, nely), bool)
    solid[:, :t_y] = True
    solid[:t_x, :] = True
    solid[nelx - t_x:, :] = True
    void = np.zeros((nelx, nely), bool)
    # the opening: 1-based rows 2*nely/5..end, columns 2*nelx/5..nelx-nelx/5
    void[2 * nelx // 5 - 1:nelx - nelx // 5, 2 * nely // 5 - 1:] = True
    passive[E[solid]] = 1
    passive[E[void & ~solid]] = -1
    return F, fixed, passive


def initial_design(nel, volfrac, passive=None):
    """Initial design of the paper's PRE.6: x = (volfrac (nEl - |P0|) - |P1|) / |A|
    on active elements, 1 on passive solid, 0 on passive void."""
    if passive is None:
        return np.full(nel, float(volfrac))
    pas = np.asarray(passive)
    nS, nV = int(np.sum(pas == 1)), int(np.sum(pas == -1))
    x = np.full(nel, (volfrac * (nel - nV) - nS) / (nel - nS - nV))
    x[pas == 1] = 1.0
    x[pas == -1] = 0.0
    return x


def random_design(nel, seed, kind="uniform", lo=0.0, hi=1.0):
    """Seeded element field in [lo, hi].

    kind = "uniform": i.i.d. uniform; "binary": mostly 0/1 with a band of
    intermediate values, the value mix of a converged SIMP design.
    """
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return lo + (hi - lo) * rng.random(nel)
    if kind == "binary":
        v = (rng.random(nel) < 0.4).astype(np.float64)
        mid = rng.random(nel) < 0.2
        v[mid] = rng.random(int(mid.sum()))
        return lo + (hi - lo) * v
    raise ValueError(kind)


def random_vector(n, seed, scale=1.0):
    """Seeded standard-normal vector of length n times scale."""
    return scale * np.random.default_rng(seed).standard_normal(n)


@dataclass
class Instance2D:
    """One problem of the batched 2D workload."""
    nelx: int
    nely: int
    volfrac: float
    rmin: float
    F: np.ndarray = field(repr=False)
    fixed: np.ndarray = field(repr=False)


def batched_instances(count=256, seed=20050543, nelx_range=(60, 480)):
    """Uneven batch of independent 2D problems.

    nelx ~ U{lo..hi}, aspect nelx:nely ~ U[2, 4], volfrac ~ U[0.2, 0.5],
    rmin = 0.02 * nelx, 1-3 unit point loads of random direction on random
    boundary nodes, 1-2 clamped boundary segments (both DOFs) of >= 2 nodes.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nelx = int(rng.integers(nelx_range[0], nelx_range[1] + 1))
        aspect = float(rng.uniform(2.0, 4.0))
        nely = max(2, int(round(nelx / aspect)))
        volfrac = float(rng.uniform(0.2, 0.5))
        rmin = 0.02 * nelx
        _, _, _, ndof = counts(nelx, nely)
        boundary = _boundary_nodes(nelx, nely)
        F = np.zeros(ndof)
        for _ in range(int(rng.integers(1, 4))):
            n = boundary[int(rng.integers(len(boundary)))]
            th = float(rng.uniform(0.0, 2.0 * math.pi))
            F[2 * n] += math.cos(th)
            F[2 * n + 1] += math.sin(th)
        fixed = np.zeros(ndof, np.uint8)
        for _ in range(int(rng.integers(1, 3))):
            L = len(boundary)
            start = int(rng.integers(L))
            length = int(rng.integers(2, max(3, L // 8)))
            for k in range(length):
                n = boundary[(start + k) % L]
                fixed[2 * n:2 * n + 2] = 1
        F[fixed.astype(bool)] = 0.0
        if not np.any(F):
            # keep at least one load on a free node
            free_nodes = [n for n in boundary if not fixed[2 * n]]
            F[2 * free_nodes[len(free_nodes) // 2] + 1] = -1.0
        out.append(Instance2D(nelx, nely, volfrac, rmin, F, fixed))
    return out


def _boundary_nodes(nelx, nely):
    """Boundary nodes walked once around the rectangle."""
    nodes = []
    for ix in range(nelx + 1):
        nodes.append(node_id(0, ix, nely=nely))
    for iy in range(1, nely + 1):
        nodes.append(node_id(iy, nelx, nely=nely))
    for ix in range(nelx - 1, -1, -1):
        nodes.append(node_id(nely, ix, nely=nely))
    for iy in range(nely - 1, 0, -1):
        nodes.append(node_id(iy, 0, nely=nely))
    return nodes
