"""Micro-benchmark of the matrix-free K u kernel through the C ABI.

    python -m paper_2005_05436_gb300.kernel_bench --grid 256x128x128 --precision fp64 --reps 3

Builds a cantilever grid with a seeded SIMP-like design and launches the
operator kernel reps + 1 times (one warm-up) on the current stream; prints the
average device time per launch and the achieved rate. Used as the target of
the ncu captures summarised under profiles/.
"""
import argparse
import json
import math

import torch

from . import TO_FP64, TO_MIXED, build as B, default_params, inputs as I
from .topopt import Grid


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", default="256x128x128")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    B.build()
    nelx, nely, nelz = (int(v) for v in a.grid.split("x"))
    dim = 3 if nelz else 2
    F, fixed = I.cantilever_3d(nelx, nely, nelz) if dim == 3 else I.mbb_half_beam(nelx, nely)
    prec = TO_FP64 if a.precision == "fp64" else TO_MIXED
    p = default_params(dim, nelx, nely, nelz, precision=prec, rmin=math.sqrt(3.0))
    g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda())
    x = torch.from_numpy(I.random_design(g.nel, 1, "binary").clip(1e-3, 1.0)).cuda()
    us = g.time_apply_K(x, prec, reps=a.reps)
    if prec == TO_FP64:
        rate = {"TFLOP/s": 2.0 * (24 if dim == 3 else 8) ** 2 * g.nel / (us * 1e-6) / 1e12}
    else:
        rate = {"GB/s": 4.0 * (2 * g.ndof + g.nel) / (us * 1e-6) / 1e9}
    print(json.dumps({"grid": a.grid, "precision": a.precision, "nel": g.nel, "ndof": g.ndof,
                      "us_per_launch": round(us, 3), **{k: round(v, 3) for k, v in rate.items()}}))


if __name__ == "__main__":
    main()
