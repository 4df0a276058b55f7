"""Micro-benchmarks through the C ABI (the targets of the ncu captures
summarised under profiles/).

    python -m paper_2005_05436_gb300.kernel_bench --grid 256x128x128 --precision fp64 --reps 3
    python -m paper_2005_05436_gb300.kernel_bench --what batch --count 256 --steps 3
    python -m paper_2005_05436_gb300.kernel_bench --what net --shape 52x28x28 --reps 10

ku: builds a cantilever grid with a seeded SIMP-like design and launches the
operator kernel reps + 1 times (one warm-up) on the current stream; prints the
average device time per launch and the achieved rate.
batch: the batched workload (256 uneven 2D instances, nelx ~ U{60..480},
seed 20050543): autotunes the tile shapes, then times design iterations.
net: forward pass and one training step (forward, backward, Adam) of the
warm-start network on an [N][D][H][W] input.
"""
import argparse
import json
import math
import time

import numpy as np
import torch

from . import TO_FP64, TO_MIXED, TO_PC_GMG, build as B, default_params, inputs as I


def bench_ku(a):
    from .topopt import Grid
    nelx, nely, nelz = (int(v) for v in a.grid.split("x"))
    dim = 3 if nelz else 2
    F, fixed = I.cantilever_3d(nelx, nely, nelz) if dim == 3 else I.mbb_half_beam(nelx, nely)
    prec = TO_FP64 if a.precision == "fp64" else TO_MIXED
    p = default_params(dim, nelx, nely, nelz, precision=prec, rmin=math.sqrt(3.0),
                       ku_impl={"auto": 0, "node": 1, "tc": 2, "walsh": 3, "pair": 4}[a.ku_impl])
    g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda())
    x = torch.from_numpy(I.random_design(g.nel, 1, "binary").clip(1e-3, 1.0)).cuda()
    us = g.time_apply_K(x, prec, reps=a.reps)
    if prec == TO_FP64:
        rate = {"TFLOP/s": 2.0 * (24 if dim == 3 else 8) ** 2 * g.nel / (us * 1e-6) / 1e12}
    else:
        rate = {"GB/s": 4.0 * (2 * g.ndof + g.nel) / (us * 1e-6) / 1e9,
                "TFLOP/s": 2.0 * (24 if dim == 3 else 8) ** 2 * g.nel / (us * 1e-6) / 1e12}
    print(json.dumps({"grid": a.grid, "precision": a.precision, "ku_impl": a.ku_impl, "nel": g.nel,
                      "ndof": g.ndof,
                      "us_per_launch": round(us, 3), **{k: round(v, 3) for k, v in rate.items()}}))


def bench_oc(a):
    """OC update (to_oc_update) with the bisection (paper tolerance 1e-4), the
    explicit primal-dual iteration and the bisection on the physical volume
    (filter and fixed-threshold projection per candidate, ft = 2), on a seeded
    SIMP-like state of the grid; wall
    time per call (each call reads lambda back, so it includes one synchronisation)."""
    from . import TO_OC_BISECTION, TO_OC_PHYSICAL_VOLUME, TO_OC_PRIMAL_DUAL
    from .topopt import Grid
    nelx, nely, nelz = (int(v) for v in a.grid.split("x"))
    dim = 3 if nelz else 2
    F, fixed = I.cantilever_3d(nelx, nely, nelz) if dim == 3 else I.mbb_half_beam(nelx, nely)
    out = {"grid": a.grid}
    for name, m in (("bisection", TO_OC_BISECTION), ("primal_dual", TO_OC_PRIMAL_DUAL),
                    ("physical_volume", TO_OC_PHYSICAL_VOLUME)):
        p = default_params(dim, nelx, nely, nelz, volfrac=0.3, move=0.2, oc_method=m, ft=2, eta=0.5, beta=2.0)
        g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda())
        r = np.random.default_rng(1)
        x0 = torch.from_numpy(np.clip(0.3 + 0.2 * r.standard_normal(g.nel), 0, 1)).cuda()
        dc = torch.from_numpy(-np.abs(r.standard_normal(g.nel)) * 10 ** r.uniform(-4, 1, g.nel)).cuda()
        dV0 = torch.full((g.nel,), 1.0 / (g.nel * 0.3), dtype=torch.float64, device="cuda")
        x = x0.clone()
        g.oc_update(x, dc, dV0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.reps):
            x.copy_(x0)
            lm = g.oc_update(x, dc, dV0)
        torch.cuda.synchronize()
        out[name] = {"ms_per_call": round((time.perf_counter() - t0) / a.reps * 1e3, 3), "lm": lm}
        g.close()
    print(json.dumps(out))


def bench_frame(a):
    """The frame-reinforcement workload of Sec. 3.5 at the paper's size
    (nelx = nely = 900, volfrac 0.2, penal 3, rmin 8, ft 3, eta 0.5, beta 2, no
    continuation): design iterations through to_step, timed with CUDA events
    after two untimed ones; both load orientations."""
    from . import TO_FP64, TO_MIXED, TO_PC_GMG
    from .topopt import Design, Grid
    nelx, nely = (int(v) for v in a.grid.split("x")[:2])
    prec = TO_FP64 if a.precision == "fp64" else TO_MIXED
    out = {"grid": f"{nelx}x{nely}", "precision": a.precision, "paper_s_per_iteration": 10.8}
    for sign in (-1.0, 1.0):
        F, fixed, pas = I.frame_reinforcement(nelx, nely, sign)
        p = default_params(2, nelx, nely, 0, volfrac=0.2, penal=3.0, rmin=8.0, ft=3, eta=0.5, beta=2.0,
                           precision=prec, precond=TO_PC_GMG, mg_nu=1, cg_rtol=1e-8, cg_maxit=50000,
                           penal_cnt=(1, 3.0, 1000, 0.0), beta_cnt=(1, 2.0, 1000, 0.0))
        g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda(),
                 torch.from_numpy(pas).cuda())
        d = Design(g, torch.from_numpy(I.initial_design(g.nel, 0.2, pas)).cuda())
        for _ in range(2):
            d.step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        infos = [d.step() for _ in range(a.steps)]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        out["left" if sign < 0 else "right"] = {
            "ms_per_iteration": round(ms, 2), "n_cg": [i["n_cg"] for i in infos],
            "c": infos[-1]["c"], "V": infos[-1]["V"], "speedup_vs_paper": round(10.8e3 / ms, 1)}
        g.close()
    print(json.dumps(out))


def bench_pae(a):
    """The convergence study of Sec. 3.6 (Table 2) on the half MBB beam (300 x 100,
    f = 0.5, rmin = 8.75, penal 3, no continuation): T1 density filter (ft 1), T2
    filter + volume-preserving projection (ft 3, beta 2); each without and with
    periodic Anderson extrapolation (q0 = 20, q = 4, m_r = 4, alpha 0.9, zeta 1),
    run until ||xPhys_k - xPhys_k-1|| / sqrt(m) < 1e-6 or 2500 design iterations
    (FP64 + GMG state solves to 1e-8)."""
    from . import TO_FP64, TO_PC_GMG
    from .topopt import Design, Grid
    nelx, nely = (int(v) for v in a.grid.split("x")[:2])
    F, fixed = I.mbb_half_beam(nelx, nely)
    out = {"grid": f"{nelx}x{nely}", "paper_iterations": {"T1": 2500, "T1-PAE": 828, "T2": 2500, "T2-PAE": 352}}
    for case, ft in (("T1", 1), ("T2", 3)):
        for pae in (False, True):
            p = default_params(2, nelx, nely, 0, volfrac=0.5, penal=3.0, rmin=8.75, ft=ft, eta=0.5, beta=2.0,
                               precision=TO_FP64, precond=TO_PC_GMG, mg_nu=1, cg_rtol=1e-8, cg_maxit=50000,
                               penal_cnt=(1, 3.0, 1000000, 0.0), beta_cnt=(1, 2.0, 1000000, 0.0),
                               pae_q0=20 if pae else 0, pae_q=4, pae_m=4, pae_alpha=0.9, pae_zeta=1.0)
            g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda())
            d = Design(g, torch.from_numpy(I.initial_design(g.nel, 0.5)).cuda())
            t0 = time.perf_counter()
            info = None
            while True:
                info = d.step()
                if info["ch"] < 1e-6 or info["loop"] >= a.steps:
                    break
            dt = time.perf_counter() - t0
            out[case + ("-PAE" if pae else "")] = {"iterations": info["loop"], "c": round(info["c"], 2),
                                                   "ch": info["ch"], "s": round(dt, 2),
                                                   "ms_per_iteration": round(1e3 * dt / info["loop"], 2)}
            g.close()
    print(json.dumps(out))


def bench_batch(a):
    """Under torchrun each rank advances its share of the instances (balanced by
    element count, no collective in the data path); rank 0 prints the whole-job
    rate over the slowest rank's time."""
    from . import replicas as R
    from .topopt import Batch
    rank, local, world = R.env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(local)
    insts = I.batched_instances(a.count, seed=20050543)
    if world > 1:
        insts = [insts[i] for i in R.shard([q.nelx * q.nely for q in insts], world)[rank]]
    p = default_params(2, 8, 4, precision=TO_MIXED, precond=TO_PC_GMG, mg_nu=1, penal=3.0, beta=2.0,
                       cg_rtol=1e-8, cg_maxit=100000, penal_cnt=(1, 3.0, 25, 0.25), beta_cnt=(1, 16.0, 25, 2.0, 1))
    F = torch.from_numpy(np.concatenate([q.F for q in insts])).cuda()
    fixed = torch.from_numpy(np.concatenate([q.fixed for q in insts])).cuda()
    x0 = torch.from_numpy(np.concatenate([I.initial_design(q.nelx * q.nely, q.volfrac) for q in insts])).cuda()
    b = Batch(p, [(q.nelx, q.nely, q.volfrac, q.rmin) for q in insts], F, fixed, x0)
    tune = b.autotune(reps=5) if a.autotune else None
    steps = []
    for _ in range(a.steps):
        info = b.step()
        steps.append({k: info[k] for k in ("loop", "ms", "max_refinements", "max_inner_iters", "inner_passes",
                                           "newton_passes", "oc_passes", "max_rel_res", "kernels")})
    ms = [s["ms"] for s in steps[1:]] or [steps[0]["ms"]]
    t_max = R.max_over_ranks(sum(ms) / len(ms) / 1000.0, world, device="cuda")
    nel_all = R.sum_over_ranks(b.nel, world, device="cuda")
    if rank == 0:
        print(json.dumps({"instances": a.count, "ranks": world, "elements": int(nel_all), "dofs_rank0": b.ndof,
                          "tiles": tune and {"node": tune["node"], "elem": tune["elem"]},
                          "design_iterations_per_s": round(1.0 / t_max, 3),
                          "elements_per_s": round(R.whole_job_rate(nel_all, t_max), 1), "steps": steps}))


def bench_net(a):
    from .learned import Net, he_init
    D, H, W = (int(v) for v in a.shape.split("x"))
    net = Net(base=16, bf16=True)
    net.set_params(he_init(16, seed=1))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((a.batch, D, H, W, 4), device="cuda", generator=g)
    t = torch.randn((a.batch, D, H, W, 3), device="cuda", generator=g)
    m = torch.ones((a.batch, D, H, W), dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    net.forward(x)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.reps):
        net.forward(x)
    e1.record()
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / a.reps
    net.accumulate(x, t, m)
    net.adam(1e-4)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.reps):
        net.accumulate(x, t, m)
        net.adam(1e-4)
    e1.record()
    torch.cuda.synchronize()
    trn = e0.elapsed_time(e1) / a.reps
    print(json.dumps({"shape": [a.batch, D, H, W], "params": net.n_params, "forward_ms": round(fwd, 3),
                      "train_step_ms": round(trn, 3)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", default="ku", choices=["ku", "batch", "net", "oc", "frame", "pae"])
    ap.add_argument("--grid", default="256x128x128")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--ku-impl", default="auto", choices=["auto", "node", "tc", "walsh", "pair"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--shape", default="52x28x28")
    ap.add_argument("--batch", type=int, default=1)
    a = ap.parse_args()
    B.build()
    {"ku": bench_ku, "batch": bench_batch, "net": bench_net, "oc": bench_oc, "frame": bench_frame,
     "pae": bench_pae}[a.what](a)


if __name__ == "__main__":
    main()
