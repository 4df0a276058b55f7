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


def bench_mma(a):
    """Cost of one tcgen05.mma kind::tf32 (K = 8) by shape, issuing threads per
    block and blocks per SM (to_time_tf32_mma): the instruction the tensor-core
    FP32 operator is built from."""
    import ctypes as C
    from . import _lib as L
    lib = L.load()
    cases = [(128, 32, 1, 1), (128, 64, 1, 1), (128, 128, 1, 1), (128, 256, 1, 1), (64, 32, 1, 1), (64, 256, 1, 1),
             (128, 32, 2, 1), (128, 32, 4, 1), (128, 32, 8, 1), (128, 64, 4, 1), (128, 32, 1, 2), (128, 32, 1, 4),
             (128, 32, 2, 2), (128, 64, 2, 2), (128, 256, 1, 2)]
    for m, n, iss, bps in cases:
        cyc, mac = C.c_double(), C.c_double()
        L.check(lib.to_time_tf32_mma(m, n, iss, bps, a.reps, C.byref(cyc), C.byref(mac)))
        print(json.dumps({"m": m, "n": n, "k": 8, "issuers_per_block": iss, "blocks_per_sm": bps,
                          "cycles_per_mma_per_issuer": round(cyc.value, 1),
                          "mac_per_cycle_per_sm": round(mac.value, 1)}))


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
    """The convergence study of Sec. 3.6 (Table 2) on the half MBB beam (f = 0.5,
    rmin = 8.75, FP64 + GMG state solves to 1e-8), each case without and with
    periodic Anderson extrapolation (q = 4, m_r = 4, alpha 0.9, zeta 1), run until
    ||xPhys_k - xPhys_k-1|| / sqrt(m) < 1e-6 or --steps design iterations:
    T1 density filter alone (ft 1, p = 3, q0 = 20); T2 + volume-preserving
    projection (ft 3, beta 2, q0 = 20); T3 as T2 with continuation betaCnt =
    {250, 16, 25, 2}, penalCnt = {50, 3, 25, 0.25} from p = 1 (q0 = 500); T4 as T2
    on 600 x 200. --cases selects them, --ftbc the filter padding."""
    from . import TO_FP64, TO_PC_GMG
    from .topopt import Design, Grid
    paper = {"T1": (2500, 252.7), "T1-PAE": (828, 258.9), "T2": (2500, 246.1), "T2-PAE": (352, 253.9),
             "T3": (2500, 199.6), "T3-PAE": (752, 197.5), "T4": (2500, 191.8), "T4-PAE": (818, 192.1)}
    out = {"ftBC": a.ftbc, "paper_iterations_c": paper}
    for case in a.cases.split(","):
        nelx, nely = (600, 200) if case == "T4" else (300, 100)
        F, fixed = I.mbb_half_beam(nelx, nely)
        ft = 1 if case == "T1" else 3
        penal, pcnt, bcnt, q0 = 3.0, (1, 3.0, 10 ** 6, 0.0), (1, 2.0, 10 ** 6, 0.0), 20
        if case == "T3":
            penal, pcnt, bcnt, q0 = 1.0, (50, 3.0, 25, 0.25), (250, 16.0, 25, 2.0), 500
        for pae in (False, True):
            p = default_params(2, nelx, nely, 0, volfrac=0.5, penal=penal, rmin=8.75, ft=ft, ftBC=a.ftbc, eta=0.5,
                               beta=2.0, precision=TO_FP64, precond=TO_PC_GMG, mg_nu=1, cg_rtol=1e-8,
                               cg_maxit=50000, penal_cnt=pcnt, beta_cnt=bcnt,
                               pae_q0=q0 if pae else 0, pae_q=4, pae_m=4, pae_alpha=0.9, pae_zeta=1.0)
            g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda())
            d = Design(g, torch.from_numpy(I.initial_design(g.nel, 0.5)).cuda())
            t0 = time.perf_counter()
            info = None
            while True:
                info = d.step()
                if info["ch"] < 1e-6 or info["loop"] >= a.steps:
                    break
            dt = time.perf_counter() - t0
            x = d.xPhys
            mnd = float(100.0 * 4.0 * (x * (1.0 - x)).mean())  # non-discreteness measure of Sec. 3.6
            out[case + ("-PAE" if pae else "")] = {"iterations": info["loop"], "c": round(info["c"], 2),
                                                   "ch": info["ch"], "m_ND": round(mnd, 4), "penal": info["penal"],
                                                   "beta": info["beta"], "s": round(dt, 2),
                                                   "ms_per_iteration": round(1e3 * dt / info["loop"], 2)}
            g.close()
    print(json.dumps(out))


def bench_mbb(a):
    """The 2D half MBB beam of Sec. 3 / Table 3 on the grids of --grids, each with
    the plain FP64 path and the mixed path (GMG-PCG to 1e-8 either way):
    config2 = volfrac 0.3, penal 1 -> 3 (+0.25 every 25 iterations), beta 2 -> 16
    (doubling every 25), rmin 0.03 nelx, ft 3; paper = the setting of Table 3
    (volfrac 0.5, penal 3, rmin = nelx / 75, i.e. 4, 8, 16, ft 3, beta 2, no
    continuation). Times design iterations warmup+1 .. warmup+steps with CUDA
    events, and one forward filter application."""
    from . import TO_CNT_MUL, TO_FP64, TO_MIXED, TO_PC_GMG
    from .topopt import Design, Grid
    out = {"variant": a.variant, "grids": {}}
    for spec in a.grids.split(","):
        nelx, nely = (int(v) for v in spec.split("x"))
        F, fixed = I.mbb_half_beam(nelx, nely)
        if a.variant == "config2":
            kw = dict(volfrac=0.3, penal=1.0, rmin=0.03 * nelx, penal_cnt=(1, 3.0, 25, 0.25),
                      beta_cnt=(1, 16.0, 25, 2.0, TO_CNT_MUL))
        else:
            kw = dict(volfrac=0.5, penal=3.0, rmin=nelx / 75.0, penal_cnt=(1, 3.0, 10 ** 6, 0.0),
                      beta_cnt=(1, 2.0, 10 ** 6, 0.0))
        res = {}
        for name, prec in (("fp64_gmg", TO_FP64), ("mixed_gmg", TO_MIXED)):
            p = default_params(2, nelx, nely, 0, ft=3, eta=0.5, beta=2.0, move=0.2, cg_rtol=1e-8, cg_maxit=100000,
                               precision=prec, precond=TO_PC_GMG, mg_nu=1, inner_rtol=1e-4, **kw)
            g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda())
            d = Design(g, torch.from_numpy(I.initial_design(g.nel, p.volfrac)).cuda())
            for _ in range(a.warmup):
                d.step()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            infos = [d.step() for _ in range(a.steps)]
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / a.steps
            xt = torch.empty_like(d.xPhys)
            g.filter(d.x, xt)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(5):
                g.filter(d.x, xt)
            e1.record()
            torch.cuda.synchronize()
            res[name] = {"design_it_per_s": round(1e3 / ms, 3), "ms_per_iteration": round(ms, 3),
                         "iterations": f"{a.warmup + 1}..{a.warmup + a.steps}",
                         "n_cg": [i["n_cg"] for i in infos], "rel_res_max": max(i["rel_res"] for i in infos),
                         "c_last": infos[-1]["c"],
                         "mean_ms": {k: round(sum(i[k] for i in infos) / len(infos), 3)
                                     for k in ("t_filter_ms", "t_solve_ms", "t_sens_ms", "t_oc_ms")},
                         "filter_us": round(1e3 * e0.elapsed_time(e1) / 5, 2)}
            g.close()
        res["rmin"] = kw["rmin"]
        res["mixed_speedup"] = round(res["fp64_gmg"]["ms_per_iteration"] / res["mixed_gmg"]["ms_per_iteration"], 2)
        res["c_rel_diff_last"] = abs(res["mixed_gmg"]["c_last"] - res["fp64_gmg"]["c_last"]) / abs(res["fp64_gmg"]["c_last"])
        out["grids"][spec] = res
    print(json.dumps(out))


def bench_learned(a):
    """The learned warm start at the scale of the 160x80x80 workload: samples
    (xPhys, F, and the converged compliance for the energy objective) from
    --runs seeded cantilever-family runs of the method on 40x20x20, 60x30x30 and
    80x40x40 grids (every design iteration after --warmup, --iters per run), a
    BF16 network with 16 base channels trained on the GPU for --epochs, then
    --steps design iterations of the 160x80x80 cantilever (volfrac 0.12, penal
    3, rmin sqrt(3), beta 2 -> 16 doubling every 25, mixed precision + GMG-PCG to
    1e-8) with and without the network from the same state, and the first state
    solve from U = 0 with and without it."""
    from . import TO_CNT_MUL, TO_MIXED, TO_PC_GMG, learned as Lr
    from .topopt import Design, Grid
    t0 = time.perf_counter()
    shapes = [(40, 20, 20), (60, 30, 30), (80, 40, 40)]
    samples, grids = Lr.generate_energy(shapes, runs=a.runs, iters=a.iters, seed=100, warmup=a.warmup)
    t_gen = time.perf_counter() - t0
    net = Lr.Net(base=16, bf16=True)
    net.set_params(Lr.he_init(16, seed=1))
    t0 = time.perf_counter()
    hist = Lr.train_energy(net, samples, grids, epochs=a.epochs, lr=2e-3, lr_final=1e-4, batch=4)
    t_train = time.perf_counter() - t0
    n_samples = len(samples)
    for g in grids:
        g.close()
    del samples, grids
    torch.cuda.empty_cache()
    nelx, nely, nelz = (int(v) for v in a.grid.split("x"))
    F, fixed = I.cantilever_3d(nelx, nely, nelz)
    p = default_params(3, nelx, nely, nelz, volfrac=0.12, penal=3.0, rmin=math.sqrt(3.0), ft=3, beta=2.0,
                       cg_rtol=1e-8, cg_maxit=50000, precision=TO_MIXED, precond=TO_PC_GMG, mg_nu=1,
                       inner_rtol=1e-4, penal_cnt=(1, 3.0, 25, 0.25), beta_cnt=(1, 16.0, 25, 2.0, TO_CNT_MUL))
    g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda())
    d = Design(g, torch.from_numpy(I.initial_design(g.nel, 0.12)).cuda())
    # the first state solve from U = 0, without and with the network
    first = {}
    snap = [t.clone() for t in (d.x, d.xPhys, d.xOld, d.U)], (d.st.eta, d.st.penal, d.st.beta, d.st.loop)
    for mode in ("plain", "learned"):
        for t, s in zip((d.x, d.xPhys, d.xOld, d.U), snap[0]):
            t.copy_(s)
        d.st.eta, d.st.penal, d.st.beta, d.st.loop = snap[1]
        Lr.attach(g, net if mode == "learned" else None)
        info = d.step()
        first[mode] = {"n_cg": info["n_cg"], "warm_err": info["warm_err"], "c": info["c"],
                       "t_solve_ms": round(info["t_solve_ms"], 2)}
    Lr.attach(g, None)
    for _ in range(a.warmup):
        d.step()
    snap = [t.clone() for t in (d.x, d.xPhys, d.xOld, d.U)], (d.st.eta, d.st.penal, d.st.beta, d.st.loop)
    runs = {}
    for mode in ("plain", "learned"):
        for t, s in zip((d.x, d.xPhys, d.xOld, d.U), snap[0]):
            t.copy_(s)
        d.st.eta, d.st.penal, d.st.beta, d.st.loop = snap[1]
        Lr.attach(g, net if mode == "learned" else None)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        infos = [d.step() for _ in range(a.steps)]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        runs[mode] = {"design_it_per_s": round(1e3 / ms, 3), "n_cg": [i["n_cg"] for i in infos],
                      "warm_err": [round(i["warm_err"], 6) for i in infos],
                      "warm_err_prev": [round(i["warm_err_prev"], 6) for i in infos],
                      "rel_res_max": max(i["rel_res"] for i in infos), "c_last": infos[-1]["c"]}
    Lr.attach(g, None)
    g.close()
    print(json.dumps({"grid": a.grid, "training_samples": n_samples, "training_shapes": shapes,
                      "runs": a.runs, "generate_s": round(t_gen, 1), "train_s": round(t_train, 1),
                      "epochs": a.epochs, "energy_loss_first_last": [round(hist[0], 4), round(hist[-1], 4)],
                      "first_solve": first, "iterations": f"{a.warmup + 2}..{a.warmup + 1 + a.steps}",
                      "runs_from_same_state": runs,
                      "c_rel_diff": abs(runs["learned"]["c_last"] - runs["plain"]["c_last"]) /
                      abs(runs["plain"]["c_last"])}))


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
        info = b.step(check=False)
        if info["status"] not in (0, 4):  # 4: TO_ENOTCONV (an instance stopped above cg_rtol), reported
            raise RuntimeError(f"batched step failed with status {info['status']}")
        steps.append({k: info[k] for k in ("loop", "status", "ms", "max_refinements", "max_inner_iters",
                                           "inner_passes", "newton_passes", "oc_passes", "max_rel_res", "stalled",
                                           "kernels")})
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
    ap.add_argument("--what", default="ku", choices=["ku", "batch", "net", "oc", "frame", "pae", "mbb", "learned", "mma"])
    ap.add_argument("--runs", type=int, default=100)
    ap.add_argument("--iters", type=int, default=54)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--grids", default="300x100,600x200,1200x400")
    ap.add_argument("--variant", default="config2", choices=["config2", "paper"])
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--cases", default="T1,T2,T3,T4")
    ap.add_argument("--ftbc", default="N", choices=["N", "D"])
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
     "pae": bench_pae, "mbb": bench_mbb, "learned": bench_learned, "mma": bench_mma}[a.what](a)


if __name__ == "__main__":
    main()
