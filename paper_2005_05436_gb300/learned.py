"""Learned warm start of the state solve: the network handle and its training
and inference calls (marshalling only; the network runs in libtopopt's kernels).

Net wraps a to_net handle: parameters, forward, gradient accumulation and Adam
steps on CUDA float32 tensors laid out [N][D][H][W][C].
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib as L


def layer_shapes(base=16, cin=4, cout=3):
    """(cin, cout) of the 11 convolutions, in parameter order."""
    c = base
    return [(cin, c), (c, c), (c, 2 * c), (2 * c, 2 * c), (2 * c, 4 * c), (4 * c, 4 * c),
            (4 * c, 2 * c), (2 * c, 2 * c), (2 * c, c), (c, c), (c, cout)]


def he_init(base=16, seed=0):
    """He-normal weights and zero biases from a seeded numpy generator (FP32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in layer_shapes(base):
        parts.append(rng.standard_normal(27 * a * b) * np.sqrt(2.0 / (27 * a)))
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


def _fp(t, name, n=None, dtype=torch.float32):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements")
    return C.c_void_p(t.data_ptr())


class Net:
    def __init__(self, base=16, bf16=True, stream=None, tensor_cores=True):
        self.lib = L.load()
        self.base = base
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = L.NetCfg(int(base), 1 if bf16 else 0, 4, 3, 0 if tensor_cores else 1, 0)
        h = C.c_void_p()
        L.check(self.lib.to_net_create(C.byref(cfg), C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.n_params = int(self.lib.to_net_param_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.to_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        t = torch.as_tensor(np.ascontiguousarray(theta, np.float32)).cuda() \
            if not isinstance(theta, torch.Tensor) else theta.to(torch.float32).contiguous()
        L.check(self.lib.to_net_set_params(self.h, _fp(t, "theta", self.n_params)))

    def params(self):
        t = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        L.check(self.lib.to_net_get_params(self.h, _fp(t, "theta")))
        return t

    def grad(self):
        t = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        L.check(self.lib.to_net_get_grad(self.h, _fp(t, "grad")))
        return t

    def zero_grad(self):
        L.check(self.lib.to_net_zero_grad(self.h))

    def forward(self, x):
        N, D, H, W, Cin = x.shape
        assert Cin == 4
        y = torch.empty((N, D, H, W, 3), dtype=torch.float32, device="cuda")
        L.check(self.lib.to_net_forward(self.h, _fp(x, "x"), N, D, H, W, _fp(y, "y")))
        return y

    def accumulate(self, x, target, mask):
        N, D, H, W, _ = x.shape
        loss = C.c_double()
        L.check(self.lib.to_net_accumulate(self.h, _fp(x, "x"), _fp(target, "target", N * D * H * W * 3),
                                           _fp(mask, "mask", N * D * H * W, torch.uint8), N, D, H, W,
                                           C.byref(loss)))
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0):
        L.check(self.lib.to_net_adam(self.h, float(lr), float(beta1), float(beta2), float(eps), float(grad_scale)))


# ------------------------------------------------------------- grid interface

def features(grid, xPhys, out=None):
    """Network input of a 3D Grid at xPhys (library kernel): [1, D, H, W, 4]."""
    dims = (C.c_int32 * 3)()
    L.check(grid.lib.to_learned_features(grid.h, None, None, dims))
    D, H, W = dims
    if out is None:
        out = torch.empty((1, D, H, W, 4), dtype=torch.float32, device="cuda")
    L.check(grid.lib.to_learned_features(grid.h, C.c_void_p(xPhys.data_ptr()), _fp(out, "x", D * H * W * 4),
                                         dims))
    return out


def target(grid, U):
    """Training target U / rms(U) on the padded node grid and its node mask."""
    dims = (C.c_int32 * 3)()
    L.check(grid.lib.to_learned_features(grid.h, None, None, dims))
    D, H, W = dims
    t = torch.empty((1, D, H, W, 3), dtype=torch.float32, device="cuda")
    m = torch.empty((1, D, H, W), dtype=torch.uint8, device="cuda")
    L.check(grid.lib.to_learned_target(grid.h, C.c_void_p(U.data_ptr()), _fp(t, "t"), _fp(m, "mask", None,
                                                                                          torch.uint8)))
    return t, m


def attach(grid, net, stride=2, rule=None):
    """Use net as the warm start of every to_step of grid (None detaches); the
    network works on the node grid coarsened by stride; rule: TO_WARM_ENERGY or
    TO_WARM_RESIDUAL (how U_prev and the network's output are combined; None
    keeps the grid's rule)."""
    L.check(grid.lib.to_set_warm_start(grid.h, net.h if net is not None else None, int(stride)))
    if rule is not None:
        L.check(grid.lib.to_set_warm_start_rule(grid.h, int(rule)))


def generate(shapes, runs, iters, seed=0, every=1, warmup=2, stride=2, **params):
    """(features, target, mask) triples from runs of the method itself: for each
    run a cantilever-family problem (inputs.cantilever_family) on one of the
    given grid shapes is advanced by to_step (mixed precision + multigrid) and
    every `every`-th design after `warmup` iterations is recorded. Returns a
    dict shape -> list of (x, t, m) CUDA tensors."""
    from . import TO_MIXED, TO_PC_GMG, default_params, inputs as I
    from .topopt import Design, Grid
    out = {}
    for r in range(runs):
        nelx, nely, nelz = shapes[r % len(shapes)]
        F, fixed, vf = I.cantilever_family(nelx, nely, nelz, seed + r)
        kw = dict(precision=TO_MIXED, precond=TO_PC_GMG, volfrac=vf, rmin=math.sqrt(3.0), beta=2.0,
                  beta_cnt=(1, 16.0, 10, 2.0, 1), cg_rtol=1e-8, cg_maxit=5000)
        kw.update(params)
        p = default_params(3, nelx, nely, nelz, **kw)
        g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda())
        attach(g, None, stride)
        d = Design(g, torch.full((g.nel,), vf, dtype=torch.float64, device="cuda"))
        for k in range(iters):
            d.step()
            if k >= warmup and (k - warmup) % every == 0:
                x = features(g, d.xPhys)
                t, m = target(g, d.U)
                out.setdefault((nelx, nely, nelz), []).append((x, t, m))
        g.close()
    return out


def train(net, data, epochs, lr=2e-3, batch=4, seed=0, log=None, lr_final=None):
    """Adam on the masked MSE over mini-batches of equal-shape samples; the
    learning rate decays geometrically from lr to lr_final (default lr)."""
    rng = np.random.default_rng(seed)
    groups = []
    for shape, items in data.items():
        for i in range(0, len(items), batch):
            groups.append(items[i:i + batch])
    hist = []
    lr_final = lr if lr_final is None else lr_final
    for ep in range(epochs):
        lr_ep = lr * (lr_final / lr) ** (ep / max(1, epochs - 1))
        tot, cnt = 0.0, 0
        for gi in rng.permutation(len(groups)):
            grp = groups[gi]
            x = torch.cat([a for a, _, _ in grp])
            t = torch.cat([b for _, b, _ in grp])
            m = torch.cat([c for _, _, c in grp])
            net.zero_grad()
            loss = net.accumulate(x, t, m)
            net.adam(lr_ep)
            tot += loss * len(grp)
            cnt += len(grp)
        hist.append(tot / max(cnt, 1))
        if log:
            log(ep, hist[-1])
    return hist


def generate_energy(shapes, runs, iters, seed=0, every=1, warmup=2, stride=2, **params):
    """Samples for the energy objective: for each run a cantilever-family
    problem is advanced by to_step; recorded are the network input, the design
    xPhys and its converged compliance, with the run's Grid (which holds F and
    the supports) kept open for the training-time operator products."""
    from . import TO_MIXED, TO_PC_GMG, default_params, inputs as I
    from .topopt import Design, Grid
    samples, grids = [], []
    for r in range(runs):
        nelx, nely, nelz = shapes[r % len(shapes)]
        F, fixed, vf = I.cantilever_family(nelx, nely, nelz, seed + r)
        kw = dict(precision=TO_MIXED, precond=TO_PC_GMG, volfrac=vf, rmin=math.sqrt(3.0), beta=2.0,
                  beta_cnt=(1, 16.0, 10, 2.0, 1), cg_rtol=1e-8, cg_maxit=5000)
        kw.update(params)
        p = default_params(3, nelx, nely, nelz, **kw)
        g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda())
        attach(g, None, stride)
        d = Design(g, torch.full((g.nel,), vf, dtype=torch.float64, device="cuda"))
        for k in range(iters):
            info = d.step()
            if k >= warmup and (k - warmup) % every == 0:
                samples.append((len(grids), features(g, d.xPhys), d.xPhys.clone(), float(info["c"]),
                                float(d.st.penal)))
        grids.append(g)
    return samples, grids


def train_energy(net, samples, grids, epochs, lr=1e-3, lr_final=None, batch=4, seed=0, log=None):
    """Adam on the mean relative energy error of the network direction
    (to_learned_energy_grad) over mini-batches of samples of one grid shape."""
    rng = np.random.default_rng(seed)
    by_shape = {}
    for i, s in enumerate(samples):
        by_shape.setdefault(tuple(s[1].shape), []).append(i)
    groups = []
    for idx in by_shape.values():
        for k in range(0, len(idx), batch):
            groups.append(idx[k:k + batch])
    lr_final = lr if lr_final is None else lr_final
    hist = []
    for ep in range(epochs):
        lr_ep = lr * (lr_final / lr) ** (ep / max(1, epochs - 1))
        tot = 0.0
        for gi in rng.permutation(len(groups)):
            grp = groups[gi]
            x = torch.cat([samples[i][1] for i in grp])
            N, D, H, W, _ = x.shape
            y = net.forward(x)
            gy = torch.empty_like(y)
            net.zero_grad()
            for b, i in enumerate(grp):
                gi_, _, xphys, c, penal = samples[i]
                g = grids[gi_]
                g.set_scalars(penal, g.params.beta, g.params.eta)
                loss = C.c_double()
                L.check(g.lib.to_learned_energy_grad(g.h, C.c_void_p(xphys.data_ptr()), C.c_void_p(y[b].data_ptr()),
                                                     float(c), C.c_void_p(gy[b].data_ptr()), C.byref(loss)))
                tot += loss.value
            L.check(net.lib.to_net_backward(net.h, _fp(gy, "gy"), N, D, H, W))
            net.adam(lr_ep, grad_scale=1.0 / len(grp))
        hist.append(tot / len(samples))
        if log:
            log(ep, hist[-1])
    return hist
