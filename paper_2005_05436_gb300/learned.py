"""Learned warm start of the state solve: the network handle and its training
and inference calls (marshalling only; the network runs in libtopopt's kernels).

Net wraps a to_net handle: parameters, forward, gradient accumulation and Adam
steps on CUDA float32 tensors laid out [N][D][H][W][C].
"""
from __future__ import annotations

import ctypes as C

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
    def __init__(self, base=16, bf16=True, stream=None):
        self.lib = L.load()
        self.base = base
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = L.NetCfg(int(base), 1 if bf16 else 0, 4, 3)
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
