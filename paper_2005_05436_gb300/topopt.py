"""Python face of the C ABI: one object per grid handle, torch tensors in and out.

Marshalling only: shapes, dtypes and devices are checked, pointers and the
current torch stream are passed to libtopopt.so, and results come back in the
caller's tensors. Nothing here computes any part of the method.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L


def _ptr(t, dtype, n, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class Grid:
    """A to_grid handle (to_init_grid ... to_destroy)."""

    def __init__(self, params: L.Params, F, fixed, passive=None, stream=None):
        self.lib = L.load()
        self.params = params
        dim = params.dim
        self.nel = params.nelx * params.nely * (params.nelz if dim == 3 else 1)
        self.nnodes = (params.nelx + 1) * (params.nely + 1) * ((params.nelz + 1) if dim == 3 else 1)
        self.ndof = dim * self.nnodes
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        L.check(self.lib.to_init_grid(
            C.byref(params), _ptr(F, torch.float64, self.ndof, "F"),
            _ptr(fixed, torch.uint8, self.ndof, "fixed"),
            _ptr(passive, torch.int8, self.nel, "passive"),
            C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.to_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scalars(self, penal, beta, eta):
        L.check(self.lib.to_set_scalars(self.h, penal, beta, eta))

    def apply_K(self, xPhys, u, y, masked=True):
        L.check(self.lib.to_apply_K(self.h, _ptr(xPhys, torch.float64, self.nel, "xPhys"),
                                    _ptr(u, torch.float64, self.ndof, "u"),
                                    _ptr(y, torch.float64, self.ndof, "y"), int(masked)))
        return y

    def solve(self, xPhys, U, F=None, check=True):
        info = L.SolveInfo()
        st = self.lib.to_solve(self.h, _ptr(xPhys, torch.float64, self.nel, "xPhys"),
                               _ptr(F, torch.float64, self.ndof, "F"),
                               _ptr(U, torch.float64, self.ndof, "U"), C.byref(info))
        if check:
            L.check(st)
        return info

    def filter(self, x, out, dprj=None):
        L.check(self.lib.to_filter(self.h, _ptr(x, torch.float64, self.nel, "in"),
                                   _ptr(out, torch.float64, self.nel, "out"),
                                   _ptr(dprj, torch.float64, self.nel, "dprj")))
        return out

    def project(self, xTilde, xPhys, dprj, eta, volume_preserving=True):
        e = C.c_double(eta)
        L.check(self.lib.to_project(self.h, _ptr(xTilde, torch.float64, self.nel, "xTilde"),
                                    _ptr(xPhys, torch.float64, self.nel, "xPhys"),
                                    _ptr(dprj, torch.float64, self.nel, "dprj"), C.byref(e),
                                    int(volume_preserving)))
        return e.value

    def sensitivity(self, xPhys, U, dc):
        c = C.c_double()
        L.check(self.lib.to_sensitivity(self.h, _ptr(xPhys, torch.float64, self.nel, "xPhys"),
                                        _ptr(U, torch.float64, self.ndof, "U"),
                                        _ptr(dc, torch.float64, self.nel, "dc"), C.byref(c)))
        return c.value

    def oc_update(self, x, dc, dV0):
        lm = C.c_double()
        L.check(self.lib.to_oc_update(self.h, _ptr(x, torch.float64, self.nel, "x"),
                                      _ptr(dc, torch.float64, self.nel, "dc"),
                                      _ptr(dV0, torch.float64, self.nel, "dV0"), C.byref(lm)))
        return lm.value

    def time_apply_K(self, xPhys, precision=L.TO_FP64, reps=20):
        """Average device microseconds of one K u kernel launch (instrumentation)."""
        us = C.c_double()
        L.check(self.lib.to_time_apply_K(self.h, _ptr(xPhys, torch.float64, self.nel, "xPhys"),
                                         int(precision), int(reps), C.byref(us)))
        return us.value

    def assemble_lower(self, xPhys):
        """Returns (row_ptr int32 [nDof+1], col int32 [nnz], val float64 [nnz]) on the GPU."""
        nnz = C.c_int64(0)
        L.check(self.lib.to_assemble_lower(self.h, None, C.byref(nnz), None, None, None))
        dev = xPhys.device
        row_ptr = torch.empty(self.ndof + 1, dtype=torch.int32, device=dev)
        col = torch.empty(nnz.value, dtype=torch.int32, device=dev)
        val = torch.empty(nnz.value, dtype=torch.float64, device=dev)
        L.check(self.lib.to_assemble_lower(self.h, _ptr(xPhys, torch.float64, self.nel, "xPhys"),
                                           C.byref(nnz), _ptr(row_ptr, torch.int32, None, "row_ptr"),
                                           _ptr(col, torch.int32, None, "col"),
                                           _ptr(val, torch.float64, None, "val")))
        return row_ptr, col, val


class Design:
    """Design state (x, xPhys, xOld, U and the continuation scalars) for Grid.step."""

    def __init__(self, grid: Grid, x0, passive=None):
        dev = x0.device
        self.grid = grid
        self.x = x0.clone()
        self.xPhys = x0.clone()
        self.xOld = torch.ones(grid.nel, dtype=torch.float64, device=dev)
        self.U = torch.zeros(grid.ndof, dtype=torch.float64, device=dev)
        p = grid.params
        self.st = L.State(self.x.data_ptr(), self.xPhys.data_ptr(), self.xOld.data_ptr(),
                          self.U.data_ptr(), p.eta, p.penal, p.beta, 0, 0)

    def step(self, check=True):
        info = L.IterInfo()
        s = self.grid.lib.to_step(self.grid.h, C.byref(self.st), C.byref(info))
        if check:
            L.check(s)
        return info.as_dict()

    @property
    def loop(self):
        return self.st.loop


class Batch:
    """A to_batch handle: uneven 2D instances advanced together (to_batch_init ...
    to_batch_destroy). F and fixed are concatenated over the instances' DOFs;
    the state tensors x, xPhys, xOld, U are created here in the same layout."""

    def __init__(self, params: L.Params, instances, F, fixed, x0, stream=None):
        self.lib = L.load()
        self.params = params
        self.count = len(instances)
        arr = (L.Instance * self.count)()
        for k, (nelx, nely, volfrac, rmin) in enumerate(instances):
            arr[k] = L.Instance(int(nelx), int(nely), float(volfrac), float(rmin))
        self.instances = arr
        self.nel = sum(int(a) * int(b) for a, b, _, _ in instances)
        self.ndof = sum(2 * (int(a) + 1) * (int(b) + 1) for a, b, _, _ in instances)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.F = F
        self.fixed = fixed
        h = C.c_void_p()
        L.check(self.lib.to_batch_init(C.byref(params), self.count, arr,
                                       _ptr(F, torch.float64, self.ndof, "F"),
                                       _ptr(fixed, torch.uint8, self.ndof, "fixed"),
                                       C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        el = (C.c_int64 * (self.count + 1))()
        dof = (C.c_int64 * (self.count + 1))()
        L.check(self.lib.to_batch_offsets(self.h, el, dof))
        self.el_off = list(el)
        self.dof_off = list(dof)
        dev = F.device
        _ptr(x0, torch.float64, self.nel, "x0")
        self.x = x0.clone()
        self.xPhys = x0.clone()
        self.xOld = torch.ones(self.nel, dtype=torch.float64, device=dev)
        self.U = torch.zeros(self.ndof, dtype=torch.float64, device=dev)

    def close(self):
        if getattr(self, "h", None):
            self.lib.to_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, reps=10):
        info = L.TileInfo()
        L.check(self.lib.to_batch_autotune(self.h, int(reps), C.byref(info)))
        n = info.n_candidates
        return {"node": (info.node_ty, info.node_tx), "elem": (info.elem_ty, info.elem_tx),
                "candidates": [(info.cand_ty[k], info.cand_tx[k]) for k in range(n)],
                "node_us": [info.node_us[k] for k in range(n)], "elem_us": [info.elem_us[k] for k in range(n)]}

    def step(self, check=True):
        info = L.BatchInfo()
        s = self.lib.to_batch_step(self.h, C.c_void_p(self.x.data_ptr()), C.c_void_p(self.xPhys.data_ptr()),
                                   C.c_void_p(self.xOld.data_ptr()), C.c_void_p(self.U.data_ptr()),
                                   C.byref(info))
        if check:
            L.check(s)
        return {k: getattr(info, k) for k, _ in L.BatchInfo._fields_ if not k.startswith("_")}

    def results(self):
        n = self.count
        c, V, ch, eta, lm, rr = ((C.c_double * n)() for _ in range(6))
        it, ref = (C.c_int32 * n)(), (C.c_int32 * n)()
        L.check(self.lib.to_batch_results(self.h, c, V, ch, eta, lm, it, ref, rr))
        return {"c": list(c), "V": list(V), "ch": list(ch), "eta": list(eta), "lm": list(lm),
                "inner_iters": list(it), "refinements": list(ref), "rel_res": list(rr)}

    def instance(self, k, t):
        """The slice of a concatenated element (nEl-long) or DOF (nDof-long) tensor for instance k."""
        off = self.el_off if t.numel() == self.nel else self.dof_off
        return t[off[k]:off[k + 1]]
