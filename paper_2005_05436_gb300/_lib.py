"""ctypes binding of the C ABI in include/topopt.h (argument marshalling only).

Arrays are torch CUDA tensors; their device pointers and the current torch
stream are passed straight through. Every step of the method runs in the CUDA
library; if it is missing this module raises instead of computing anything.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtopopt.so")

TO_OK, TO_EINVAL, TO_ENOMEM, TO_ECUDA, TO_ENOTCONV, TO_ENAN, TO_ETIMEOUT = range(7)
STATUS_NAMES = {0: "TO_OK", 1: "TO_EINVAL", 2: "TO_ENOMEM", 3: "TO_ECUDA", 4: "TO_ENOTCONV",
                5: "TO_ENAN", 6: "TO_ETIMEOUT"}
TO_FP64, TO_MIXED = 0, 1
TO_PC_JACOBI, TO_PC_GMG = 0, 1
TO_CNT_ADD, TO_CNT_MUL = 0, 1
TO_OC_BISECTION, TO_OC_PRIMAL_DUAL, TO_OC_PHYSICAL_VOLUME = 0, 1, 2
TO_REFINE_RELIABLE, TO_REFINE_FLEXIBLE = 0, 1
TO_WARM_ENERGY, TO_WARM_RESIDUAL = 0, 1


class Continuation(C.Structure):
    _fields_ = [("istart", C.c_int32), ("isteps", C.c_int32), ("maxpar", C.c_double),
                ("delta", C.c_double), ("kind", C.c_int32), ("_pad", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nelx", C.c_int32), ("nely", C.c_int32), ("nelz", C.c_int32),
                ("E0", C.c_double), ("Emin", C.c_double), ("nu", C.c_double),
                ("volfrac", C.c_double), ("penal", C.c_double), ("rmin", C.c_double),
                ("ft", C.c_int32), ("ftBC", C.c_int32),
                ("eta", C.c_double), ("beta", C.c_double), ("move", C.c_double),
                ("penal_cnt", Continuation), ("beta_cnt", Continuation),
                ("newton_tol", C.c_double), ("newton_maxit", C.c_int32), ("oc_maxit", C.c_int32),
                ("oc_tol", C.c_double), ("cg_rtol", C.c_double), ("cg_maxit", C.c_int32),
                ("precision", C.c_int32), ("precond", C.c_int32), ("mg_levels", C.c_int32),
                ("deadline_cycles", C.c_int64), ("inner_rtol", C.c_double),
                ("mg_omega", C.c_double), ("mg_nu", C.c_int32), ("ku_impl", C.c_int32),
                ("loop_mode", C.c_int32), ("mg_coarse_every", C.c_int32), ("oc_method", C.c_int32),
                ("pae_q0", C.c_int32), ("pae_q", C.c_int32), ("pae_m", C.c_int32), ("pae_alpha", C.c_double),
                ("pae_zeta", C.c_double), ("inner_maxit", C.c_int32), ("refine", C.c_int32),
                ("mg_unfused", C.c_int32), ("pdl_off", C.c_int32),
                ("mg_nu_fine", C.c_int32), ("_pad5", C.c_int32), ("mg_omega_coarse", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("refinements", C.c_int32), ("rel_res", C.c_double),
                ("status", C.c_int32), ("fallback", C.c_int32), ("t_setup_ms", C.c_double),
                ("t_krylov_ms", C.c_double), ("t_resid_ms", C.c_double)]


class State(C.Structure):
    _fields_ = [("x", C.c_void_p), ("xPhys", C.c_void_p), ("xOld", C.c_void_p), ("U", C.c_void_p),
                ("eta", C.c_double), ("penal", C.c_double), ("beta", C.c_double),
                ("loop", C.c_int32), ("_pad", C.c_int32)]


class IterInfo(C.Structure):
    _fields_ = [("loop", C.c_int32), ("n_cg", C.c_int32), ("n_refine", C.c_int32),
                ("n_newton", C.c_int32), ("n_bisect", C.c_int32), ("status", C.c_int32),
                ("c", C.c_double), ("V", C.c_double), ("ch", C.c_double), ("penal", C.c_double),
                ("beta", C.c_double), ("eta", C.c_double), ("lm", C.c_double),
                ("rel_res", C.c_double), ("t_filter_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("t_sens_ms", C.c_double), ("t_oc_ms", C.c_double), ("t_setup_ms", C.c_double),
                ("t_krylov_ms", C.c_double), ("t_resid_ms", C.c_double), ("t_warm_ms", C.c_double), ("warm_a", C.c_double), ("warm_b", C.c_double),
                ("warm_err_prev", C.c_double), ("warm_err", C.c_double), ("pae", C.c_int32), ("fallback", C.c_int32),
                ("warm_res_prev", C.c_double), ("warm_res", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Instance(C.Structure):
    _fields_ = [("nelx", C.c_int32), ("nely", C.c_int32), ("volfrac", C.c_double), ("rmin", C.c_double)]


class TileInfo(C.Structure):
    _fields_ = [("node_ty", C.c_int32), ("node_tx", C.c_int32), ("elem_ty", C.c_int32), ("elem_tx", C.c_int32),
                ("n_candidates", C.c_int32), ("cand_ty", C.c_int32 * 8), ("cand_tx", C.c_int32 * 8),
                ("node_us", C.c_double * 8), ("elem_us", C.c_double * 8)]


class BatchInfo(C.Structure):
    _fields_ = [("loop", C.c_int32), ("status", C.c_int32), ("max_refinements", C.c_int32),
                ("max_inner_iters", C.c_int32), ("newton_passes", C.c_int32), ("inner_passes", C.c_int32),
                ("oc_passes", C.c_int32), ("stalled", C.c_int32), ("max_rel_res", C.c_double),
                ("penal", C.c_double), ("beta", C.c_double), ("ms", C.c_double), ("kernels", C.c_int64)]


class NetCfg(C.Structure):
    _fields_ = [("base", C.c_int32), ("bf16", C.c_int32), ("in_ch", C.c_int32), ("out_ch", C.c_int32),
                ("cuda_cores_only", C.c_int32), ("_pad", C.c_int32)]


class TopoptError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


P = C.c_void_p
_SIGS = {
    "to_last_error": (C.c_char_p, []),
    "to_sizeof_params": (C.c_size_t, []),
    "to_sizeof_state": (C.c_size_t, []),
    "to_sizeof_iter_info": (C.c_size_t, []),
    "to_params_init": (C.c_int, [C.POINTER(Params), C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "to_init_grid": (C.c_int, [C.POINTER(Params), P, P, P, P, C.POINTER(P)]),
    "to_destroy": (None, [P]),
    "to_set_scalars": (C.c_int, [P, C.c_double, C.c_double, C.c_double]),
    "to_assemble_lower": (C.c_int, [P, P, C.POINTER(C.c_int64), P, P, P]),
    "to_apply_K": (C.c_int, [P, P, P, P, C.c_int32]),
    "to_solve": (C.c_int, [P, P, P, P, C.POINTER(SolveInfo)]),
    "to_filter": (C.c_int, [P, P, P, P]),
    "to_project": (C.c_int, [P, P, P, P, C.POINTER(C.c_double), C.c_int32]),
    "to_sensitivity": (C.c_int, [P, P, P, P, C.POINTER(C.c_double)]),
    "to_oc_update": (C.c_int, [P, P, P, P, C.POINTER(C.c_double)]),
    "to_step": (C.c_int, [P, C.POINTER(State), C.POINTER(IterInfo)]),
    "to_oc_update_noalloc": (C.c_int, [C.c_int64, P, P, P, P, C.c_double, C.c_double, C.c_double,
                                       C.c_int32, C.c_int64, P, C.POINTER(C.c_double)]),
    "to_kernel_launches": (C.c_int64, []),
    "to_apply_K_fp32": (C.c_int, [P, P, P, P, C.c_int32]),
    "to_time_apply_K": (C.c_int, [P, P, C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "to_time_tf32_mma": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "to_batch_init": (C.c_int, [C.POINTER(Params), C.c_int32, C.POINTER(Instance), P, P, P, C.POINTER(P)]),
    "to_batch_offsets": (C.c_int, [P, P, P]),
    "to_batch_autotune": (C.c_int, [P, C.c_int32, C.POINTER(TileInfo)]),
    "to_batch_step": (C.c_int, [P, P, P, P, P, C.POINTER(BatchInfo)]),
    "to_batch_results": (C.c_int, [P, P, P, P, P, P, P, P, P]),
    "to_batch_destroy": (None, [P]),
    "to_sizeof_instance": (C.c_size_t, []),
    "to_sizeof_net_cfg": (C.c_size_t, []),
    "to_net_create": (C.c_int, [C.POINTER(NetCfg), P, C.POINTER(P)]),
    "to_net_param_count": (C.c_int64, [P]),
    "to_net_set_params": (C.c_int, [P, P]),
    "to_net_get_params": (C.c_int, [P, P]),
    "to_net_forward": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P]),
    "to_net_accumulate": (C.c_int, [P, P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                    C.POINTER(C.c_double)]),
    "to_net_get_grad": (C.c_int, [P, P]),
    "to_net_zero_grad": (C.c_int, [P]),
    "to_net_adam": (C.c_int, [P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]),
    "to_net_destroy": (None, [P]),
    "to_set_warm_start": (C.c_int, [P, P, C.c_int32]),
    "to_set_warm_start_rule": (C.c_int, [P, C.c_int32]),
    "to_learned_features": (C.c_int, [P, P, P, P]),
    "to_learned_target": (C.c_int, [P, P, P, P]),
    "to_learned_energy_grad": (C.c_int, [P, P, P, C.c_double, P, C.POINTER(C.c_double)]),
    "to_net_backward": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "to_sizeof_tile_info": (C.c_size_t, []),
    "to_sizeof_batch_info": (C.c_size_t, []),
}

_lib = None


def load(path=LIB_PATH):
    """Load libtopopt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2005_05436_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    assert lib.to_sizeof_params() == C.sizeof(Params), "to_params layout mismatch"
    assert lib.to_sizeof_state() == C.sizeof(State), "to_state layout mismatch"
    assert lib.to_sizeof_instance() == C.sizeof(Instance), "to_instance layout mismatch"
    assert lib.to_sizeof_net_cfg() == C.sizeof(NetCfg), "to_net_cfg layout mismatch"
    assert lib.to_sizeof_tile_info() == C.sizeof(TileInfo), "to_tile_info layout mismatch"
    assert lib.to_sizeof_batch_info() == C.sizeof(BatchInfo), "to_batch_info layout mismatch"
    assert lib.to_sizeof_iter_info() == C.sizeof(IterInfo), "to_iter_info layout mismatch"
    _lib = lib
    return lib


def check(status):
    if status != TO_OK:
        msg = _lib.to_last_error().decode() if _lib is not None else ""
        raise TopoptError(status, msg)
    return status


def default_params(dim, nelx, nely, nelz=0, **kw):
    """to_params_init defaults, then keyword overrides (ftBC may be 'N'/'D')."""
    lib = load()
    p = Params()
    check(lib.to_params_init(C.byref(p), dim, nelx, nely, nelz))
    for k, v in kw.items():
        if k == "ftBC" and isinstance(v, str):
            v = ord(v)
        if k in ("penal_cnt", "beta_cnt") and not isinstance(v, Continuation):
            istart, maxpar, isteps, delta = v[:4]
            kind = v[4] if len(v) > 4 else TO_CNT_ADD
            v = Continuation(int(istart), int(isteps), float(maxpar), float(delta), int(kind), 0)
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p
