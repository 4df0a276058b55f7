"""GB300-native (sm_103a) SIMP topology-optimisation hot path (Ferrari & Sigmund 2020).

The CUDA library ``libtopopt.so`` (C ABI in include/topopt.h) is built in-tree by
``paper_2005_05436_gb300.build.build()``; ``Grid`` / ``Design`` are thin torch
bindings of it. Importing this package does not load the library; the first
``Grid`` does, and raises if it has not been built.
"""
from ._lib import (TO_OC_BISECTION, TO_OC_PRIMAL_DUAL, TO_OC_PHYSICAL_VOLUME, TO_CNT_ADD, TO_CNT_MUL, TO_FP64, TO_MIXED, TO_PC_GMG, TO_PC_JACOBI,  # noqa: F401
                   TO_REFINE_RELIABLE, TO_REFINE_FLEXIBLE, TO_WARM_ENERGY, TO_WARM_RESIDUAL, TO_OK, TO_EINVAL, TO_ENOMEM, TO_ECUDA, TO_ENOTCONV, TO_ENAN, TO_ETIMEOUT,
                   TopoptError, default_params, load)


def __getattr__(name):
    if name in ("Grid", "Design", "Batch"):
        from . import topopt
        return getattr(topopt, name)
    raise AttributeError(name)
