"""The FP32 stiffness operators of the mixed path against the FP64 oracle.

impl 1: node-centric gather with the dense Ke (FP32 FMAs on CUDA cores);
impl 2: tcgen05 tensor cores (TF32 with split operands, FP32 accumulation in tensor
memory, streaming element slabs);
impl 3: element tiles with Ke factored in the Walsh basis of the corners (FP32
on CUDA cores); impl 4: the same product for two elements per thread in paired
FP32 instructions. All must reproduce K u to FP32-level accuracy (normwise 1e-5;
the split TF32 products carry about 21 bits).
"""
import numpy as np
import pytest

from oracle import topopt_oracle as O
from paper_2005_05436_gb300 import inputs as I
from tests._util import design_field, make_grid, rel, to_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


def _apply(g, xp, u, impl):
    from paper_2005_05436_gb300 import _lib as L
    y = torch.empty(g.ndof, dtype=torch.float64, device="cuda")
    xt, ut = to_cuda(xp), to_cuda(u)
    import ctypes as C
    L.check(g.lib.to_apply_K_fp32(g.h, C.c_void_p(xt.data_ptr()), C.c_void_p(ut.data_ptr()),
                                  C.c_void_p(y.data_ptr()), impl))
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("impl", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(7, 5, 3), (13, 9, 6), (4, 8, 4), (1, 1, 1), (24, 12, 12), (40, 33, 9),
                                   (5, 130, 17), (9, 200, 3), (6, 129, 40), (3, 2, 61), (11, 47, 23)])
def test_fp32_operator_matches_oracle(shape, impl):
    from paper_2005_05436_gb300 import TO_MIXED
    g, F, fixed = make_grid(shape, precision=TO_MIXED, penal=3.0)
    og = O.Grid(*shape)
    Ke = O.element_stiffness(3)
    xp = design_field(shape, 3, rmin=1.5)
    u = I.random_vector(g.ndof, 4)
    ref = O.apply_K(og, Ke, O.simp_modulus(xp, 3.0), u, fixed)
    got = _apply(g, xp, u, impl)
    assert rel(got, ref) <= 1e-5, rel(got, ref)
    assert np.all(got[fixed.astype(bool)] == 0)


def test_fp32_operators_agree_at_full_size():
    """96x48x48: tensor-core and CUDA-core FP32 operators agree, and sampled rows
    match the oracle's element sums."""
    from paper_2005_05436_gb300 import TO_MIXED
    shape = (96, 48, 48)
    g, F, fixed = make_grid(shape, precision=TO_MIXED, penal=3.0)
    xp = design_field(shape, 5)
    u = I.random_vector(g.ndof, 6)
    y1 = _apply(g, xp, u, 1)
    y2 = _apply(g, xp, u, 2)
    y3 = _apply(g, xp, u, 3)
    y4 = _apply(g, xp, u, 4)
    assert rel(y2, y1) <= 1e-5
    assert rel(y3, y1) <= 1e-5
    assert rel(y4, y1) <= 1e-5
    og = O.Grid(*shape)
    rows = np.random.default_rng(7).integers(0, g.ndof, 150)
    ref = O.apply_K_rows(og, O.element_stiffness(3), O.simp_modulus(xp, 3.0), u, rows, fixed)
    assert np.abs(y2[rows] - ref).max() <= 1e-5 * np.abs(ref).max()
    assert np.abs(y3[rows] - ref).max() <= 1e-5 * np.abs(ref).max()
    assert np.abs(y4[rows] - ref).max() <= 1e-5 * np.abs(ref).max()


def test_translation_invariance_exact():
    """Adding a rigid translation to u leaves the tensor-core K u bit-identical:
    each block stages its displacements relative to one of its nodes before
    rounding to TF32 parts, so with u and u + t exactly representable in FP32
    the staged differences are the same."""
    from paper_2005_05436_gb300 import TO_MIXED
    shape = (13, 9, 6)
    F, fixed = I.cantilever_3d(*shape)
    free = np.zeros_like(fixed)  # no supports: translations are null vectors of K
    g, _, _ = make_grid(shape, precision=TO_MIXED, penal=3.0, F=F, fixed=free)
    xp = design_field(shape, 8, rmin=1.5, lo=0.05)
    u = np.round(np.clip(I.random_vector(g.ndof, 9), -4, 4) * 2 ** 12) / 2 ** 12
    shift = np.tile([1024.0, -2048.0, 512.0], g.ndof // 3)
    y0 = _apply(g, xp, u, 2)
    y1 = _apply(g, xp, u + shift, 2)
    np.testing.assert_array_equal(y1, y0)
