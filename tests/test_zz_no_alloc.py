"""The OC update entry point that allocates nothing (to_oc_update_noalloc).

Some callers cannot call cudaMalloc: their device memory is already reserved by
another allocator, or they run a loop that must not take cudaMalloc's implicit
device synchronisation. to_oc_update_noalloc keeps its scratch in a file-scope
device array instead. This test calls it through the C ABI twice in a row and
compares each result with the existing handle-based to_oc_update, with the
tolerances of the OC parity tests. It lives in its own file, collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(n, seed, vf):
    rng = np.random.default_rng(seed)
    x = np.clip(vf + 0.3 * rng.standard_normal(n), 0.0, 1.0)
    dc = -np.abs(rng.standard_normal(n)) * 10 ** rng.uniform(-6, 2, n)
    dV0 = np.full(n, 1.0 / (n * vf)) * (1 + 0.1 * rng.random(n))
    return x, dc, dV0


@pytest.mark.parametrize("tol", [1e-15, 1e-4])
def test_noalloc_oc_matches_handle_entry_twice(tol):
    from paper_2005_05436_gb300 import _lib as L, build
    from tests._util import make_grid, rel
    build.build()
    lib = L.load()
    shape = (96, 48, 12)
    vf, move = 0.3, 0.2
    g, _, _ = make_grid(shape, volfrac=vf, move=move, oc_tol=tol)
    n = g.nel
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((21, 22)):
        x, dc, dV0 = _case(n, seed, vf)
        ref = torch.from_numpy(x).cuda()
        dct = torch.from_numpy(dc).cuda()
        dvt = torch.from_numpy(dV0).cuda()
        lm_ref = g.oc_update(ref, dct, dvt)
        got = torch.from_numpy(x).cuda()
        lm = C.c_double()
        torch.cuda.synchronize()
        # the first call on this device has loaded the module that holds the scratch
        # array; the second must leave the device's free memory and torch's pool as
        # they were (the property this entry point exists for)
        free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        st = lib.to_oc_update_noalloc(n, C.c_void_p(got.data_ptr()), C.c_void_p(dct.data_ptr()),
                                      C.c_void_p(dvt.data_ptr()), None, vf, move, tol, 200,
                                      2_000_000_000, C.c_void_p(stream.cuda_stream), C.byref(lm))
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_reserved() == reserved0
        assert st == L.TO_OK, (call, st, lib.to_last_error())
        assert abs(lm.value - lm_ref) <= max(tol, 1e-14) * 4 * lm_ref, (call, lm.value, lm_ref)
        assert rel(got.cpu().numpy(), ref.cpu().numpy()) <= 1e-12, call


def test_noalloc_oc_against_oracle_and_maxit():
    """Once directly against the oracle's OC bisection (parity tolerance), then
    with oc_maxit = 1: the search stops early and the call says so."""
    from oracle import topopt_oracle as O
    from paper_2005_05436_gb300 import _lib as L, build
    build.build()
    lib = L.load()
    n, vf, move = 30000, 0.3, 0.2
    x, dc, dV0 = _case(n, 31, vf)
    xr, lm_ref, _ = O.oc_update(x, dc, dV0, np.ones(n, bool), move, vf, tol=1e-15)
    got = torch.from_numpy(x).cuda()
    dct, dvt = torch.from_numpy(dc).cuda(), torch.from_numpy(dV0).cuda()
    lm = C.c_double()
    st = lib.to_oc_update_noalloc(n, C.c_void_p(got.data_ptr()), C.c_void_p(dct.data_ptr()),
                                  C.c_void_p(dvt.data_ptr()), None, vf, move, 1e-15, 200, 2_000_000_000,
                                  None, C.byref(lm))
    assert st == L.TO_OK
    assert abs(lm.value - lm_ref) <= 1e-12 * lm_ref, (lm.value, lm_ref)
    assert np.abs(got.cpu().numpy() - xr).max() <= 1e-12
    got = torch.from_numpy(x).cuda()
    st = lib.to_oc_update_noalloc(n, C.c_void_p(got.data_ptr()), C.c_void_p(dct.data_ptr()),
                                  C.c_void_p(dvt.data_ptr()), None, vf, move, 1e-15, 1, 2_000_000_000,
                                  None, C.byref(lm))
    assert st == L.TO_ENOTCONV
    assert b"oc_maxit" in lib.to_last_error()


def test_noalloc_oc_with_passive_and_size_limit():
    from paper_2005_05436_gb300 import _lib as L, build, inputs as I
    from tests._util import make_grid, rel
    build.build()
    lib = L.load()
    F, fixed, pas = I.frame_reinforcement(100, 50)
    g, _, _ = make_grid((100, 50, 0), F=F, fixed=fixed, passive=pas, volfrac=0.2, oc_tol=1e-15)
    x, dc, dV0 = _case(g.nel, 5, 0.2)
    x[pas == 1], x[pas == -1] = 1.0, 0.0
    dct, dvt = torch.from_numpy(dc).cuda(), torch.from_numpy(dV0).cuda()
    ref = torch.from_numpy(x).cuda()
    lm_ref = g.oc_update(ref, dct, dvt)
    got = torch.from_numpy(x).cuda()
    pt = torch.from_numpy(pas).cuda()
    lm = C.c_double()
    st = lib.to_oc_update_noalloc(g.nel, C.c_void_p(got.data_ptr()), C.c_void_p(dct.data_ptr()),
                                  C.c_void_p(dvt.data_ptr()), C.c_void_p(pt.data_ptr()), 0.2, 0.2,
                                  1e-15, 200, 2_000_000_000, None, C.byref(lm))
    assert st == L.TO_OK
    assert abs(lm.value - lm_ref) <= 4e-14 * lm_ref
    assert rel(got.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
    # beyond the stated maximum (1,048,576 elements) the call is rejected
    st = lib.to_oc_update_noalloc((1 << 20) + 1, C.c_void_p(got.data_ptr()), C.c_void_p(dct.data_ptr()),
                                  C.c_void_p(dvt.data_ptr()), None, 0.2, 0.2, 1e-4, 200,
                                  2_000_000_000, None, C.byref(lm))
    assert st == L.TO_EINVAL
