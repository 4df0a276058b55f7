"""Pins of the oracle's design-iteration glue (design_step) against what the
paper fixes: the initial design with passive sets (Appendix B, PRE.6), passive
densities kept through filter and projection (RL.1), the volume equation of the
OC update taken over all elements (Eq. 13, passive ones included), the order of
continuation (after the OC update, post-increment loop counter), and the wiring
of periodic Anderson extrapolation (Sec. 3.6): the damped step with alpha = 1
is the plain OC step, the damped step with alpha is x + alpha r with r the OC
step's residual, and extrapolation happens exactly on the loops of reading R23.

All checks run the oracle on grids small enough for a direct solve.
"""
import copy
import dataclasses

import numpy as np
import pytest

from oracle import topopt_oracle as O
from paper_2005_05436_gb300 import inputs as I


def _mbb(nelx, nely, **kw):
    F, fixed = I.mbb_half_beam(nelx, nely)
    kw.setdefault("volfrac", 0.5)
    kw.setdefault("rmin", 1.5)
    p = O.Params.parity(nelx=nelx, nely=nely, **kw)
    return p, F, fixed


def test_initial_design_with_passive_sets_by_hand():
    """PRE.6 on a 4 x 1 grid, one solid and one void element, volfrac 0.5:
    the active elements get (0.5 * (4 - 1) - 1) / 2 = 0.25."""
    p, F, fixed = _mbb(4, 1)
    pas = np.array([1, 0, -1, 0], np.int8)
    s = O.initial_state(p, pas)
    np.testing.assert_array_equal(s.x, [1.0, 0.25, 0.0, 0.25])
    assert s.x.mean() == 0.375  # volfrac (nEl - nV) / nEl: the void element is outside the budget
    np.testing.assert_array_equal(s.xold, np.ones(4))


@pytest.mark.parametrize("ft", [1, 2, 3])
def test_passive_densities_and_total_volume(ft):
    """Solid and void passive elements keep x = 1 / 0 and xPhys = 1 / 0 (prj(0) = 0,
    prj(1) = 1), and the OC update meets mean(x) = volfrac over all elements."""
    F, fixed, pas = I.frame_reinforcement(30, 30)
    p = O.Params.parity(nelx=30, nely=30, volfrac=0.3, rmin=1.5, ft=ft, beta=4.0, eta=0.45,
                        penal_cnt=(1, 3.0, 100, 0.0), beta_cnt=(1, 4.0, 100, 0.0))
    s = O.initial_state(p, pas)
    Ke = O.element_stiffness(2)
    for _ in range(3):
        O.design_step(p, s, F, fixed, pas, Ke)
        assert np.all(s.x[pas == 1] == 1.0) and np.all(s.x[pas == -1] == 0.0)
        assert np.all(s.xphys[pas == 1] == 1.0) and np.all(s.xphys[pas == -1] == 0.0)
        assert abs(s.x.mean() - 0.3) <= 1e-12
        assert np.all((s.x >= 0.0) & (s.x <= 1.0))


def test_continuation_acts_after_the_step():
    """With penalCnt = {1, 3, 2, +0.5} from p = 1 the first two iterations solve
    with p = 1 (the increment at loop 2 acts after that iteration's OC update),
    so their compliances equal those of a run without continuation; the third
    solves with p = 1.5 and differs."""
    p1, F, fixed = _mbb(20, 8, penal=1.0, penal_cnt=(1, 3.0, 2, 0.5), beta_cnt=(1, 2.0, 100, 0.0))
    p0, _, _ = _mbb(20, 8, penal=1.0, penal_cnt=(1, 3.0, 100, 0.0), beta_cnt=(1, 2.0, 100, 0.0))
    s1, s0 = O.initial_state(p1), O.initial_state(p0)
    Ke = O.element_stiffness(2)
    r1 = [O.design_step(p1, s1, F, fixed, None, Ke) for _ in range(3)]
    r0 = [O.design_step(p0, s0, F, fixed, None, Ke) for _ in range(3)]
    assert [r["penal"] for r in r1] == [1.0, 1.5, 1.5]
    assert r1[0]["c"] == r0[0]["c"] and r1[1]["c"] == r0[1]["c"]
    assert abs(r1[2]["c"] - r0[2]["c"]) > 1e-6 * abs(r0[2]["c"])


def test_pae_damping_one_is_the_plain_oc_step():
    """z_k = alpha r_k with alpha = 1 and no extrapolation (q larger than the run)
    is x_k + (U(x_k) - x_k) = U(x_k): the run equals the one without PAE."""
    p_on, F, fixed = _mbb(24, 8, ft=1, pae_q0=2, pae_q=10 ** 6, pae_m=4, pae_alpha=1.0)
    p_off, _, _ = _mbb(24, 8, ft=1)
    s_on, s_off = O.initial_state(p_on), O.initial_state(p_off)
    Ke = O.element_stiffness(2)
    for _ in range(6):
        a = O.design_step(p_on, s_on, F, fixed, None, Ke)
        b = O.design_step(p_off, s_off, F, fixed, None, Ke)
        # x + 1 * (U(x) - x) equals U(x) up to rounding, which the next iterations carry on
        np.testing.assert_allclose(s_on.x, s_off.x, rtol=0, atol=1e-10)
        assert abs(a["c"] - b["c"]) <= 1e-10 * abs(b["c"])


def test_pae_damped_step_is_x_plus_alpha_r():
    """For alpha = 0.5 each damped step from loop q0 on moves x half way from x_k
    towards the plain OC result U(x_k) of the same state (active elements only,
    passive ones untouched), before that loop it is the plain step."""
    F, fixed, pas = I.frame_reinforcement(20, 20)
    p = O.Params.parity(nelx=20, nely=20, volfrac=0.3, rmin=1.5, ft=1, pae_q0=3, pae_q=10 ** 6, pae_m=4,
                        pae_alpha=0.5, penal_cnt=(1, 3.0, 100, 0.0), beta_cnt=(1, 2.0, 100, 0.0))
    p_plain = dataclasses.replace(p, pae_q0=0)
    s = O.initial_state(p, pas)
    Ke = O.element_stiffness(2)
    act = pas == 0
    for k in range(1, 7):
        probe = copy.deepcopy(s)
        O.design_step(p_plain, probe, F, fixed, pas, Ke)   # U(x_k) from the same state
        x_k = s.x.copy()
        O.design_step(p, s, F, fixed, pas, Ke)
        want = probe.x.copy()
        if k >= 3:
            want[act] = np.clip(x_k[act] + 0.5 * (probe.x[act] - x_k[act]), 0.0, 1.0)
        np.testing.assert_allclose(s.x, want, rtol=0, atol=1e-15)
        assert np.all(s.x[pas == 1] == 1.0) and np.all(s.x[pas == -1] == 0.0)


def test_pae_extrapolates_on_the_loops_of_the_reading():
    """Reading R23: with it = loop - q0 the extrapolated step is taken when it >= 1
    and (it + 1) is a multiple of q. For q0 = 5, q = 4 that is loops 8, 12, 16;
    every other loop from q0 on is a damped step, earlier loops are plain."""
    p, F, fixed = _mbb(24, 8, ft=1, pae_q0=5, pae_q=4, pae_m=4, pae_alpha=0.9)
    s = O.initial_state(p)
    Ke = O.element_stiffness(2)
    kinds = {O.design_step(p, s, F, fixed, None, Ke)["loop"]: s.history[-1]["pae"] for _ in range(17)}
    assert [k for k, v in kinds.items() if v == 2] == [8, 12, 16]
    assert all(kinds[k] == 0 for k in range(1, 5))
    assert all(kinds[k] == 1 for k in range(5, 18) if k not in (8, 12, 16))
