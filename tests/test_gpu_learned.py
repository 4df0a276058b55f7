"""The learned warm start inside the design iteration.

The network is trained on (xPhys, F, U) triples that the method itself produces
(runs of to_step on seeded cantilever-family problems); attached to a grid it
provides a displacement direction, and the state solve starts from the
minimiser of the potential energy over span{U_prev, U_net}. The tests check
that the solution does not change, that the start is never worse (in the
energy norm) than the previous solution, and what the trained network gains:
energy error of the start and iteration counts against the method without it.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(16, 8, 8), (24, 12, 12)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def nets():
    """A network trained on the energy objective (to_learned_energy_grad) with
    samples from 12 runs of the method, and the same network untrained."""
    from paper_2005_05436_gb300 import learned as Lr
    samples, grids = Lr.generate_energy(SHAPES, runs=12, iters=12, seed=0, warmup=2)
    trained = Lr.Net(base=16, bf16=True)
    trained.set_params(Lr.he_init(16, seed=1))
    hist = Lr.train_energy(trained, samples, grids, epochs=30, lr=2e-3, lr_final=1e-4, batch=4)
    for g in grids:
        g.close()
    raw = Lr.Net(base=16, bf16=True)
    raw.set_params(Lr.he_init(16, seed=1))
    return trained, raw, hist


def test_mse_training_on_the_normalised_displacement():
    """The alternative objective: mean squared error to U / rms(U)."""
    from paper_2005_05436_gb300 import learned as Lr
    data = Lr.generate(SHAPES, runs=4, iters=8, seed=0, warmup=2)
    net = Lr.Net(base=8, bf16=True)
    net.set_params(Lr.he_init(8, seed=2))
    hist = Lr.train(net, data, epochs=20, lr=3e-3, lr_final=2e-4, batch=4)
    assert hist[-1] < 0.9 * hist[0], hist


def _problem(r, precision):
    from paper_2005_05436_gb300 import TO_PC_GMG, default_params, inputs as I
    from paper_2005_05436_gb300.topopt import Design, Grid
    nelx, nely, nelz = SHAPES[r % 2]
    F, fixed, vf = I.cantilever_family(nelx, nely, nelz, 1000 + r)
    p = default_params(3, nelx, nely, nelz, precision=precision, precond=TO_PC_GMG, volfrac=vf,
                       rmin=math.sqrt(3.0), beta=2.0, beta_cnt=(1, 16.0, 10, 2.0, 1), cg_rtol=1e-8,
                       cg_maxit=5000)
    g = Grid(p, torch.from_numpy(F).cuda(), torch.from_numpy(fixed).cuda())
    d = Design(g, torch.full((g.nel,), vf, dtype=torch.float64, device="cuda"))
    for _ in range(6):
        d.step()
    return g, d


def _snap(d):
    return [t.clone() for t in (d.x, d.xPhys, d.xOld, d.U)], (d.st.eta, d.st.penal, d.st.beta, d.st.loop)


def _restore(d, s):
    for a, b in zip((d.x, d.xPhys, d.xOld, d.U), s[0]):
        a.copy_(b)
    d.st.eta, d.st.penal, d.st.beta, d.st.loop = s[1]


def _steps(g, d, modes, nets, rule=None):
    from paper_2005_05436_gb300 import learned as Lr
    trained, raw, _ = nets
    s = _snap(d)
    out = {}
    for mode in modes:
        _restore(d, s)
        if mode.startswith("cold"):
            d.U.zero_()
        Lr.attach(g, trained if mode.endswith("+net") else raw if mode.endswith("+raw") else None, rule=rule)
        info = d.step()
        out[mode] = (info, d.xPhys.clone(), d.x.clone())
    Lr.attach(g, None)
    return out


def test_training_lowers_the_energy_error(nets):
    _, _, hist = nets
    assert hist[-1] < 0.95 * hist[0], hist


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warm_start_keeps_the_answer_and_never_raises_the_start_energy(nets, precision):
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED
    g, d = _problem(0, TO_FP64 if precision == "fp64" else TO_MIXED)
    out = _steps(g, d, ["warm", "warm+net", "cold+net"], nets)
    ref, xp_ref, x_ref = out["warm"]
    for mode in ("warm+net", "cold+net"):
        info, xp, x = out[mode]
        assert info["rel_res"] <= 1e-8
        assert abs(info["c"] - ref["c"]) <= 1e-7 * abs(ref["c"])
        assert float(torch.linalg.norm(xp - xp_ref) / torch.linalg.norm(xp_ref)) <= 1e-7
        assert float(torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)) <= 1e-6
        assert info["warm_err"] <= info["warm_err_prev"] + 1e-9
        assert info["t_warm_ms"] > 0
    assert out["cold+net"][0]["warm_err_prev"] == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_residual_rule_keeps_the_answer_and_never_raises_the_start_residual(nets, precision):
    """TO_WARM_RESIDUAL: the start minimises ||F - K U0|| over span{U_prev, U_net},
    so its residual (reported as warm_res) is at most that of U_prev; the
    solution is the one without the network, and both rules report both
    measures of both starts."""
    from paper_2005_05436_gb300 import TO_FP64, TO_MIXED, TO_WARM_ENERGY, TO_WARM_RESIDUAL
    g, d = _problem(1, TO_FP64 if precision == "fp64" else TO_MIXED)
    out = _steps(g, d, ["warm", "warm+net", "cold+net"], nets, rule=TO_WARM_RESIDUAL)
    ref = out["warm"][0]
    for mode in ("warm+net", "cold+net"):
        info, xp, _ = out[mode]
        assert info["rel_res"] <= 1e-8
        assert abs(info["c"] - ref["c"]) <= 1e-7 * abs(ref["c"])
        assert float(torch.linalg.norm(xp - out["warm"][1]) / torch.linalg.norm(out["warm"][1])) <= 1e-7
        assert 0.0 < info["warm_res"] <= info["warm_res_prev"] * (1 + 1e-9) + 1e-12
    assert out["cold+net"][0]["warm_res_prev"] == pytest.approx(1.0, abs=1e-9)  # U = 0: ||F|| / ||F||
    en = _steps(g, d, ["warm+net"], nets, rule=TO_WARM_ENERGY)["warm+net"][0]
    assert en["warm_err"] <= en["warm_err_prev"] + 1e-9 and en["warm_res"] > 0.0
    # the energy rule's start is the energy minimiser: the residual rule's start is not better in energy
    assert en["warm_err"] <= out["warm+net"][0]["warm_err"] + 1e-9
    g.close()


def test_what_the_trained_warm_start_gains(nets):
    """Held-out problems, after 6 design iterations: the next state solve from
    (a) U_prev (the method without the network), (b) the energy-optimal point of
    span{U_prev, U_net}, and from zero with and without the trained network.
    Energy errors are exact (relative to the zero start); the iteration counts
    are reported, and may not grow on average."""
    from paper_2005_05436_gb300 import TO_FP64
    rows = []
    for r in range(4):
        g, d = _problem(r, TO_FP64)
        out = _steps(g, d, ["warm", "warm+net", "cold", "cold+net", "cold+raw"], nets)
        rows.append({k: v[0] for k, v in out.items()})
        g.close()
    mean = lambda k, f: float(np.mean([row[k][f] for row in rows]))  # noqa: E731
    # the start actually used is far better than U_prev itself in the energy norm
    assert mean("warm+net", "warm_err") < 0.5 * mean("warm+net", "warm_err_prev")
    # from zero, the trained direction captures more energy than the untrained one
    assert mean("cold+net", "warm_err") < mean("cold+raw", "warm_err") <= 1.0 + 1e-9
    # iterations: never more on average than the method without the network
    assert mean("warm+net", "n_cg") <= mean("warm", "n_cg") + 0.5
    assert mean("cold+net", "n_cg") <= mean("cold", "n_cg") + 0.5
