"""The network kernels (forward, backward, Adam) against the FP64 network oracle."""
import numpy as np
import pytest

from oracle import net_oracle as N
from tests._util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


def _sample(seed, shape=(8, 8, 4), base=4):
    r = np.random.default_rng(seed)
    theta = N.init_params(base, seed=seed) + 0.02 * r.standard_normal(N.n_params(base))
    x = r.standard_normal(shape + (4,))
    target = r.standard_normal(shape + (3,))
    mask = r.random(shape) > 0.2
    return theta, x, target, mask


def _cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _net(base, bf16, theta):
    from paper_2005_05436_gb300.learned import Net
    net = Net(base=base, bf16=bf16)
    assert net.n_params == N.n_params(base)
    net.set_params(theta.astype(np.float32))
    return net


@pytest.mark.parametrize("bf16,tol_y,tol_g", [(False, 2e-5, 1e-4), (True, 3e-2, 8e-2)])
def test_forward_and_gradient_match_oracle(bf16, tol_y, tol_g):
    base = 4
    theta, x, target, mask = _sample(1, base=base)
    th32 = theta.astype(np.float32).astype(np.float64)  # the values the GPU holds
    net = _net(base, bf16, theta)
    y = net.forward(_cuda(x[None])).cpu().numpy()[0]
    y_ref, _ = N.forward(th32, x.astype(np.float32).astype(np.float64), base)
    assert rel(y, y_ref) <= tol_y, rel(y, y_ref)
    net.zero_grad()
    loss = net.accumulate(_cuda(x[None]), _cuda(target[None]), _cuda(mask[None], torch.uint8))
    f_ref, g_ref = N.backward(th32, x.astype(np.float32).astype(np.float64), target.astype(np.float32), mask, base)
    assert abs(loss - f_ref) <= tol_y * abs(f_ref), (loss, f_ref)
    g = net.grad().cpu().numpy()
    assert rel(g, g_ref) <= tol_g, rel(g, g_ref)


def test_batch_gradient_is_the_sum_of_sample_gradients():
    base = 4
    theta, x0, t0, m0 = _sample(2, base=base)
    _, x1, t1, m1 = _sample(3, base=base)
    net = _net(base, False, theta)
    n0, n1 = m0.sum() * 3, m1.sum() * 3
    net.zero_grad()
    net.accumulate(_cuda(x0[None]), _cuda(t0[None]), _cuda(m0[None], torch.uint8))
    g0 = net.grad().cpu().numpy().astype(np.float64)
    net.zero_grad()
    net.accumulate(_cuda(x1[None]), _cuda(t1[None]), _cuda(m1[None], torch.uint8))
    g1 = net.grad().cpu().numpy().astype(np.float64)
    net.zero_grad()
    net.accumulate(_cuda(np.stack([x0, x1])), _cuda(np.stack([t0, t1])), _cuda(np.stack([m0, m1]), torch.uint8))
    gb = net.grad().cpu().numpy()
    # batch loss = (n0 L0 + n1 L1) / (n0 + n1)
    assert rel(gb, (n0 * g0 + n1 * g1) / (n0 + n1)) <= 1e-5


@pytest.mark.parametrize("bf16", [False, True])
def test_adam_fits_one_sample(bf16):
    base = 4
    theta, x, target, mask = _sample(4, shape=(8, 8, 8), base=base)
    net = _net(base, bf16, theta)
    xs, ts, ms = _cuda(x[None]), _cuda(0.5 * target[None]), _cuda(mask[None], torch.uint8)
    net.zero_grad()
    l0 = net.accumulate(xs, ts, ms)
    for _ in range(150):
        net.adam(3e-3)
        loss = net.accumulate(xs, ts, ms)
    assert loss < 0.5 * l0, (l0, loss)
