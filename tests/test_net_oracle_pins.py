"""Pins of the network oracle (oracle/net_oracle.py) against definitions that do
not share its code: explicit loops, delta kernels, adjoint identities and
central finite differences of the full loss."""
import numpy as np
import pytest

from oracle import net_oracle as N


def _rng(s):
    return np.random.default_rng(s)


def test_conv3d_matches_the_loop_definition():
    r = _rng(1)
    x = r.standard_normal((3, 4, 2, 2))
    W = r.standard_normal((27, 2, 3))
    b = r.standard_normal(3)
    np.testing.assert_allclose(N.conv3d(x, W, b), N.conv3d_loops(x, W, b), rtol=1e-12, atol=1e-12)


def test_conv3d_delta_kernels_are_identity_and_shift():
    r = _rng(2)
    x = r.standard_normal((4, 3, 5, 2))
    W = np.zeros((27, 2, 2))
    W[13] = np.eye(2)  # centre tap (0, 0, 0)
    np.testing.assert_array_equal(N.conv3d(x, W, np.zeros(2)), x)
    W = np.zeros((27, 2, 2))
    t = N.TAPS.index((1, 0, 0))  # reads x[d + 1]
    W[t] = np.eye(2)
    y = N.conv3d(x, W, np.zeros(2))
    np.testing.assert_array_equal(y[:-1], x[1:])
    np.testing.assert_array_equal(y[-1], 0.0)


def test_pool_up_adjoints():
    r = _rng(3)
    x = r.standard_normal((4, 6, 2, 3))
    g = r.standard_normal((2, 3, 1, 3))
    np.testing.assert_allclose(np.sum(N.pool(x) * g), np.sum(x * N.pool_backward(g)), rtol=1e-12)
    z = r.standard_normal((2, 3, 1, 3))
    G = r.standard_normal((4, 6, 2, 3))
    np.testing.assert_allclose(np.sum(N.up(z) * G), np.sum(z * N.up_backward(G)), rtol=1e-12)
    np.testing.assert_allclose(N.pool(N.up(z)), z, rtol=1e-15)


def test_conv3d_backward_adjoint_and_weight_gradient():
    r = _rng(4)
    x = r.standard_normal((3, 3, 4, 2))
    W = r.standard_normal((27, 2, 3))
    b = r.standard_normal(3)
    gy = r.standard_normal((3, 3, 4, 3))
    gx, gW, gb = N.conv3d_backward(x, W, gy)
    # <conv(x) - b, gy> = <x, gx> (the data gradient is the adjoint)
    np.testing.assert_allclose(np.sum((N.conv3d(x, W, b) - b) * gy), np.sum(x * gx), rtol=1e-12)
    # weight and bias gradients by central differences of f(W) = <conv(x, W, b), gy>
    f = lambda W_, b_: np.sum(N.conv3d(x, W_, b_) * gy)  # noqa: E731
    for (t, i, o) in [(0, 0, 0), (13, 1, 2), (26, 1, 1), (7, 0, 2)]:
        E = np.zeros_like(W)
        E[t, i, o] = 1e-6
        fd = (f(W + E, b) - f(W - E, b)) / 2e-6
        assert abs(fd - gW[t, i, o]) <= 1e-6 * max(1.0, abs(fd))
    eb = np.zeros(3)
    eb[1] = 1e-6
    assert abs((f(W, b + eb) - f(W, b - eb)) / 2e-6 - gb[1]) <= 1e-6


@pytest.mark.parametrize("seed", [5, 6])
def test_network_gradient_matches_central_differences(seed):
    base = 2
    r = _rng(seed)
    theta = N.init_params(base, seed=seed) + 0.05 * r.standard_normal(N.n_params(base))
    x = r.standard_normal((4, 4, 4, 4))
    target = r.standard_normal((4, 4, 4, 3))
    mask = np.ones((4, 4, 4), bool)
    mask[3, :, :] = False  # padding voxels do not count
    f, g = N.backward(theta, x, target, mask, base)
    assert f == pytest.approx(N.loss(N.forward(theta, x, base)[0], target, mask), rel=1e-14)
    idx = r.choice(theta.size, 24, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fp = N.loss(N.forward(theta + e, x, base)[0], target, mask)
        fm = N.loss(N.forward(theta - e, x, base)[0], target, mask)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1e-3, abs(fd)), (i, fd, g[i])
    # a small step against the gradient lowers the loss
    assert N.loss(N.forward(theta - 1e-3 * g / np.linalg.norm(g), x, base)[0], target, mask) < f


def test_parameter_layout():
    assert N.n_params(16) == sum(27 * a * b + b for a, b in N.layer_shapes(16))
    th = np.arange(N.n_params(2), dtype=float)
    np.testing.assert_array_equal(N.pack(N.unpack(th, 2)), th)
