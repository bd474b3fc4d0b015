"""Pins of the FP64 reference network (oracle/nn_oracle.py): the convolution
against scipy's correlation, GELU' and the whole backward pass against central
finite differences."""
import numpy as np
import scipy.signal

from oracle import nn_oracle as N


def test_conv1d_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 23, 3))
    W = rng.standard_normal((4, 5, 3))
    b = rng.standard_normal(4)
    y = N.conv1d(x, W, b, stride=2, pad=2)
    assert y.shape == (2, N.conv_out_len(23, 5, 2, 2), 4)
    for bb in range(2):
        for o in range(4):
            full = np.zeros(23 + 4)
            for c in range(3):
                xp = np.pad(x[bb, :, c], (2, 2))
                full[:len(xp) - 4] += scipy.signal.correlate(xp, W[o, :, c], mode="valid")
            ref = full[: 23 + 4 - 4][::2][: y.shape[1]] + b[o]
            np.testing.assert_allclose(y[bb, :, o], ref, rtol=1e-12, atol=1e-12)


def test_gelu_grad_fd():
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (N.gelu(z + h) - N.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(N.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_network_backward_fd():
    net = N.Net(C_in=3, L_in=20, channels=5, n_conv=2, ksize=5, stride=2, pad=2, hidden=7, n_out=4)
    params = [p.astype(np.float64) for p in net.init(1)]
    rng = np.random.default_rng(2)
    params = [p + 0.1 * rng.standard_normal(p.shape) for p in params]  # nonzero biases
    x = rng.standard_normal((3, 20, 3))
    t = rng.standard_normal((3, 4))
    y, cache = net.forward(params, x)
    loss, dy = N.mse(y, t)
    grads = net.backward(params, cache, dy)
    h = 1e-6
    for pi, p in enumerate(params):
        flat = p.ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = N.mse(net.forward(params, x)[0], t)[0]
            flat[idx] = old - h
            lm = N.mse(net.forward(params, x)[0], t)[0]
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            g = grads[pi].ravel()[idx]
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (pi, idx, fd, g)
