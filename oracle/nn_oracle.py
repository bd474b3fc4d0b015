"""FP64 NumPy reference of the learned initialiser's network.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): a plain, slow,
obviously correct forward and backward pass of the 1-D convolution + MLP that
the CUDA kernels train in BF16.  It shares no code with the CUDA path.

The network is not in the paper (its sections describe the inverse problem
the network initialises, Sec. II-D); parity of this part is pinned by finite
differences of this reference and by the direct definition of a
convolution, not by a passage of the paper.

Conventions shared with the CUDA path because they define the parameters:
activations are [batch, length, channels]; a convolution weight is
[C_out, ksize, C_in]; y[b, l, o] = bias[o] + sum_{k, c} W[o, k, c]
x[b, stride*l + k - pad, c] (zero outside); flatten order (length, channel);
GELU(z) = z Phi(z) with the standard normal CDF Phi.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def conv_out_len(L, ks, stride, pad):
    return (L + 2 * pad - ks) // stride + 1


def conv1d(x, W, b, stride, pad):
    """Direct definition, loops over taps."""
    B, L, C = x.shape
    Co, ks, Ci = W.shape
    Lo = conv_out_len(L, ks, stride, pad)
    y = np.tile(b, (B, Lo, 1)).astype(np.float64)
    for k in range(ks):
        for lo in range(Lo):
            j = stride * lo + k - pad
            if 0 <= j < L:
                y[:, lo, :] += x[:, j, :] @ W[:, k, :].T
    return y


def conv1d_backward(x, W, dy, stride, pad):
    """Gradients of conv1d with respect to x, W and the bias."""
    B, L, C = x.shape
    Co, ks, Ci = W.shape
    Lo = dy.shape[1]
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for k in range(ks):
        for lo in range(Lo):
            j = stride * lo + k - pad
            if 0 <= j < L:
                dx[:, j, :] += dy[:, lo, :] @ W[:, k, :]
                dW[:, k, :] += dy[:, lo, :].T @ x[:, j, :]
    db = dy.sum(axis=(0, 1))
    return dx, dW, db


class Net:
    """n_conv convolutions (ksize, stride, pad, channels) + GELU, flatten,
    a hidden dense layer + GELU and a linear output layer."""

    def __init__(self, C_in, L_in, channels=64, n_conv=4, ksize=5, stride=2, pad=2, hidden=256, n_out=43):
        self.C_in, self.L_in = C_in, L_in
        self.channels, self.n_conv, self.ksize, self.stride, self.pad = channels, n_conv, ksize, stride, pad
        self.hidden, self.n_out = hidden, n_out
        self.lens = [L_in]
        for _ in range(n_conv):
            self.lens.append(conv_out_len(self.lens[-1], ksize, stride, pad))
        self.flat = self.lens[-1] * channels

    def shapes(self):
        s = []
        cin = self.C_in
        for _ in range(self.n_conv):
            s.append((self.channels, self.ksize, cin))
            s.append((self.channels,))
            cin = self.channels
        s += [(self.hidden, self.flat), (self.hidden,), (self.n_out, self.hidden), (self.n_out,)]
        return s

    def init(self, seed):
        """He-style initialisation (a seeded input of both paths)."""
        rng = np.random.default_rng(seed)
        ps = []
        for shp in self.shapes():
            if len(shp) == 1:
                ps.append(np.zeros(shp))
            else:
                fan_in = int(np.prod(shp[1:]))
                ps.append(rng.standard_normal(shp) * math.sqrt(2.0 / fan_in))
        return [p.astype(np.float32) for p in ps]

    def forward(self, params, x):
        params = [np.asarray(p, np.float64) for p in params]
        a = np.asarray(x, np.float64)
        cache = []
        for i in range(self.n_conv):
            W, b = params[2 * i], params[2 * i + 1]
            z = conv1d(a, W, b, self.stride, self.pad)
            cache.append((a, z))
            a = gelu(z)
        B = a.shape[0]
        f = a.reshape(B, -1)
        W1, b1, W2, b2 = params[2 * self.n_conv:]
        z1 = f @ W1.T + b1
        h = gelu(z1)
        y = h @ W2.T + b2
        cache.append((f, z1, h))
        return y, cache

    def backward(self, params, cache, dy):
        params = [np.asarray(p, np.float64) for p in params]
        W1, b1, W2, b2 = params[2 * self.n_conv:]
        f, z1, h = cache[-1]
        grads = [None] * len(params)
        grads[-1] = dy.sum(axis=0)
        grads[-2] = dy.T @ h
        dz1 = (dy @ W2) * gelu_grad(z1)
        grads[-3] = dz1.sum(axis=0)
        grads[-4] = dz1.T @ f
        da = (dz1 @ W1).reshape(f.shape[0], self.lens[-1], self.channels)
        for i in reversed(range(self.n_conv)):
            a_in, z = cache[i]
            dz = da * gelu_grad(z)
            dx, dW, db = conv1d_backward(a_in, params[2 * i], dz, self.stride, self.pad)
            grads[2 * i], grads[2 * i + 1] = dW, db
            da = dx
        return grads


def mse(y, t):
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size
