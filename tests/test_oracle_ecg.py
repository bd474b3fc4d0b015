"""Pins of the oracle's ECG (Sec. II-D, Eq. tanh_waveform, Eq. inverse_ecg)."""
import math

import numpy as np

from oracle import oracle as O
from paper_2308_08410_gb300 import synth as S


def test_single_node_closed_form():
    """One lead-field column: V_l(t) = L_l U(t - phi) with
    U(xi) = K0 + (K1 - K0)/2 (1 + tanh(2 xi / tau)); the paper's rabbit
    template K0=-85, K1=30, tau=1 (Sec. III-B)."""
    tm = S.Template(K0=-85.0, K1=30.0, tau=1.0, t0=100.0, dt=0.5, T=130)
    L = np.zeros((3, 5), np.float32)
    L[:, 2] = [0.5, -1.25, 2.0]
    phi = np.array([np.inf, 1.0, 132.7, 0.0, 200.0])
    V = O.ecg(L, phi, tm)
    for l in range(3):
        for s in range(tm.T):
            t = tm.t0 + s * tm.dt
            u = -85.0 + 57.5 * (1 + math.tanh(2 * (t - 132.7) / 1.0))
            assert abs(V[l, s] - float(L[l, 2]) * u) <= 1e-12 * abs(u) + 1e-12


def test_unreached_vertex_rests_at_K0_and_linearity():
    tm = S.Template(T=40)
    rng = np.random.default_rng(1)
    L1 = rng.normal(size=(4, 50)).astype(np.float32)
    L2 = rng.normal(size=(4, 50)).astype(np.float32)
    phi = rng.uniform(0, 40, 50)
    phi[7] = np.inf
    a = O.ecg(L1, phi, tm)
    b = O.ecg(L2, phi, tm)
    c = O.ecg((L1 + L2).astype(np.float32), phi, tm)
    np.testing.assert_allclose(a + b, c, rtol=1e-5, atol=1e-9)  # L1+L2 rounded to float32
    e = np.zeros((4, 50), np.float32)
    e[:, 7] = 1.0
    np.testing.assert_allclose(O.ecg(e, phi, tm), np.full((4, 40), tm.K0), rtol=0, atol=0)


def test_loss_and_phi_gradient_fd():
    """loss = 1/(N T) sum (V - Vhat)^2 and lam = d loss / d phi against central
    differences of the full ECG + loss in phi (Sec. II-D)."""
    tm = S.Template(T=60)
    rng = np.random.default_rng(2)
    N, n = 5, 40
    L = rng.normal(size=(N, n)).astype(np.float32)
    phi = rng.uniform(5, 50, n)
    tgt = rng.normal(scale=20, size=(N, tm.T)).astype(np.float32)
    V = O.ecg(L, phi, tm)
    loss, lam = O.loss_grad_phi(L, phi, tm, V, tgt)
    np.testing.assert_allclose(loss, np.mean((V - tgt.astype(float)) ** 2), rtol=1e-14)
    h = 1e-6
    for k in range(n):
        def f(dh):
            p = phi.copy()
            p[k] += dh
            Vp = O.ecg(L, p, tm)
            return np.mean((Vp - tgt.astype(float)) ** 2)
        fd = O.fd_probe(f, h)
        assert abs(fd - lam[k]) <= 1e-6 * max(abs(lam[k]), 1e-3 * np.abs(lam).max())
