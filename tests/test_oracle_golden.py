"""The oracle reproduces its committed regression fixture (written by
tests/golden/make_golden.py from the oracle alone), and the paper's printed
template constants give the values Eq. (tanh_waveform) prescribes."""
import json
import math
import os
import sys

import numpy as np

from oracle import oracle as O
from paper_2308_08410_gb300 import synth as S

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
import make_golden  # noqa: E402


def test_regression_fixture():
    with open(os.path.join(HERE, "oracle_tiny.json")) as f:
        g = json.load(f)
    p = make_golden.tiny_problem()
    r = O.forward_backward(p.mesh, p.fib, p.cf, p.ct, p.onsets, p.L, p.tmpl, p.extra["target"])
    np.testing.assert_allclose(r["phi"], g["phi"], rtol=1e-12)
    np.testing.assert_array_equal(r["parent"], g["parent"])
    np.testing.assert_allclose(r["loss"], g["loss"], rtol=1e-11)
    for k in ("lam", "d_cf", "d_ct", "d_t", "d_x"):
        ref = np.asarray(g[k])
        np.testing.assert_allclose(r[k], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_paper_template_constants():
    """Sec. III-B prints K0 = -85 mV, K1 = 30 mV, tau = 1 ms: U spans
    [K0, K1], U(0) is the midpoint and U'(0) = (K1 - K0)/tau."""
    with open(os.path.join(HERE, "paper_constants.json")) as f:
        c = json.load(f)["rabbit_template"]
    tm = S.Template(K0=c["K0_mV"], K1=c["K1_mV"], tau=c["tau_ms"], t0=-50.0, dt=0.5, T=201)
    L = np.ones((1, 1), np.float32)
    V = O.ecg(L, np.array([0.0]), tm)[0]
    assert abs(V[0] - c["K0_mV"]) < 1e-9 and abs(V[-1] - c["K1_mV"]) < 1e-9
    mid = (c["K0_mV"] + c["K1_mV"]) / 2
    assert abs(V[100] - mid) < 1e-12
    h = 1e-6
    tm2 = S.Template(K0=c["K0_mV"], K1=c["K1_mV"], tau=c["tau_ms"], t0=-h, dt=2 * h, T=2)
    v = O.ecg(L, np.array([0.0]), tm2)[0]
    assert math.isclose((v[1] - v[0]) / (2 * h), (c["K1_mV"] - c["K0_mV"]) / c["tau_ms"], rel_tol=1e-6)
