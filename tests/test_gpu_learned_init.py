"""The learned initialiser end to end at reduced size: data from the forward
model on the GPU, training with the project's BF16 kernels, and the gain over
plain Geodesic-BP from the default start on held-out ECGs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2308_08410_gb300 import learned_init as LI  # noqa: E402

pytestmark = pytest.mark.gpu


def test_learned_init_beats_default_start():
    res = LI.run_experiment(n_train=2048, n_test=256, epochs=12, n_eval=4, iters=60, log=lambda *_: None)
    m = res["median"]
    # the network's start already explains the ECG better than the default start
    assert m["learned_loss0"] < m["plain_loss0"], m
    # and it reaches the plain method's best misfit (over 60 iterations) sooner
    assert res["reached"] >= 2, res["cases"]
    assert m["learned_time"] < m["plain_time"], m
