"""Write the oracle regression fixtures of this folder.

Calls only the seeded generators and ``oracle/``; nothing here comes from the
CUDA path.  Re-run (python tests/golden/make_golden.py) only when a change to
the oracle's arithmetic is justified by a passage of the paper, and name that
passage in the commit message.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2308_08410_gb300 import synth as S  # noqa: E402


def tiny_problem():
    """5^3-vertex cube, c1 fibres, per-tet velocities jittered by 5 %, two
    element onsets, 4 electrodes, T = 40."""
    p = S.make_c1(n=5, n_leads=4, T=40)
    rng = np.random.default_rng(77)
    p.cf = (p.cf * (1 + 0.05 * rng.standard_normal(p.mesh.n_t))).astype(np.float32)
    p.ct = (p.ct * (1 + 0.05 * rng.standard_normal(p.mesh.n_t))).astype(np.float32)
    p.onsets = S.onsets_element(p.mesh, 2, seed=78, tmin=0.0, tmax=4.0)
    ek = O.eikonal(p.mesh, p.fib, (p.cf * 1.1).astype(np.float32), p.ct, p.onsets)
    p.extra["target"] = S.add_noise(O.ecg(p.L, ek["phi"], p.tmpl), 0.05, 79)
    return p


def main():
    p = tiny_problem()
    r = O.forward_backward(p.mesh, p.fib, p.cf, p.ct, p.onsets, p.L, p.tmpl, p.extra["target"])
    out = {
        "what": "oracle regression fixture: tiny_problem() of make_golden.py",
        "phi": r["phi"].tolist(),
        "parent": r["parent"].tolist(),
        "loss": r["loss"],
        "lam": r["lam"].tolist(),
        "d_cf": r["d_cf"].tolist(),
        "d_ct": r["d_ct"].tolist(),
        "d_t": r["d_t"].tolist(),
        "d_x": r["d_x"].tolist(),
    }
    with open(os.path.join(HERE, "oracle_tiny.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
