"""Writes the oracle trajectory of the two-cube workload (two 7^3-cell
Neo-Hookean cubes, 4,116 tets, 1 cm gap, E = 1e5, h = 1/30 s, dhat = 1e-3 m,
gravity), ten steps, Newton tolerance 1e-8: positions and velocities after each
step, Newton iterations and convergence flags, and Algorithm 1's decision log
(|A|, |A'| and sigma at every Newton iterate). Calls only oracle/ (the FP64 CPU
reference with dense Cholesky solves).

    python tests/golden/make_two_cubes_trajectory.py   # ~10 min on one core
"""
import os
import sys

import numpy as np

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), "..", ".."))
sys.path.insert(0, ROOT)

from oracle import bal, system  # noqa: E402
from paper_2407_00046_b300 import scenes  # noqa: E402

STEPS = 10
NEWTON_TOL = 1e-8
NEWTON_MAX = 400


def main():
    sc = scenes.two_cubes()
    m = system.make_model(sc)
    x, v = sc.X.copy(), sc.V0.copy()
    xs, vs, iters, conv, nA, logs = [], [], [], [], [], []
    for k in range(STEPS):
        x, v, info = bal.time_step(m, x, v, bal.Params(newton_tol=NEWTON_TOL, newton_max=NEWTON_MAX))
        keys, _ = bal.active_pairs(m, x)
        xs.append(x.copy())
        vs.append(v.copy())
        iters.append(info["iters"])
        conv.append(bool(info["converged"]))
        nA.append(len(keys))
        # Algorithm 1's decisions at every Newton iterate: |A|, |A'| and sigma
        logs.append([(r["nA"], r["nAp"], r["sigma"]) for r in info["log"]])
        print(k, info["iters"], info["converged"], len(keys), flush=True)
    L = max(len(lg) for lg in logs)
    log_len = np.array([len(lg) for lg in logs])
    log_nA = np.full((STEPS, L), -1, dtype=np.int64)
    log_nAp = np.full((STEPS, L), -1, dtype=np.int64)
    log_sigma = np.full((STEPS, L), np.nan)
    for k, lg in enumerate(logs):
        for i, (a, ap, sg) in enumerate(lg):
            log_nA[k, i], log_nAp[k, i], log_sigma[k, i] = a, ap, sg
    out = os.path.join(os.path.dirname(__file__), "two_cubes_trajectory.npz")
    np.savez_compressed(out, x=np.array(xs), v=np.array(vs), newton_iters=np.array(iters),
                        converged=np.array(conv), n_active=np.array(nA), newton_tol=NEWTON_TOL,
                        newton_max=NEWTON_MAX, log_len=log_len, log_nA=log_nA, log_nAp=log_nAp,
                        log_sigma=log_sigma)


if __name__ == "__main__":
    main()
