"""The two-cube workload (two 7^3-cell Neo-Hookean cubes, 4,116 tets, 1 cm
gap, E = 1e5, ten steps) through the C ABI against the oracle's trajectory,
stored by tests/golden/make_two_cubes_trajectory.py (FP64 CPU, dense Cholesky
solves): Algorithm 1's decision log and the positions after every step while
the oracle's steps converge."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_00046_b300 import bal, scenes  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "two_cubes_trajectory.npz")


def test_two_cubes_trajectory_matches_the_oracle_golden_file():
    """All ten stored oracle steps converged (Newton tolerance 1e-8). Per
    step, while the GPU follows the oracle's path: Algorithm 1's decision log
    (|A|, |A'| and sigma at every Newton iterate) identical to the stored one,
    and positions equal to 1e-8 m. If a step's log differs (the decisions
    compare d_min with a threshold, and rounding-level differences of the
    atomic FP64 sums can tip one), that GPU step and every later one must be
    a solution of its step under the GPU's own AL state (oracle residual).
    Every GPU step converges."""
    from oracle import system
    from gpu_common import gpu_step_is_solution
    g = np.load(GOLD)
    sc = scenes.two_cubes()
    m = system.make_model(sc)
    newton_max = int(g["newton_max"])
    assert bool(np.all(g["converged"])) and len(g["x"]) == 10
    S = bal.Scene(sc, bal.default_params(newton_tol=float(g["newton_tol"]), newton_max_iter=newton_max,
                                         pcg_tol=1e-12, pcg_max_iter=20000))
    x = torch.tensor(sc.X, dtype=torch.float64, device="cuda")
    v = torch.tensor(sc.V0, dtype=torch.float64, device="cuda")
    compared, same = 0, True
    for k in range(len(g["x"])):
        x_t, v_t = x.clone(), v.clone()
        S.step_begin(x, v)
        log, converged = [], False
        for _ in range(newton_max):
            ni = S.newton_step(x)
            log.append((ni["n_active"], ni["n_ap"], ni["sigma"]))
            if ni["converged"]:
                converged = True
                break
        v.copy_((x - x_t) * (1.0 / sc.h))
        assert converged, k
        n = int(g["log_len"][k])
        ref = [(int(g["log_nA"][k, i]), int(g["log_nAp"][k, i]), float(g["log_sigma"][k, i])) for i in range(n)]
        same = same and len(log) == n and all(
            a == ra and ap == rap and abs(sg - rsg) <= 1e-12 * rsg for (a, ap, sg), (ra, rap, rsg) in zip(log, ref))
        if same:
            assert np.abs(x.cpu().numpy() - g["x"][k]).max() < 1e-8, k
            assert np.abs(v.cpu().numpy() - g["v"][k]).max() < 1e-8 / sc.h * 10, k
            compared += 1
        else:
            gpu_step_is_solution(m, x_t.cpu().numpy(), v_t.cpu().numpy(), x.cpu().numpy(), S.get_al_state())
    assert compared >= 1     # at least the first step follows the oracle's path exactly
