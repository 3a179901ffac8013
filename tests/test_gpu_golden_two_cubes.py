"""The two-cube workload (two 7^3-cell Neo-Hookean cubes, 4,116 tets, 1 cm
gap, E = 1e5, ten steps) through the C ABI against the oracle's trajectory,
stored by tests/golden/make_two_cubes_trajectory.py (FP64 CPU, dense Cholesky
solves): positions after every step while the oracle's steps converge."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_00046_b300 import bal, scenes  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "two_cubes_trajectory.npz")


def test_two_cubes_trajectory_matches_the_oracle_golden_file():
    """Equal to the stored trajectory while the GPU follows the oracle's path;
    if a step ends elsewhere (the augmented-Lagrangian decisions compare d_min
    with a threshold, and rounding-level differences of the atomic FP64 sums
    can tip one), that GPU step and every later one must be a solution of its
    step under the GPU's own AL state (oracle residual)."""
    from oracle import system
    from gpu_common import gpu_step_is_solution
    g = np.load(GOLD)
    sc = scenes.two_cubes()
    m = system.make_model(sc)
    S = bal.Scene(sc, bal.default_params(newton_tol=float(g["newton_tol"]), newton_max_iter=int(g["newton_max"]),
                                         pcg_tol=1e-12, pcg_max_iter=20000))
    x = torch.tensor(sc.X, dtype=torch.float64, device="cuda")
    v = torch.tensor(sc.V0, dtype=torch.float64, device="cuda")
    compared, same = 0, True
    for k in range(len(g["x"])):
        x_t, v_t = x.cpu().numpy().copy(), v.cpu().numpy().copy()
        info = S.time_step(x, v, check=False)
        if not g["converged"][k]:
            break                                # past an unconverged oracle step the states may part
        assert info["converged"] == 1, k
        err = np.abs(x.cpu().numpy() - g["x"][k]).max()
        same = same and err < 1e-8
        if same:
            assert np.abs(v.cpu().numpy() - g["v"][k]).max() < 1e-8 / sc.h * 10, k
            compared += 1
        else:
            gpu_step_is_solution(m, x_t, v_t, x.cpu().numpy(), S.get_al_state())
    assert compared >= 1
