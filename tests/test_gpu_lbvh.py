"""GPU parity of the LBVH broad phase (Sec. 5.3) through the C ABI: the
candidate set equals the oracle's brute-force box enumeration, static and
swept, on scenes spanning several bodies; the grid and the LBVH both contain
every close pair; and a time step with LBVH + cubic CCD matches the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bal as obal  # noqa: E402
from oracle import contact, system  # noqa: E402
from paper_2407_00046_b300 import bal, scenes  # noqa: E402

from gpu_common import close_cubes, compare_trajectory  # noqa: E402

DEV = "cuda"


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _keys(pairs):
    return sorted(bal.pair_key(*k) for k in pairs)


def _gpu(S, x, r, dirv=None):
    out = S.find_candidates(T(x).view(-1), r, None if dirv is None else T(dirv).view(-1))
    return sorted(int(k) for k in out.cpu().numpy().astype(np.uint64))


@pytest.mark.parametrize("name", ["two_cubes_small", "cube_stack_small"])
@pytest.mark.parametrize("r", [1e-3, 4e-3])
def test_lbvh_candidates_equal_brute_force_boxes(name, r):
    sc = scenes.scene_by_name(name)
    rng = np.random.default_rng(2)
    x = sc.X + 2e-4 * rng.normal(size=sc.X.shape)
    S = bal.Scene(sc, bal.default_params(broad_phase=bal.BROAD_LBVH))
    got = _gpu(S, x, r)
    ref = _keys(contact.box_candidates(x, sc, r))
    assert len(ref) > 0
    assert got == ref


def test_lbvh_swept_candidates_equal_brute_force_boxes():
    sc = close_cubes(n=4)
    rng = np.random.default_rng(3)
    x = sc.X.copy()
    x[sc.body == 1, 1] += 3e-3
    dirv = 1e-4 * rng.normal(size=x.shape)
    dirv[sc.body == 1] += [0.0, -4e-3, 0.0]
    S = bal.Scene(sc, bal.default_params(broad_phase=bal.BROAD_LBVH))
    got = _gpu(S, x, 1e-3, dirv)
    ref = _keys(contact.box_candidates(x, sc, 1e-3, dirv))
    assert len(ref) > 0 and got == ref


def test_grid_and_lbvh_contain_every_close_pair():
    sc = close_cubes(n=4)
    rng = np.random.default_rng(4)
    x = sc.X + 3e-4 * rng.normal(size=sc.X.shape)
    r = 2e-3
    cand = contact.candidate_pairs(x, sc, r)
    d, _, _ = contact.pair_distances(x, cand, sc)
    close = set(_keys([k for k, dd in zip(cand, d) if dd < r]))
    assert close
    for bp in (bal.BROAD_GRID, bal.BROAD_LBVH):
        S = bal.Scene(sc, bal.default_params(broad_phase=bp))
        assert close <= set(_gpu(S, x, r))


@pytest.mark.parametrize("mode", ["ccd", "ca"])
def test_time_step_with_lbvh_matches_oracle(mode):
    sc = close_cubes(n=2, gap=5e-4)
    S = bal.Scene(sc, bal.default_params(newton_tol=1e-8, pcg_tol=1e-12, pcg_max_iter=20000,
                                         step_mode=bal.STEP_CCD if mode == "ccd" else bal.STEP_CA,
                                         broad_phase=bal.BROAD_LBVH))
    m = system.make_model(sc)
    compare_trajectory(S, m, sc, 2, obal.Params(newton_tol=1e-8, step_mode=mode, broad_phase="lbvh"), T)
