"""GPU parity of the cubic CCD step bound (Sec. 5.3) through the C ABI: per
pair and over a candidate set against the oracle's conservative time of
impact, and a trajectory with the CCD line search."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bal as obal  # noqa: E402
from oracle import ccd, contact, system  # noqa: E402
from paper_2407_00046_b300 import bal  # noqa: E402

from gpu_common import close_cubes, compare_trajectory  # noqa: E402

DEV = "cuda"


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def crossing_case():
    """Two close cubes; the upper one is pushed through the lower along a
    random direction field, so many stencils cross their planes in [0, 1]."""
    sc = close_cubes(n=3)
    rng = np.random.default_rng(21)
    x = sc.X + 1e-4 * rng.normal(size=sc.X.shape) * (sc.pinned == 0)[:, None]
    p = 2e-3 * rng.normal(size=sc.X.shape)
    p[sc.body == 1] += np.array([0.0, -3e-3, 0.0])
    p[sc.pinned == 1] = 0.0
    m = system.make_model(sc)
    r = m.dhat + 2.0 * np.sqrt((p ** 2).sum(1)).max()
    cand = contact.candidate_pairs(x, sc, r)
    S = bal.Scene(sc, bal.default_params())
    S.step_begin(T(sc.X), T(sc.V0))
    return sc, m, S, x, p, cand


def test_ccd_toi_per_pair_matches_oracle(crossing_case):
    sc, m, S, x, p, cand = crossing_case
    nodes = contact.stencil_nodes(cand, sc)
    eta = bal.default_params().step_bound
    refs = np.array([ccd.pair_toi(x[nodes[i]], p[nodes[i]], cand[i][0] == 1, m.dhat, eta)
                     for i in range(len(cand))])
    act = np.flatnonzero(refs < 1.0)
    rng = np.random.default_rng(5)
    rest = rng.choice(np.flatnonzero(refs == 1.0), size=min(150, int((refs == 1.0).sum())), replace=False)
    idx = np.concatenate([act[:150], rest])
    assert len(act) >= 10        # enough pairs actually bound the step
    xg, pg = T(x).view(-1), T(p).view(-1)
    for i in idx:
        k = cand[int(i)]
        got = S.step_bound(xg, pg, [bal.pair_key(*k)], bal.STEP_CCD)
        assert got == pytest.approx(refs[i], rel=1e-12, abs=1e-15), (k, got, refs[i])


def test_ccd_step_bound_over_all_candidates(crossing_case):
    sc, m, S, x, p, cand = crossing_case
    ref = ccd.step_bound(m, x, p, cand, bal.default_params().step_bound)
    keys = [bal.pair_key(*k) for k in cand]
    got = S.step_bound(T(x).view(-1), T(p).view(-1), keys, bal.STEP_CCD)
    assert ref < 1.0
    assert got == pytest.approx(ref, rel=1e-12)
    # conservative advancement on the same pairs, for comparison with its oracle
    got_ca = S.step_bound(T(x).view(-1), T(p).view(-1), keys, bal.STEP_CA)
    assert got_ca == pytest.approx(obal.step_bound(m, x, p, cand, obal.Params()), rel=1e-9)


def test_ccd_bound_is_one_without_pairs(crossing_case):
    sc, m, S, x, p, cand = crossing_case
    assert S.step_bound(T(x).view(-1), T(p).view(-1), [], bal.STEP_CCD) == 1.0


def test_time_step_with_ccd_matches_oracle():
    sc = close_cubes(n=2, gap=5e-4)
    S = bal.Scene(sc, bal.default_params(newton_tol=1e-8, pcg_tol=1e-12, pcg_max_iter=20000,
                                         step_mode=bal.STEP_CCD))
    m = system.make_model(sc)
    compare_trajectory(S, m, sc, 2, obal.Params(newton_tol=1e-8, step_mode="ccd"), T)
