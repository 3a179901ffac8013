"""Pins of the oracle's brute-force box broad phase (the reference for the
LBVH): it contains every pair closer than r, it follows the box rule on a
hand-made case, and the swept form contains every pair that comes within r
along the step."""
import numpy as np

from oracle import contact
from paper_2407_00046_b300 import scenes


def _close_pairs(x, sc, r):
    cand = contact.candidate_pairs(x, sc, r)
    if not cand:
        return set()
    d, _, _ = contact.pair_distances(x, cand, sc)
    return {k for k, dd in zip(cand, d) if dd < r}


def _scene():
    sc = scenes.two_cubes(n=3)
    sc.X[sc.body == 1, 1] -= 0.01 - 4e-4
    sc.X[sc.body == 1, 0] += 0.013
    return sc


def test_box_candidates_contain_every_close_pair():
    sc = _scene()
    rng = np.random.default_rng(0)
    x = sc.X + 1e-4 * rng.normal(size=sc.X.shape)
    for r in (1e-3, 5e-3):
        box = set(contact.box_candidates(x, sc, r))
        close = _close_pairs(x, sc, r)
        assert close and close <= box


def test_box_rule_on_a_hand_made_case():
    sc = _scene()
    x = sc.X.copy()
    r = 1e-3
    box = set(contact.box_candidates(x, sc, r))
    # the upper cube sits 0.4 mm above the lower one: faces within r give pairs;
    # lifting it by 1.5 r more separates every box by more than r
    assert any(k[0] == 0 for k in box) and any(k[0] == 1 for k in box)
    x2 = x.copy()
    x2[sc.body == 1, 1] += 1.5 * r
    cross = [k for k in contact.box_candidates(x2, sc, r)
             if len({int(sc.body[v]) for v in contact.stencil_nodes([k], sc)[0]}) > 1]
    assert cross == []


def test_swept_boxes_contain_every_pair_reaching_r_along_the_step():
    sc = _scene()
    rng = np.random.default_rng(1)
    x = sc.X.copy()
    x[sc.body == 1, 1] += 3e-3                 # 3.4 mm apart
    dirv = np.zeros_like(x)
    dirv[sc.body == 1] = [0.0, -4e-3, 0.0]     # falls 4 mm over the step
    dirv += 1e-4 * rng.normal(size=x.shape)
    r = 1e-3
    swept = set(contact.box_candidates(x, sc, r, dirv))
    reach = set()
    for t in np.linspace(0.0, 1.0, 21):
        reach |= _close_pairs(x + t * dirv, sc, r)
    assert reach and reach <= swept
    assert not (reach <= set(contact.box_candidates(x, sc, r)))   # the static boxes miss them
