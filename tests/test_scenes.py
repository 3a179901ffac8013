"""Input generators: the seeded scenes start valid for the method (positive
tets, no pair within dhat) and have the advertised sizes."""
import numpy as np
import pytest

from oracle import contact, elastic
from paper_2407_00046_b300 import scenes


@pytest.mark.parametrize("name", ["two_cubes_small", "cube_stack_small", "chain_net_shells_small",
                                  "cube_on_slab_small"])
def test_small_scenes_start_feasible(name):
    sc = scenes.scene_by_name(name)
    Dm_inv, vol = elastic.rest_data(sc.X, sc.tets)
    a, b, c, d = (sc.X[sc.tets[:, k]] for k in range(4))
    assert np.all(np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a) > 0)
    cand = contact.candidate_pairs(sc.X, sc, sc.dhat)
    dist, _, _ = contact.pair_distances(sc.X, cand, sc)
    assert dist.size == 0 or dist.min() > sc.dhat


def test_sizes():
    sc = scenes.two_cubes()
    assert (sc.n_tets, sc.n_verts) == (4116, 1024)
    assert sc.pinned.sum() == 64
    assert scenes.cube_stack(n_cubes=2, n=4).n_tets == 2 * 6 * 64


def test_chain_net_link_separation_full_resolution():
    # full-resolution links and a shell: nothing within dhat at rest
    sc = scenes.chain_net_shells(nx=2, nz=2, n_shells=1, shell_m=16, n_spikes=16)
    cand = contact.candidate_pairs(sc.X, sc, sc.dhat)
    dist, _, _ = contact.pair_distances(sc.X, cand, sc)
    assert dist.size == 0 or dist.min() > sc.dhat


def test_seeded_reproducible():
    a, b = scenes.cube_stack(n_cubes=3, n=3), scenes.cube_stack(n_cubes=3, n=3)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.E, b.E)
