"""Pins of the plain inexact Newton ablation in the oracle: sigma stays at
sigma0 and A' stays empty where Algorithm 1 grows sigma and builds A', and the
step stays intersection-free."""
from oracle import bal, system
from paper_2407_00046_b300 import scenes


def _scene():
    sc = scenes.two_cubes(n=2)
    sc.X[sc.body == 1, 1] -= 0.01 - 5e-4
    return sc


def test_plain_newton_keeps_sigma_and_no_augmentation():
    sc = _scene()
    m = system.make_model(sc)
    xa, va, ia = bal.time_step(m, sc.X.copy(), sc.V0.copy(), bal.Params(newton_tol=1e-8))
    xp, vp, ip = bal.time_step(m, sc.X.copy(), sc.V0.copy(), bal.Params(newton_tol=1e-8, al_mode="plain"))
    assert ia["converged"] and ip["converged"]
    # Algorithm 1 augments (A' non-empty at some iterate) and grows sigma here
    assert any(rec["nAp"] > 0 for rec in ia["log"]) and ia["sigma"] > ia["sigma0"]
    assert all(rec["nAp"] == 0 for rec in ip["log"])
    assert ip["sigma"] == ip["sigma0"] and ip["Ap"] == {}
    for x in (xa, xp):
        keys, d = bal.active_pairs(m, x)
        assert len(d) > 0 and d.min() > 0.0
