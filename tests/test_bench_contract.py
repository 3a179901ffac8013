"""The benchmark's measurement contract on CPU: the dominant kernel's
algorithmic bytes, the roofline fraction, the DRAM-traffic record and its
source-hash guard, the measured peak, the defaults of a run, and the
time-step phase's summary and wall-clock budget (on a host stand-in scene)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_df64_spmv_bytes_are_the_symmetric_storage_read_once():
    nv, nL, nC = 433336, 2454448, 3136
    name, b = bench.spmv_kernel_bytes("df64", nv, nL, nC)
    nb = nL + nC
    # D and L/C blocks as 8-byte double-floats (72 B), one column index per block,
    # the row pointer, one read of p and one write of q (24 B each per vertex)
    assert b == (nv + nb) * 72 + nb * 4 + (nv + 1) * 4 + 2 * 24 * nv
    assert name.startswith("k_dd_spmv")
    _, b32 = bench.spmv_kernel_bytes("fp32", nv, nL, nC)
    _, b64 = bench.spmv_kernel_bytes("fp64", nv, nL, nC)
    assert b32 < b64


def test_roofline_fraction():
    e = bench.roofline_entry("df64", "k", 3000.0, 6000.0, "measured", 1, 0.08, 10, 1, 1, 0, None)
    assert e["frac"] == 0.5 and e["bound"] == "hbm" and e["unit"] == "GB/s"


def test_traffic_record_is_guarded_by_the_kernel_sources(tmp_path, monkeypatch):
    assert bench.ncu_traffic("df64", "no_such_scene") is None
    rec = bench.NCU_TRAFFIC[("df64", "chain_net_shells")]
    assert rec["bytes"] > 240e6                      # at least the algorithmic bytes
    # a record whose source hash does not match the tree reads as unknown
    stale = {("df64", "chain_net_shells"): dict(rec, sources={k: "0" * 16 for k in rec["sources"]})}
    monkeypatch.setattr(bench, "NCU_TRAFFIC", stale)
    assert bench.ncu_traffic("df64", "chain_net_shells") is None


def test_peak_is_the_measured_copy_bandwidth():
    peak, kind = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == 6400.0


def test_default_run_is_one_gpu_a_few_steps():
    import argparse
    captured = {}

    def fake_parse(self, args=None, namespace=None):
        captured["defaults"] = {a.dest: a.default for a in self._actions}
        raise SystemExit(0)

    with pytest.MonkeyPatch.context() as mp:
        mp.setattr(argparse.ArgumentParser, "parse_args", fake_parse)
        with pytest.raises(SystemExit):
            bench.main()
    d = captured["defaults"]
    assert d["gpus"] == 1 and d["warmup"] >= 3 and 1 <= d["steps"] <= 20
    assert d["sigma_rule"] == "printed" and d["newton_max"] >= 200 and d["time_steps"] >= 2
    assert d["scene"] == "chain_net_shells" and d["precision"] == "df64"


class _FakeScene:
    """Host stand-in for a scene: Algorithm 1 converges at iteration `conv`."""

    def __init__(self, conv, sleep=0.0):
        self.conv, self.sleep, self.calls, self.ended = conv, sleep, 0, False

    def step_begin(self, x, v, stream=None):
        self.calls = 0

    def step_end(self, x, v, stream=None):
        self.ended = True

    def get_al_state(self):
        return {"sigma": 2.0 * (1 + self.calls), "sigma0": 2.0}

    def get_params(self):
        class P:
            newton_max_iter = 50
        return P()

    def newton_step(self, x, stream=None, check=True):
        import time
        time.sleep(self.sleep)
        self.calls += 1
        return {"status": 0, "converged": int(self.calls > self.conv), "pcg_iters": 10, "n_active": self.calls,
                "dmin": 1.0 / self.calls, "ms_assemble": 1.0, "ms_solve": 2.0, "ms_line_search": 0.5,
                "ms_contact": 0.25}


def test_budgeted_time_step_matches_the_time_step_summary():
    S = _FakeScene(conv=4)
    out = bench.budgeted_time_step(S, None, None, None, budget_s=1e9)
    # four iterations that do not pass the test, then the one that does
    assert out["converged"] == 1 and out["status"] == 0 and out["newton_iters"] == 4
    assert out["pcg_iters_total"] == 50 and out["max_active"] == 5 and out["min_distance"] == 0.2
    assert out["ms_solve"] == 10.0 and out["sigma0"] == 2.0 and out["sigma_final"] == 12.0
    assert S.ended and out["budget_hit"] == 0


def test_budgeted_time_step_stops_at_the_budget_and_the_cap():
    S = _FakeScene(conv=10 ** 6, sleep=0.02)
    out = bench.budgeted_time_step(S, None, None, None, budget_s=0.05)
    assert out["budget_hit"] == 1 and out["converged"] == 0 and out["status"] == 3
    assert 1 <= out["newton_iters"] < 50 and S.ended
    S = _FakeScene(conv=10 ** 6)
    out = bench.budgeted_time_step(S, None, None, None, budget_s=1e9)
    assert out["newton_iters"] == 50 and out["converged"] == 0 and out["budget_hit"] == 0


def test_pcg_iteration_bytes_are_the_spmv_plus_two_fused_vector_passes():
    nv, nL, nC = 433336, 2454448, 0
    _, spmv = bench.spmv_kernel_bytes("df64", nv, nL, nC)
    b = bench.pcg_iteration_bytes(nv, nL, nC)
    assert b - spmv == 312 * nv                   # 7 vector accesses + D^-1, then z, p read and p written
    assert 375e6 < b < 376e6                      # the chain net's 1.77M-tet system
    e = bench.pcg_iteration_roofline("df64", nv, nL, nC, 9000.0, 6500.0, "measured")
    assert e["frac"] == round(b * 9000.0 / 1e9 / 6500.0, 4) and e["bound"] == "hbm"
    assert bench.pcg_iteration_roofline("mixed", nv, nL, nC, 9000.0, 6500.0, "measured") is None
