"""The benchmark's measurement contract on CPU: the dominant kernel's
algorithmic bytes, the roofline fraction, the DRAM-traffic record and its
source-hash guard, the measured peak, and the defaults of a run."""
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
