"""bench.py's contract on the CPU: the reference arm (the FP64 oracle on the
host cores) prints one JSON line with the keys the driver reads, and the
recorded DRAM traffic is reported only for the configuration and sources it
was measured with."""
import json

import pytest

import bench


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)

    class A:
        steps, warmup, gpus, nr, ntheta = 2, 1, 1, 64, 64
    assert bench.run_reference(A) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "64x" in d["config"]["workload"]


def test_traffic_is_reported_only_for_its_capture():
    cap = bench.TRAFFIC_CAPTURES[0]
    sha = bench.kernel_sources_sha256()
    got = bench.measured_traffic(cap["variant"], cap["nr"], cap["ntheta"])
    assert got == (cap["bytes"] if cap["sources_sha256"] == sha else None)
    assert bench.measured_traffic(cap["variant"], cap["nr"] // 2, cap["ntheta"]) is None
    assert bench.measured_traffic(cap["variant"] + 100, cap["nr"], cap["ntheta"]) is None
    # the capture is within a few per cent of the algorithmic 272 B per site
    assert cap["bytes"] == pytest.approx(272 * cap["nr"] * cap["ntheta"], rel=0.05)
