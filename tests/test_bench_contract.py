"""The headline JSON line of bench.py carries every key of the benchmark contract, computed as
stated: the device timing helpers are replaced by stand-ins (no GPU here), everything else --
argument handling, roofline arithmetic, the source-hashed traffic record, the line's layout --
is the bench's own."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _fake_variant(lbm, variant, steps, warmup, world, tile=None, min_seconds=0.0, max_repeats=200):
    cells = 256 ** 3
    bpp = 8 if variant.startswith("fp64") else (2 if "dev" in variant else 4)
    sweep_ms = 0.4
    alg = 2 * 19 * bpp * cells
    return {"mlups": cells / (sweep_ms + 0.004) / 1e3, "ms_per_step": sweep_ms + 0.004, "sweep_ms": sweep_ms,
            "fill_ms": 0.0, "sweep_share": 1.0, "sweep_gbs": alg / (sweep_ms / 1e3) / 1e9,
            "alg_bytes_per_sweep": alg, "launches": steps,
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 4},
            "info": {"cells": cells, "fluid_cells": cells, "bytes_per_pdf": bpp}, "finite": True, "mass": float(cells),
            "repeats": 7 if min_seconds > 0 else 1}


def _fake_error(lbm, variant, steps=2000):
    return {"steps": steps, "pdf": 1e-9, "deviation": 1e-7, "u": 1e-6, "against": "oracle column"}


def _fake_e2e(lbm, variant, steps, world):
    return {"value": 30000.0, "unit": "MLUPS", "h2d_bytes_per_step": 268435, "d2h_bytes_per_step": 268499}


def test_headline_line_has_the_contract_keys(monkeypatch, capsys):
    pytest.importorskip("torch")
    monkeypatch.setattr(bench, "time_variant", _fake_variant)
    monkeypatch.setattr(bench, "time_e2e", _fake_e2e)
    monkeypatch.setattr(bench, "time_diag_sweep", lambda lbm, variant: {"diag_ms": 1.1, "plain_ms": 1.0})
    monkeypatch.setattr(bench, "variant_error", _fake_error)
    monkeypatch.setattr(bench, "measure_workloads", lambda args: {"c1_taylor_green": {"value": 1.0}})
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    bench.main(["--steps", "20", "--warmup", "3", "--no-cpu-baseline"])
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 20, 3)
    assert d["unit"] == "MLUPS" and d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["vs_baseline"] is None and d["dtype"] == "f32" and "workload" in d["config"]
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert r["achieved"] == pytest.approx(2 * 19 * 4 * 256 ** 3 / 0.4e-3 / 1e9, rel=1e-3)
    # traffic: the committed record of the current sweep source, or null when the source changed
    assert r["traffic"] == bench.recorded_traffic("fp32-twogrid")
    assert set(d["e2e"]) == {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert d["gpu_launches"] == 20
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    assert set(d["variants"]) == set(bench.VARIANTS)
    assert d["variants"]["fp64-twogrid"]["fp64_pipe"] == bench.fp64_pipe("fp64-twogrid", 256 ** 3, 0.4)
    # every variant states its error against the oracle; the headline's is repeated at the top
    assert all(v["error_vs_oracle"]["steps"] == 2000 for v in d["variants"].values())
    assert d["stated_error"] == d["variants"]["fp32-twogrid"]["error_vs_oracle"]
    # the headline's timed region was repeated for the clock sampler (median repeat reported)
    assert d["timing"]["repeats"] == 7
    assert d["workloads"] == {"c1_taylor_green": {"value": 1.0}}


def test_no_workloads_flag(monkeypatch, capsys):
    pytest.importorskip("torch")
    monkeypatch.setattr(bench, "time_variant", _fake_variant)
    monkeypatch.setattr(bench, "time_e2e", _fake_e2e)
    monkeypatch.setattr(bench, "time_diag_sweep", lambda lbm, variant: {"diag_ms": 1.1, "plain_ms": 1.0})
    monkeypatch.setattr(bench, "variant_error", _fake_error)
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    bench.main(["--steps", "20", "--warmup", "3", "--no-cpu-baseline", "--no-workloads", "--headline-only"])
    d = json.loads([l for l in capsys.readouterr().out.splitlines() if l.strip()][0])
    assert "workloads" not in d and d["stated_error"] is None
