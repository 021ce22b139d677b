"""The bench's roofline records: a traffic, instruction or FP64-instruction figure from
profiles/ is used only while the hash of the kernel sources it was measured on matches the
current sources (otherwise the bench reports null), and the FP64-pipe fraction is computed from
it as stated."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.fixture
def records(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "a.md").write_text(
        "# summary\n"
        "TRAFFIC variant=fp32-twogrid bytes_per_launch=2529778000 source=aaaa\n"
        "TRAFFIC variant=fp32-aa bytes_per_launch=2500000000 source=bbbb\n"
        "FP64OPS variant=fp64-twogrid per_cell=193.0 source=aaaa\n")
    (tmp_path / "profiles" / "b.md").write_text("INSTR kernel=closure-mlp-aa-128 per_cell=1146.9 source=cccc\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: "aaaa")
    monkeypatch.setattr(bench, "closure_source_hash", lambda: "cccc")
    return tmp_path


def test_records_match_only_the_current_source(records, monkeypatch):
    assert bench.recorded_traffic("fp32-twogrid") == 2529778000.0
    assert bench.recorded_traffic("fp32-aa") is None          # taken on other sources
    assert bench.recorded_traffic("fp16dev-twogrid") is None  # never taken
    assert bench.recorded_fp64_ops("fp64-twogrid") == 193.0
    assert bench.recorded_instructions("closure-mlp-aa-128") == 1146.9
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: "dddd")  # the sweep changed since
    assert bench.recorded_traffic("fp32-twogrid") is None
    assert bench.recorded_fp64_ops("fp64-twogrid") is None
    assert bench.fp64_pipe("fp64-twogrid", 1 << 24, 6.0) is None


def test_fp64_pipe_fraction(records):
    cells, ms = 256 ** 3, 6.0993
    r = bench.fp64_pipe("fp64-twogrid", cells, ms)
    achieved = 193.0 * cells / (ms / 1e3) / 1e9
    assert r["achieved"] == round(achieved, 1)
    assert bench.FP64_PIPE_PEAK_GINST == pytest.approx(2 * 152 * 2.070)
    assert r["frac"] == round(achieved / bench.FP64_PIPE_PEAK_GINST, 4)
    assert 0.8 < r["frac"] < 0.9
    assert bench.fp64_pipe("fp64-aa", cells, ms) is None


def test_committed_records_name_existing_variants():
    """Every record line in the committed profiles names a variant or kernel the bench knows."""
    import glob
    import re
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            m = re.search(r"(TRAFFIC|FP64OPS) variant=(\S+)", line)
            if m:
                assert m.group(2) in bench.VARIANTS, (path, line)
            m = re.search(r"INSTR kernel=(\S+)", line)
            if m:
                assert m.group(1).startswith("closure-"), (path, line)


def test_oracle_baselines_of_the_other_workloads_run_bounded():
    """The CPU-baseline legs of the turbulence and porous workloads (the oracle as it stands on
    a bounded sample) at small sizes: at least one step, a positive rate, the keys the bench
    reports."""
    for r, unit in ((bench.cpu_baseline_turbulence(min_seconds=0.0, n=16), "MLUPS"),
                    (bench.cpu_baseline_porous(min_seconds=0.0, nb=2), "MFLUPS")):
        assert r["kind"] == "oracle" and r["unit"] == unit and r["value"] > 0 and r["cores"] >= 1
        assert r["sample"].startswith("1 oracle steps")
