"""bench.py's host-side accounting, on CPU: the algorithmic abs-diff count of
the roofline (checked against a count by enumeration), the executed-work
split, and the rule that the recorded DRAM traffic is used only while the
kernel sources it was captured on are unchanged."""
import os
import shutil

import numpy as np
import pytest

import bench
from paper_2506_19656_gb300 import synth

REPO = bench.ROOT


def _enumerated_ad(cfg, T):
    """Abs-diffs of the full integer search counted by walking the padded
    frame: every P-frame, group, PU, candidate vector and PU sample."""
    G = (cfg.bands + 2) // 3
    Hp = int(np.ceil(cfg.H / cfg.ctu)) * cfg.ctu
    Wp = int(np.ceil(cfg.W / cfg.ctu)) * cfg.ctu
    pus = sum(1 for _ in range(0, Hp, cfg.ctu) for _ in range(0, Wp, cfg.ctu))
    vectors = sum(1 for dy in range(-cfg.R, cfg.R + 1) for dx in range(-cfg.R, cfg.R + 1))
    return (T - 1) * G * pus * vectors * cfg.ctu * cfg.ctu


@pytest.mark.parametrize("workload", ["tiny", "deepextremecubes", "dynamicearthnet", "era5"])
def test_algorithmic_abs_diffs_match_an_enumeration(workload):
    cfg = synth.WORKLOADS[workload]
    for T in (cfg.sub_T or (cfg.T,)):
        assert bench.algorithmic_ad(cfg, T) == _enumerated_ad(cfg, T)


def test_deepextremecubes_step_count():
    """One step (three encodes of 4 groups, 255 P-frames, 64 PUs of 16 x 16,
    65 x 65 vectors) is 2.12e11 abs-diffs."""
    cfg = synth.WORKLOADS["deepextremecubes"]
    assert 3 * bench.algorithmic_ad(cfg, cfg.T) == 3 * 4 * 255 * 64 * 256 * 65 * 65 == 211_820_544_000


def test_executed_work_splits_exact_and_bound_terms():
    cfg = synth.WORKLOADS["deepextremecubes"]
    full = 3 * 4 * 255 * 64 * 65 * 65
    none = bench.executed_ad(cfg, 0, full)
    assert none["exact_ad"] == 0 and none["ad"] == none["bound_ad"] > 0
    # every vector column of 65 is covered by 9 units of 8 (72 lanes), 8 bounds
    # of (16 / 4)^2 terms each per unit and vector row
    assert none["bound_ad"] == 3 * 4 * 255 * 64 * 65 * 9 * 8 * 16
    some = bench.executed_ad(cfg, full // 100, full)
    assert some["exact_ad"] == (full // 100) * 256
    assert some["ad"] == some["exact_ad"] + some["bound_ad"]
    assert some["exact_fraction"] == pytest.approx(0.01, rel=1e-6)
    # bounds cost well below the full search, which is what pruning buys
    assert none["bound_ad"] < 0.15 * 3 * bench.algorithmic_ad(cfg, cfg.T)


def test_whole_job_value_counts_every_rank():
    assert bench.whole_job_value(10.0, 4, 2, 200.0) == pytest.approx(2 * 10 * 4 / 0.2)


def test_default_qps():
    assert bench.default_qps("deepextremecubes") == (22, 27, 32)
    assert bench.default_qps("era5") == (22,)
    assert bench.default_qps("dynamicearthnet") == (27,)


def _tree(tmp_path, sha):
    """A copy of the kernel sources with a traffic record keyed by `sha`."""
    for f in bench.PERSIST_SOURCES:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(REPO, f), dst)
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / "k_persist_deepextremecubes_traffic.txt").write_text(
        "# comment = ignored\nsources_sha = %s\ndram_bytes_per_launch = 123456\n" % sha)


def test_recorded_traffic_only_for_the_same_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path, "0" * 16)
    assert bench.recorded_traffic() is None
    _tree(tmp_path, bench.kernel_sources_sha())
    assert bench.recorded_traffic() == 123456.0
    # any change to a kernel source drops it
    src = tmp_path / bench.PERSIST_SOURCES[1]
    src.write_text(src.read_text() + "\n// edited\n")
    assert bench.recorded_traffic() is None


def test_recorded_traffic_absent(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic() is None
