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


def _tree(tmp_path, sha, name="k_persist_32"):
    """A copy of the kernel sources with a traffic record keyed by `sha`."""
    for f in bench.kernel_sources("persist", 32):
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(REPO, f), dst)
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / f"{name}_traffic.txt").write_text(
        "# comment = ignored\nsources_sha = %s\ndram_bytes_per_item = 15400\n" % sha)


def test_recorded_traffic_only_for_the_same_sources(tmp_path, monkeypatch):
    files = bench.kernel_sources("persist", 32)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path, "0" * 16)
    assert bench.recorded_traffic("k_persist_32", files) is None
    _tree(tmp_path, bench.kernel_sources_sha(files))
    assert bench.recorded_traffic("k_persist_32", files) == 15400.0
    # any change to a kernel source drops it
    src = tmp_path / files[1]
    src.write_text(src.read_text() + "\n// edited\n")
    assert bench.recorded_traffic("k_persist_32", files) is None


def test_recorded_traffic_absent(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k_persist_32", bench.kernel_sources("persist", 32)) is None


def test_kernel_sources_name_the_compiled_files():
    """The persistent kernel's record depends on its CTU's translation unit and
    the device headers; the per-frame kernels' on k_frame.cu and the headers."""
    p = bench.kernel_sources("persist", 32)
    f = bench.kernel_sources("frames", 32)
    assert any(x.endswith("k_batch_ctu32.cu") for x in p) and not any(x.endswith("k_frame.cu") for x in p)
    assert any(x.endswith("k_frame.cu") for x in f)
    for x in p + f:
        assert os.path.exists(os.path.join(REPO, x)), x


def test_work_items_era5():
    """ERA5-shaped sub-cube of T frames at CTU 32: 2 groups x T x 23 x 45 PUs."""
    cfg = synth.WORKLOADS["era5"]
    assert bench.work_items(cfg, 24) == 2 * 24 * 23 * 45


def _butterfly(x, N, T, count, inverse=False):
    """An N-point partial butterfly written out in Python (forward y = T x,
    inverse x = T^T c), counting its multiplications by matrix entries."""
    if N == 2:
        count[0] += 2
        return [64 * (x[0] + x[1]), 64 * (x[0] - x[1])]
    h = N // 2
    if not inverse:
        e = [x[k] + x[N - 1 - k] for k in range(h)]
        o = [x[k] - x[N - 1 - k] for k in range(h)]
        ye = _butterfly(e, h, T[::2, :h], count)
        y = [0] * N
        y[::2] = ye
        for k in range(1, N, 2):
            y[k] = sum(int(T[k, n]) * o[n] for n in range(h))
            count[0] += h
        return y
    ee = _butterfly(x[::2], h, T[::2, :h], count, True)
    out = [0] * N
    for n in range(h):
        o = sum(int(T[2 * i + 1, n]) * x[2 * i + 1] for i in range(h))
        count[0] += h
        out[n], out[N - 1 - n] = ee[n] + o, ee[n] - o
    return out


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_butterfly_multiply_count(N):
    """The partial butterfly reproduces the oracle's matrix product exactly
    (forward and inverse) with bench.butterfly_mults(N) multiplications,
    against N^2 for the matrix form."""
    import oracle
    oracle.build()
    T = oracle.transform_matrix(N).astype(np.int64)
    x = np.random.default_rng(N).integers(-512, 512, N)
    for inverse in (False, True):
        count = [0]
        y = _butterfly([int(v) for v in x], N, T, count, inverse)
        want = (T.T @ x) if inverse else (T @ x)
        assert np.array_equal(np.array(y), want)
        assert count[0] == bench.butterfly_mults(N) < N * N


def test_transform_work_per_step():
    """DeepExtremeCubes-shaped step: 3 encodes x 4 groups x 256 frames x 3
    channels x 128^2 samples, TU 4 / 8 / 16 forward and back: 38.5
    multiply-adds per sample by butterflies, 112 by the matrix form."""
    cfg = synth.WORKLOADS["deepextremecubes"]
    samples = 3 * 4 * 256 * 3 * 128 * 128
    b, m = (3 * v for v in bench.transform_macs(cfg, cfg.T))
    assert b * 2 == samples * 77 and m == samples * 112


def test_cpu_baseline_all_cores_and_one_thread():
    import oracle
    oracle.build()
    cfg = synth.WORKLOADS["tiny"]
    cube = synth.make_cube("tiny")
    before = oracle.max_threads()
    got = bench.cpu_baseline(cube, cfg, frames=4, single_frames=2)
    assert got["kind"] == "oracle" and got["cores"] == before and got["value"] > 0
    assert got["single_thread"]["cores"] == 1 and got["single_thread"]["value"] > 0
    assert "first 2 of 8 frames" in got["single_thread"]["sample"]
    assert oracle.max_threads() == before          # the thread count is restored


def test_parse_tune_log():
    got = bench.parse_tune_log("ctu32 nt128 per4 161.250;ctu32 nt128 per3 170.000;frames 180.500;")
    assert got == {"ctu32 nt128 per4": 161.25, "ctu32 nt128 per3": 170.0, "frames": 180.5}
