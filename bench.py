#!/usr/bin/env python3
"""Throughput of the encoder-analysis path on GB300, one JSON line.

Workload (default): the ERA5-shaped batch -- six float32 variables on the
721 x 1440 grid, six sub-cubes of T = 24, 53, 82, 110, 139 and 168 frames
(synthetic -- see paper_2506_19656_gb300/synth.py), each encoded at QP 22
(CTU 32, search range 16, TU 4/8/16/32) in ONE batched C-ABI call,
xv_encode_batch (captured graphs: one persistent launch over all sub-cubes,
or the jobs as per-frame chains on concurrent streams, whichever the
autotuner timed faster).  One step is the whole path for the six sub-cubes --
min/max, quantise/pack, motion search, transform / quantise / reconstruct,
PSNR and rate.  The metric counts pixels x bands x frames per second.

  value   inputs resident in HBM, device time of K steps (CUDA events)
  e2e     one xv_encode_batch_from_host call per step: the cubes copied from
          pinned host memory by the library, the host results read back
  plain   the per-frame launch path (xv_encode_cube per sub-cube), same work,
          one encode after another and on concurrent streams
  roofline  the dominant kernel (the persistent kernel, or the per-frame
          chains in that mode): integer-search abs-diffs per launch / its
          event-timed duration, against the measured ALU peak
  cpu_baseline  the CPU oracle on a bounded sample (the whole T = 24
          sub-cube), on every host core (and, in `single_thread`, on one)
  deepextremecubes  the DeepExtremeCubes-shaped step (QP 22/27/32) beside it

--workload selects another workload; --impl reference times the CPU oracle
(the reference arm of this tier) on bounded samples of the same workload.
Under torchrun each rank runs its own replica (the path has no exchange
step); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpx·band/s of ME+transform/quant/recon (bit-exact), batched vs plain; p50/p99"
WORKLOAD = "era5"
QPS = (22, 27, 32)
CTU = 0  # 0: the workload's own CTU size; else the --ctu override


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, dist_mod=None, device=None):
    """The timed region's length as the slowest rank saw it (no-op on one rank)."""
    if dist_mod is None or not dist_mod.is_available() or not dist_mod.is_initialized() \
            or dist_mod.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(work_per_rank, steps, world_size, max_total_ms):
    """Units all ranks processed / the slowest rank's time (weak scaling: every
    rank runs its own replica of the workload)."""
    return world_size * work_per_rank * steps / (max_total_ms / 1e3)


def executed_ad(cfg, exact_cand, full_cand):
    """Abs-diffs the integer search executed in one launch: the candidates
    evaluated exactly (N^2 each) plus the sub-block bound pass (8 bounds of
    (N/SB)^2 terms per 8-wide unit of vectors, every unit, every P-frame PU).
    The box-sum table build (additions, not abs-diffs) is not counted."""
    N, R = cfg.ctu, cfg.R
    sb = 4 if N <= 16 else (8 if N == 32 else 16)
    side = 2 * R + 1
    ngxa = side // 8 + 1 if side % 8 == 1 else (side + 7) // 8
    pu_frames = full_cand // (side * side)
    bound = pu_frames * side * ngxa * 8 * (N // sb) ** 2
    exact = exact_cand * N * N
    return {"ad": exact + bound, "exact_ad": exact, "bound_ad": bound,
            "exact_candidates": exact_cand, "full_candidates": full_cand,
            "exact_fraction": exact_cand / full_cand if full_cand else None}


def work_items(cfg, T):
    """Work items of one encode: one per PU (= CU) and frame of every group."""
    G = (cfg.bands + 2) // 3
    Hp = -(-cfg.H // cfg.ctu) * cfg.ctu
    Wp = -(-cfg.W // cfg.ctu) * cfg.ctu
    return G * T * (Hp // cfg.ctu) * (Wp // cfg.ctu)


def algorithmic_ad(cfg, T):
    """Integer-search abs-diffs of one encode: N^2 (2R+1)^2 per PU and P-frame."""
    G = (cfg.bands + 2) // 3
    Hp = -(-cfg.H // cfg.ctu) * cfg.ctu
    Wp = -(-cfg.W // cfg.ctu) * cfg.ctu
    npu = (Hp // cfg.ctu) * (Wp // cfg.ctu)
    return G * (T - 1) * npu * cfg.ctu ** 2 * (2 * cfg.R + 1) ** 2


def butterfly_mults(n):
    """Multiply-adds of one n-point 1-D transform by partial butterflies (the
    kernels' form, forward or inverse): the even half recursively, the odd
    half as an (n/2) x (n/2) product; 2 at n = 2.  The matrix form takes n^2."""
    return 2 if n == 2 else butterfly_mults(n // 2) + (n // 2) ** 2


def transform_macs(cfg, T):
    """Transform multiply-adds of one encode: every TU size of the mask tiles
    every CU of every channel, group and frame, and each is transformed
    forward and back (the RD choice compares the reconstructions), i.e.
    4 M(n) / n per sample and size.  Returns (butterfly count, matrix-form
    count); the matrix form takes 4 n per sample and size."""
    G = (cfg.bands + 2) // 3
    Hp = -(-cfg.H // cfg.ctu) * cfg.ctu
    Wp = -(-cfg.W // cfg.ctu) * cfg.ctu
    samples = G * T * 3 * Hp * Wp
    sizes = [n for n in cfg.tu_sizes if n <= cfg.ctu]
    bfly = sum(samples * 4 * butterfly_mults(n) // n for n in sizes)
    matrix = sum(samples * 4 * n for n in sizes)
    return bfly, matrix


# The sources a dominant kernel is compiled from: the persistent encode
# kernel's translation unit for its CTU size, or the per-frame kernels', and
# the device headers they include.  A recorded DRAM traffic figure holds only
# while these are unchanged.
_CSRC = "paper_2506_19656_gb300/csrc/"


def kernel_sources(mode, ctu):
    base = (_CSRC + "me.cuh", _CSRC + "tqr.cuh", _CSRC + "xv_dev.cuh", _CSRC + "xv_internal.h")
    if mode == "persist":
        return (_CSRC + f"k_batch_ctu{ctu}.cu", _CSRC + "batch.cuh", _CSRC + "dec.cuh") + base
    return (_CSRC + "k_frame.cu",) + base


def kernel_sources_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(name, files):
    """DRAM bytes (read + written) per work item (one PU of one frame) of a
    kernel, from the committed ncu summary profiles/<name>_traffic.txt, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"{name}_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                vals[k.strip()] = v.strip()
    if vals.get("sources_sha") != kernel_sources_sha(files):
        return None
    try:
        return float(vals["dram_bytes_per_item"])
    except (KeyError, ValueError):
        return None


def cpu_sample_frames(workload, cfg):
    """The oracle's bounded sample of a workload, as frames of its first cube:
    the T = 24 ERA5-shaped sub-cube in full, the first 8 frames of the
    DynamicEarthNet-shaped cube, 192 of the 256 DeepExtremeCubes-shaped frames
    (about 10-30 s of host time each), the whole tiny cube."""
    return {"era5": cfg.sub_T[0] if cfg.sub_T else cfg.T, "dynamicearthnet": 8,
            "deepextremecubes": 192}.get(workload, cfg.T)


def cpu_baseline(cube, cfg, frames=16, single_frames=0, whole=False):
    """The oracle, as it stands, on the first `frames` frames at each QP, with
    its OpenMP threads on every host core; with single_frames > 0 also on one
    thread over the first `single_frames` frames.  whole: the sample is a whole
    sub-cube of the workload (its own min/max), not a causal prefix."""
    import oracle
    oracle.build()

    def run(n, is_whole):
        n = min(n, cube.shape[1])
        sample = cube[:, :n].copy()
        t0 = time.perf_counter()
        for qp in QPS:
            oracle.encode_cube(sample, cfg.ctu, cfg.R, cfg.tu_mask, qp, want_levels=True)
        dt = time.perf_counter() - t0
        work = len(QPS) * cfg.bands * n * cfg.H * cfg.W / 1e6
        what = (f"the whole T = {n} sub-cube" if is_whole else
                f"first {n} of {cfg.T} frames (causal prefix) of the same cube")
        return work / dt, f"{what} at QP {QPS}, {dt:.1f} s"

    value, sample = run(frames, whole)
    out = {"value": value, "unit": "Mpx·band/s", "cores": oracle.max_threads(), "kind": "oracle",
           "sample": sample}
    if single_frames:
        threads = oracle.max_threads()
        oracle.set_threads(1)
        try:
            v1, s1 = run(single_frames, False)
        finally:
            oracle.set_threads(threads)
        out["single_thread"] = {"value": v1, "unit": "Mpx·band/s", "cores": 1, "sample": s1}
    return out


def plain_concurrent(jobs, stream, flush, k):
    """The per-frame path with the encodes as concurrent chains: one context,
    stream and host thread per encode (xv_encode_cube is synchronous on its
    stream).  Device time per step from events: the streams start after an
    event on the launching stream, which then waits for each of them."""
    import statistics
    from concurrent.futures import ThreadPoolExecutor

    import torch

    from paper_2506_19656_gb300 import xv
    ctxs = [xv.Context(0) for _ in jobs]
    streams = [torch.cuda.Stream() for _ in jobs]

    def run():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        for s in streams:
            s.wait_event(e0)
        with ThreadPoolExecutor(len(jobs)) as ex:
            list(ex.map(lambda i: xv.xv_encode_cube(ctxs[i], jobs[i], streams[i]), range(len(jobs))))
        for s in streams:
            ev = torch.cuda.Event()
            ev.record(s)
            stream.wait_event(ev)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)
    run()
    ms = [run() for _ in range(k)]
    for c in ctxs:
        c.close()
    return {"ms_per_step": statistics.mean(ms),
            "path": "xv_encode_cube per encode, the encodes on concurrent streams (a context and host thread each)"}


def default_qps(workload):
    """The QPs one step encodes when --qps is not given: 22, 27 and 32 for the
    DeepExtremeCubes-shaped cube, the workload's own QPs otherwise (22 for the
    ERA5-shaped sub-cubes)."""
    from paper_2506_19656_gb300 import synth
    return (22, 27, 32) if workload == "deepextremecubes" else tuple(synth.WORKLOADS[workload].qps)


def workload_jobs(workload, frames=0, device=None, qps=None):
    """The encodes one step runs: for each sub-cube (the ERA5-shaped workload is
    six causal prefixes of one generated cube, each in its own contiguous
    buffer) and each QP (default: QPS, which main() sets from --qps or
    default_qps), device buffers and an xv_job.  Returns (cfg, lengths, cube,
    srcs, jobs, bufs): cube = the generated host cube, srcs = the device
    sub-cubes, bufs[i] = job i's buffers plus "src", "qp" and "T"."""
    import dataclasses

    import torch

    from paper_2506_19656_gb300 import synth, xv
    cfg = synth.WORKLOADS[workload]
    if frames:
        cfg = dataclasses.replace(cfg, T=frames)
    if CTU:
        cfg = dataclasses.replace(cfg, ctu=CTU)
    lengths = list(cfg.sub_T) if cfg.sub_T and not frames else [cfg.T]
    cube = synth.make_cube(workload, T=max(lengths))
    full = torch.from_numpy(cube)
    srcs = [full[:, :T].contiguous().to(device) for T in lengths]
    del full
    jobs, bufs = [], []
    for T, src in zip(lengths, srcs):
        for qp in (QPS if qps is None else qps):
            p = xv.xv_params_init(cfg.ctu, cfg.R, cfg.tu_mask, qp)
            b = xv.alloc_cube_buffers(cfg.bands, T, cfg.H, cfg.W, p, device=device)
            b.update(src=src, qp=qp, T=T)
            jobs.append(xv.make_job(src, p, b["planes"], b["recon"], minmax=b["minmax"], mv=b["mv"], cost=b["cost"],
                                    levels=b["levels"], tu_log2=b["tu_log2"], bits=b["bits"]))
            bufs.append(b)
    return cfg, lengths, cube, srcs, jobs, bufs


def run_reference(args):
    """Reference arm: the CPU oracle on bounded samples of the workload (the
    ERA5-shaped sub-cubes by default: each step encodes the first 3 frames of
    the T = 24 sub-cube; the DeepExtremeCubes-shaped cube: its first 8 frames
    at each QP)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import dataclasses

    import numpy as np

    import oracle
    from paper_2506_19656_gb300 import synth
    oracle.build()
    cfg = synth.WORKLOADS[args.workload]
    if CTU:
        cfg = dataclasses.replace(cfg, ctu=CTU)
    frames = {"era5": 3, "dynamicearthnet": 2, "tiny": cfg.T}.get(args.workload, 8)
    cube = synth.make_cube(args.workload, T=max(frames, cfg.sub_T[0] if cfg.sub_T else frames))
    cube = np.ascontiguousarray(cube[:, :frames])
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for qp in QPS:
            oracle.encode_cube(cube, cfg.ctu, cfg.R, cfg.tu_mask, qp)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    work = len(QPS) * cfg.bands * frames * cfg.H * cfg.W / 1e6
    ms = 1e3 * sum(times) / len(times)
    value = work / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpx·band/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": cfg.name, "qps": list(QPS), "ctu": cfg.ctu, "search_range": cfg.R,
                   "tu_sizes": list(cfg.tu_sizes), "sample_frames": frames},
        "cpu_baseline": {"value": value, "unit": "Mpx·band/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"first {frames} frames of the workload's first (sub-)cube at QP {QPS} per step"},
        "e2e": {"value": value, "unit": "Mpx·band/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_decode(args):
    """Decode run: the workload's encodes (QP 22/27/32 for the DeepExtremeCubes
    shape) are encoded once, untimed; each timed step decodes all of them in
    one xv_decode_batch, writing the reconstruction planes and the cube in its
    own units (float32), checked equal to the encoder's reconstruction."""
    import statistics

    import numpy as np
    import torch

    from paper_2506_19656_gb300 import build, xv
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cfg, lengths, _, _, jobs, bufs = workload_jobs(args.workload, args.frames, dev)
    ctx = xv.Context(0)
    if args.block_size:
        xv.xv_debug_force_block_size(ctx, args.block_size)
    djobs, outs = [], []
    for b in bufs:
        p = xv.xv_params_init(cfg.ctu, cfg.R, cfg.tu_mask, b["qp"])
        G, Tn = b["levels"].shape[:2]
        o = dict(recon=torch.empty_like(b["recon"]), bits=torch.zeros((G, Tn), dtype=torch.int64, device=dev),
                 dst=torch.empty((cfg.bands, b["T"], cfg.H, cfg.W), dtype=torch.float32, device=dev))
        djobs.append(xv.make_djob(p, b["levels"], b["mv"], b["tu_log2"], o["recon"], bits=o["bits"],
                                  minmax=b["minmax"], dst=o["dst"], bands=cfg.bands, H=cfg.H, W=cfg.W))
        outs.append(o)
    enc = xv.xv_encode_batch(ctx, jobs)  # untimed: the coded data to decode
    work_mpx = len(QPS) * sum(cfg.bands * T * cfg.H * cfg.W for T in lengths) / 1e6
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def timed(step, k):
        ms, extra = [], []
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            extra.append(out)
        return ms, extra

    def batched():
        xv.xv_decode_batch(ctx, djobs)
        return xv.xv_last_batch_kernel_ms(ctx)

    for _ in range(args.warmup):
        batched()
    torch.cuda.synchronize()
    for b, o, r in zip(bufs, outs, enc):  # bit-exact before anything is timed
        assert torch.equal(o["recon"].view(torch.int16), b["recon"].view(torch.int16)), "decode != encoder recon"
        assert torch.equal(o["bits"], b["bits"]) and int(o["bits"].sum()) == r["total_bits"], "decoded rate differs"
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = xv.xv_ctx_launches(ctx)
    torch.cuda.synchronize()
    step_ms, kern_ms = timed(batched, args.steps)
    torch.cuda.synchronize()
    launches = xv.xv_ctx_launches(ctx) - launches0
    clk = clocks.stop()
    value = work_mpx / (sum(step_ms) / args.steps / 1e3)

    # plain: per-frame decode launches, then unpack, per encode
    def plain_step():
        for dj, b, o in zip(djobs, bufs, outs):
            G, Tn, _, Hp, Wp = b["levels"].shape
            fsz = 3 * Hp * Wp
            ncu = b["tu_log2"].shape[2]
            o["bits"].zero_()
            for t in range(Tn):
                xv.xv_decode_frame(ctx, b["levels"][:, t], o["recon"][:, t - 1] if t else None, b["mv"][:, t],
                                   b["tu_log2"][:, t], G, Tn * fsz, Hp, Wp, dj.p, Tn * ncu, o["recon"][:, t],
                                   o["bits"][:, t], Tn)
            xv.xv_unpack(ctx, o["recon"], cfg.bands, cfg.H, cfg.W, b["minmax"], o["dst"])
    plain = None
    if not args.no_plain:
        plain_step()
        pm, _ = timed(plain_step, max(3, min(args.steps, 5)))
        for b, o in zip(bufs, outs):
            assert torch.equal(o["recon"].view(torch.int16), b["recon"].view(torch.int16))
        plain = {"value": work_mpx / (statistics.mean(pm) / 1e3), "ms_per_step": statistics.mean(pm),
                 "path": "xv_decode_frame per frame (one launch for all groups) + xv_unpack, per encode"}

    # end to end: the coded data from pinned host memory, the float cube back to the host
    hosts = [{k: b[k].cpu().pin_memory() for k in ("levels", "mv", "tu_log2")} for b in bufs]
    backs = [torch.empty(o["dst"].shape, dtype=torch.float32).pin_memory() for o in outs]

    def e2e_step():
        for h, b in zip(hosts, bufs):
            for k in ("levels", "mv", "tu_log2"):
                b[k].copy_(h[k], non_blocking=True)
        xv.xv_decode_batch(ctx, djobs)
        for o, bk in zip(outs, backs):
            bk.copy_(o["dst"], non_blocking=True)
        torch.cuda.synchronize()
    e2e_step()
    em, _ = timed(e2e_step, max(3, min(args.steps, 5)))
    h2d = sum(sum(h[k].numel() * h[k].element_size() for k in h) for h in hosts)
    d2h = sum(bk.numel() * bk.element_size() for bk in backs)
    e2e = {"value": work_mpx / (statistics.mean(em) / 1e3), "unit": "Mpx·band/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h)}

    # HBM roofline of the persistent decode: per plane sample the levels read
    # (2 B), the reference read by motion compensation (2 B) and the
    # reconstruction written (2 B); vectors and TU sizes are negligible
    samples = sum(b["levels"].numel() for b in bufs)
    algo = 6 * samples
    kms = statistics.mean(kern_ms)
    peak = 6660.3
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass
    achieved = algo / (kms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": f"k_persist<{cfg.ctu}> in decode mode", "kernel_ms": kms,
                "work_per_launch": f"{algo:.4g} B (levels read, reference read, recon written: 6 B per plane sample)",
                "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    line = {
        "metric": "Mpx·band/s of decode (levels, vectors, TU sizes -> recon -> cube units; bit-exact)",
        "value": value, "unit": "Mpx·band/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(step_ms) / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": cfg.name, "qps": list(QPS), "ctu": cfg.ctu, "frames": lengths if len(lengths) > 1 else cfg.T,
                   "bands": cfg.bands, "path": "xv_decode_batch (persistent kernel, decode mode) + unpack",
                   "block_size": xv.xv_last_batch_block_size(ctx),
                   "l2": "flushed before every step (256 MB write)", "parallelism": "replicas1"},
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "plain": plain, "e2e": e2e, "roofline": roofline, "clocks": clk, "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_options(args):
    """Intra / deblocking run: each step encodes the workload's cubes through
    xv_encode_cube with XV_INTRA | XV_DEBLOCK (frame 0 intra predicted, every
    frame deblocked before it becomes a reference); "plain" is the same
    per-frame path without the options.  Also timed alone: the deblocking of
    every frame (HBM roofline: per plane sample the levels read and the
    reconstruction read and written, 6 B) and the intra frame 0."""
    import statistics

    import numpy as np
    import torch

    from paper_2506_19656_gb300 import build, xv
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cfg, lengths, _, _, jobs, bufs = workload_jobs(args.workload, args.frames, dev)
    ctx = xv.Context(0)
    opt_jobs = []
    for j in jobs:
        oj = xv.xv_job.from_buffer_copy(j)
        oj.p.flags = xv.XV_INTRA | xv.XV_DEBLOCK
        opt_jobs.append(oj)
    work_mpx = len(QPS) * sum(cfg.bands * T * cfg.H * cfg.W for T in lengths) / 1e6
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def timed(step, k, before=None):
        ms = []
        for _ in range(k):
            if before:
                before()
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    def with_options():
        return [xv.xv_encode_cube(ctx, j) for j in opt_jobs]

    for _ in range(args.warmup):
        with_options()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = xv.xv_ctx_launches(ctx)
    step_ms = timed(with_options, args.steps)
    launches = xv.xv_ctx_launches(ctx) - launches0
    clk = clocks.stop()
    value = work_mpx / (sum(step_ms) / args.steps / 1e3)
    res = with_options()

    plain = None
    if not args.no_plain:
        for _ in range(2):
            [xv.xv_encode_cube(ctx, j) for j in jobs]
        pm = timed(lambda: [xv.xv_encode_cube(ctx, j) for j in jobs], max(3, min(args.steps, 5)))
        plain = {"value": work_mpx / (statistics.mean(pm) / 1e3), "ms_per_step": statistics.mean(pm),
                 "path": "xv_encode_cube per encode without the options (flat frame 0, no loop filter)"}
    # the encodes are independent chains: run concurrently (plain_concurrent)
    k = max(3, min(args.steps, 5))
    cm = plain_concurrent(opt_jobs, stream, flush, k)["ms_per_step"]
    cp = plain_concurrent(jobs, stream, flush, k)["ms_per_step"]
    conc = {"value": work_mpx / (cm / 1e3), "ms_per_step": cm, "plain_value": work_mpx / (cp / 1e3),
            "plain_ms_per_step": cp,
            "path": "the encodes on concurrent streams (one context and host thread each), with and without the options"}
    with_options()  # the buffers hold the options' coded data again

    # deblocking alone: the frames of every encode as the "groups" of
    # xv_deblock_frame calls, on a fresh copy of the reconstruction
    db = []
    for b, j in zip(bufs, opt_jobs):
        G, Tn, _, Hp, Wp = b["recon"].shape
        npu = b["tu_log2"].shape[2]
        db.append(dict(src=b["recon"].reshape(G * Tn, 3, Hp, Wp), work=torch.empty_like(b["recon"]).reshape(G * Tn, 3, Hp, Wp),
                       tu=b["tu_log2"].reshape(G * Tn, npu), lev=b["levels"].reshape(G * Tn, 3, Hp, Wp),
                       mv=b["mv"].reshape(G * Tn, npu, 2), n=G * Tn, Hp=Hp, Wp=Wp, npu=npu, p=j.p))

    def refresh():
        for d in db:
            d["work"].copy_(d["src"])

    def deblock_all():  # in calls of at most 255 frames (the per-call group limit)
        for d in db:
            for a in range(0, d["n"], 255):
                b_ = min(d["n"], a + 255)
                xv.xv_deblock_frame(ctx, d["work"][a:b_], b_ - a, 3 * d["Hp"] * d["Wp"], d["Hp"], d["Wp"], d["p"],
                                    d["npu"], d["tu"][a:b_], d["lev"][a:b_], d["mv"][a:b_], False)
    refresh()
    deblock_all()
    dm = timed(deblock_all, max(3, min(args.steps, 10)), before=refresh)
    samples = sum(d["work"].numel() for d in db)
    algo = 6 * samples
    dms = statistics.mean(dm)
    peak = 6660.3
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass
    achieved = algo / (dms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "k_cbf + k_deblock<vertical> + k_deblock<horizontal> (deblocking)",
                "kernel_ms": dms,
                "work_per_launch": f"{algo:.4g} B for {sum(d['n'] for d in db)} frames (levels read, reconstruction "
                                   f"read and written: 6 B per plane sample)",
                "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}

    # the intra frame 0 of every encode alone
    def intra_all():
        for b, j in zip(bufs, opt_jobs):
            G, Tn, _, Hp, Wp = b["recon"].shape
            npu = b["tu_log2"].shape[2]
            b["bits"][:, 0].zero_()
            xv.xv_intra_frame(ctx, b["planes"][:, 0], G, Tn * 3 * Hp * Wp, Hp, Wp, j.p, Tn * npu, b["recon"][:, 0],
                              b["levels"][:, 0], b["tu_log2"][:, 0], b["mv"][:, 0], b["bits"][:, 0], Tn)
    intra_all()
    im = timed(intra_all, max(3, min(args.steps, 10)))
    intra_mpx = len(QPS) * len(lengths) * cfg.bands * cfg.H * cfg.W / 1e6
    line = {
        "metric": "Mpx·band/s of ME+transform/quant/recon with frame-0 intra prediction and in-loop deblocking "
                  "(bit-exact), per-frame path",
        "value": value, "unit": "Mpx·band/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(step_ms) / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": cfg.name, "qps": list(QPS), "ctu": cfg.ctu, "frames": lengths if len(lengths) > 1 else cfg.T,
                   "bands": cfg.bands, "path": "xv_encode_cube with XV_INTRA | XV_DEBLOCK",
                   "l2": "flushed before every step (256 MB write)", "parallelism": "replicas1"},
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "plain": plain, "concurrent": conc, "roofline": roofline,
        "intra_frame": {"ms_per_step": statistics.mean(im), "value": intra_mpx / (statistics.mean(im) / 1e3),
                        "unit": "Mpx·band/s", "what": "frame 0 of every encode through xv_intra_frame"},
        "psnr_mean": [r["psnr_mean"] for r in res], "bpppb": [r["bpppb"] for r in res],
        "clocks": clk, "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_metrics(args):
    """Quality-metric run: the workload's encodes are made once, untimed; each
    timed step computes SSIM per band (xv_ssim) and the mean spectral angle
    (xv_sa) of every encode's reconstruction against the cube."""
    import statistics

    import numpy as np
    import torch

    from paper_2506_19656_gb300 import build, xv
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cfg, lengths, _, _, jobs, bufs = workload_jobs(args.workload, args.frames, dev)
    srcs = [b["src"] for b in bufs]
    ctx = xv.Context(0)
    xv.xv_encode_batch(ctx, jobs)  # untimed: the reconstructions to score
    work_mpx = len(QPS) * sum(cfg.bands * T * cfg.H * cfg.W for T in lengths) / 1e6
    windows = len(QPS) * sum(cfg.bands * T * max(cfg.H - 10, 0) * max(cfg.W - 10, 0) for T in lengths)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        out = []
        for src, b in zip(srcs, bufs):
            s = xv.xv_ssim(ctx, src, b["recon"], b["minmax"])
            a, _ = xv.xv_sa(ctx, src, b["recon"], b["minmax"])
            out.append((s["ssim_mean"], a))
        return out

    def ssim_only():
        for src, b in zip(srcs, bufs):
            xv.xv_ssim(ctx, src, b["recon"], b["minmax"])

    def timed(fn, k):
        ms, res = [], None
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, res

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = xv.xv_ctx_launches(ctx)
    step_ms, res = timed(step, args.steps)
    launches = xv.xv_ctx_launches(ctx) - launches0
    clk = clocks.stop()
    ssim_ms, _ = timed(ssim_only, max(3, min(args.steps, 5)))
    value = work_mpx / (statistics.mean(step_ms) / 1e3)
    # SSIM kernel: per window 121 taps x 9 FP32 operations (3 deviations and
    # their weighted products, 3 accumulations) plus about 100 for the means
    # and the index; the FP32 peak is 152 SMs x 128 lanes x 2 (FMA) x 2.07 GHz
    flops = windows * (121 * 9 + 100)
    peak = 152 * 128 * 2 * 2.07e9
    ach = flops / (statistics.mean(ssim_ms) / 1e3)
    roofline = {"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": "k_ssim (FP32)", "kernel_ms": statistics.mean(ssim_ms),
                "work_per_launch": f"{flops:.4g} FP32 operations over {windows:.4g} windows (all encodes)",
                "peak_basis": "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz"}
    line = {
        "metric": "Mpx·band/s of SSIM per band + mean spectral angle of the reconstructions",
        "value": value, "unit": "Mpx·band/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg.name, "qps": list(QPS), "frames": lengths if len(lengths) > 1 else cfg.T,
                   "bands": cfg.bands, "path": "xv_ssim + xv_sa per encode",
                   "l2": "flushed before every step (256 MB write)", "parallelism": "replicas1"},
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "ssim_mean_by_qp": [r[0] for r in res], "sa_rad_by_qp": [r[1] for r in res],
        "roofline": roofline, "clocks": clk, "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_pca(args):
    """PCA run on the workload's cube: each timed step fits the PCA over its
    bands (xv_pca_fit), projects it onto all but the last component (the
    paper's "PCA - 9 bands" packing of ten bands into three videos) and
    inverts the projection; the round trip is checked against the cube."""
    import statistics

    import numpy as np
    import torch

    from paper_2506_19656_gb300 import build, synth, xv
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cfg = synth.WORKLOADS[args.workload]
    T = args.frames or cfg.T
    cube = synth.make_cube(args.workload, T=T)
    src = torch.from_numpy(np.ascontiguousarray(cube)).to(dev)
    bands = cube.shape[0]
    npc = max(1, bands - 1)
    ctx = xv.Context(0)
    z = torch.empty((npc,) + cube.shape[1:], dtype=torch.float32, device=dev)
    back = torch.empty(cube.shape, dtype=torch.float32, device=dev)
    npix = int(np.prod(cube.shape[1:]))
    work_mpx = bands * npix / 1e6
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    state = {}

    def step():
        m, c, v = xv.xv_pca_fit(ctx, src)
        xv.xv_pca_project(ctx, src, m, c, npc, z)
        xv.xv_pca_inverse(ctx, z, m, c, back)
        state.update(m=m, c=c, v=v)

    def proj_inv():
        xv.xv_pca_project(ctx, src, state["m"], state["c"], npc, z)
        xv.xv_pca_inverse(ctx, z, state["m"], state["c"], back)

    def timed(fn, k):
        ms = []
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the dropped component's variance is the round trip's mean square error per pixel
    err = (back.double() - src.double()).pow(2).sum(dim=0).mean().item()
    assert abs(err - state["v"][-1]) <= 1e-3 * state["v"][-1] + 1e-9 * state["v"][0], (err, state["v"][-1])
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = xv.xv_ctx_launches(ctx)
    step_ms = timed(step, args.steps)
    launches = xv.xv_ctx_launches(ctx) - launches0
    clk = clocks.stop()
    pi_ms = timed(proj_inv, max(3, min(args.steps, 5)))
    esz = src.element_size()
    algo = npix * (bands * esz + npc * 4) + npix * (npc * 4 + bands * 4)  # project, then inverse
    kms = statistics.mean(pi_ms)
    peak = 6660.3
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass
    ach = algo / (kms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                "kernel": "k_pca_project + k_pca_inverse", "kernel_ms": kms,
                "work_per_launch": f"{algo:.4g} B (bands and components read and written once each)",
                "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    line = {
        "metric": "Mpx·band/s of PCA over bands (fit + project to bands-1 components + inverse)",
        "value": work_mpx / (statistics.mean(step_ms) / 1e3), "unit": "Mpx·band/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 fit, f32 transform",
        "data": "synthetic",
        "config": {"workload": cfg.name, "frames": T, "bands": bands, "components_kept": npc,
                   "path": "xv_pca_fit + xv_pca_project + xv_pca_inverse",
                   "l2": "flushed before every step (256 MB write)", "parallelism": "replicas1"},
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "variance_kept": float(sum(state["v"][:npc]) / sum(state["v"])), "roundtrip_mse": err,
        "roofline": roofline, "clocks": clk, "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_pca_all(args):
    """The paper's "PCA - all bands" test (Sec. 3, Tab. 5) on the workload's
    cube: each timed step fits the PCA over all bands, projects the cube onto
    every component, packs the components three to a group and encodes every
    group at its own QP (xv_split_groups + one xv_encode_batch; the i-th group
    at base QP + 5 i, later components at lower quality), then rebuilds the
    cube: the groups' reconstructions back to component units (xv_unpack)
    and the inverse projection.  The line reports the step's throughput and
    the rebuilt cube's PSNR per band against the original (peak = the band's
    maximum, as the codec's PSNR), beside one QP for all groups."""
    import statistics

    import numpy as np
    import torch

    from paper_2506_19656_gb300 import build, synth, xv
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cfg = synth.WORKLOADS[args.workload]
    T = args.frames or cfg.T
    cube = synth.make_cube(args.workload, T=T)
    src = torch.from_numpy(np.ascontiguousarray(cube)).to(dev)
    bands = cube.shape[0]
    G = (bands + 2) // 3
    base = QPS[0]
    qps_all = [base + 5 * g for g in range(G)]
    ctx = xv.Context(0)
    z = torch.empty(cube.shape, dtype=torch.float32, device=dev)
    zr = torch.empty(cube.shape, dtype=torch.float32, device=dev)
    back = torch.empty(cube.shape, dtype=torch.float32, device=dev)
    p = xv.xv_params_init(cfg.ctu, cfg.R, cfg.tu_mask, base)
    buf = xv.alloc_cube_buffers(bands, T, cfg.H, cfg.W, p, device=dev)
    whole = xv.make_job(z, p, buf["planes"], buf["recon"], minmax=buf["minmax"], mv=buf["mv"], cost=buf["cost"],
                        levels=buf["levels"], tu_log2=buf["tu_log2"], bits=buf["bits"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(qps):
        mean, comps, var = xv.xv_pca_fit(ctx, src)
        xv.xv_pca_project(ctx, src, mean, comps, bands, z)
        res = xv.xv_encode_batch(ctx, xv.xv_split_groups(whole, qps))
        xv.xv_unpack(ctx, buf["recon"], bands, cfg.H, cfg.W, buf["minmax"], zr)
        xv.xv_pca_inverse(ctx, zr, mean, comps, back)
        return res

    def timed(qps, k):
        ms = []
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = step(qps)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, res

    def quality(res):
        x = src.double()
        e = (back.double() - x).pow(2).mean(dim=(1, 2, 3))
        peak = x.amax(dim=(1, 2, 3))
        psnr = (10 * torch.log10(peak * peak / e)).tolist()
        bits = sum(r["total_bits"] for r in res)
        return {"psnr_band": psnr, "psnr_mean": float(np.mean(psnr)), "bpppb": bits / (bands * T * cfg.H * cfg.W)}

    for _ in range(args.warmup):
        step(qps_all)
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = xv.xv_ctx_launches(ctx)
    step_ms, res = timed(qps_all, args.steps)
    launches = xv.xv_ctx_launches(ctx) - launches0
    clk = clocks.stop()
    q_all = quality(res)
    for _ in range(2):
        step([base] * G)
    one_ms, res1 = timed([base] * G, max(3, min(args.steps, 5)))
    q_one = quality(res1)
    work_mpx = bands * T * cfg.H * cfg.W / 1e6
    line = {
        "metric": "Mpx·band/s of PCA over all bands + per-group-QP encode of the components + rebuild (\"PCA - all bands\")",
        "value": work_mpx / (statistics.mean(step_ms) / 1e3), "unit": "Mpx·band/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32 encode, f64 fit, f32 projections", "data": "synthetic",
        "config": {"workload": cfg.name, "frames": T, "bands": bands, "group_qps": qps_all, "ctu": cfg.ctu,
                   "path": "xv_pca_fit + xv_pca_project + xv_split_groups + xv_encode_batch + xv_unpack + "
                           "xv_pca_inverse", "l2": "flushed before every step (256 MB write)", "parallelism": "replicas1"},
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "per_group_qp": q_all,
        "one_qp": dict(q_one, qp=base, ms_per_step=statistics.mean(one_ms)),
        "clocks": clk, "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_serve(args):
    """Serving run: a stream of requests with Poisson arrivals, kinds drawn
    uniformly from the four workloads, through xv_serve_*; against the plain
    per-request path (xv_encode_cube on each request in arrival order).  With
    --util U, a second labelled run at the arrival rate that offers U times
    the first run's saturated throughput (the same requests, the arrival gaps
    rescaled)."""

    import numpy as np
    import torch

    from paper_2506_19656_gb300 import build, synth, xv
    build.build()
    torch.cuda.set_device(0)
    reqs = synth.serving_requests(seed=4000, n=args.requests, mean_interval_s=1.0 / args.rate)
    # host pools in pinned memory: causal prefixes of one long cube serve the
    # shorter draws of a workload (every prefix is itself a valid cube)
    t0 = time.time()
    pools = {"tiny": [torch.from_numpy(synth.make_cube("tiny", cube=i)).pin_memory() for i in range(4)]}
    for name in ("deepextremecubes", "dynamicearthnet", "era5"):
        if any(r["workload"] == name for r in reqs):
            T = max(r["T"] for r in reqs if r["workload"] == name)
            pools[name] = [torch.from_numpy(synth.make_cube(name, T=T)).pin_memory()]
    gen_s = time.time() - t0
    work = []
    prefixes = {}  # one contiguous pinned copy per (workload, pool cube, T), shared by every request of that shape
    for r in reqs:
        c = synth.WORKLOADS[r["workload"]]
        pool = pools[r["workload"]]
        key = (r["workload"], r["cube"] % len(pool), r["T"])
        host = prefixes.get(key)
        if host is None:
            host = pool[key[1]][:, : r["T"]]
            if not host.is_contiguous():
                host = host.contiguous().pin_memory()
            prefixes[key] = host
        p = xv.xv_params_init(c.ctu, c.R, c.tu_mask, r["qp"])
        work.append((r, host, p, c.bands * r["T"] * c.H * c.W / 1e6))
    total_mpx = sum(w[3] for w in work)
    ctx = xv.Context(0, mem_budget_bytes=120 << 30)

    def serve(arrivals):
        """One pass of the request stream at the given arrival times."""
        xv.xv_serve_start(ctx, 64, args.frames_per_tick)
        seen = set()  # warm-up: one request of each kind, alone
        for r, host, p, _ in work:
            if r["workload"] in seen:
                continue
            seen.add(r["workload"])
            t = xv.xv_serve_submit(ctx, xv.make_request(host, p))
            while not xv.xv_serve_poll(ctx, t)[0]:
                time.sleep(0.001)
        stats0 = xv.xv_serve_stats(ctx)
        lat, done_at, pending = {}, {}, {}
        start = time.perf_counter()
        i = 0
        while len(lat) < len(work):
            now = time.perf_counter() - start
            while i < len(work) and arrivals[i] <= now:
                r, host, p, _ = work[i]
                pending[xv.xv_serve_submit(ctx, xv.make_request(host, p))] = i
                i += 1
            for t in list(pending):
                ok, res = xv.xv_serve_poll(ctx, t)
                if ok:
                    k = pending.pop(t)
                    assert res["status"] == 0, res
                    lat[k] = res["latency_s"]
                    done_at[k] = time.perf_counter() - start
            time.sleep(0.0005)
        makespan = max(done_at.values()) - arrivals[0]
        stats = xv.xv_serve_stats(ctx)
        xv.xv_serve_stop(ctx)
        lats = np.array([lat[k] for k in range(len(work))])
        return {"value": total_mpx / makespan, "p50_s": float(np.percentile(lats, 50)),
                "p99_s": float(np.percentile(lats, 99)), "makespan_s": makespan,
                "ticks": stats["ticks"] - stats0["ticks"], "peak_resident": stats["peak_resident"]}

    arrivals = [w[0]["arrival_s"] for w in work]
    main = serve(arrivals)

    # plain per-request path: measured service time of each request (upload,
    # xv_encode_cube, results), then a FIFO timeline over the same arrivals
    bufs = {}
    service = []
    for r, host, p, _ in work:
        key = (r["workload"], r["T"])
        c = synth.WORKLOADS[r["workload"]]
        if key not in bufs:
            bufs[key] = (torch.empty(host.shape, dtype=host.dtype, device="cuda"),
                         xv.alloc_cube_buffers(c.bands, r["T"], c.H, c.W, p, levels=False))
        dsrc, b = bufs[key]
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        dsrc.copy_(host, non_blocking=True)
        job = xv.make_job(dsrc, p, b["planes"], b["recon"], minmax=b["minmax"], mv=b["mv"], bits=b["bits"])
        xv.xv_encode_cube(ctx, job)
        service.append(time.perf_counter() - s0)
    del bufs
    torch.cuda.empty_cache()

    def plain_timeline(arr):
        finish, lat = 0.0, []
        for a_, sv in zip(arr, service):
            finish = max(finish, a_) + sv
            lat.append(finish - a_)
        mk = finish - arr[0]
        return {"value": total_mpx / mk, "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "makespan_s": mk,
                "path": "xv_encode_cube per request in arrival order (measured service times, FIFO timeline)"}

    under = None
    if args.util > 0:
        # the rate at which the offered work is `util` x the saturated throughput
        rate2 = args.util * main["value"] / (total_mpx / len(work))
        scale = args.rate / rate2
        arr2 = [a_ * scale for a_ in arrivals]
        under = serve(arr2)
        under.update(label=f"secondary run: arrivals at {rate2:.2f}/s, offering {args.util:.0%} of the first run's "
                           "saturated throughput", rate_per_s=rate2, plain=plain_timeline(arr2))
    ctx.close()
    kinds = {k: sum(1 for r in reqs if r["workload"] == k) for k in synth.WORKLOADS}
    line = {
        "metric": METRIC, "value": main["value"], "unit": "Mpx·band/s", "n_gpus": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "serving mix of the four workloads", "requests": len(work),
                   "arrivals": f"Poisson, mean {args.rate:g}/s", "kinds": kinds, "budget_gb": 120,
                   "max_resident": 64, "frames_per_tick": args.frames_per_tick,
                   "host_pool": "pinned; one cube per workload (four for the tiny one), shorter draws use causal "
                                "prefixes", "generation_s": round(gen_s, 1)},
        "p50_s": main["p50_s"], "p99_s": main["p99_s"], "makespan_s": main["makespan_s"], "total_mpx_band": total_mpx,
        "ticks": main["ticks"], "peak_resident": main["peak_resident"],
        "plain": plain_timeline(arrivals),
        "under_load": under,
    }
    print(json.dumps(line), flush=True)


def parse_tune_log(log):
    """The autotuner's candidate timings as {candidate: ms} ("ctu32 nt128 per4"
    = a CTU-32 persistent launch of 128-thread blocks, 4 resident per SM;
    "frames" = the per-frame mode)."""
    out = {}
    for item in log.split(";"):
        item = item.strip()
        if item:
            name, ms = item.rsplit(" ", 1)
            out[name] = float(ms)
    return out


def measured_peaks(ctx):
    """The device's measured rates of the roofline's instruction sequences
    (xv_measure_peak): abs-diff-accumulates as sad, on the FP32 pipe and as
    their mix, and 32-bit integer multiply-adds."""
    from paper_2506_19656_gb300 import xv
    out = {}
    for kind, name in xv.PEAK_KINDS.items():
        rate, ms = xv.xv_measure_peak(ctx, kind)
        out[name] = {"per_s": rate, "ms": ms}
    out["absdiff_best"] = max(out[k]["per_s"] for k in ("sad", "fp32_absdiff", "sad_fp32_mix"))
    return out


def kernels_alone(ctx, cfg, bufs, flush, stream, reps=3):
    """The motion search and the transform chain each timed on their own, as
    the per-frame kernels over every P-frame of every encode at once: frames
    1..T-1 of a group are the "groups" of one call (plane stride one frame),
    the encode's own reconstructions are the references and, for the
    transform, its vectors the motion.  The outputs must equal the batched
    encode's bit for bit (checked), so the times are of the same work."""
    import torch
    from paper_2506_19656_gb300 import xv
    calls = []
    for b in bufs:
        G, T, _, Hp, Wp = b["planes"].shape
        if T < 2:
            continue
        npu = b["mv"].shape[2]
        p = xv.xv_params_init(cfg.ctu, cfg.R, cfg.tu_mask, b["qp"])
        o = dict(mv=torch.zeros_like(b["mv"]), recon=torch.zeros_like(b["recon"]),
                 levels=torch.zeros_like(b["levels"]), tu=torch.zeros_like(b["tu_log2"]),
                 bits=torch.zeros_like(b["bits"]))
        calls.append((b, o, p, G, T, Hp, Wp, npu))

    def chunks(T):  # frames 1..T-1 as calls of at most 255 "groups" (the entry points' limit)
        return [(f0, min(255, T - f0)) for f0 in range(1, T, 255)]

    def run_me():
        for b, o, p, G, T, Hp, Wp, npu in calls:
            for g in range(G):
                for f0, n in chunks(T):
                    xv.xv_motion_search(ctx, b["planes"][g, f0], b["recon"][g, f0 - 1], n, 3 * Hp * Wp, Hp, Wp, p,
                                        o["mv"][g, f0], pu_gstride=npu)

    def run_tqr():
        for b, o, p, G, T, Hp, Wp, npu in calls:
            o["bits"].zero_()  # the transform adds each CU's bits to its frame's total
            for g in range(G):
                for f0, n in chunks(T):
                    xv.xv_transform_quant_recon(ctx, b["planes"][g, f0], b["recon"][g, f0 - 1], b["mv"][g, f0], n,
                                                3 * Hp * Wp, Hp, Wp, p, npu, o["recon"][g, f0], o["levels"][g, f0],
                                                o["tu"][g, f0], o["bits"][g, f0], 1)

    def timed(fn):
        best = None
        for _ in range(reps + 1):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None or ms < best else best
        return best
    me_ms, tqr_ms = timed(run_me), timed(run_tqr)
    for b, o, *_ in calls:  # the same results as the batched encode
        assert torch.equal(o["mv"][:, 1:], b["mv"][:, 1:]), "motion search alone differs from the encode"
        for k, kb in (("recon", "recon"), ("levels", "levels"), ("tu", "tu_log2"), ("bits", "bits")):
            assert torch.equal(o[k][:, 1:], b[kb][:, 1:]), f"transform alone: {k} differs from the encode"
    launches = sum(c[3] * len(chunks(c[4])) for c in calls)
    del calls
    torch.cuda.empty_cache()
    return me_ms, tqr_ms, launches


def tune_ctu(dev, candidates=(16, 32, 64), reps=3):
    """The CTU size for a workload whose configuration leaves it open (the
    ERA5-shaped sub-cubes): the T = 24 sub-cube encoded through
    xv_encode_batch at each candidate size (each after its own autotuning
    call), the fastest encode section (median of `reps`) wins.  The choice
    changes the output (the CTU is part of the encode's definition), so the
    encode is then run, and checked, at the chosen size."""
    import torch
    from paper_2506_19656_gb300 import synth, xv
    global CTU
    cfg = synth.WORKLOADS["era5"]
    times = {}
    saved = CTU
    try:
        for ctu in candidates:
            CTU = ctu
            c, lengths, _, _, jobs, bufs = workload_jobs("era5", frames=cfg.sub_T[0], device=dev)
            ctx = xv.Context(dev.index or 0)
            xv.xv_encode_batch(ctx, jobs)  # tunes this shape
            ms = []
            for _ in range(reps):
                xv.xv_encode_batch(ctx, jobs)
                ms.append(xv.xv_last_batch_kernel_ms(ctx))
            times[ctu] = statistics.median(ms)
            ctx.close()
            del jobs, bufs
            torch.cuda.empty_cache()
    finally:
        CTU = saved
    best = min(times, key=times.get)
    return best, {"encode_section_ms": {str(k): v for k, v in times.items()}, "chosen": best,
                  "sample": f"the T = {cfg.sub_T[0]} sub-cube, median of {reps} batched encodes per CTU size"}


def secondary_line(ctx, dev, flush, stream, steps=10):
    """The DeepExtremeCubes-shaped step (QP 22, 27 and 32 through
    xv_encode_batch) beside the headline: device time per step, value and the
    search's effective ALU fraction."""
    from paper_2506_19656_gb300 import xv
    import torch
    global CTU
    saved, CTU = CTU, 0  # the workload's own CTU size (16), not the headline's tuned one
    try:
        cfg, lengths, _, _, jobs, bufs = workload_jobs("deepextremecubes", 0, dev, qps=(22, 27, 32))
    finally:
        CTU = saved
    assert cfg.ctu == 16
    for _ in range(3):
        xv.xv_encode_batch(ctx, jobs)
    torch.cuda.synchronize()
    ms, kms = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = xv.xv_encode_batch(ctx, jobs)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        kms.append(xv.xv_last_batch_kernel_ms(ctx))
    block_size = xv.xv_last_batch_block_size(ctx)
    tune_log = xv.xv_last_tune_log(ctx)
    # the last step's outputs against the per-cube path's (bit-exact)
    recon = [b["recon"].clone() for b in bufs]
    for j, b, r, rec in zip(jobs, bufs, res, recon):
        want = xv.xv_encode_cube(ctx, j)
        assert want["total_bits"] == r["total_bits"] and torch.equal(b["recon"], rec), \
            "the DeepExtremeCubes-shaped batch differs from the per-cube path"
    work_mpx = 3 * sum(cfg.bands * T * cfg.H * cfg.W for T in lengths) / 1e6
    ad = 3 * sum(algorithmic_ad(cfg, T) for T in lengths)
    k = statistics.mean(kms)
    out = {"workload": cfg.name, "qps": [22, 27, 32], "value": work_mpx / (statistics.mean(ms) / 1e3),
           "unit": "Mpx·band/s", "ms_per_step": statistics.mean(ms), "steps": steps,
           "block_size": block_size, "encode_section_ms": k,
           "search_effective_gad_s": ad / (k / 1e3) / 1e9,
           "autotune_ms": parse_tune_log(tune_log) if tune_log else None,
           "checked": "the last step's reconstruction and rates equal xv_encode_cube's"}
    del jobs, bufs
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="xv", choices=["xv", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-alone", action="store_true",
                    help="skip timing the motion search and the transform chain on their own")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the DeepExtremeCubes-shaped line reported beside the ERA5-shaped headline")
    ap.add_argument("--qps", default="",
                    help="QPs of the encodes in one step (default: 22,27,32 for the DeepExtremeCubes-shaped cube, "
                         "the workload's own otherwise)")
    ap.add_argument("--frames", type=int, default=0, help="encode only the first F frames (profiling cases)")
    ap.add_argument("--ctu", type=int, default=0, choices=[0, 8, 16, 32, 64],
                    help="CTU size instead of the workload's own (the encode changes with it)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["tiny", "deepextremecubes", "dynamicearthnet", "era5"],
                    help="the ERA5-shaped sub-cubes (default: six uneven-length sub-cubes in one batch), the "
                         "DeepExtremeCubes-shaped cube, the DynamicEarthNet-shaped uint16 cube or the tiny cube")
    ap.add_argument("--serve", action="store_true", help="the serving run (request stream) instead")
    ap.add_argument("--decode", action="store_true", help="the decode run (the workload's coded data) instead")
    ap.add_argument("--metrics", action="store_true", help="the SSIM / spectral-angle run instead")
    ap.add_argument("--pca", action="store_true", help="the PCA (fit, project, inverse) run instead")
    ap.add_argument("--pca-all", action="store_true",
                    help="the PCA over all bands with one QP per component group (encode and rebuild) instead")
    ap.add_argument("--options", action="store_true",
                    help="the per-frame path with frame-0 intra prediction and in-loop deblocking instead")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--util", type=float, default=0.0,
                    help="serving: also run at the arrival rate that offers this fraction of the saturated throughput")
    ap.add_argument("--rate", type=float, default=200.0, help="mean arrivals per second")
    ap.add_argument("--frames-per-tick", type=int, default=8)
    ap.add_argument("--block-size", type=int, default=0,
                    help="the batched path's execution mode instead of the autotuner's choice: a persistent-kernel "
                         "block size (128/192/256/512) or 1 for the per-frame mode, e.g. to profile the variant an "
                         "uninstrumented run picks")
    args = ap.parse_args()
    globals()["CTU"] = args.ctu
    globals()["QPS"] = tuple(int(q) for q in args.qps.split(",")) if args.qps else default_qps(args.workload)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.decode:
        return run_decode(args)
    if args.metrics:
        return run_metrics(args)
    if args.pca:
        return run_pca(args)
    if args.pca_all:
        return run_pca_all(args)
    if args.options:
        return run_options(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            dist.barrier()

    from paper_2506_19656_gb300 import build, xv
    build.build()
    dev = torch.device("cuda", local)
    ctu_tuning = None
    if args.workload == "era5" and not args.ctu and not args.frames:
        # the configuration leaves the ERA5-shaped batch's CTU open: tune it
        chosen, ctu_tuning = tune_ctu(dev)
        globals()["CTU"] = chosen
    ctx = xv.Context(local)
    if args.block_size:
        xv.xv_debug_force_block_size(ctx, args.block_size)
    cfg, lengths, cube, srcs, jobs, bufs = workload_jobs(args.workload, args.frames, dev)
    src = srcs[0] if len(srcs) == 1 else None
    work_mpx = len(QPS) * sum(cfg.bands * T * cfg.H * cfg.W for T in lengths) / 1e6
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # larger than the 129 MB L2
    stream = torch.cuda.current_stream()

    def timed(step, k):
        """k steps, each bracketed by events on the launching stream, L2 flushed before each."""
        ms, extra = [], []
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            extra.append(out)
        return ms, extra

    def batched():
        xv.xv_encode_batch(ctx, jobs)
        return xv.xv_last_batch_kernel_ms(ctx)

    # warm-up (also builds the tuner / allocates scratch)
    for _ in range(args.warmup):
        batched()
    torch.cuda.synchronize()
    tune_log = xv.xv_last_tune_log(ctx)  # the first batch of this shape tuned it
    peaks = measured_peaks(ctx)

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = xv.xv_ctx_launches(ctx)
    barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms = timed(batched, args.steps)
    torch.cuda.synchronize()
    barrier()
    launches = xv.xv_ctx_launches(ctx) - launches0
    block_size = xv.xv_last_batch_block_size(ctx)
    _, blocks_per_sm = xv.xv_last_batch_config(ctx, cfg.ctu)
    exact_cand, full_cand = xv.xv_last_batch_search_stats(ctx)
    # step latency percentiles over at least 20 repeats: the K timed steps,
    # topped up when K < 20 by further steps timed the same way, still inside
    # the clock sampling (they do not enter `value`)
    extra_ms = timed(batched, 20 - len(step_ms))[0] if len(step_ms) < 20 else []
    lat_ms = list(step_ms) + extra_ms
    clk = clocks.stop()

    total_ms = max_over_ranks(sum(step_ms), dist if ws > 1 else None, dev)
    value = whole_job_value(work_mpx, args.steps, ws, total_ms)

    # plain per-frame path, same work
    plain = None
    if not args.no_plain:
        for _ in range(2):
            for j in jobs:
                xv.xv_encode_cube(ctx, j)
        pm, _ = timed(lambda: [xv.xv_encode_cube(ctx, j) for j in jobs], max(3, min(args.steps, 5)))
        plain = {"value": work_mpx / (statistics.mean(pm) / 1e3), "ms_per_step": statistics.mean(pm),
                 "path": "xv_encode_cube per encode: one motion-search and one transform launch per frame"}
        plain["concurrent"] = plain_concurrent(jobs, stream, flush, max(3, min(args.steps, 5)))
        plain["concurrent"]["value"] = work_mpx / (plain["concurrent"]["ms_per_step"] / 1e3)

    # end to end: one C-ABI call per step that takes the cubes from pinned host
    # memory (the library copies them in) and returns the host results (PSNR,
    # rate) read back from the device
    hosts = [torch.from_numpy(cube[:, :T].copy()).pin_memory() for T in lengths]
    host_of_job = [hosts[lengths.index(b["T"])] if i % len(QPS) == 0 else None for i, b in enumerate(bufs)]

    def e2e_step():
        return xv.xv_encode_batch_from_host(ctx, jobs, host_of_job)

    for _ in range(2):
        e2e_step()
    em, _ = timed(e2e_step, max(3, min(args.steps, 5)))
    G = (cfg.bands + 2) // 3
    d2h = len(jobs) * cfg.bands * (32 + 48) + len(jobs) * 8 + 4 * 24
    e2e = {"value": work_mpx / (statistics.mean(em) / 1e3), "unit": "Mpx·band/s",
           "h2d_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hosts)),
           "d2h_bytes_per_step": int(d2h)}

    # roofline of the dominant kernel(s): the persistent encode, or in the
    # per-frame mode (block size 1) the motion-search and transform launches
    # of the concurrent chains; the peak is measured on this device now
    frames_mode = block_size == 1
    ad = len(QPS) * sum(algorithmic_ad(cfg, T) for T in lengths)
    kms = statistics.mean(kern_ms)
    achieved = ad / (kms / 1e3)
    executed = executed_ad(cfg, exact_cand, full_cand)
    tmac = [len(QPS) * sum(transform_macs(cfg, T)[i] for T in lengths) for i in (0, 1)]
    items = len(QPS) * sum(work_items(cfg, T) for T in lengths)
    if frames_mode:
        per = [recorded_traffic(f"k_{k}_frame_{cfg.ctu}", kernel_sources("frames", cfg.ctu)) for k in ("me", "tqr")]
        per_item = None if None in per else sum(per)
    else:
        per_item = recorded_traffic(f"k_persist_{cfg.ctu}", kernel_sources("persist", cfg.ctu))
    traffic = per_item * items if per_item is not None else None
    traffic_note = (f"ncu dram bytes read + written per work item ({per_item:.0f} B, a capture of the same kernel "
                    f"sources on a short prefix) x {items} items of this launch" if per_item is not None else
                    "none: no ncu DRAM capture of the current kernel sources is recorded for this kernel")
    peak_ad = peaks["absdiff_best"]
    peak_mac = peaks["imad"]["per_s"]
    me_ms, tqr_ms, alone_launches = kernels_alone(ctx, cfg, bufs, flush, stream) if not args.no_alone else (None,) * 3
    window_tma = None
    if frames_mode and not args.no_alone:
        # the per-frame mode's search windows by TMA (the default) against the
        # threads' own 16-byte loads: the encode section both ways
        def section_ms(k=3):
            out = []
            for _ in range(k):
                flush.zero_()
                xv.xv_encode_batch(ctx, jobs)
                out.append(xv.xv_last_batch_kernel_ms(ctx))
            return statistics.median(out)
        xv.xv_debug_set_window_wait(ctx, -1)
        xv.xv_encode_batch(ctx, jobs)  # captures the variant's graphs
        off_ms = section_ms()
        xv.xv_debug_set_window_wait(ctx, 0)
        xv.xv_encode_batch(ctx, jobs)
        on_ms = section_ms()
        window_tma = {"tma_ms": on_ms, "loads_ms": off_ms,
                      "what": "encode section (median of 3) with the search windows by TMA vs by 16-byte loads"}
    alone = None
    if me_ms:
        alone = {
            "search": {"ms": me_ms, "effective_gad_s": ad / (me_ms / 1e3) / 1e9,
                       "frac": ad / (me_ms / 1e3) / peak_ad,
                       "kernel": f"k_me_frame<{cfg.ctu}> over every P-frame at once ({alone_launches} launches)"},
            "transform": {"ms": tqr_ms, "butterfly_gmac_s": tmac[0] / (tqr_ms / 1e3) / 1e9,
                          "frac": tmac[0] / (tqr_ms / 1e3) / peak_mac,
                          "matrix_form_gmac_s": tmac[1] / (tqr_ms / 1e3) / 1e9,
                          "kernel": f"k_tqr_frame<{cfg.ctu}> over every P-frame at once ({alone_launches} launches), "
                                    "motion compensation and the RD choice over every TU size included"},
            "note": "each timed alone on the encode's own references and vectors (outputs checked equal to the "
                    "batched encode's); peaks: the measured abs-diff and multiply-add rates",
        }
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_ad / 1e9, "unit": "GAD/s",
                "frac": achieved / peak_ad, "traffic": traffic, "traffic_note": traffic_note,
                "effective": "achieved/frac count the full search's abs-diffs (the method's definition); the kernel "
                             "skips candidates that the exact sub-block bound excludes, so frac can exceed 1",
                "executed": executed["ad"] / (kms / 1e3) / 1e9,
                "executed_frac": executed["ad"] / (kms / 1e3) / peak_ad,
                "executed_work": executed,
                "kernel": (f"k_me_frame<{cfg.ctu}> + k_tqr_frame<{cfg.ctu}> (the jobs as per-frame chains on "
                           f"concurrent streams)" if frames_mode else
                           f"k_persist<{cfg.ctu}> (motion search + refinement + transform/quant/recon, fused)"),
                "work_per_launch": f"{ad:.4g} integer-search abs-diffs ({cfg.ctu}^2 x {2 * cfg.R + 1}^2 per PU "
                                   f"and P-frame) over {items} work items",
                "kernel_ms": kms,
                "transform": {"butterfly_mac": tmac[0], "matrix_form_mac": tmac[1],
                              "butterfly_gmac_s_lower_bound": tmac[0] / (kms / 1e3) / 1e9,
                              "note": "forward + inverse of every allowed TU size over every sample (the RD "
                                      "choice); the rate divides by the whole encode section, search included"},
                "alone": alone,
                "window_tma": window_tma,
                "peak_basis": "measured now on this device (xv_measure_peak): the fastest abs-diff-accumulate "
                              "sequence of sad / FP32 / their mix; MEASURED_PEAKS.json holds no integer-pipe peak",
                "peaks_measured": peaks}

    line = {
        "metric": METRIC, "value": value, "unit": "Mpx·band/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": cfg.name, "qps": list(QPS), "ctu": cfg.ctu, "search_range": cfg.R,
                   "tu_sizes": list(cfg.tu_sizes), "frames": lengths if len(lengths) > 1 else cfg.T,
                   "bands": cfg.bands,
                   "path": "xv_encode_batch (" + ("per-frame chains on concurrent streams, the autotuner's choice"
                                                  if frames_mode else "persistent kernel") + ")",
                   "block_size": block_size, "blocks_per_sm": blocks_per_sm or "as many as fit",
                   "autotune_ms": parse_tune_log(tune_log) if tune_log else "forced (--block-size)",
                   "ctu_autotune": ctu_tuning,
                   "l2": "flushed before every step (256 MB write); "
                   f"the float32 input ({sum(t.numel() * 4 for t in srcs) / 1e9:.2f} GB) is also larger than L2",
                   "parallelism": f"replicas{ws}"},
        "p50_ms": statistics.median(lat_ms), "p99_ms": float(np.percentile(lat_ms, 99)),
        "latency_samples": len(lat_ms), "latency_samples_extra": len(extra_ms),
        "stage_ms": {"search_and_transform": kms, "rest": statistics.mean(step_ms) - kms,
                     "rest_is": "min/max, quantise/pack, PSNR, rate totals and the results read-back (the step's "
                                "time outside the encode section)"},
        "plain": plain, "e2e": e2e, "roofline": roofline, "clocks": clk,
        "gpu_launches": int(launches),
    }
    if rank == 0 and ws == 1 and not args.no_extra and args.workload == "era5" and not args.frames:
        line["deepextremecubes"] = secondary_line(ctx, dev, flush, stream)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cube, cfg, frames=cpu_sample_frames(args.workload, cfg),
                                            single_frames={"era5": 2, "deepextremecubes": 8}.get(args.workload, 2),
                                            whole=args.workload == "era5" and not args.frames)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
