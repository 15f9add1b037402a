"""Benchmark of the SparStencil GB300 hot path (one JSON line on rank 0).

Workload: Box-2D9P, 4096 x 4096 FP32 grid, periodic boundary, 100 time steps, seeded
random positive weights normalised to 1 (the paper's Table-2 2D workload at a size that a
single run covers).  One bench "step" is one full run of the 100 time steps through the C
ABI (sparstencil_run: copy into the padded grid + ceil(100/t) sparse tensor-core sweeps).

  value     GStencil/s = 100 * 4096^2 / run time (device-resident input, L2 flushed
            before every timed run by writing a 512 MiB buffer), BF16 split operands
            (rel-L2 <= 1e-5 against the FP64 oracle, checked on sampled points)
  e2e       the same metric through sparstencil_run_host (pinned host buffers, H2D copy of
            the input and D2H copy of the result inside the timed region)
  roofline  the sweep kernel's algorithmic HBM bytes (8 B per output per sweep) over its
            device time (CUDA events around each launch), against the measured copy
            bandwidth in MEASURED_PEAKS.json
  variants  the single-word BF16 path and the plain FP32 CUDA-core direct stencil on the
            same workload, each with its rel-L2 against the oracle
  cpu_baseline / --impl reference   the FP64 C oracle on the host cores, on a bounded
            sample of the workload (test infrastructure, not the product path)

--gpus N runs under torchrun with one process per GPU: every rank runs its own replica of
the workload (the paper's method is single-GPU; replicas only), value = all ranks' work /
max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CFG_NAME = "box2d9p_4096"
METRIC = "GStencil/s per GB300, sparse-TCU vs plain FP32 at stated L2 err; p99 latency"
FALLBACK_HBM_GBS = 6800.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _profile_traffic():
    """Per-launch DRAM bytes of the sweep kernel from the committed ncu summary, if the
    summary was taken on the current kernel source (sweep2d.cu + kernels.h; else None)."""
    csrc = os.path.join(ROOT, "paper_2506_22969_gb300", "csrc")
    prof = os.path.join(ROOT, "profiles", "sweep2d_box9_4096.md")
    try:
        h = hashlib.sha256()
        for name in ("sweep2d.cu", "kernels.h"):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(f.read())
        sha = h.hexdigest()[:16]
        with open(prof) as f:
            text = f.read()
        m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", text)
        m_tr = re.search(r"dram_bytes_per_launch_scaled:\s*([0-9.eE+]+)", text)
        if m_sha and m_tr and m_sha.group(1) == sha:
            return float(m_tr.group(1))
    except OSError:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.samples.append([x.strip() for x in line.split(",")])

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                smax.append(float(s[2]))
                for name, v in zip(names, s[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _workload():
    from paper_2506_22969_gb300 import inputs
    cfg = inputs.CONFIGS[CFG_NAME]
    w = inputs.stencil_weights(cfg["shape"], 2, cfg["radius"], cfg["recipe"], seed=cfg["seed"])
    u = inputs.make_grid(cfg["grid"], cfg["seed"], cfg["dims"])
    return cfg, w, u


def cpu_oracle_sample(target_s: float = 15.0):
    """Times the FP64 oracle on a bounded sample of the workload (the full 4096^2 grid,
    as many of the 100 steps as fit in about target_s seconds) on all host cores."""
    import oracle
    cfg, w, u = _workload()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.run(u, w, cfg["bc"], 1, threads=cores)
    one = time.perf_counter() - t0
    steps = int(max(1, min(cfg["steps"], target_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(u, w, cfg["bc"], steps, threads=cores)
    dt = time.perf_counter() - t0
    pts = steps * u.size
    return {"value": pts / dt / 1e9, "unit": "GStencil/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 C oracle, OpenMP, full {u.shape[0]}x{u.shape[1]} grid, {steps} of {cfg['steps']} "
                      f"steps ({dt:.1f} s)"}


def run_reference(args):
    """--impl reference: the FP64 oracle as it stands, on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    cfg, w, u = _workload()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.run(u, w, cfg["bc"], 1, threads=cores)
    # each step: a bounded sample (4 time steps on the full grid) of the 100-step workload
    sample_steps = 4
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(u, w, cfg["bc"], sample_steps, threads=cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = args.steps * sample_steps * u.size / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GStencil/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "grid": list(cfg["dims"]), "steps_per_run": cfg["steps"],
                       "sample_steps": sample_steps, "l2_flush": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": "GStencil/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample_steps} of {cfg['steps']} steps on the full grid per bench step"},
            "e2e": {"value": val, "unit": "GStencil/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ncu_case(spec: str, t: int):
    """Small profiling case: 3 runs of one fused sweep each (copy-in + 1 sweep kernel)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_22969_gb300 import binding, inputs
    prec, side = spec.split(":")
    side = int(side)
    cfg = inputs.CONFIGS[CFG_NAME]
    w = inputs.stencil_weights(cfg["shape"], 2, cfg["radius"], cfg["recipe"], seed=cfg["seed"])
    u = inputs.make_grid(cfg["grid"], cfg["seed"], (side, side))
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    plan = binding.Plan(w, (side, side), dtype=prec, bc="periodic", fusion_depth=t)
    for _ in range(3):
        plan.run(x, y, t)
    torch.cuda.synchronize()
    assert binding.device_status() == 0


def trace_case():
    """Prints the CTA-0 timeline (microseconds from the first TMA issue) of one sweep for
    each precision and fused depth of the workload.  Needs a library built with
    SPARSTENCIL_DEBUG_TRACE=1."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_22969_gb300 import binding
    cfg, w, u = _workload()
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    for dtype in ("bf16_split", "bf16"):
        for t in (1, 2, 3):
            plan = binding.Plan(w, cfg["dims"], dtype=dtype, bc=cfg["bc"], fusion_depth=t, shape=cfg["shape"])
            plan.run(x, y, t)
            torch.cuda.synchronize()
            binding.trace(True)
            c_ms, s_ms, n = plan.run_profiled(x, y, t)
            tr, ch, pub = binding.trace_read()
            binding.trace(False)
            t0 = int(np.min(tr[tr > 0])) if np.any(tr > 0) else 0
            ntile = int(np.sum(tr[1, :, 0] > 0))
            print(f"== {dtype} t={t}: sweep {s_ms * 1e3:.1f} us, CTA 0 tiles {ntile}")
            names = ["tma", "mma", "gather", "epi"]
            for li in range(ntile):
                row = " ".join(f"{names[r]} {(tr[r, li, 0] - t0) / 1e3:7.2f}-{(tr[r, li, 1] - t0) / 1e3:7.2f}"
                               if tr[r, li, 1] else (f"{names[r]} {(tr[r, li, 0] - t0) / 1e3:7.2f}"
                                                     if tr[r, li, 0] else f"{names[r]}    -   ")
                               for r in range(4))
                print(f"  tile {li}: {row}")
            c0 = ch[0, 0, 0]
            for kc in range(16):
                if ch[0, kc, 0]:
                    g = " | ".join(f"w{s}: start {ch[s, kc, 0] - c0:6d} loaded {ch[s, kc, 1] - c0:6d} "
                                   f"free {ch[s, kc, 2] - c0:6d} pub {ch[s, kc, 3] - c0:6d}" for s in (0, 1))
                    print(f"  tile 1 chunk {kc:2d}: {g} | mma ready {ch[2, kc, 0] - c0:6d} "
                          f"issued {ch[2, kc, 1] - c0:6d} (cycles)")
                    print("      stored  by gather warp: " + " ".join(f"{pub[1, w, kc] - c0:6d}" for w in range(16)))
                    print("      publish by gather warp: " + " ".join(f"{pub[0, w, kc] - c0:6d}" for w in range(16)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sparstencil", choices=["sparstencil", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fusion", type=int, default=0, help="fusion depth t (0: autotune over 1..3)")
    ap.add_argument("--trace", action="store_true",
                    help="print the sweep kernel's CTA-0 timeline for single sweeps of the workload and exit")
    ap.add_argument("--ncu-case", default=None,
                    help="profiling case for ncu: '<precision>:<side>' runs a few single sweeps of Box-2D9P "
                         "on a side x side periodic grid and exits (no JSON line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case:
        return ncu_case(args.ncu_case, args.fusion or 1)
    if args.trace:
        return trace_case()

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_22969_gb300 import binding

    cfg, w, u = _workload()
    H, W = cfg["dims"]
    T = cfg["steps"]
    pts = T * H * W
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed_runs(fn, k, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(k):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts

    # autotune the fusion depth per precision (the paper's layout search rebuilt as a
    # measured search over the fused depth t)
    candidates = [args.fusion] if args.fusion > 0 else [1, 2, 3]
    tune = {}

    def autotune(dtype):
        best = None
        tune[dtype] = {}
        for t in candidates:
            pl = binding.Plan(w, (H, W), dtype=dtype, bc=cfg["bc"], fusion_depth=t, shape=cfg["shape"])
            ms = min(timed_runs(lambda: pl.run(x, y, T), 2, 1))
            tune[dtype][str(t)] = ms
            if best is None or ms < best[1]:
                best = (t, ms, pl)
        return best

    # clocks: sampled every 20 ms from the start of the fusion-depth search (about a second
    # of the same sweeps) to the end of the timed runs, so that short timed regions still
    # get samples
    clocks = ClockSampler(local)
    clocks.start()
    t_best, _, plan = autotune("bf16_split")
    info = plan.info()

    # accuracy of the timed configuration (sampled points against the dependence-cone oracle)
    def sampled_rel_l2(out_t, n=16):
        import oracle
        rng = np.random.default_rng(1)
        pts_ = [tuple(int(v) for v in rng.integers(0, H, 2)) for _ in range(n)]
        ref = np.array([oracle.point(u, w, cfg["bc"], T, p) for p in pts_])
        got = out_t.cpu().numpy().astype(np.float64)
        vals = np.array([got[p] for p in pts_])
        return float(np.sqrt(np.sum((vals - ref) ** 2) / np.sum(ref ** 2)))

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    run_ms = timed_runs(lambda: plan.run(x, y, T), args.steps, args.warmup)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    clock_info["window"] = "fusion-depth search + warm-up + timed runs, 20 ms period"
    if dist is not None:
        dist.barrier()
    tot = sum(run_ms)
    if dist is not None:
        tt = torch.tensor([tot], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        tot = float(tt.item())
    value = world * args.steps * pts / (tot / 1e3) / 1e9
    status = binding.device_status()

    # per-kernel device time of the sweeps (events around each launch)
    sw_ms, nsw, cin_ms = [], 0, []
    for _ in range(3):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        c_ms, s_ms, n = plan.run_profiled(x, y, T)
        cin_ms.append(c_ms)
        sw_ms.append(s_ms)
        nsw = n
    sweep_ms = min(sw_ms) / nsw
    alg_bytes = 8.0 * H * W  # read 4 B + write 4 B per output per sweep
    achieved = alg_bytes / (sweep_ms / 1e3) / 1e9
    peak, peak_kind = _peaks()
    traffic = _profile_traffic()

    rel_split = sampled_rel_l2(y)

    # e2e through the host-buffer entry point (pinned), copies inside the timed region
    hx = torch.from_numpy(u).pin_memory()
    hy = torch.empty((H, W), dtype=torch.float32).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.run_host(hx, hy, T)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_ms.append(dt * 1e3)
    e2e_val = world * len(e2e_ms) * pts / (sum(e2e_ms) / 1e3) / 1e9

    # variants: single-word BF16 and the plain FP32 CUDA-core direct stencil
    t1, _, plan1 = autotune("bf16")
    ms1 = timed_runs(lambda: plan1.run(x, y, T), max(2, args.steps // 2), 1)
    rel_single = sampled_rel_l2(y)
    work = torch.empty_like(x)
    msd = timed_runs(lambda: binding.direct_run(w, x, y, work, T, bc=cfg["bc"]), 2, 1)
    rel_direct = sampled_rel_l2(y)
    variants = {
        "bf16_split_sparse_tc": {"gstencil_s": args.steps * pts / (tot / 1e3) / 1e9, "rel_l2_sampled": rel_split,
                                 "fusion_depth": t_best},
        "bf16_single_sparse_tc": {"gstencil_s": pts / (statistics.median(ms1) / 1e3) / 1e9,
                                  "rel_l2_sampled": rel_single, "fusion_depth": t1},
        "fp32_direct_cuda_core": {"gstencil_s": pts / (statistics.median(msd) / 1e3) / 1e9,
                                  "rel_l2_sampled": rel_direct, "fusion_depth": 1},
    }

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_oracle_sample()
        line = {
            "metric": METRIC, "value": value, "unit": "GStencil/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": cfg["name"], "grid": [H, W], "steps_per_run": T, "boundary": cfg["bc"],
                       "stencil": "box 3x3 (9-point), seeded random positive weights summing to 1",
                       "precision": "bf16_split (weights 3 BF16 pieces, data hi+lo)", "fusion_depth": t_best,
                       "crush": [info.r1, info.r2], "kpad": info.kpad, "mma_terms": info.mma_terms,
                       "l2_flush": "512 MiB write before every timed run", "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_val, "unit": "GStencil/s", "h2d_bytes_per_step": H * W * 4,
                    "d2h_bytes_per_step": H * W * 4},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "sweep2d_kernel", "alg_bytes_per_launch": alg_bytes,
                         "launch_ms": sweep_ms},
            "cpu_baseline": cpu,
            "gpu_launches": args.steps * (1 + nsw),
            "clocks": clock_info,
            "variants": variants,
            "autotune_ms_per_run": tune,
            "rel_l2_sampled": rel_split,
            "device_status": status,
            "planner_ms": info.planner_ms,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
