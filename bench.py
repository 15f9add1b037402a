"""Benchmark of the SparStencil GB300 hot path (one JSON line on rank 0).

Headline workload: Box-2D49P (7 x 7 box, Gaussian-decay weights, sigma 1.5, normalised to
1), 8192 x 8192 FP32 grid uniform on [0, 1), periodic boundary, 200 time steps (the
paper's Table-2 high-order 2D workload at a size one run covers; the largest single-GPU
configuration of the workload set).  One bench "step" is one full run of the 200 time
steps through the C ABI (sparstencil_run: copy into the padded grid + ceil(200/t) sparse
tensor-core sweeps).

  value     GStencil/s = 200 * 8192^2 / run time (device-resident input; the two 256 MiB
            grids are larger than the 129 MB L2, and a 512 MiB buffer is written before
            every timed run), BF16 split operands, autotuned fusion depth
  accuracy  rel-L2 and rel-Linf of the timed run's output at 64 sampled points (random,
            tile corners, grid corners) against the FP64 oracle's dependence cones
  e2e       the same metric through the host-buffer entry points (pinned host buffers, H2D copy of
            the input and D2H copy of the result inside the timed region; consecutive runs
            pipelined over two plans and two streams, and one run at a time as serial_value)
  roofline  the sweep kernel's algorithmic HBM bytes (8 B per output per sweep) over its
            device time (CUDA events around the sweeps of a run), against the measured copy
            bandwidth in MEASURED_PEAKS.json
  serving   the job server on the C5 trace (Poisson arrivals of mixed 2D / 3D jobs): p50,
            p99, throughput, and a sample of jobs compared bit for bit with lone runs
  variants  the single-word BF16 path and the plain FP32 CUDA-core direct stencil on the
            same workload (same sampled points), and Box-2D9P 4096^2 (100 steps)
  cpu_baseline / --impl reference   the FP64 C oracle on the host cores, on a bounded
            sample of the workload (test infrastructure, not the product path)

Other modes: --suite (every workload configuration, sparse against FP32), --batch (64 grids in
one multi-grid launch per sweep index), --serve (the C5 trace alone), --ablation (dense vs
sparse tensor-core MMAs), --correction (the optional FP64 correction step against its
period), --ncu-case / --ncu-kernels (profiling cases).

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

CFG_NAME = "box2d49p_8192"
C2_NAME = "box2d9p_4096"
METRIC = "GStencil/s per GB300, sparse-TCU vs plain FP32 at stated L2 err; p99 latency"
FALLBACK_HBM_GBS = 6800.0


def _peak_bf16_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _profile_traffic(depth: int, profile: str = "sweep2d_box49_8192.md", patch: int = 16):
    """Per-launch DRAM bytes of the sweep kernel from a committed ncu summary, if the summary
    was taken on the current kernel source (sweep2d.cu + kernels.h) at the timed fusion depth
    and 2D patch shape (else None).  A summary may list one figure per patch shape
    ('dram_bytes_per_launch_scaled_patch8:' for 8 x 16 patches)."""
    csrc = os.path.join(ROOT, "paper_2506_22969_gb300", "csrc")
    prof = os.path.join(ROOT, "profiles", profile)
    try:
        h = hashlib.sha256()
        for name in ("sweep2d.cu", "kernels.h"):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(f.read())
        sha = h.hexdigest()[:16]
        with open(prof) as f:
            text = f.read()
        m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", text)
        key = "dram_bytes_per_launch_scaled" + ("" if patch == 16 else f"_patch{patch}")
        m_tr = re.search(key + r":\s*([0-9.eE+]+)", text)
        m_t = re.search(r"fusion_depth:\s*([0-9]+)", text)
        if m_sha and m_tr and m_t and m_sha.group(1) == sha and int(m_t.group(1)) == depth:
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


def _workload(name: str = CFG_NAME):
    from paper_2506_22969_gb300 import inputs
    cfg = inputs.CONFIGS[name]
    w = inputs.stencil_weights(cfg["shape"], cfg["ndim"], cfg["radius"], cfg["recipe"], seed=cfg["seed"])
    u = inputs.make_grid(cfg["grid"], cfg["seed"], cfg["dims"])
    return cfg, w, u


def _oracle_slab(target_s: float, cores: int):
    """A bounded sample of the headline workload for the FP64 oracle: one time step on the
    first `rows` rows of the grid (a full-width slab, periodic), with rows sized from a
    64-row probe so that the step takes about target_s seconds.  Returns (rows, seconds,
    point-steps per second)."""
    import oracle
    cfg, w, u = _workload()
    H = u.shape[0]
    probe = 64
    t0 = time.perf_counter()
    oracle.run(u[:probe], w, cfg["bc"], 1, threads=cores)
    per_row = (time.perf_counter() - t0) / probe
    rows = int(max(probe, min(H, target_s / max(per_row, 1e-9))))
    t0 = time.perf_counter()
    oracle.run(u[:rows], w, cfg["bc"], 1, threads=cores)
    dt = time.perf_counter() - t0
    return rows, dt, rows * u.shape[1] / dt


def cpu_oracle_sample(target_s: float = 15.0):
    """Times the FP64 oracle on a bounded sample of the workload (one time step on a
    full-width slab of the 8192^2 grid, about target_s seconds) on all host cores."""
    cores = os.cpu_count() or 1
    rows, dt, rate = _oracle_slab(target_s, cores)
    cfg = _workload()[0]
    return {"value": rate / 1e9, "unit": "GStencil/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 C oracle, OpenMP, one time step on a {rows} x {cfg['dims'][1]} slab of the "
                      f"{cfg['dims'][0]} x {cfg['dims'][1]} grid ({dt:.1f} s); the workload has {cfg['steps']} steps"}


def replica_throughput(local_ms_total, runs, points_per_run, dist=None, device="cpu"):
    """Whole-job GStencil/s of N independent replicas (no data-path collective): every rank
    timed `runs` runs of `points_per_run` point-steps; the slowest rank's total time counts
    (max over ranks).  Returns (GStencil/s, that time in ms)."""
    import torch
    tot = float(local_ms_total)
    world = 1
    if dist is not None:
        world = dist.get_world_size()
        t = torch.tensor([tot], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot = float(t.item())
    return world * runs * points_per_run / (tot / 1e3) / 1e9, tot


def run_reference(args):
    """--impl reference: the FP64 oracle as it stands, on the host cores (rank 0 only).  Each
    bench step is one time step of the workload's stencil on a full-width slab of the grid
    (rows sized once so that a step takes about 1.5 s)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    cfg, w, u = _workload()
    cores = os.cpu_count() or 1
    rows, _, _ = _oracle_slab(1.5, cores)
    slab = np.ascontiguousarray(u[:rows])
    for _ in range(args.warmup):
        oracle.run(slab, w, cfg["bc"], 1, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(slab, w, cfg["bc"], 1, threads=cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = args.steps * slab.size / tot / 1e9
    sample = f"one time step on a {rows} x {u.shape[1]} slab of the {u.shape[0]} x {u.shape[1]} grid per bench step"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GStencil/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "grid": list(cfg["dims"]), "steps_per_run": cfg["steps"],
                       "sample_rows": rows, "l2_flush": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": "GStencil/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GStencil/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ncu_case(spec: str, t: int, patch: int = 16):
    """Small profiling case: 3 runs of one fused sweep each (copy-in + 1 sweep kernel).
    spec = '<workload>:<precision>[:<side>]', e.g. 'box2d49p_8192:bf16_split' (side: a
    side x side grid instead of the workload's); patch: the 2D patch shape (16: 16 x 8,
    8: 8 x 16)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_22969_gb300 import binding
    parts = spec.split(":")
    name, prec = parts[0], parts[1]
    cfg, w, u = _workload(name)
    if len(parts) > 2:
        side = int(parts[2])
        u = np.ascontiguousarray(u[:side, :side])
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    plan = binding.Plan(w, u.shape, dtype=prec, bc=cfg["bc"], fusion_depth=t, shape=cfg["shape"],
                        layout=(patch, -1) if u.ndim == 2 else None)
    for _ in range(3):
        plan.run(x, y, t)
    torch.cuda.synchronize()
    assert binding.device_status() == 0


def ncu_kernels_case():
    """Profiling case covering every kernel of the library once or twice, each on inputs larger
    than L2 where the kernel streams a grid: the 3D sweep (Heat-3D 384^3, FP16, with its copy-in
    and, periodic, its ghost refresh; fused two steps with a zero Dirichlet boundary, with the
    3D band), the 1D sweep (Heat-1D 2^26, BF16 split, t = 8, two sweeps with the ghost refresh
    between them), the 2D sweep with 8 x 16 patches
    and the Dirichlet band of a fused 2D sweep (Heat-2D 8192^2, t = 3), a batch launch of four
    grids, the FP32 direct kernels (1D, 2D radius 1 and 3, 3D radius-1 star and box), two FP64
    correction steps (Box-2D9P 4096^2) and the FP64 error norms."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_22969_gb300 import binding, inputs
    cases = [("star", 3, 1, "random", (384, 384, 384), "fp16", "periodic", 1, 2, None),
             ("star", 3, 1, "random", (384, 384, 384), "fp16", "dirichlet", 2, 2, None),
             ("star", 1, 1, "heat", (1 << 26,), "bf16_split", "periodic", 8, 16, None),
             ("star", 2, 1, "heat", (8192, 8192), "bf16", "dirichlet", 3, 3, (8, -1))]
    for shape, nd, r, recipe, dims, dt, bc, t, steps, layout in cases:
        w = inputs.stencil_weights(shape, nd, r, recipe, seed=1)
        x = torch.from_numpy(inputs.uniform01(1, dims)).cuda()
        y = torch.empty_like(x)
        plan = binding.Plan(w, dims, dtype=dt, bc=bc, fusion_depth=t, shape=shape, layout=layout)
        plan.run(x, y, steps)
        binding.direct_run(w, x, y, torch.empty_like(x), 1, bc=bc)
        if len(dims) == 2:
            w3 = inputs.stencil_weights("box", 2, 3, "gaussian", seed=1)
            binding.direct_run(w3, x, y, torch.empty_like(x), 1, bc=bc)
        if len(dims) == 3 and bc == "periodic":
            w27 = inputs.stencil_weights("box", 3, 1, "random", seed=1)
            binding.direct_run(w27, x, y, torch.empty_like(x), 1, bc=bc)
        binding.error_norms(y, x)
        del x, y
        torch.cuda.synchronize()
    # the FP64 correction step: two steps of the 9-point box on 4096^2, both in FP64 (the first
    # writes the padded ping-pong grid, the second the caller's grid)
    w = inputs.stencil_weights("box", 2, 1, "random", seed=1)
    x = torch.from_numpy(inputs.uniform01(1, (4096, 4096))).cuda()
    y = torch.empty_like(x)
    plan = binding.Plan(w, (4096, 4096), dtype="bf16", bc="periodic", fusion_depth=1)
    plan.set_fp64_correction(1)
    plan.run(x, y, 2)
    torch.cuda.synchronize()
    del x, y, plan
    # a batch: four 2048^2 grids, one multi-grid launch per sweep index
    w = inputs.stencil_weights("box", 2, 3, "gaussian", seed=1)
    xs = [torch.from_numpy(inputs.uniform01(k, (2048, 2048))).cuda() for k in range(4)]
    ys = [torch.empty_like(x) for x in xs]
    plans = [binding.Plan(w, (2048, 2048), dtype="bf16", bc="periodic", fusion_depth=2) for _ in xs]
    binding.run_batch(plans, xs, ys, [4] * 4)
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
            try:
                plan = binding.Plan(w, cfg["dims"], dtype=dtype, bc=cfg["bc"], fusion_depth=t, shape=cfg["shape"])
            except binding.SparStencilError:
                continue
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
                    g = " | ".join(f"w{s}: start {ch[s, kc, 0] - c0:6d} free {ch[s, kc, 1] - c0:6d} "
                                   f"stored {ch[s, kc, 2] - c0:6d} pub {ch[s, kc, 3] - c0:6d}" for s in (0, 1))
                    print(f"  tile 1 chunk {kc:2d}: {g} | mma ready {ch[2, kc, 0] - c0:6d} "
                          f"issued {ch[2, kc, 1] - c0:6d} (cycles)")
                    print("      stored  by gather warp: " + " ".join(f"{pub[1, w, kc] - c0:6d}" for w in range(16)))
                    print("      publish by gather warp: " + " ".join(f"{pub[0, w, kc] - c0:6d}" for w in range(16)))


def _sample_points(dims, n=64, tile=128, seed=1):
    """n output points of a 2D grid: the four grid corners, the four cells around two tile
    corners, and seeded random points."""
    H, W = dims
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1)]
    for ty, tx in ((tile, tile), (H // 2 // tile * tile, W // 2 // tile * tile)):
        pts += [(ty - 1, tx - 1), (ty - 1, tx), (ty, tx - 1), (ty, tx)]
    rng = np.random.default_rng(seed)
    while len(pts) < n:
        pts.append((int(rng.integers(0, H)), int(rng.integers(0, W))))
    return pts


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sparstencil", choices=["sparstencil", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="leave out the C5 serving trace")
    ap.add_argument("--no-variants", action="store_true", help="leave out the variant workloads")
    ap.add_argument("--fusion", type=int, default=0, help="fusion depth t (0: autotune)")
    ap.add_argument("--patch", type=int, default=16, help="--ncu-case: 2D patch shape (16: 16 x 8, 8: 8 x 16)")
    ap.add_argument("--trace", action="store_true",
                    help="print the sweep kernel's CTA-0 timeline for single sweeps of the workload and exit")
    ap.add_argument("--ncu-case", default=None,
                    help="profiling case for ncu: '<workload>:<precision>[:<side>]' runs a few single sweeps "
                         "(depth --fusion) and exits (no JSON line)")
    ap.add_argument("--suite", action="store_true",
                    help="configs C1, C2, C3, C4a/b and Heat-1D / 1D5P (one JSON line each) and exit")
    ap.add_argument("--batch", action="store_true", help="config C4c (64 grids in one CUDA graph) and exit")
    ap.add_argument("--serve", action="store_true", help="config C5 (Poisson-arrival job server) and exit")
    ap.add_argument("--ncu-kernels", action="store_true",
                    help="profiling case: one launch or two of every kernel of the library, then exit")
    ap.add_argument("--correction", action="store_true",
                    help="run time and accuracy of the optional FP64 correction step against its period")
    ap.add_argument("--ablation", action="store_true",
                    help="dense versus sparse tensor-core MMAs on Box-2D49P at several sizes and exit")
    args = ap.parse_args()
    if args.suite:
        return suite_mode()
    if args.batch:
        return batch_mode()
    if args.serve:
        return serve_mode()
    if args.correction:
        return correction_mode()
    if args.ablation:
        return ablation_mode()
    if args.ncu_kernels:
        return ncu_kernels_case()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case:
        return ncu_case(args.ncu_case, args.fusion or 1, args.patch)
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
    import oracle
    from paper_2506_22969_gb300 import binding

    cfg, w, u = _workload()
    H, W = cfg["dims"]
    T = cfg["steps"]
    pts = T * H * W
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # accuracy: the timed run's output at sampled points against the FP64 oracle (computed on
    # the host cores after the GPU measurements, so that it does not compete with them)
    sample = _sample_points((H, W))

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

    # the fusion depth per precision, measured (the paper's layout search rebuilt as a
    # search over the fused depth t; depths whose tables do not fit TMEM or shared memory
    # are rejected by the planner and skipped)
    candidates = [args.fusion] if args.fusion > 0 else [1, 2, 3, 4, 5, 6]
    tune = {}

    # the Sec. 3.3 cost model beside the measured search: sparse tensor rate = 2 x the measured
    # dense BF16 rate, HBM = the measured copy bandwidth, shared memory = 128 B per clock per SM
    model_rates = (2.0 * _peak_bf16_tflops() * 1e12, _peaks()[0] * 1e9, 128.0 * 152 * 1.9e9)
    model = {}

    def autotune(dtype, wl=(cfg, w, x, y)):
        """The layout search over fusion depth x 2D patch shape (16 x 8, 8 x 16), timed here
        (the library's fusion_depth-0 search does the same on a plan's first run)."""
        c, ww, xx, yy = wl
        best = None
        tune.setdefault(c["name"], {})[dtype] = {}
        model.setdefault(c["name"], {})[dtype] = {}
        for t in candidates:
            for r1 in (16, 8):
                try:
                    pl = binding.Plan(ww, c["dims"], dtype=dtype, bc=c["bc"], fusion_depth=t, shape=c["shape"],
                                      layout=(r1, -1))
                except binding.SparStencilError:
                    continue
                ms = min(timed_runs(lambda: pl.run(xx, yy, c["steps"]), 2, 1))
                tune[c["name"]][dtype][f"t={t} patch={r1}x{128 // r1}"] = ms
                if r1 == 16:
                    model[c["name"]][dtype][str(t)] = pl.cost_model(t, *model_rates) * c["steps"] * 1e3
                if best is None or ms < best[1]:
                    best = (t, ms, pl)
        return best

    # clocks: sampled every 20 ms from the start of the fusion-depth search to the end of
    # the timed runs
    clocks = ClockSampler(local)
    clocks.start()
    t_best, _, plan = autotune("bf16_split")
    info = plan.info()

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    run_ms = timed_runs(lambda: plan.run(x, y, T), args.steps, args.warmup)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    clock_info["window"] = "fusion-depth search + warm-up + timed runs, 20 ms period"
    if dist is not None:
        dist.barrier()
    value, tot = replica_throughput(sum(run_ms), args.steps, pts, dist, "cuda")
    status = binding.device_status()
    got = y.cpu().numpy()

    # per-launch device time of the sweeps (events around the sweeps of a run)
    sw_ms, nsw = [], 0
    for _ in range(3):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        c_ms, s_ms, n = plan.run_profiled(x, y, T)
        sw_ms.append(s_ms)
        nsw = n
    sweep_ms = min(sw_ms) / nsw
    alg_bytes = 8.0 * H * W  # read 4 B + write 4 B per output per sweep
    achieved = alg_bytes / (sweep_ms / 1e3) / 1e9
    peak, peak_kind = _peaks()
    traffic = _profile_traffic(t_best, patch=info.r1)

    # e2e through the host-buffer entry points from pinned host memory, every run's host->
    # device copy of its input and device->host copy of its result inside the timed region.
    # Consecutive runs are independent jobs: two plans alternate on two streams
    # (sparstencil_run_host_async), so run i+1's input copy and run i-1's result copy (copy
    # engines) overlap run i's sweeps.  The serial figure (sparstencil_run_host, one run at a
    # time, L2 flushed before each) is reported beside it.
    hx = [torch.from_numpy(u).pin_memory() for _ in range(2)]
    hy = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
    plan2 = binding.Plan(w, cfg["dims"], dtype="bf16_split", bc=cfg["bc"], fusion_depth=t_best, shape=cfg["shape"],
                         layout=(info.r1, -1))
    plans2, streams2 = [plan, plan2], [torch.cuda.Stream(), torch.cuda.Stream()]

    def e2e_runs(n):
        for i in range(n):
            plans2[i % 2].run_host_async(hx[i % 2], hy[i % 2], T, stream=streams2[i % 2])

    e2e_runs(args.warmup)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_runs(args.steps)
    torch.cuda.synchronize()
    e2e_total_ms = (time.perf_counter() - t0) * 1e3
    if dist is not None:
        dist.barrier()
    e2e_val, _ = replica_throughput(e2e_total_ms, args.steps, pts, dist, "cuda")
    e2e_same = bool(torch.equal(hy[0], hy[1]))  # both plans computed the same run
    serial_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.run_host(hx[0], hy[0], T)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            serial_ms.append(dt * 1e3)
    e2e_serial, _ = replica_throughput(sum(serial_ms), len(serial_ms), pts, dist, "cuda")
    del hx, hy, plan2, plans2

    def acc(out_np, ref):
        vals = np.array([float(out_np[p]) for p in sample])
        d = vals - ref
        return {"rel_l2": float(np.sqrt(np.sum(d * d) / np.sum(ref * ref))),
                "rel_linf": float(np.max(np.abs(d)) / np.max(np.abs(ref))), "points": len(sample)}

    variants = {}
    if not args.no_variants and rank == 0:
        # single-word BF16 and the plain FP32 CUDA-core direct stencil on the same workload
        t1, _, plan1 = autotune("bf16")
        ms1 = timed_runs(lambda: plan1.run(x, y, T), max(2, args.steps // 2), 1)
        got_single = y.cpu().numpy()
        work = torch.empty_like(x)
        msd = timed_runs(lambda: binding.direct_run(w, x, y, work, T, bc=cfg["bc"]), 2, 1)
        got_direct = y.cpu().numpy()
        del work
        # Box-2D9P 4096^2, 100 steps (the 9-point workload), BF16 split, autotuned depth
        del x, y
        torch.cuda.empty_cache()
        c2, w2, u2 = _workload(C2_NAME)
        x2 = torch.from_numpy(u2).cuda()
        y2 = torch.empty_like(x2)
        t2, _, plan2 = autotune("bf16_split", (c2, w2, x2, y2))
        ms2 = timed_runs(lambda: plan2.run(x2, y2, c2["steps"]), args.steps, 1)
        g2 = y2.cpu().numpy()
        del x2, y2
        torch.cuda.empty_cache()

    serving = None
    if not args.no_serving and rank == 0:
        serving = serve_trace()

    accuracy = None
    if rank == 0:
        ref = oracle.points(u, w, cfg["bc"], T, sample)
        accuracy = acc(got, ref)
    if not args.no_variants and rank == 0:
        variants["bf16_split_sparse_tc"] = {"gstencil_s": value / world, "fusion_depth": t_best, **accuracy}
        variants["bf16_single_sparse_tc"] = {"gstencil_s": pts / (statistics.median(ms1) / 1e3) / 1e9,
                                             "fusion_depth": t1, **acc(got_single, ref)}
        variants["fp32_direct_cuda_core"] = {"gstencil_s": pts / (statistics.median(msd) / 1e3) / 1e9,
                                             "fusion_depth": 1, **acc(got_direct, ref)}
        sample2 = _sample_points(c2["dims"], n=16)
        ref2 = oracle.points(u2, w2, c2["bc"], c2["steps"], sample2)
        v2 = np.array([float(g2[p]) for p in sample2])
        pts2 = c2["steps"] * c2["dims"][0] * c2["dims"][1]
        variants["box2d9p_4096_bf16_split_sparse_tc"] = {
            "workload": c2["name"], "gstencil_s": pts2 / (statistics.median(ms2) / 1e3) / 1e9, "fusion_depth": t2,
            "rel_l2": float(np.sqrt(np.sum((v2 - ref2) ** 2) / np.sum(ref2 ** 2))),
            "rel_linf": float(np.max(np.abs(v2 - ref2)) / np.max(np.abs(ref2))), "points": len(sample2)}

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_oracle_sample()
        line = {
            "metric": METRIC, "value": value, "unit": "GStencil/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": cfg["name"], "grid": [H, W], "steps_per_run": T, "boundary": cfg["bc"],
                       "stencil": "box 7x7 (49-point), Gaussian-decay weights (sigma 1.5) normalised to 1",
                       "precision": f"bf16_split ({info.mma_terms - 1} BF16 weight pieces, data hi+lo)",
                       "fusion_depth": t_best, "crush": [info.r1, info.r2], "pairing": info.pairing,
                       "kpad": info.kpad,
                       "mma_terms": info.mma_terms,
                       "l2_flush": "grids (2 x 256 MiB) larger than L2, plus a 512 MiB write before every timed run",
                       "parallelism": f"replicas x{world}"},
            "accuracy": {**accuracy, "tolerance_rel_l2": 1e-5, "tolerance_rel_linf": 1e-4,
                         "reference": "FP64 oracle, dependence cones of the sampled points"},
            "e2e": {"value": e2e_val, "unit": "GStencil/s", "h2d_bytes_per_step": H * W * 4,
                    "d2h_bytes_per_step": H * W * 4,
                    "mode": "independent runs from pinned host buffers, two plans on two streams "
                            "(sparstencil_run_host_async): copies of neighbouring runs overlap a run's sweeps",
                    "serial_value": e2e_serial, "pipelined_results_equal": e2e_same},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "sweep2d_kernel", "alg_bytes_per_launch": alg_bytes,
                         "launch_ms": sweep_ms},
            "cpu_baseline": cpu,
            "gpu_launches": args.steps * (1 + nsw),
            "clocks": clock_info,
            "serving": serving,
            "variants": variants,
            "autotune_ms_per_run": tune,
            "cost_model_ms_per_run": model,
            "device_status": status,
            "planner_ms": info.planner_ms,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------------------
# Extra workloads (not the headline JSON line): --suite, --batch, --serve print one JSON
# line per workload on stdout.
# ---------------------------------------------------------------------------------------
def _time_runs(fn, k=3, warm=1, flush=None):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(k):
        if flush is not None:
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return min(ts), statistics.median(ts)


def _rel_l2_gpu(binding, x, ref):
    l2, linf, _ = binding.error_norms(x, ref)
    return l2, linf


def _rel(vals, ref):
    """(rel-L2, rel-Linf) of sampled values against their reference values."""
    d = np.asarray(vals, dtype=np.float64) - np.asarray(ref, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    return float(np.sqrt(np.sum(d * d) / np.sum(r * r))), float(np.max(np.abs(d)) / np.max(np.abs(r)))


def suite_mode():
    """Configs C1, C3, C4a/b and the 1D workloads: GStencil/s of the sparse path (single and split, fusion depth
    autotuned) and of the plain FP32 direct kernel, with rel-L2 against the FP64 oracle (C1:
    full grid; C3: sampled points, plus the whole grid against the FP32 direct result) or
    against the FP32 direct result (C4)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2506_22969_gb300 import binding, inputs
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for name in ("heat2d_512", "box2d9p_4096", "star2d13p_8192", "box2d49p_8192", "box3d27p_256", "heat3d_512", "heat1d",
                 "1d5p"):
        cfg = inputs.CONFIGS[name]
        dims, T, bc = cfg["dims"], cfg["steps"], cfg["bc"]
        w = inputs.stencil_weights(cfg["shape"], cfg["ndim"], cfg["radius"], cfg["recipe"], seed=cfg["seed"])
        u = inputs.make_grid(cfg["grid"], cfg["seed"], dims)
        x = torch.from_numpy(u).cuda()
        y = torch.empty_like(x)
        work = torch.empty_like(x)
        pts = T * int(np.prod(dims))
        line = {"workload": cfg["name"], "points": list(dims), "steps": T}
        ref_gpu = torch.empty_like(x)
        ms_d, _ = _time_runs(lambda: binding.direct_run(w, x, ref_gpu, work, T, bc=bc), 2, 1, flush)
        line["fp32_direct_gstencil_s"] = pts / ms_d / 1e6
        sample, sample_ref = None, None
        if cfg["ndim"] != 2:
            # 1D and 3D: sampled points against the FP64 oracle's dependence cones, and the
            # whole grid against the FP32 direct kernel
            rng = np.random.default_rng(0)
            sample = [tuple(int(rng.integers(0, d)) for d in dims) for _ in range(6)]
            u64 = u.astype(np.float64)
            sample_ref = np.array([oracle.point(u64, w, bc, T, p) for p in sample])
            del u64

            def sampled_l2(t):
                got = t.cpu().numpy()
                vals = np.array([float(got[p]) for p in sample])
                return float(np.sqrt(np.sum((vals - sample_ref) ** 2) / np.sum(sample_ref ** 2)))

            line["fp32_direct_rel_l2_sampled_vs_oracle"] = sampled_l2(ref_gpu)
        if name == "heat2d_512":
            dtypes = ("fp16",)
        elif cfg["ndim"] == 3:
            dtypes = ("fp16", "bf16", "fp16_split", "bf16_split")
        elif cfg["ndim"] == 1:
            dtypes = ("fp16", "bf16", "fp16_split", "bf16_split")
        else:
            dtypes = ("bf16", "bf16_split")
        full_ref = oracle.run(u, w, bc, T) if name == "heat2d_512" else None
        for dt in dtypes:
            try:
                plan = binding.Plan(w, dims, dtype=dt, bc=bc, fusion_depth=0, shape=cfg["shape"])
            except binding.SparStencilError as e:
                line[f"{dt}_sparse"] = f"unsupported: {e}"
                continue
            plan.run(x, y, T)  # fixes the autotuned depth (and 2D patch shape)
            ms, med = _time_runs(lambda: plan.run(x, y, T), 3, 1, flush)
            line[f"{dt}_sparse_gstencil_s"] = pts / ms / 1e6
            line[f"{dt}_fusion_depth"] = plan.info().fusion_depth
            if cfg["ndim"] == 2:
                line[f"{dt}_patch"] = f"{plan.info().r1}x{plan.info().r2}"
            if cfg["ndim"] == 3 and plan.info().fusion_depth > 1:
                # the unfused sweep beside the fused one the search chose
                p1 = binding.Plan(w, dims, dtype=dt, bc=bc, fusion_depth=1, shape=cfg["shape"])
                p1.run(x, y, T)
                ms1, _ = _time_runs(lambda: p1.run(x, y, T), 3, 1, flush)
                line[f"{dt}_t1_sparse_gstencil_s"] = pts / ms1 / 1e6
                plan.run(x, y, T)
            if dt.endswith("split"):
                line[f"{dt}_low_accumulator"] = plan.info().low_accumulator
            if sample is not None:
                line[f"{dt}_rel_l2_sampled_vs_oracle"] = sampled_l2(y)
            if name == "heat2d_512":
                # latency-bound: also the run replayed from a CUDA graph (no host work per run)
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    plan.run(x, y, T)
                gms, _ = _time_runs(graph.replay, 5, 2, flush)
                line[f"{dt}_graph_us_per_run"] = gms * 1e3
                line[f"{dt}_graph_gstencil_s"] = pts / gms / 1e6
                line[f"{dt}_us_per_run"] = ms * 1e3
                graph.replay()
            if full_ref is not None:
                l2, linf = oracle.rel_errors(y.cpu().numpy().astype(np.float64), full_ref)
                line[f"{dt}_rel_l2_vs_oracle"] = l2
                line[f"{dt}_rel_linf_vs_oracle"] = linf
            else:
                l2, linf = _rel_l2_gpu(binding, y, ref_gpu)
                line[f"{dt}_rel_l2_vs_fp32_direct"] = l2
                line[f"{dt}_rel_linf_vs_fp32_direct"] = linf
        print(json.dumps(line), flush=True)
        del x, y, work, ref_gpu
        torch.cuda.empty_cache()


def ablation_mode():
    """Dense versus sparse tensor-core MMAs on the same morphed A' (the paper's breakdown of
    CUDA cores -> dense tensor cores -> sparse tensor cores -> optimised): Box-2D49P, Gaussian
    weights, periodic, 200 steps, BF16 single words, at several grid sizes.  One JSON line per
    size: GStencil/s of the FP32 direct kernel, the dense and the sparse sweep at t = 1, and the
    sparse sweep at the autotuned depth, with rel-L2 against the FP32 direct result."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_22969_gb300 import binding, inputs
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    w = inputs.stencil_weights("box", 2, 3, "gaussian", seed=4)
    T = 200
    for side in (1024, 2048, 4096, 8192):
        dims = (side, side)
        u = inputs.uniform01(4, dims)
        x = torch.from_numpy(u).cuda()
        y = torch.empty_like(x)
        ref = torch.empty_like(x)
        work = torch.empty_like(x)
        pts = T * side * side
        line = {"workload": f"Box-2D 49-point {side}^2, periodic, {T} steps, BF16", "points": [side, side], "steps": T}
        ms, _ = _time_runs(lambda: binding.direct_run(w, x, ref, work, T, bc="periodic"), 2, 1, flush)
        line["fp32_direct_gstencil_s"] = pts / ms / 1e6
        for name, kw in (("dense_tc_t1", dict(fusion_depth=1, dense=True)), ("sparse_tc_t1", dict(fusion_depth=1)),
                         ("sparse_tc_autotuned", dict(fusion_depth=0))):
            try:
                plan = binding.Plan(w, dims, dtype="bf16", bc="periodic", shape="box", **kw)
            except binding.SparStencilError as e:
                line[name] = f"unsupported: {e}"
                continue
            plan.run(x, y, T)
            ms, _ = _time_runs(lambda: plan.run(x, y, T), 3, 1, flush)
            line[f"{name}_gstencil_s"] = pts / ms / 1e6
            line[f"{name}_fusion_depth"] = plan.info().fusion_depth
            line[f"{name}_rel_l2_vs_fp32_direct"] = _rel_l2_gpu(binding, y, ref)[0]
        print(json.dumps(line), flush=True)
        del x, y, ref, work
        torch.cuda.empty_cache()
    # the other dimensionalities at one size each: Box-2D9P 4096^2 (100 steps), Heat-3D 512^3
    # (50 steps, FP16), Heat-1D 10,240,000 (1000 steps)
    for name, dtype, T2 in (("box2d9p_4096", "bf16", 100), ("heat3d_512", "fp16", 50), ("heat1d", "bf16", 1000)):
        cfg = inputs.CONFIGS[name]
        dims = cfg["dims"]
        nd = len(dims)
        w2 = inputs.stencil_weights(cfg["shape"], nd, cfg["radius"], cfg["recipe"], seed=cfg["seed"])
        x = torch.from_numpy(inputs.make_grid(cfg["grid"], cfg["seed"], dims)).cuda()
        y, ref, work = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
        pts = T2 * int(np.prod(dims))
        line = {"workload": f"{cfg['name'].split(',')[0]}, {cfg['bc']}, {T2} steps, {dtype}", "points": list(dims),
                "steps": T2}
        ms, _ = _time_runs(lambda: binding.direct_run(w2, x, ref, work, T2, bc=cfg["bc"]), 2, 1, flush)
        line["fp32_direct_gstencil_s"] = pts / ms / 1e6
        for tag, kw in (("dense_tc_t1", dict(fusion_depth=1, dense=True)), ("sparse_tc_t1", dict(fusion_depth=1)),
                        ("sparse_tc_autotuned", dict(fusion_depth=0))):
            try:
                plan = binding.Plan(w2, dims, dtype=dtype, bc=cfg["bc"], shape=cfg["shape"], **kw)
            except binding.SparStencilError as e:
                line[tag] = f"unsupported: {e}"
                continue
            plan.run(x, y, T2)
            ms, _ = _time_runs(lambda: plan.run(x, y, T2), 3, 1, flush)
            line[f"{tag}_gstencil_s"] = pts / ms / 1e6
            line[f"{tag}_fusion_depth"] = plan.info().fusion_depth
            line[f"{tag}_rel_l2_vs_fp32_direct"] = _rel_l2_gpu(binding, y, ref)[0]
        print(json.dumps(line), flush=True)
        del x, y, ref, work
        torch.cuda.empty_cache()


def _c4c_jobs(n=64, seed=4):
    """64 grids, side log-uniform in [256, 2048] rounded to 128, alternating Star-2D13P and
    Box-2D49P (Gaussian weights), 200 steps, periodic."""
    from paper_2506_22969_gb300 import inputs
    z = inputs.uniform01(seed, (n,)).astype(np.float64)
    sides = np.exp(np.log(256) + z * (np.log(2048) - np.log(256)))
    sides = (np.round(sides / 128) * 128).astype(int)
    jobs = []
    for i in range(n):
        shape = "star" if i % 2 == 0 else "box"
        w = inputs.stencil_weights(shape, 2, 3, "gaussian", seed=seed)
        jobs.append((shape, w, (int(sides[i]), int(sides[i])), 200))
    return jobs


def correction_mode():
    """The optional FP64 correction step (every k-th time step in FP64 on the CUDA cores): run
    time and accuracy against k.  Box-2D9P 4096^2, 100 steps, BF16 single and split words at
    t = 6, rel-L2 / rel-Linf against the FP32 direct result; Heat-1D 10,240,000, 1000 steps,
    BF16 single words at t = 8, against 8 points of the FP64 oracle (the 1D FP32 direct kernel
    itself drifts by about 1e-6 there).  One JSON line per workload and precision."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2506_22969_gb300 import binding, inputs
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    cases = (("box2d9p_4096", "bf16", 6, 100), ("box2d9p_4096", "bf16_split", 6, 100), ("heat1d", "bf16", 8, 1000))
    for name, dtype, t, T in cases:
        cfg = inputs.CONFIGS[name]
        dims = cfg["dims"]
        nd = len(dims)
        w = inputs.stencil_weights(cfg["shape"], nd, cfg["radius"], cfg["recipe"], seed=cfg["seed"])
        u = inputs.make_grid(cfg["grid"], cfg["seed"], dims)
        x = torch.from_numpy(u).cuda()
        y = torch.empty_like(x)
        pts = T * int(np.prod(dims))
        line = {"workload": f"{cfg['name'].split(',')[0]}, {cfg['bc']}, {T} steps", "dtype": dtype, "fusion_depth": t}
        if nd == 1:
            rng = np.random.default_rng(3)
            sample = [(int(v),) for v in rng.integers(0, dims[0], 8)]
            ref = oracle.points(u, w, cfg["bc"], T, sample)
        else:
            ref_t, work = torch.empty_like(x), torch.empty_like(x)
            binding.direct_run(w, x, ref_t, work, T, bc=cfg["bc"])
        for k in (0, 50, 10, 2, 1):
            plan = binding.Plan(w, dims, dtype=dtype, bc=cfg["bc"], fusion_depth=t, shape=cfg["shape"])
            plan.set_fp64_correction(k)
            plan.run(x, y, T)
            ms, _ = _time_runs(lambda: plan.run(x, y, T), 2, 1, flush)
            if nd == 1:
                got = y.cpu().numpy()
                l2, linf = _rel(np.array([float(got[s]) for s in sample]), ref)
            else:
                l2, linf = _rel_l2_gpu(binding, y, ref_t)
            line[f"k{k}"] = {"gstencil_s": pts / ms / 1e6, "ms_per_run": ms, "rel_l2": l2, "rel_linf": linf}
            del plan
        print(json.dumps(line), flush=True)
        del x, y
        torch.cuda.empty_cache()


def batch_mode():
    """Config C4c: 64 mixed grids in one CUDA graph (sparstencil_run_batch) against the same
    jobs run one after another; per-grid rel-L2 against the FP32 direct kernel."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_22969_gb300 import binding, inputs
    jobs = _c4c_jobs()
    plans, xs, ys = [], [], []
    for k, (shape, w, dims, T) in enumerate(jobs):
        u = inputs.uniform01(100 + k, dims)
        plans.append(binding.Plan(w, dims, dtype="bf16", bc="periodic", fusion_depth=0, shape=shape))
        xs.append(torch.from_numpy(u).cuda())
        ys.append(torch.empty(dims, device="cuda"))
    steps = [j[3] for j in jobs]
    pts = sum(T * d[0] * d[1] for (_, _, d, T) in jobs)
    # first call: plan preparation (fusion-depth search), capture, instantiation and launch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    binding.run_batch(plans, xs, ys, steps)
    torch.cuda.synchronize()
    first_ms = (time.perf_counter() - t0) * 1e3
    # later calls replay the kept graph
    ms_b, med_b = _time_runs(lambda: binding.run_batch(plans, xs, ys, steps), 5, 1)
    ms_s, _ = _time_runs(lambda: [p.run(x, y, T) for p, x, y, T in zip(plans, xs, ys, steps)], 3, 1)
    worst = 0.0
    for (shape, w, dims, T), x, y in zip(jobs, xs, ys):
        ref = torch.empty_like(x)
        work = torch.empty_like(x)
        binding.direct_run(w, x, ref, work, T, bc="periodic")
        worst = max(worst, _rel_l2_gpu(binding, y, ref)[0])
    # the four smallest grids against the FP64 oracle, whole grid
    import oracle
    oracle_checks = []
    for k in sorted(range(len(jobs)), key=lambda i: jobs[i][2][0])[:4]:
        shape, w, dims, T = jobs[k]
        l2, linf = oracle.rel_errors(ys[k].cpu().numpy(), oracle.run(xs[k].cpu().numpy(), w, "periodic", T))
        oracle_checks.append({"grid": list(dims), "stencil": shape, "rel_l2": l2, "rel_linf": linf})
    print(json.dumps({"workload": "C4c: 64 grids 256^2-2048^2, Star-2D13P / Box-2D49P alternating, 200 steps, BF16",
                      "oracle_whole_grid": oracle_checks,
                      "grids": len(jobs), "point_steps": pts, "first_call_ms": first_ms,
                      "graph_replay_ms": ms_b, "graph_replay_gstencil_s": pts / ms_b / 1e6,
                      "sequential_ms": ms_s, "sequential_gstencil_s": pts / ms_s / 1e6,
                      "worst_rel_l2_vs_fp32_direct": worst,
                      "depths": sorted({p.info().fusion_depth for p in plans})}), flush=True)


def _c5_jobs(n=512, seed=5):
    """Config C5: stencil uniform over 5/9/13/49-point 2D and 7/27-point 3D; 2D side
    log-uniform 128-4096, 3D side 64-256 (multiples of 8); steps uniform in [10, 500];
    tolerance class 2e-3 (single-word operands) or 1e-5 (split operands) with probability 1/2:
    BF16 for 2D jobs, FP16 for 3D jobs."""
    from paper_2506_22969_gb300 import inputs
    r = inputs.uniform01(seed, (n, 4)).astype(np.float64)
    kinds = [("star", 2, 1, "heat"), ("box", 2, 1, "random"), ("star", 2, 3, "gaussian"), ("box", 2, 3, "gaussian"),
             ("star", 3, 1, "random"), ("box", 3, 1, "random")]
    jobs = []
    for i in range(n):
        shape, nd, rad, recipe = kinds[min(5, int(r[i, 0] * 6))]
        lo, hi = (128, 4096) if nd == 2 else (64, 256)
        side = int(np.exp(np.log(lo) + r[i, 1] * (np.log(hi) - np.log(lo))) // 8 * 8)
        dims = (side,) * nd
        T = 10 + int(r[i, 2] * 491)
        split = r[i, 3] < 0.5
        if nd == 3:
            # 3D: FP16 operands (BF16 single words miss 2e-3 on 3D grids; FP16 split carries the
            # low-order accumulator), one step per sweep
            dtype, fusion = ("fp16_split" if split else "fp16"), 1
        else:
            dtype = "bf16_split" if split else "bf16"
            fusion = 1 if (rad == 3 and split) else (3 if rad == 1 else 1)
        w = inputs.stencil_weights(shape, nd, rad, recipe, seed=seed + i % 3)
        jobs.append(dict(shape=shape, w=w, dims=dims, T=T, dtype=dtype, fusion=fusion))
    return jobs


def serve_mode():
    """--serve: the C5 trace (512 jobs), one JSON line."""
    import __graft_entry__
    __graft_entry__.build()
    print(json.dumps(serve_trace()), flush=True)


def serve_trace(n_jobs=512, budget=120 << 30, slots=8):
    """Config C5: Poisson arrivals at 0.8 of the measured capacity into the library's job
    server (HBM budget 120 GB, 8 slots); p50/p99 of completion minus arrival, throughput, and a
    sample of jobs re-run alone (bit-exact equality with their result in the mix).  Returns a
    dict."""
    import torch
    from paper_2506_22969_gb300 import binding, inputs
    t_start = time.perf_counter()
    jobs = _c5_jobs(n_jobs)
    base2 = inputs.uniform01(5, (4096, 4096))
    base3 = inputs.uniform01(6, (256, 256, 256))
    npool = 3 * slots
    pool_in = [torch.empty(4096 * 4096, dtype=torch.float32).pin_memory() for _ in range(npool)]
    pool_out = [torch.empty(4096 * 4096, dtype=torch.float32).pin_memory() for _ in range(npool)]

    def grid_of(j):
        d = j["dims"]
        return base2[:d[0], :d[1]] if len(d) == 2 else base3[:d[0], :d[1], :d[2]]

    keep = set(range(0, n_jobs, 37))  # jobs whose results are re-checked alone

    def run_trace(srv, idx, arrivals):
        free = list(range(npool))
        inflight = {}
        t0 = srv.clock()
        results = {}
        for k, i in enumerate(idx):
            j = jobs[i]
            while not free:  # wait for a buffer pair (backpressure only when far over capacity)
                jid, (bi, ii) = next(iter(inflight.items()))
                srv.wait(jid)
                if ii in keep:
                    results[ii] = pool_out[bi][:int(np.prod(jobs[ii]["dims"]))].clone()
                free.append(bi)
                del inflight[jid]
            bi = free.pop()
            size = int(np.prod(j["dims"]))
            hin = pool_in[bi][:size].view(*j["dims"])
            hin.copy_(torch.from_numpy(np.ascontiguousarray(grid_of(j))))
            hout = pool_out[bi][:size].view(*j["dims"])
            while srv.clock() < t0 + arrivals[k]:
                time.sleep(0.0002)
            jid = srv.submit(j["w"], hin, hout, j["T"], dtype=j["dtype"], bc="periodic", fusion_depth=j["fusion"],
                             shape=j["shape"], arrival_s=t0 + arrivals[k])
            inflight[jid] = (bi, i)
        for jid, (bi, i) in list(inflight.items()):
            srv.wait(jid)
            if i in keep:
                results[i] = pool_out[bi][:int(np.prod(jobs[i]["dims"]))].clone()
        return results

    # capacity: the first 48 jobs submitted at once
    srv = binding.Server(budget, slots)
    cal = list(range(48))
    t_a = time.perf_counter()
    run_trace(srv, cal, [0.0] * len(cal))
    cal_s = time.perf_counter() - t_a
    work_cal = sum(jobs[i]["T"] * int(np.prod(jobs[i]["dims"])) for i in cal)
    srv.close()
    cap = work_cal / cal_s  # point-steps per second
    mean_work = np.mean([j["T"] * int(np.prod(j["dims"])) for j in jobs])
    lam = 0.8 * cap / mean_work
    rng = np.random.default_rng(5)
    arrivals = np.cumsum(rng.exponential(1.0 / lam, n_jobs))
    srv = binding.Server(budget, slots)
    results = run_trace(srv, list(range(n_jobs)), list(arrivals))
    st = srv.stats()
    srv.close()
    # alone vs mix on a sample of 2D and 3D jobs
    same = True
    checked = 0
    for i in sorted(keep):
        j = jobs[i]
        x = torch.from_numpy(np.ascontiguousarray(grid_of(j))).cuda()
        y = torch.empty_like(x)
        p = binding.Plan(j["w"], j["dims"], dtype=j["dtype"], bc="periodic", fusion_depth=j["fusion"],
                         shape=j["shape"])
        p.run(x, y, j["T"])
        same &= bool(torch.equal(y.cpu().reshape(-1), results[i].reshape(-1)))
        checked += 1
    return {"workload": f"C5: {n_jobs} Poisson-arrival jobs, 2D 5/9/13/49-pt 128-4096^2, "
                        "3D 7/27-pt 64-256^3, 10-500 steps, periodic",
            "budget_bytes": budget, "slots": slots, "arrival_rate_per_s": lam,
            "capacity_gstencil_s": cap / 1e9, "completed": st.completed, "failed": st.failed,
            "p50_s": st.p50_s, "p99_s": st.p99_s, "mean_s": st.mean_s, "max_s": st.max_s,
            "throughput_gstencil_s": st.gstencil_per_s, "peak_device_bytes": st.peak_bytes,
            "pool_high_bytes": st.pool_high_bytes, "pool_resident_bytes": st.pool_reserved_bytes,
            "alone_equals_mix": same, "alone_checked": checked,
            "wall_s": time.perf_counter() - t_start}


if __name__ == "__main__":
    main()
