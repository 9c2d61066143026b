"""Benchmark: chi^2 + gradient evaluations of non-gridding MEM on one GB300.

One step = one mem_objective_grad call over the whole data set: attenuation
and operand preparation, forward operator with fused residual / chi^2,
adjoint (chi^2 gradient), entropy, gradient assembly and projection.  The
metric is vis*pixel/s = Z * N^2 * steps / s.  Default workload: the
256 x 256, 999,600-visibility single-channel data set (50 antennas, 1 km
disk, 816 Earth-rotation dumps), split-FP16 (3-term) tensor-core form, tile
shapes picked by the library's autotuner before the timed region.  Beside
it, in the same JSON line: the same evaluation on the largest single-image
workload (1024 x 1024, 2.0e7 visibilities) with its own roofline, a
fixed-iteration MEM solve timed in the same form and in the FP64 direct
form, the paper's gridded forward, and the FP64 oracle on the host cores
(all cores and one thread).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config 1..5] [--precision fp16x3|bf16x3|fp32_direct|fp64_direct]
                  [--solve-iters I] [--no-solve] [--large-steps L]

--impl reference times the FP64 CPU oracle on this machine's host cores:
every step is one evaluation on the same bounded visibility sample at full
image size, whose rate is the whole workload's (the cost is exactly Z N^2;
the line says so with "extrapolated": true).
Multi-GPU: replicas only (each rank evaluates its own copy of the workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "chi2+gradient evals/s as vis*pixel/s"
UNIT = "vis*pixel/s"
WORKLOADS = {
    1: "64x64 image, 10,260 vis (20 ant, 300 m, 27 dumps + conjugates)",
    2: "256x256 image, 999,600 vis (50 ant, 1 km, 816 dumps)",
    3: "512x512 image, 10,000,900 vis (50 ant, 2 km, 8,164 dumps)",
    4: "64-channel cube of 256x256 images, log-uniform 2e5-2e6 vis per channel (50 ant, 500 m)",
    5: "1024x1024 image, 19,998,720 vis (64 ant, 3 km, 9,920 dumps)",
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu: int, path: str | None = None):
        import tempfile
        self.gpu = gpu
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"memsynth_clocks_gpu{gpu}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(1.0)  # let the sampler start before the timed region
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu record, or None when the
    kernel's sources changed since the capture (or there is no record)."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return rec["bytes_per_launch"] if h.hexdigest()[:16] == rec["source_sha"] else None
    except (OSError, KeyError, ValueError):
        return None


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value (replicas: each rank times its own copy)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units: int, world: int, ms_step: float) -> float:
    """Whole-job throughput: every rank processes `units` per step."""
    return units * world / (ms_step * 1e-3)


def make_data(config: int, shared_image: bool = False):
    """The config's synthetic data set; shared_image: one image for all its
    channels (the multi-frequency mode of Eq. chi2-multi), the channel mean of
    the cube as its stand-in sky."""
    import dataclasses
    from paper_1703_02920_gb300 import synth
    ds = synth.make(config)
    if shared_image:
        ds = dataclasses.replace(ds, shared_image=True,
                                 truth=np.mean(ds.truth, axis=0, keepdims=True).astype(np.float32))
    return ds


def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_sample(ds, z: int):
    """The data set restricted to z evenly spaced visibilities of its first
    channel, at full image size (the oracle's cost is exactly Z N^2)."""
    import oracle
    P = oracle.Problem.from_dataset(ds)
    idx = np.linspace(0, int(ds.offsets[1]) - 1, z).astype(np.int64)
    return oracle.Problem(ds.N, ds.dx, ds.dy, P.u[idx], P.v[idx], P.vo[idx], P.sigma[idx], P.pb[:1],
                          np.array([0, z]), P.G, P.lam)


def _size_sample(ds, img, target_s: float) -> int:
    """Largest visibility count (doubling from 64) whose oracle evaluation
    takes about target_s with the current thread count."""
    import oracle
    z, zmax = 64, int(ds.offsets[1])
    while True:
        sub = _oracle_sample(ds, z)
        t0 = time.perf_counter()
        oracle.objective_grad(sub, img[:1])
        dt = time.perf_counter() - t0
        if dt > target_s / 2 or z >= zmax:
            return z
        z = min(zmax, int(z * max(2.0, min(8.0, target_s / max(dt, 1e-3)))))


def _time_oracle(ds, img, budget_s: float):
    import oracle
    z = _size_sample(ds, img, budget_s / 4)
    sub = _oracle_sample(ds, z)
    evals = 0
    t0 = time.perf_counter()
    while True:
        oracle.objective_grad(sub, img[:1])
        evals += 1
        if time.perf_counter() - t0 >= budget_s / 2:
            break
    dt = time.perf_counter() - t0
    return z * ds.N * ds.N * evals / dt, z, evals, dt


def cpu_baseline(ds, budget_s: float = 12.0, single_budget_s: float = 6.0):
    """FP64 oracle (as it stands) on a visibility subsample at full image
    size: all host cores (OpenMP) and one thread."""
    import oracle
    img = np.maximum(ds.truth.astype(np.float64), ds.G)
    cores = oracle.num_threads()
    value, z, evals, dt = _time_oracle(ds, img, budget_s)
    single = None
    if single_budget_s > 0:
        oracle.set_num_threads(1)
        try:
            v1, z1, e1, d1 = _time_oracle(ds, img, single_budget_s)
        finally:
            oracle.set_num_threads(cores)
        single = {"value": v1, "unit": UNIT, "cores": 1,
                  "sample": f"{e1} evaluation(s) on {z1} of {ds.Z} visibilities in {d1:.1f} s"}
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{evals} objective+gradient evaluation(s) on {z} of {ds.Z} visibilities "
                      f"(evenly spaced) at full {ds.N}x{ds.N} in {dt:.1f} s, FP64 factored order, OpenMP; "
                      f"the rate extrapolates to the whole workload exactly (cost is Z N^2)",
            "single_thread": single, "cpu_model": cpu_model(), "os_cpu_count": os.cpu_count()}


def run_reference(args, rank, world):
    """The oracle as the reference arm: every step is one FP64 objective +
    gradient evaluation on the same bounded visibility sample (full image
    size), timed on the host's cores.  value = the sampled vis*pixel / the
    step's wall time, which is the whole workload's rate (the cost is exactly
    Z N^2); ms_per_step is the sampled step's wall time as run."""
    if rank != 0:
        return 0
    t_start = time.perf_counter()
    ds = make_data(args.config, args.shared_image)
    import oracle
    oracle.build()
    img = np.maximum(ds.truth.astype(np.float64), ds.G)
    per_step_s = min(3.0, 60.0 / max(1, args.warmup + args.steps))
    z = _size_sample(ds, img, per_step_s)
    sub = _oracle_sample(ds, z)
    ms = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.objective_grad(sub, img[:1])
        dt = (time.perf_counter() - t0) * 1e3
        if k >= args.warmup:
            ms.append(dt)
    ms_step = statistics.mean(ms)
    sampled_units = z * ds.N * ds.N
    value = sampled_units / (ms_step * 1e-3)
    wall = time.perf_counter() - t_start
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config] + (
                ", one image shared by all channels (Eq. chi2-multi)" if args.shared_image else ""),
                "precision": "fp64 oracle (CPU)"},
            "extrapolated": True,
            "sample": {"visibilities": z, "of": ds.Z, "image": f"{ds.N}x{ds.N}",
                       "vis_pixel_per_step": sampled_units,
                       "full_workload_ms_per_step": ds.Z * ds.N * ds.N / value * 1e3,
                       "wall_s": wall},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"each step: one objective+gradient evaluation on {z} of {ds.Z} "
                                       f"visibilities (evenly spaced) at full {ds.N}x{ds.N}, FP64, OpenMP",
                             "cpu_model": cpu_model(), "os_cpu_count": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def roofline(kprof: dict, units: int, config: int) -> dict:
    """Roofline object of the dominant kernel from per-launch CUDA-event times.
    Each launch is timed alone (events around it), so the split forms are held
    against the burst bf16 peak; the fp16 dense rate is the same."""
    peaks, src = _peaks()
    dom = max(kprof.items(), key=lambda kv: kv[1][0]) if kprof else ("none", (0.0, 1))
    name, (tot_ms, cnt) = dom
    avg_ms = tot_ms / max(cnt, 1)
    # algorithmic work: 4 flops per (visibility, pixel) pair for each operator pass
    flops = 4.0 * units
    if name.startswith(("fwd", "adj")) and not name.endswith("reduce"):
        achieved = flops / (avg_ms * 1e-3) / 1e12
        if name in ("fwd_tc", "fwd_rs", "adj_tc"):
            peak = peaks.get("bf16_tflops")
            sus = peaks.get("bf16_tflops_sustained", peak)
            return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": _traffic(name) if config == 2 else None,
                    "executed_frac": 3 * achieved / peak, "algorithmic_cap": 1.0 / 3.0,
                    "note": f"{name}{' (+ slice combination)' if name == 'fwd_rs' else ''}: "
                            f"{avg_ms:.3f} ms/launch, 4 algorithmic flops per vis*pixel "
                            f"(12 executed in the 3-term split, so the algorithmic fraction is capped at 1/3: "
                            f"executed {3 * achieved:.0f} TFLOP/s); peak = {src} burst bf16 "
                            f"(of sustained: {achieved / sus:.3f})"}
        if name.endswith("direct_f32"):
            # one SFU sine and one SFU cosine per (visibility, pixel) pair; peak
            # derived from the unit counts and clocks: 152 SMs x 16 SFU results
            # per clock x 2.07 GHz = 5.03 Top/s
            sfu = 2.0 * units / (avg_ms * 1e-3) / 1e12
            peak = 152 * 16 * 2.07e9 / 1e12
            return {"bound": "alu", "achieved": sfu, "peak": peak, "unit": "Top/s (SFU)", "frac": sfu / peak,
                    "traffic": None, "note": f"{name}: {avg_ms:.3f} ms/launch, 2 SFU operations per vis*pixel; "
                                             "peak derived (152 SMs x 16 SFU/clk x 2.07 GHz)"}
        return {"bound": "alu", "achieved": achieved, "peak": None, "unit": "TFLOP/s",
                "frac": None, "traffic": None, "note": f"{name}: {avg_ms:.3f} ms/launch (FP64 pipe)"}
    return {"bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
            "frac": None, "traffic": None, "note": name}


def large_block(precision: str, steps: int, warmup: int = 3, config: int = 5) -> dict:
    """Device-timed evaluations of the largest single-image workload (1024^2,
    2.0e7 visibilities), with its own per-kernel roofline; L2 flushed between
    steps (its inputs are also larger than L2)."""
    import torch
    from paper_1703_02920_gb300 import memsynth
    ds = make_data(config)
    units = ds.Z * ds.N * ds.N
    ctx = memsynth.Context(ds, precision=precision)
    img = torch.from_numpy(np.maximum(ds.truth, ds.G)).cuda()
    grad = torch.empty_like(img)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tiles = list(ctx.autotune(img, reps=1)) if precision in ("bf16x3", "fp16x3") else None
    for _ in range(warmup):
        memsynth.mem_objective_grad(ctx.handle, img, grad, 0, want_scalars=False)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    l0 = ctx.launches()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(ctx.stream)
        memsynth.mem_objective_grad(ctx.handle, img, grad, 0, want_scalars=False)
        ev[k][1].record(ctx.stream)
    torch.cuda.synchronize()
    launches = ctx.launches() - l0
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    ctx.profile(True)
    ctx.profile_read()
    for _ in range(2):
        flush.zero_()
        memsynth.mem_objective_grad(ctx.handle, img, grad, 0, want_scalars=False)
    kprof = ctx.profile_read()
    ctx.profile(False)
    ctx.close()
    return {"workload": WORKLOADS[config], "precision": precision, "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT, "gpu_launches": launches,
            "tiles": tiles, "roofline": roofline(kprof, units, config),
            "kernels": {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1]} for k, v in kprof.items()}}


def run_sweep(args):
    """Evaluation rate over image size and visibility count on seeded random
    problems (one JSON line per size); L2 flushed between evaluations, median
    of CUDA-event times on the library's stream, autotuned tiling."""
    import torch
    from paper_1703_02920_gb300 import memsynth, synth
    torch.cuda.set_device(0)
    memsynth.load()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for N in (128, 256, 512, 1024):
        for Z in (100_000, 1_000_000, 10_000_000):
            ds = synth.random_problem(N, Z, 11, lam=3.0)
            ctx = memsynth.Context(ds, precision=args.precision)
            img = torch.from_numpy(ds.truth).cuda()
            g = torch.empty_like(img)
            if args.precision in ("bf16x3", "fp16x3"):
                ctx.autotune(img, reps=2)
            for _ in range(3):
                memsynth.mem_objective_grad(ctx.handle, img, g, 0, want_scalars=False)
            steps = max(3, min(50, int(2e13 / (Z * N * N)) + 3))
            ts = []
            for _ in range(steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(ctx.stream)
                memsynth.mem_objective_grad(ctx.handle, img, g, 0, want_scalars=False)
                b.record(ctx.stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            t = float(np.median(ts))
            print(json.dumps({"sweep": True, "precision": args.precision, "N": N, "visibilities": Z,
                              "ms_per_evaluation": t, "value": Z * N * N / (t * 1e-3), "unit": UNIT,
                              "tiling": list(ctx.tiling()) if args.precision in ("bf16x3", "fp16x3") else None}),
                  flush=True)
            ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--precision", default="fp16x3", choices=["bf16x3", "fp16x3", "fp32_direct", "fp64_direct"])
    ap.add_argument("--solve-iters", type=int, default=4)
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--clock-log", default=None, help="CSV file for the nvidia-smi samples (default: a temp file)")
    ap.add_argument("--tiling", default=None,
                    help="kernel,cols,fwd_stages,adj_stages (e.g. resident,256,6,3): fixed tiling, no autotuning")
    ap.add_argument("--profile-run", action="store_true",
                    help="only W + K objective+gradient evaluations with the default tiling (for ncu captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--large-steps", type=int, default=10,
                    help="device-timed steps of the 1024^2, 2e7-visibility workload reported beside the "
                         "main line (0: skip)")
    ap.add_argument("--shared-image", action="store_true",
                    help="one image for all channels (multi-frequency mode); meaningful for the cube config 4")
    ap.add_argument("--sweep", action="store_true",
                    help="evaluation rate over N in 128..1024 and 1e5..1e7 visibilities (one line per size)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.sweep:
        return run_sweep(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1703_02920_gb300 import memsynth

    memsynth.load()
    ds = make_data(args.config, args.shared_image)
    N, Z = ds.N, ds.Z
    units = Z * N * N
    ctx = memsynth.Context(ds, precision=args.precision)
    stream = ctx.stream
    img = torch.from_numpy(np.maximum(ds.truth, ds.G)).cuda()
    grad = torch.empty_like(img)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    def step():
        memsynth.mem_objective_grad(ctx.handle, img, grad, 0, want_scalars=False)

    fixed = None
    if args.tiling and args.precision in ("bf16x3", "fp16x3"):
        k, c_, f_, a_ = args.tiling.split(",")
        fixed = (k, int(c_), int(f_), int(a_))
        ctx.set_tiling(*fixed)
    if args.profile_run:
        for _ in range(args.warmup + args.steps):
            step()
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "precision": args.precision, "evaluations": args.warmup + args.steps,
                          "tiling": ctx.tiling(), "launches": ctx.launches()}))
        ctx.close()
        return 0

    tiles = None
    if args.precision in ("bf16x3", "fp16x3"):
        kern, bn, fs, ast = fixed if fixed else ctx.autotune(img)
        tiles = {"fwd_kernel": kern, "fwd_cols": bn, "fwd_stages": fs, "adj_stages": ast}
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-timed region: CUDA events on the context stream per step, L2
    # flushed between steps; each step replays the captured CUDA graph
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launches()
    with ClockSampler(local, args.clock_log) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches = ctx.launches() - launches0
    ctx.sync()
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = max_over_ranks(sum(ms) / len(ms), dist, "cuda")
    value = job_value(units, world, ms_step)

    # ---- per-kernel durations: the same steps again with every launch bracketed
    # by CUDA events on the context stream (direct launches, no graph)
    ctx.profile(True)
    ctx.profile_read()
    for k in range(args.steps):
        flush.zero_()
        step()
    kprof = ctx.profile_read()
    ctx.profile(False)

    # ---- end to end through the host-buffer entry point (pinned host memory)
    himg = torch.from_numpy(np.maximum(ds.truth, ds.G).astype(np.float32)).pin_memory().numpy()
    hgrad = torch.empty(himg.shape, dtype=torch.float32).pin_memory().numpy()
    for _ in range(2):
        ctx.objective_grad_host(himg)
    e2e_ms = []
    for _ in range(max(3, min(50, args.steps // 2))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        memsynth.mem_objective_grad_host(ctx.handle, himg, hgrad, 0)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_val = job_value(units, world, max_over_ranks(statistics.mean(e2e_ms), dist, "cuda"))

    # ---- roofline of the dominant kernel (algorithmic flops per launch / event time)
    roof = roofline(kprof, units, args.config)
    kernels = {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1],
                   "share": v[0] / max(sum(x[0] for x in kprof.values()), 1e-30)} for k, v in kprof.items()}

    # ---- the paper's gridded forward (FFT + bilinear) beside the exact one:
    # time per pass and its error against the exact model visibilities
    gridded = None
    if not args.no_solve:
        vex = ctx.forward(img).double()
        gridded = {}
        for pad in (2, 4):
            vg = ctx.forward_gridded(img, pad)  # warm-up (plan, buffers)
            torch.cuda.synchronize()
            gms = []
            for _ in range(5):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                memsynth.mem_forward_gridded(ctx.handle, img, pad, vg)
                b.record(stream)
                torch.cuda.synchronize()
                gms.append(a.elapsed_time(b))
            err = float((vg.double() - vex).norm(dim=1).max() / vex.norm(dim=1).max())
            gridded[f"pad{pad}"] = {"ms": statistics.mean(gms), "max_rel_err_vs_exact": err}
        gridded["exact_forward_ms"] = kprof.get("fwd_tc", kprof.get("fwd_rs", (0.0, 1)))[0] / max(
            kprof.get("fwd_tc", kprof.get("fwd_rs", (0.0, 1)))[1], 1)

    # ---- MEM solve from I = G: a few CG iterations in this form and in the
    # FP64 direct form (same algorithm, same start)
    solve = None
    if not args.no_solve and args.solve_iters > 0:
        I0 = torch.full_like(img, float(ds.G))
        solve = {}
        # the FP64 form takes about a minute per iteration at 256 x 256 and 1e6
        # visibilities: one timed iteration, no warm-up (its set-up is negligible)
        legs = [("form", args.precision, args.solve_iters, True)]
        if units <= 2e11:  # the FP64 iteration is about a minute at 6.5e10 vis*pixel
            legs.append(("fp64", "fp64_direct", 1, False))
        for key, prec, iters, warm in legs:
            sctx = ctx if prec == args.precision else memsynth.Context(ds, precision=prec)
            if warm:
                sctx.solve(I0, 1)  # warm-up (graph capture, buffers)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, rep, _ = sctx.solve(I0, iters)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            solve[key] = {"precision": prec, "iterations": rep.iterations, "s": dt,
                          "ms_per_iter": dt * 1e3 / max(rep.iterations, 1),
                          "evaluations": rep.evaluations, "phi": rep.phi}
            if sctx is not ctx:
                sctx.close()
        if "fp64" in solve:
            solve["speedup_vs_fp64_per_iter"] = solve["fp64"]["ms_per_iter"] / solve["form"]["ms_per_iter"]
        else:
            solve["fp64"] = "not run: over a minute per iteration at this size"

    large = None
    if args.large_steps > 0 and args.config != 5 and not args.shared_image:
        large = large_block(args.precision, args.large_steps)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ds)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": {"bf16x3": "bf16x3", "fp16x3": "f16x3", "fp32_direct": "f32", "fp64_direct": "f64"}[args.precision],
                "data": "synthetic",
                "config": {"workload": WORKLOADS[args.config] + (
                               ", one image shared by all channels (Eq. chi2-multi)" if args.shared_image else ""),
                           "precision": args.precision,
                           "image": f"{N}x{N}", "visibilities": Z, "parallelism": f"replicas x{world}",
                           "l2": "flushed between timed steps (256 MB write)", "tiles": tiles},
                # per step: the image up; the gradient, the objective scalars
                # (3 totals + 3 per image, FP64) and the 4-byte status word down
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(img.numel() * 4),
                        "d2h_bytes_per_step": int(img.numel() * 4 + (3 + 3 * ctx.n_images) * 8 + 4)},
                "gpu_launches": launches,
                "roofline": roof, "kernels": kernels,
                "clocks": clk.summary(), "cpu_baseline": cpu, "solve": solve, "gridded_forward": gridded,
                "largest_single_image": large}
        print(json.dumps(line))
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
