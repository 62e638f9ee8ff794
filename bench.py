"""Throughput of the resampling F-statistic on the search-sized workload.

Workload (one step): 10 days of heterodyned complex64 data at dt = 0.5 s
(1,728,000 samples) with 10 % of the samples in gap blocks of 1-6 h, and
8192 templates = 1024 sky points (Fibonacci sphere) x 8 spindowns in
[-1e-9, 0] Hz/s, each resampled with an 8-tap Lanczos-windowed sinc onto its
barycentric grid and transformed with a 2^22-point FFT: 3.4e10 2F values per
step, written to HBM.  Metric: 2F values per second (templates x frequency
bins / wall time), device-timed with CUDA events over the timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank takes its own 8192 templates (weak scaling, no
collective on the data path; a barrier and a max-reduction of the timing
only).  The reference arm (``--impl reference``) is the FP64 CPU oracle run
on the host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

N_SKY, N_FDOT = 1024, 8
GAP_FRAC = 0.10
BATCH = 64            # templates per fstat_compute call (the 2F ring buffer)
KINDS = ("timemap", "resample", "fft_cols", "fft_rows", "grad_fwd", "grad_adj", "persistent", "sums")


def workload(rank: int = 0, world: int = 1):
    """The search-sized workload; under N ranks the sky grid has N x 1024
    points and each rank takes its contiguous share of the N x 8192
    templates (weak scaling)."""
    from paper_0912_4255_gb300.shard import shard
    desc = synth.search_plan(max_templates=BATCH)
    seed = synth.SEED_BASE + 1
    gaps = synth.gap_intervals(desc.n_data, GAP_FRAC, 7200, 43200, seed=seed)
    x = synth.zero_gaps(synth.complex_noise(desc.n_data, desc.sigma2, seed), gaps)
    a, d = synth.fibonacci_sky(N_SKY * world)
    fd = np.linspace(-1e-9, 0.0, N_FDOT)
    tm = synth.make_templates(np.repeat(a, N_FDOT), np.repeat(d, N_FDOT), np.tile(fd, N_SKY * world),
                              0, desc.n_data, 0, len(gaps))
    tm, _ = shard(tm, rank, world)
    return desc, x, tm, gaps


PRECISION_GPU = "mixed (FP64 time map/phase at knots, FP32 samples, FP32 FFT)"
PRECISION_ORACLE = "FP64 NumPy oracle (complex128 FFT), the same algorithm"


def config_dict(desc, n_templates, world, precision=PRECISION_GPU):
    return {
        "workload": ("search-sized: 10 d at dt=0.5 s (1,728,000 complex64 samples), 10% gaps in "
                     "1-6 h blocks, 1024 sky x 8 fdot = 8192 templates per GPU, 8-tap Lanczos sinc, "
                     "FFT 2^22, 2F in every bin"),
        "templates_per_gpu": int(n_templates),
        "n_data": int(desc.n_data),
        "n_fft": int(desc.n_fft),
        "dt": desc.dt,
        "interp": "sinc8-lanczos",
        "precision": precision,
        "parallelism": f"replicas x{world} (template shards, no data-path collective)",
        "l2": ("each step writes 137 GB of 2F per GPU (>> 129 MB L2); the 13.8 MB input "
               "series stays L2-resident across templates by design"),
    }


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
                pw.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- peaks

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def fp32_peak_tflops(sm_mhz: float) -> float:
    """FP32 FMA peak: 152 SMs x 128 FP32 lanes x 2 flop per clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def algorithmic_per_template(desc, fused=True, l1=None):
    """(FLOPs, design bytes) of one template in each kernel.

    FLOPs, counted from the algorithm:
    * FFTs: 5 N log2 N per complex transform of length N, two series (F_a,
      F_b); the first pass does the log2 N1 part, the second the log2 N2 part;
      the inter-pass twiddle is one complex multiply per element and series;
    * resampling, per grid point: K taps x (4 flop complex MAC + 5 flop
      weight) + 16 flop (phase rotation, a/b weights, sums A, B, C);
    * 2F: 12 flop per bin.
    Design bytes, the HBM traffic the four-step design needs (N_d data
    samples ~ N_b grid points, N = n_fft):
    * time map: an 80-byte knot record per 2^10 grid points;
    * resample (split): read x_h 8 N_d, write w_a, w_b 16 N_b;
    * first pass: read w_a, w_b 16 N_b (split) or x_h 8 N_d (fused), write the
      intermediate 16 N;
    * second pass: read the intermediate 16 N, write 2F 4 N.
    The path's own algorithmic bytes are 8 N_d + 4 N (path_bytes)."""
    n = int(desc.n_fft)
    L = int(math.log2(n))
    if l1 is None:
        l1 = max(6, min(12, L - 6))       # the library's default factorisation
    l2 = L - l1
    taps = desc.taps if desc.interp == 1 else 1
    nd = float(desc.n_data)
    fft_a = 2 * 5 * n * l1 + 2 * 6 * n
    res = nd * (taps * 9 + 16)
    rows = 2 * 5 * n * l2 + 12 * n
    out = {"fft_rows": (rows, 16.0 * n + 4.0 * n), "timemap": (0.0, 80.0 * (n >> 10)), "sums": (0.0, 0.0),
           "persistent": (fft_a + res + rows, 8.0 * nd + 32.0 * n + 4.0 * n)}
    if fused:
        out["fft_cols"] = (fft_a + res, 8.0 * nd + 16.0 * n)
    else:
        out["resample"] = (res, 8.0 * nd + 16.0 * nd)
        out["fft_cols"] = (fft_a, 16.0 * nd + 16.0 * n)
    return out


def path_bytes(desc):
    """Algorithmic bytes of the whole path per template: read x_h once, write 2F."""
    return 8.0 * desc.n_data + 4.0 * desc.n_fft


def ncu_traffic(kernel: str, templates_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary
    (profiles/traffic.md), scaled by templates per launch, or None if the
    path kernels changed since that capture (digest mismatch)."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    try:
        from paper_0912_4255_gb300 import build as fsbuild
        digest = fsbuild.path_digest()
        txt = open(path).read()
        if f"path digest: {digest}" not in txt:
            return None
        for line in txt.splitlines():
            p = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(p) >= 3 and p[0] == kernel:
                return float(p[1]) * templates_per_launch
    except (OSError, ValueError):
        return None
    return None


# ---------------------------------------------------------------- CPU oracle

def _oracle_one(args):
    desc, x, tmpl, gaps = args
    sys.path.insert(0, ROOT)
    from oracle import fstat as F
    t0 = time.perf_counter()
    F.resample_two_f(x.astype(np.complex128), tmpl, gaps, desc)
    return time.perf_counter() - t0


def cpu_oracle_rate(desc, x, tm, gaps, n_templates=None, workers=None):
    """2F values/s of the FP64 oracle on a bounded sample of templates, run
    in a spawn-started process pool over the host cores."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    workers = workers or max(1, min(cores, 8))
    n_templates = n_templates or 2 * workers
    sel = np.linspace(0, len(tm) - 1, n_templates).astype(int)
    jobs = [(desc, x, tm[i], gaps) for i in sel]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_one, jobs)
    wall = time.perf_counter() - t0
    value = n_templates * desc.n_fft / wall
    return {"value": value, "unit": "2F values/s", "cores": workers, "kind": "oracle",
            "sample": (f"{n_templates} of the workload's templates (evenly spaced in the grid), "
                       f"FP64 NumPy oracle, {workers} spawn workers, {wall:.1f} s wall")}


# ---------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--templates", type=int, default=N_SKY * N_FDOT,
                    help="templates per GPU per step (default: the whole 8192-template grid)")
    ap.add_argument("--batch", type=int, default=BATCH,
                    help="templates per fstat_compute call (size of the 2F ring buffer)")
    ap.add_argument("--mode", default="split", choices=["fused", "split", "persistent", "plain"],
                    help="library execution mode")
    ap.add_argument("--chunk", type=int, default=0,
                    help="templates per internal launch (0: the library's default)")
    ap.add_argument("--log2-n1", type=int, default=0,
                    help="log2 of the first-pass FFT length (0: the library's default)")
    ap.add_argument("--copy-streams", type=int, default=4,
                    help="streams the end-to-end leg splits each batch's device-to-host copy over")
    ap.add_argument("--workload", default="search",
                    choices=["search", "batch", "montecarlo", "frontend", "demod"],
                    help="search: the 8192-template grid (the metric's workload); batch: 4096 "
                         "templates with uneven spans, own gap lists and FFT lengths; montecarlo: "
                         "noise-only realizations of the 12 h nearest-neighbour configuration; frontend: "
                         "the SFT front end making the search's 10 d series from 1800 s SFTs; demod: the "
                         "SFT-domain demodulation F-statistic against resampling on the same data")
    ap.add_argument("--realizations", type=int, default=1 << 20,
                    help="Monte Carlo realizations (--workload montecarlo), noise only and with signals")
    ap.add_argument("--mc-h0", type=float, default=0.12,
                    help="injected amplitude of the Monte Carlo with signals (sigma^2 = 1; mean rho^2 ~ 100)")
    ap.add_argument("--topk", type=int, default=16,
                    help="candidates per band returned by the e2e leg (0: return every 2F value)")
    ap.add_argument("--topk-band", type=int, default=65536, help="bins per candidate band")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "montecarlo":
        return run_montecarlo(args)
    if args.workload == "frontend":
        return run_frontend(args)
    if args.workload == "demod":
        return run_demod(args)

    import torch
    import torch.distributed as dist
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300 import build as fsbuild
    fsbuild.build()

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    desc, x_np, tm, gaps_np = workload(rank, world)
    tm = tm[:args.templates]
    batch = max(1, min(args.batch, len(tm)))
    desc = desc.replace(max_templates=batch)
    n_t = len(tm)
    n_fft = int(desc.n_fft)

    # CPU baseline first (spawned pool, before heavy GPU allocation)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(desc, x_np, tm, gaps_np)

    plan = fs.Plan(desc, device=dev)
    mode = {"fused": fs.MODE_FUSED, "split": fs.MODE_SPLIT, "persistent": fs.MODE_PERSISTENT,
            "plain": fs.MODE_PLAIN}[args.mode]
    if args.chunk or args.log2_n1 or mode != fs.MODE_SPLIT:
        plan.set_tuning(mode=mode, chunk=args.chunk, log2_n1=args.log2_n1)
    stream = torch.cuda.Stream(device=dev)
    x = torch.from_numpy(x_np.astype(np.complex64)).to(dev)
    gaps = torch.from_numpy(gaps_np.reshape(-1).copy()).to(dev)
    tmpl = fs.pack_templates(tm, device=dev)
    tsize = fs.TEMPLATE_DTYPE.itemsize
    out = torch.empty(batch * n_fft, dtype=torch.float32, device=dev)

    def step(s):
        for b0 in range(0, n_t, batch):
            nb = min(batch, n_t - b0)
            fs.fstat_compute(plan, x, tmpl[b0 * tsize:(b0 + nb) * tsize], gaps, out, stream=s)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(stream)
    stream.synchronize()
    fs.fstat_status(plan, stream)
    fs.fstat_profile_read(plan)          # clear counters

    # ---- timed region (device time, CUDA events on the launching stream)
    fs.fstat_profile(plan, True)
    clk = ClockSampler(dev.index if dev.index is not None else 0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            step(stream)
    ev1.record(stream)
    stream.synchronize()
    clocks = clk.stop()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    prof = fs.fstat_profile_read(plan)
    fs.fstat_profile(plan, False)
    fs.fstat_status(plan, stream)
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    values_per_step = n_t * n_fft * world
    value = values_per_step / (ms_per_step / 1e3)

    # ---- roofline of the dominant kernel
    peak_gbs, peak_kind = measured_peaks()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak_tf = fp32_peak_tflops(sm_mhz)
    per_tpl = algorithmic_per_template(desc, fused=mode in (fs.MODE_FUSED, fs.MODE_PERSISTENT),
                                       l1=plan.tuning()["log2_n1"])
    kernels = {}
    for k in ("timemap", "resample", "fft_cols", "fft_rows", "persistent", "sums"):
        k_ms, k_n = prof[k]
        if not k_n:
            continue
        tpl_per_launch = n_t * args.steps / k_n
        t_launch = k_ms / k_n / 1e3
        flops, nbytes = per_tpl[k]
        kernels[k] = {"launches": int(k_n), "ms_per_launch": k_ms / k_n,
                      "templates_per_launch": tpl_per_launch,
                      "tflops": flops * tpl_per_launch / t_launch / 1e12,
                      "design_bytes_per_launch": nbytes * tpl_per_launch,
                      "design_gbs": nbytes * tpl_per_launch / t_launch / 1e9}
    dom = max(kernels, key=lambda k: prof[k][0])
    kd = kernels[dom]
    traffic = ncu_traffic(dom, kd["templates_per_launch"])
    # the dominant kernel against the HBM roofline on the path's algorithmic
    # bytes (x_h read once, 2F written once per template)
    alg_launch = path_bytes(desc) * kd["templates_per_launch"]
    alg_gbs = alg_launch / (kd["ms_per_launch"] / 1e3) / 1e9
    # whole path: algorithmic and design bytes per template at the measured rate
    tpl_per_s = n_t * world / (ms_per_step / 1e3)
    design_tpl = sum(per_tpl[k][1] for k in kernels if k in per_tpl)
    launches = sum(v[1] for v in prof.values())
    kernel_ms = {k: round(v[0] / args.steps, 3) for k, v in prof.items() if v[1]}
    # ---- end to end through the public API: pinned host in, pinned host out
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(fs, plan, desc, x_np, tm, gaps_np, dev, args, world, batch,
                      copy_streams=max(1, args.copy_streams))

    line = {
        "metric": "2F values/sec (templates x freq bins) at rel err <= 1e-4",
        "value": value, "unit": "2F values/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 time map)",
        "data": "synthetic (seeded complex Gaussian noise with gaps; analytic ephemeris)",
        "config": config_dict(desc, n_t, world),
        "kernel_ms_per_step": kernel_ms,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": alg_gbs, "peak": peak_gbs,
                     "unit": "GB/s", "frac": alg_gbs / peak_gbs,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                     "bytes": ("algorithmic bytes of the path (8 N_d + 4 N per template: read x_h, "
                               "write 2F) x templates per launch of the dominant kernel"),
                     "bytes_per_launch": alg_launch,
                     "traffic": traffic,
                     "design_achieved": kd["design_gbs"], "design_frac": kd["design_gbs"] / peak_gbs,
                     "design_bytes_per_launch": kd["design_bytes_per_launch"],
                     "alu": {"achieved": kd["tflops"], "peak": peak_tf, "unit": "TFLOP/s",
                             "frac": kd["tflops"] / peak_tf,
                             "peak_source": f"FP32 FMA: 152 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz"}},
        "path": {"alg_bytes_per_template": path_bytes(desc),
                 "alg_gbs": path_bytes(desc) * tpl_per_s / 1e9,
                 "alg_frac": path_bytes(desc) * tpl_per_s / 1e9 / peak_gbs,
                 "design_bytes_per_template": design_tpl,
                 "design_gbs": design_tpl * tpl_per_s / 1e9,
                 "design_frac": design_tpl * tpl_per_s / 1e9 / peak_gbs},
        "kernels": kernels,
        "clocks": clocks, "gpu_launches": int(launches), "tuning": plan.tuning(),
    }
    # the headline e2e is the search as a user runs it: inputs in, every 2F
    # computed on the device, the step's result (the loudest bins of every
    # band) out; the transfer of every 2F value to the host is kept beside it
    e2e_cand = None
    if not args.no_e2e and args.topk > 0:
        e2e_cand = run_e2e_candidates(fs, plan, desc, x_np, tm, gaps_np, dev, args, world,
                                      batch, args.topk_band, args.topk)
        e2e_cand["result"] = (f"the {args.topk} loudest bins of every {args.topk_band}-bin band "
                              "(values and bins)")
    if e2e_cand is not None:
        line["e2e"] = e2e_cand
        if e2e is not None:
            e2e["result"] = "every 2F value"
            line["e2e_full_2f"] = e2e
    elif e2e is not None:
        line["e2e"] = e2e
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def run_e2e(fs, plan, desc, x_np, tm, gaps_np, dev, args, world, batch, copy_streams=4):
    """Same metric with host buffers: per step the input series, templates and
    gap list go host->device and every 2F value comes back device->host into
    pinned memory (double-buffered, copies overlapped with compute; each
    batch's copy is split over copy_streams streams so that several copy
    engines move it)."""
    import torch
    n_t = len(tm)
    n_fft = int(desc.n_fft)
    tsize = fs.TEMPLATE_DTYPE.itemsize
    x_h = torch.from_numpy(x_np.astype(np.complex64)).pin_memory()
    g_h = torch.from_numpy(gaps_np.reshape(-1).copy()).pin_memory()
    t_h = fs.pack_templates(tm, device=None).pin_memory()
    x_d = torch.empty_like(x_h, device=dev)
    g_d = torch.empty_like(g_h, device=dev)
    t_d = torch.empty_like(t_h, device=dev)
    outs = [torch.empty(batch * n_fft, dtype=torch.float32, device=dev) for _ in range(2)]
    host = [torch.empty(batch * n_fft, dtype=torch.float32).pin_memory() for _ in range(2)]
    cs = torch.cuda.Stream(device=dev)
    xss = [torch.cuda.Stream(device=dev) for _ in range(copy_streams)]
    done = [torch.cuda.Event() for _ in range(2)]
    copied = [[torch.cuda.Event() for _ in xss] for _ in range(2)]
    for ev in copied:
        for e, xs in zip(ev, xss):
            e.record(xs)

    def step():
        with torch.cuda.stream(cs):
            x_d.copy_(x_h, non_blocking=True)
            g_d.copy_(g_h, non_blocking=True)
            t_d.copy_(t_h, non_blocking=True)
            for i, b0 in enumerate(range(0, n_t, batch)):
                nb = min(batch, n_t - b0)
                j = i & 1
                for e in copied[j]:
                    cs.wait_event(e)
                fs.fstat_compute(plan, x_d, t_d[b0 * tsize:(b0 + nb) * tsize], g_d, outs[j], stream=cs)
                done[j].record(cs)
                total = nb * n_fft
                part = (total + len(xss) - 1) // len(xss)
                for k, xs in enumerate(xss):
                    a0, a1 = k * part, min(total, (k + 1) * part)
                    xs.wait_event(done[j])
                    if a1 > a0:
                        with torch.cuda.stream(xs):
                            host[j][a0:a1].copy_(outs[j][a0:a1], non_blocking=True)
                    copied[j][k].record(xs)

    step()                                   # warm-up: pinned buffers and copy streams in use
    torch.cuda.synchronize(dev)
    steps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize(dev)
    wall = (time.perf_counter() - t0) / steps
    h2d = x_h.numel() * 8 + g_h.numel() * 8 + t_h.numel()
    d2h = n_t * n_fft * 4
    return {"value": n_t * n_fft * world / wall, "unit": "2F values/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": wall * 1e3, "steps": steps}


def run_e2e_candidates(fs, plan, desc, x_np, tm, gaps_np, dev, args, world, batch, band_len, k):
    """End to end through the public API for a search that keeps candidates:
    per step the inputs go host->device, every 2F value is computed in device
    memory, fstat_topk keeps the k loudest bins of every band, and only those
    (values and bins) come back to pinned host memory.  The top-k of one
    chunk runs on a second stream while the next chunk is computed (two 2F
    buffers): its HBM streaming overlaps the compute-bound kernels."""
    import torch
    n_t = len(tm)
    n_fft = int(desc.n_fft)
    tsize = fs.TEMPLATE_DTYPE.itemsize
    x_h = torch.from_numpy(x_np.astype(np.complex64)).pin_memory()
    g_h = torch.from_numpy(gaps_np.reshape(-1).copy()).pin_memory()
    t_h = fs.pack_templates(tm, device=None).pin_memory()
    x_d, g_d, t_d = (torch.empty_like(h, device=dev) for h in (x_h, g_h, t_h))
    outs = [torch.empty(batch * n_fft, dtype=torch.float32, device=dev) for _ in range(2)]
    n_bands = n_fft // band_len
    dv = [torch.empty((batch, n_bands, k), dtype=torch.float32, device=dev) for _ in range(2)]
    db = [torch.empty((batch, n_bands, k), dtype=torch.int32, device=dev) for _ in range(2)]
    hv = torch.empty((n_t, n_bands, k), dtype=torch.float32).pin_memory()
    hb = torch.empty((n_t, n_bands, k), dtype=torch.int32).pin_memory()
    # compute at the higher priority: the top-k blocks fill what it leaves
    cs = torch.cuda.Stream(device=dev, priority=-1)         # compute
    ts = torch.cuda.Stream(device=dev, priority=0)          # selection and result copies
    ready = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    for e in freed:
        e.record(ts)

    def step():
        with torch.cuda.stream(cs):
            x_d.copy_(x_h, non_blocking=True)
            g_d.copy_(g_h, non_blocking=True)
            t_d.copy_(t_h, non_blocking=True)
        for i, b0 in enumerate(range(0, n_t, batch)):
            nb = min(batch, n_t - b0)
            j = i & 1
            cs.wait_event(freed[j])
            fs.fstat_compute(plan, x_d, t_d[b0 * tsize:(b0 + nb) * tsize], g_d, outs[j], stream=cs)
            ready[j].record(cs)
            ts.wait_event(ready[j])
            with torch.cuda.stream(ts):
                fs.fstat_topk(outs[j][:nb * n_fft], band_len, k, n_rows=nb, stream=ts, val=dv[j], bins=db[j])
                hv[b0:b0 + nb].copy_(dv[j][:nb], non_blocking=True)
                hb[b0:b0 + nb].copy_(db[j][:nb], non_blocking=True)
            freed[j].record(ts)

    step()
    torch.cuda.synchronize(dev)
    steps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize(dev)
    wall = (time.perf_counter() - t0) / steps
    return {"value": n_t * n_fft * world / wall, "unit": "2F values/s",
            "h2d_bytes_per_step": int(x_h.numel() * 8 + g_h.numel() * 8 + t_h.numel()),
            "d2h_bytes_per_step": int(hv.numel() * 4 + hb.numel() * 4),
            "ms_per_step": wall * 1e3, "steps": steps, "band_len": band_len, "k": k}


def run_frontend(args):
    """The SFT front end (Sec. III.B) at the search workload's size: 10 d of
    1800 s SFTs of 256 Hz data (480 slots, 10 % missing in runs of 1-3),
    3648 stored bins around f_h = 100 Hz, a 2 Hz output band (3600 bins per
    SFT, dt_out = 0.5 s), 33 Dirichlet terms, a 101-bin running median and a
    5 % Tukey taper; the output is the search's 1,728,000-sample series.
    SFT noise bins are drawn directly (white noise: independent complex
    Gaussian bins).  Device-timed with CUDA events over K passes, inputs
    resident; e2e adds the host-to-device copy of the SFTs and the
    device-to-host copy of the series."""
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300 import build as fsbuild
    fsbuild.build()
    dev = torch.device("cuda", 0)
    n_slots, t_len, fs_raw = 480, 1800.0, 256.0
    n1, dk, pad, k_h = 3600, 16, 8, 180000
    d = synth.SftDesc(sft_len=int(t_len * fs_raw), dt_raw=1.0 / fs_raw, k_lo=k_h - n1 // 2 - dk - pad,
                      n_bins=n1 + 2 * (dk + pad), k_het=k_h, band_bins=n1, dirichlet_terms=dk,
                      median_window=101, tukey_frac=0.05)
    slots = synth.sft_slots(n_slots, n_slots // 10, synth.SEED_BASE + 80)
    X_h = synth.sft_noise(len(slots), d.n_bins, d.sft_len, 1.0, synth.SEED_BASE + 81)
    t_sft = slots * t_len
    n_out = n_slots * n1
    X = torch.from_numpy(X_h).to(dev)
    x = torch.empty(n_out, dtype=torch.complex64, device=dev)
    ws = torch.empty(fs.fstat_sft_workspace(d, len(slots)) + 256, dtype=torch.uint8, device=dev)
    for _ in range(max(args.warmup, 1)):
        fs.fstat_sft_series(d, X, t_sft, 0.0, n_out, x_h=x, workspace=ws)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fs.fstat_sft_series(d, X, t_sft, 0.0, n_out, x_h=x, workspace=ws)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    # end to end: SFTs from pinned host memory, series back to pinned host memory
    Xp = torch.from_numpy(X_h).pin_memory()
    xp = torch.empty(n_out, dtype=torch.complex64).pin_memory()
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(args.steps):
        X.copy_(Xp, non_blocking=True)
        fs.fstat_sft_series(d, X, t_sft, 0.0, n_out, x_h=x, workspace=ws)
        xp.copy_(x, non_blocking=True)
    e1.record()
    torch.cuda.synchronize(dev)
    ms_e2e = e0.elapsed_time(e1) / args.steps
    chunks = synth_chunks(t_sft, t_len)
    n_chunks = len(chunks)
    # the library groups chunks by at most 32 chunks and 65535 SFTs per launch
    groups, i = 0, 0
    while i < n_chunks:
        rows, n = 0, 0
        while i + n < n_chunks and n < 32 and rows + chunks[i + n][1] <= 65535:
            rows += chunks[i + n][1]
            n += 1
        groups += 1
        i += n
    print(json.dumps({
        "workload": "frontend",
        "config": "10 d of 1800 s SFTs at 256 Hz (480 slots, 48 missing), 3648 stored bins, f_h = 100 Hz, "
                  "2 Hz band (3600 bins per SFT), dk = 16, median window 101, Tukey 5 %",
        "sfts": int(len(slots)), "chunks": n_chunks, "x_h_samples": n_out,
        "ms": ms, "x_h_samples_per_s": n_out / (ms / 1e3),
        "sft_bins_per_s": len(slots) * d.n_bins / (ms / 1e3),
        "e2e": {"ms": ms_e2e, "h2d_bytes": int(X_h.nbytes), "d2h_bytes": int(n_out * 8)},
        "gpu_launches_per_pass": 1 + 5 * groups,            # normalisation + 5 per group of chunks
        "steps": args.steps, "warmup": args.warmup}))


def run_demod(args):
    """The speed comparison of Sec. IV.A on one GPU: the SFT-domain
    demodulation F-statistic (the earlier method) and resampling on the same
    10 d data set (432 normalised 1800 s SFTs; for resampling the series the
    front end makes from them), the same frequency grid (the search plan's:
    N = 2^22 at dt = 0.5 s, f_h = 100 Hz) and templates of the search grid.
    Demodulation: 8 templates x 65536 bins around f_h, device-timed.
    Resampling: 64 templates x all 2^22 bins, device-timed, default tuning.
    Reports both rates in 2F values/s and their ratio, with the paper's
    operation-count estimate N_SFT / log2 N beside it."""
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300 import build as fsbuild
    fsbuild.build()
    dev = torch.device("cuda", 0)
    n_slots, t_len, fs_raw = 480, 1800.0, 256.0
    n1, dk, pad, k_h = 3600, 16, 8, 180000
    sd = synth.SftDesc(sft_len=int(t_len * fs_raw), dt_raw=1.0 / fs_raw, k_lo=k_h - n1 // 2 - dk - pad,
                       n_bins=n1 + 2 * (dk + pad), k_het=k_h, band_bins=n1, dirichlet_terms=dk,
                       median_window=101, tukey_frac=0.05)
    slots = synth.sft_slots(n_slots, n_slots // 10, synth.SEED_BASE + 80)
    X = torch.from_numpy(synth.sft_noise(len(slots), sd.n_bins, sd.sft_len, 1.0, synth.SEED_BASE + 81)).to(dev)
    t_sft = slots * t_len
    Xn = fs.fstat_sft_normalize(sd, X)
    a, d = synth.random_sky(64, synth.SEED_BASE + 82)
    desc = synth.tiny_plan(dt=0.5, n_data=n_slots * n1, n_fft=1 << 22, f_het=k_h / t_len, interp=synth.SINC,
                           taps=8, max_templates=64)
    plan = fs.Plan(desc, device=dev)
    tm = synth.make_templates(a, d, np.linspace(-1e-9, 0, 64), 0, desc.n_data)
    # demodulation
    n_t, n_q = 8, 65536
    q0 = desc.n_fft // 2 - n_q // 2
    td8 = fs.pack_templates(tm[:n_t], device=dev)
    tsd = torch.from_numpy(np.asarray(t_sft, np.float64)).to(dev)
    ws = torch.empty(int(plan.lib.fstat_sft_demod_workspace(len(slots), n_t)) + 256, dtype=torch.uint8, device=dev)
    out = torch.empty((n_t, n_q), dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 1)):
        fs.fstat_sft_demod(plan, sd, Xn, tsd, td8, q0, n_q, twoF=out, workspace=ws)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fs.fstat_sft_demod(plan, sd, Xn, tsd, td8, q0, n_q, twoF=out, workspace=ws)
    e1.record()
    torch.cuda.synchronize(dev)
    ms_dm = e0.elapsed_time(e1) / args.steps
    rc_dm = fs.fstat_status(plan, raise_error=False)
    dm_rate = n_t * n_q / (ms_dm / 1e3)
    # resampling on the series the front end makes from the same SFTs
    x = fs.fstat_sft_series(sd, X, t_sft, 0.0, desc.n_data)
    td = fs.pack_templates(tm, device=dev)
    two = torch.empty(64 * desc.n_fft, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 1)):
        fs.fstat_compute(plan, x, td, None, two)
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(args.steps):
        fs.fstat_compute(plan, x, td, None, two)
    e1.record()
    torch.cuda.synchronize(dev)
    ms_rs = e0.elapsed_time(e1) / args.steps
    rs_rate = 64 * desc.n_fft / (ms_rs / 1e3)
    print(json.dumps({
        "workload": "demod",
        "config": "10 d: 432 of 480 normalised 1800 s SFTs at 256 Hz, 3648 stored bins, f_h = 100 Hz; "
                  "demodulation with 2 x 16 + 1 Dirichlet terms; resampling on the front end's series "
                  "(N_d = 1,728,000, N = 2^22, 8-tap Lanczos)",
        "demod": {"templates": n_t, "bins": n_q, "ms": ms_dm, "two_f_values_per_s": dm_rate, "status": rc_dm},
        "resampling": {"templates": 64, "bins": desc.n_fft, "ms": ms_rs, "two_f_values_per_s": rs_rate},
        "speedup": rs_rate / dm_rate,
        "paper_op_count_estimate": {"n_sft_over_log2_n": len(slots) / 22.0,
                                    "note": "Sec. IV.A: ratio ~ N_SFTs / log N; the paper reports ~10 for "
                                            "Einstein@Home and up to ~2000 for multi-month searches"},
        "steps": args.steps, "warmup": args.warmup}))


def synth_chunks(t_sft, t_len):
    """Contiguous runs of SFT start times (host bookkeeping for the report)."""
    out, a = [], 0
    for i in range(1, len(t_sft) + 1):
        if i == len(t_sft) or abs(t_sft[i] - t_sft[i - 1] - t_len) > 1e-6:
            out.append((a, i - a))
            a = i
    return out


def run_montecarlo(args):
    """The paper's validation at its scale (Sec. IV.B: 2F is chi^2_4 in
    Gaussian noise, non-central chi^2_4 with a signal): R noise-only
    realizations of the 12 h configuration (86,400 samples, nearest
    neighbour, FFT 2^17), 4096 per call as consecutive spans of one series
    (one template per span), Gaussian noise drawn on the GPU from a seeded
    generator; reports the mean and variance of 2F and its tail
    probabilities against chi^2_4's closed forms and the rate (noise
    generation included); then R realizations with one injected signal
    each, standardized against the non-central chi^2_4."""
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300 import build as fsbuild
    fsbuild.build()
    dev = torch.device("cuda", 0)
    span, per = 86400, 4096
    total = max(per, (args.realizations // per) * per)
    desc = synth.tiny_plan(n_data=span * per, max_templates=per)
    plan = fs.Plan(desc, device=dev)
    a, d = synth.random_sky(1, synth.SEED_BASE + 33)
    tm = fs.pack_templates(synth.make_templates(np.repeat(a, per), float(d[0]), 0.0,
                                                np.arange(per) * span, span), device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.SEED_BASE + 34)
    raw = torch.empty(2 * span * per, dtype=torch.float32, device=dev)
    x = raw.view(torch.complex64)
    out = torch.empty(per * desc.n_fft, dtype=torch.float32, device=dev)
    thr = (10.0, 20.0, 30.0)
    acc = torch.zeros(6, dtype=torch.float64, device=dev)     # count, sum, sum of squares, tail counts
    hist_edges = 40                                           # unit-width bins of 2F on [0, 40)
    hist = torch.zeros(hist_edges, dtype=torch.float64, device=dev)
    scale = math.sqrt(desc.sigma2 / 2.0)

    def batch():
        raw.normal_(0.0, scale, generator=gen)
        fs.fstat_compute(plan, x, tm, None, out)
        fs.fstat_stats(out, acc, thr, hist, 1.0)                # one pass: moments, tails, histogram

    batch()                                   # warm-up (not counted)
    torch.cuda.synchronize(dev)
    acc.zero_()
    hist.zero_()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(total // per):
        batch()
    ev1.record()
    torch.cuda.synchronize(dev)
    rc = fs.fstat_status(plan, raise_error=False)
    ms = ev0.elapsed_time(ev1)
    n = float(acc[0])                                           # finite 2F values (all, unless a template failed)
    mean = float(acc[1]) / n
    var = float(acc[2]) / n - mean * mean
    tails = {f"P(2F>{int(t)})": {"measured": float(acc[3 + i]) / n,
                                 "chi2_4": math.exp(-t / 2) * (1 + t / 2)}
             for i, t in enumerate((10.0, 20.0, 30.0))}
    # histogram against chi^2_4: P(a <= 2F < a + 1) = G(a) - G(a + 1), G(x) = e^{-x/2}(1 + x/2)
    sf = [math.exp(-a / 2) * (1 + a / 2) for a in range(hist_edges + 1)]
    h = hist.cpu().numpy() / n
    p_bin = np.array([sf[a] - sf[a + 1] for a in range(hist_edges)])
    sig = np.sqrt(p_bin * (1 - p_bin) / n)
    noise_only = {"realizations": total, "two_f_values": float(total) * desc.n_fft, "finite_values": n, "ms": ms,
                  "two_f_values_per_s": float(total) * desc.n_fft / (ms / 1e3),
                  "mean": mean, "var": var, "chi2_4": {"mean": 4.0, "var": 8.0}, "tails": tails,
                  "histogram": {"bins": "unit width on [0, 40)",
                                "max_rel_dev_bins_0_20": float(np.max(np.abs(h[:20] / p_bin[:20] - 1))),
                                "max_dev_in_binomial_sigma": float(np.max(np.abs(h - p_bin) / sig)),
                                "note": "neighbouring bins of a zero-padded FFT are correlated, so the "
                                        "binomial sigma understates the scatter"}}

    # --- with signals: every realization carries one injection (isotropic
    # sky and orientation, h0 = args.mc_h0, frequency on bin q) added on the
    # GPU by fstat_inject and searched with its own template; the expected
    # non-centrality lambda is 2F of the noise-free injection at bin q
    # (resampling loss included), and z = (2F - lambda - 4) / sqrt(8 + 4 lambda)
    # has mean 0 and variance 1 for a non-central chi^2_4.
    q_off = 3000
    q = desc.n_fft // 2 + q_off
    df = q_off / (desc.n_fft * desc.dt)
    n_b = total // per
    recs = [synth.random_injection_records(per, synth.SEED_BASE + 1000 + b, df, args.mc_h0, span)
            for b in range(n_b)]
    inj_dev = torch.cat([fs.pack_injections(r, device=None)[0] for r in recs]).to(dev)
    tm_dev = torch.cat([fs.pack_templates(synth.make_templates(r["alpha"], r["delta"], 0.0, r["span_start"],
                                                               span), device=None) for r in recs]).to(dev)
    ib, tb = fs.INJECTION_DTYPE.itemsize * per, synth.TEMPLATE_DTYPE.itemsize * per
    sig = torch.empty(span * per, dtype=torch.complex64, device=dev)
    acc2 = torch.zeros(5, dtype=torch.float64, device=dev)   # sum z, sum z^2, sum (2F - 4), sum lambda, n(lambda > 0)
    f_all = torch.empty(n_b * per, dtype=torch.float64, device=dev)     # 2F and lambda at bin q, for the
    lam_all = torch.empty(n_b * per, dtype=torch.float64, device=dev)   # non-central histogram

    def sbatch(b):
        rb, tmb = inj_dev[b * ib:(b + 1) * ib], tm_dev[b * tb:(b + 1) * tb]
        sig.zero_()
        fs.fstat_inject(plan, sig, rb, span)
        fs.fstat_compute(plan, sig, tmb, None, out)
        lam = out.view(per, -1)[:, q].double()
        raw.normal_(0.0, scale, generator=gen)
        fs.fstat_inject(plan, x, rb, span)
        fs.fstat_compute(plan, x, tmb, None, out)
        f = out.view(per, -1)[:, q].double()
        z = (f - lam - 4.0) / torch.sqrt(8.0 + 4.0 * lam)
        acc2[0] += z.sum()
        acc2[1] += (z * z).sum()
        acc2[2] += (f - 4.0).sum()
        acc2[3] += lam.sum()
        acc2[4] += (lam > 0).sum()
        f_all[b * per:(b + 1) * per] = f
        lam_all[b * per:(b + 1) * per] = lam

    sbatch(0)                                 # warm-up (not counted)
    torch.cuda.synchronize(dev)
    acc2.zero_()
    ev0.record()
    for b in range(n_b):
        sbatch(b)
    ev1.record()
    torch.cuda.synchronize(dev)
    rc = rc or fs.fstat_status(plan, raise_error=False)
    ms2 = ev0.elapsed_time(ev1)
    zm = float(acc2[0]) / total
    # probability integral transform u = CDF_{ncx2(4, lambda)}(2F): uniform on
    # [0, 1) when 2F is non-central chi^2_4 with the noise-free 2F as lambda
    try:
        from scipy.stats import ncx2
        u = ncx2.cdf(f_all.cpu().numpy(), 4, lam_all.cpu().numpy())
        hu, _ = np.histogram(u, bins=20, range=(0.0, 1.0))
        pit = {"bins": 20, "max_rel_dev": float(np.max(np.abs(hu / (total / 20) - 1))),
               "binomial_rel_sigma": float(math.sqrt(19 / total)),
               "ks_stat": float(np.max(np.abs(np.sort(u) - (np.arange(total) + 0.5) / total)))}
    except ImportError:
        pit = None
    with_signal = {"realizations": total, "h0": args.mc_h0, "bin": q_off, "ms": ms2,
                   "mean_lambda": float(acc2[3]) / total,
                   "z_mean": zm, "z_var": float(acc2[1]) / total - zm * zm,
                   "sum_2F_minus_4_over_sum_lambda": float(acc2[2]) / float(acc2[3]),
                   "pit_histogram": pit,
                   "expected": {"z_mean": 0.0, "z_var": 1.0, "ratio": 1.0}}
    print(json.dumps({
        "workload": "montecarlo",
        "config": "12 h at dt = 0.5 s (86,400 samples), nearest neighbour, FFT 2^17, 4096 realizations "
                  "per call as consecutive spans of one series, noise drawn on the GPU; with signals: "
                  "injections by fstat_inject, lambda from the noise-free run",
        "noise_only": noise_only, "with_signal": with_signal, "status": rc}))


def run_batch(args):
    """The ragged batch: 4096 templates over one 10 d series, spans uniform in
    1-10 d, own gap lists (0-20 %), random sky, fdot in [-1e-9, 0], each with
    the FFT length next_pow2(N_b); one split-mode plan per FFT length
    (--mode split, the default) or one persistent launch (--mode
    persistent), both replayed from a CUDA graph.  Metric: sum of N_f over
    the batch / time."""
    import torch
    import paper_0912_4255_gb300 as fs
    from paper_0912_4255_gb300 import build as fsbuild
    from paper_0912_4255_gb300.batch import RaggedBatch
    fsbuild.build()
    dev = torch.device("cuda", 0)
    n = min(args.templates, 4096)
    desc = synth.batch_plan(max_templates=n)
    x_np = synth.complex_noise(desc.n_data, desc.sigma2, synth.SEED_BASE + 2)
    tm, gaps_np = synth.batch_templates(n, desc.n_data, desc.dt, synth.SEED_BASE + 2)
    probe = fs.Plan(desc.replace(max_templates=1), device=dev)
    nb = fs.fstat_template_nb(probe, tm)
    probe.close()
    nf = np.array([max(synth.next_pow2(int(v)), 1 << 12) for v in nb], np.int64)
    tm["n_fft"] = nf
    tm["out_off"] = np.concatenate([[0], np.cumsum(nf)[:-1]])
    x = torch.from_numpy(x_np.astype(np.complex64)).to(dev)
    gaps = torch.from_numpy(gaps_np.reshape(-1).copy()).to(dev)
    out = torch.empty(int(nf.sum()), dtype=torch.float32, device=dev)
    mode = "split" if args.mode == "split" else "persistent"
    if mode == "split":
        rb = RaggedBatch(desc, x, tm, gaps, out, device=dev, graph=True)
        run, stream, status = rb.run, rb.stream, rb.status
    else:
        plan = fs.Plan(desc.replace(n_fft=int(nf.max())), device=dev)
        plan.set_tuning(mode=fs.MODE_PERSISTENT)
        runner = fs.GraphRunner(plan, x, fs.pack_templates(tm, device=dev), gaps, out)
        run, stream = runner.replay, runner.stream
        status = lambda: fs.fstat_status(plan, stream, raise_error=False)
    for _ in range(max(1, args.warmup)):
        run()
    torch.cuda.synchronize(dev)
    clk = ClockSampler(0)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        run()
    ev1.record(stream)
    stream.synchronize()
    clocks = clk.stop()
    rc = status()
    ms = ev0.elapsed_time(ev1) / args.steps
    values = float(nf.sum())
    print(json.dumps({
        "metric": "2F values/sec (templates x freq bins) at rel err <= 1e-4",
        "value": values / (ms / 1e3), "unit": "2F values/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (f64 time map)", "data": "synthetic",
        "config": {"workload": f"ragged batch: {n} templates, spans 1-10 d of a 10 d series at dt=0.5 s, "
                               "own gap lists (0-20 %), FFT next_pow2(N_b) per template",
                   "mode": mode, "templates": n, "sum_n_fft": int(nf.sum()),
                   "n_fft_counts": {int(k): int(v) for k, v in zip(*np.unique(nf, return_counts=True))}},
        "status": rc, "clocks": clocks}))


def run_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores, each step a bounded sample of
    the workload (rank 0 only)."""
    if rank != 0:
        return
    desc, x, tm, gaps = workload(0, 1)
    cores = min(os.cpu_count() or 1, 8)
    per_step = cores          # one template per worker per step
    for _ in range(args.warmup if args.warmup < 1 else 1):
        cpu_oracle_rate(desc, x, tm, gaps, n_templates=per_step, workers=cores)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = cpu_oracle_rate(desc, x, tm, gaps, n_templates=per_step, workers=cores)
        vals.append(r["value"])
    wall = time.perf_counter() - t0
    value = per_step * desc.n_fft * args.steps / wall
    line = {
        "impl": "reference",
        "metric": "2F values/sec (templates x freq bins) at rel err <= 1e-4",
        "value": value, "unit": "2F values/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(desc, per_step, 1, precision=PRECISION_ORACLE),
        "cpu_baseline": {"value": value, "unit": "2F values/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} templates of the search-sized workload per step"},
        "e2e": {"value": value, "unit": "2F values/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
