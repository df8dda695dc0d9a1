"""Benchmark of the fused feature-extraction path on a 4-band 16384^2 uint16 scene.

A step is one pass of the whole path (LoG x2, zero crossings, contrast,
standard deviation, OR, hybrid median) over the 4 bands of a synthetic
multispectral scene (12-bit values, band by band, one fused launch per band).
Inputs are resident in HBM and larger than L2 (512 MiB per band).

Prints one JSON line.  Beyond metric, value, unit, timing, clocks and e2e:
  roofline    the fused kernel against the measured HBM copy bandwidth
  issue_roof  the same kernel against the SM issue rate (lane-instructions)
  batched     64 uneven scenes (uint8/uint16 mixed) in one persistent
              graph-replayed launch versus 64 plain launches
  cpu_baseline  the FP64 oracle on the host cores, on a bounded row sample

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SIDE = 16384
BANDS = 4
BYTES_PER_PX = 3  # one uint16 read + one uint8 mask write (algorithmic)
WORKLOAD = "4-band multispectral 16384x16384 uint16 (12-bit), band by band"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fx", choices=["fx", "reference"])
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-LoG mode measurement")
    ap.add_argument("--no-specialize", action="store_true",
                    help="time the precompiled first pass only (no fx_specialize)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the parameter variants (crossing-map source, median levels, grayscale median)")
    ap.add_argument("--side", type=int, default=SIDE, help="band side (default 16384)")
    ap.add_argument("--serve-duration", type=float, default=60.0,
                    help="seconds of the Poisson serving run at 200 requests/s (0 skips it)")
    ap.add_argument("--serve-burst", type=float, default=5.0,
                    help="seconds of a second serving run at a rate that keeps the GPU busy (0 skips it)")
    return ap.parse_args()


# ------------------------------------------------------------ CPU oracle

CPU_SAMPLE_ROWS = 4096  # rows of band 0 the oracle computes per CPU measurement


def oracle_sample(band: np.ndarray, rows: int, threads: int) -> dict:
    """The FP64 oracle as it stands on `rows` rows of one band, split in row
    chunks of at least 256 rows over `threads` host threads (each chunk
    recomputes its own halo rows, a few percent at 256 rows)."""
    import oracle
    oracle.build()
    p = oracle.default_params(16.0)
    y0 = (band.shape[0] - rows) // 2
    chunk = max(256, -(-rows // threads))
    spans = [(y, min(y + chunk, y0 + rows)) for y in range(y0, y0 + rows, chunk)]
    t = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda s: oracle.extract(band, p, rows=s), spans))
    dt = time.perf_counter() - t
    px = rows * band.shape[1]
    return {"px": px, "seconds": dt, "gpx_s": px / dt / 1e9}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) != 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- profiles

KERNEL_SOURCES = ("fx_internal.h", "fx_checked.cuh", "fx_stream.cuh", "fx_stream_kernels.cuh", "fx_stream.cu", "fx_jit.cpp")


def kernel_source_sha() -> str:
    """Hash of the files that define the timed kernel (the streaming path)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1304_3992_gb300", "csrc")
    for n in KERNEL_SOURCES:
        h.update(open(os.path.join(d, n), "rb").read())
    return h.hexdigest()


def profiled(kernel_key: str, field: str):
    """A numeric field of the committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_key}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256") != kernel_source_sha():
        return None
    try:
        return float(kv[field].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


def profiled_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary (None if stale)."""
    return profiled(kernel_key, "dram_bytes_per_launch_full_size")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured", d
    return 6800.0, "fallback", {}


# ----------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from gen import scenes
    band = next(scenes.ms_bands_u16_12bit(side=args.side, bands=[0]))
    cores = host_cores()
    rows = min(band.shape[0], CPU_SAMPLE_ROWS)  # the sample of the main arm's cpu_baseline
    times = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(band, rows, cores)
        if i >= args.warmup:
            times.append(r["seconds"])
    px = rows * band.shape[1]
    v = px * len(times) / sum(times) / 1e9
    line = {
        "impl": "reference", "metric": "fused extraction throughput", "value": v, "unit": "Gpixel/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "side": args.side, "bands": BANDS,
                   "sample": f"{rows} rows x {band.shape[1]} px of band 0 per step"},
        "cpu_baseline": {"value": v, "unit": "Gpixel/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows} rows x {band.shape[1]} px of band 0 per step, row chunks of at least "
                                   f"256 rows over {cores} threads"},
        "e2e": {"value": v, "unit": "Gpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ replicas

def max_over_ranks(value: float, device) -> float:
    """The slowest rank's time (replicas: every rank runs the same workload)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gpx_s(px_per_step_per_rank: int, steps: int, elapsed_ms: float, world: int) -> float:
    """Whole-job throughput: all ranks' pixels over the slowest rank's time."""
    return world * px_per_step_per_rank * steps / (elapsed_ms * 1e-3) / 1e9


# ------------------------------------------------------------------ main

def time_band(torch, stream, call, px, warmup=3, reps=10):
    """Median event-timed duration of call() (one band) on stream."""
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    ms.sort()
    m = ms[len(ms) // 2]
    return {"ms_per_band": round(m, 4), "gpx_s": round(px / m / 1e6, 1)}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from gen import scenes
    from paper_1304_3992_gb300 import fx

    # ---- workload: 4 bands resident in HBM
    bands_np = list(scenes.ms_bands_u16_12bit(side=args.side))
    bands = [torch.from_numpy(b).to(dev) for b in bands_np]
    outs = [torch.empty(b.shape, dtype=torch.uint8, device=dev) for b in bands]
    params = fx.make_params(fx.FX_U16, 12)
    stream = torch.cuda.current_stream()
    px_step = sum(b.numel() for b in bands)

    def step(ev=None):
        for i, (b, o) in enumerate(zip(bands, outs)):
            if ev is not None:
                ev[2 * i].record(stream)
            fx.extract(b, params, out=o, stream=stream)
            if ev is not None:
                ev[2 * i + 1].record(stream)

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- the precompiled first pass, timed on band 0 before the specialisation
    generic = None
    if not args.no_specialize:
        generic = time_band(torch, stream, lambda: fx.extract(bands[0], params, out=outs[0], stream=stream),
                            bands[0].numel())
    # the first pass compiled at run time with these parameters' masks and
    # contrast thresholds as constants (fx_specialize, cached per process);
    # its masks are the precompiled kernel's
    specialized = False
    if not args.no_specialize:
        t0 = time.perf_counter()
        # uint16 for the bands, uint8 too for the batched scenes and the server
        specialized = fx.specialize(params, fx.FX_U16) and fx.specialize(params, fx.FX_U8)
        if generic is not None:
            generic["specialize_s"] = round(time.perf_counter() - t0, 2)
            ref0 = outs[0].clone()
            fx.extract(bands[0], params, out=outs[0], stream=stream)
            torch.cuda.synchronize()
            generic["identical_masks"] = bool(torch.equal(ref0, outs[0]))

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    K = args.steps
    launch_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2 * BANDS)] for _ in range(K)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(K):
            step(launch_ev[k])
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    elapsed_ms = e0.elapsed_time(e1)
    launch_ms = [launch_ev[k][2 * i].elapsed_time(launch_ev[k][2 * i + 1]) for k in range(K) for i in range(BANDS)]
    elapsed_ms = max_over_ranks(elapsed_ms, dev)
    value = aggregate_gpx_s(px_step, K, elapsed_ms, world)

    # ---- the FP32-LoG mode (non-integer masks) on the same bands
    fp32 = None
    if not args.no_fp32:
        fp32 = bench_fp32_log(fx, torch, stream, bands, outs, max(3, args.warmup), min(K, 10))

    # ---- parameter variants and the grayscale median op on band 0
    variants = None
    if not args.no_variants:
        variants = bench_variants(fx, torch, stream, bands[0], outs[0], bands_np[0])

    # ---- end to end through the C ABI on pinned host buffers
    h_in = [torch.from_numpy(b).pin_memory() for b in bands_np]
    h_out = [torch.empty(b.shape, dtype=torch.uint8).pin_memory() for b in bands_np]
    plan = fx.Plan(params, max_images=BANDS, device=local)
    host_pairs = [(h_in[i].numpy(), h_out[i].numpy()) for i in range(BANDS)]
    plan.extract_host_batch(host_pairs)  # warm-up: grows the staging buffers
    ke = max(1, min(K, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):  # one call per step: the four bands through one copy/kernel/copy pipeline
        plan.extract_host_batch(host_pairs)
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_ok = all(torch.equal(h_out[i].to(dev), outs[i]) for i in range(BANDS))
    e2e = {"value": world * px_step * ke / e2e_s / 1e9, "unit": "Gpixel/s",
           "h2d_bytes_per_step": sum(b.nbytes for b in bands_np),
           "d2h_bytes_per_step": sum(b.size for b in bands_np), "matches_device_path": bool(e2e_ok),
           "call": "fx_extract_host_batch (pinned host buffers, 4 bands per call)"}

    # ---- batched persistent launch vs 64 plain launches (uneven scenes)
    batched = None
    if not args.no_batch:
        batched = bench_batched(fx, torch, dev, params, plan_cls=fx.Plan)
    plan.close()

    # ---- continuous-batching server under a Poisson stream
    serving = None
    if args.serve_duration > 0:
        serving = bench_serving(fx, torch, dev, params, bands_np[0], args.serve_duration)
    if args.serve_burst > 0:
        burst = bench_serving(fx, torch, dev, params, bands_np[0], args.serve_burst, rate_hz=BURST_RATE_HZ,
                              check_every=500)
        serving = serving or {}
        serving["saturated"] = burst

    # ---- roofline of the fused kernel
    peak, peak_src, _ = peaks()
    avg_launch_ms = sum(launch_ms) / len(launch_ms)
    px_launch = bands[0].numel()
    achieved = BYTES_PER_PX * px_launch / (avg_launch_ms * 1e-3) / 1e9
    traffic = profiled_traffic("fused_extract_16384_u16")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "algorithmic_bytes_per_launch": BYTES_PER_PX * px_launch,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs copy)" if peak_src == "measured" else peak_src,
            "kernel_ms": avg_launch_ms}
    props = torch.cuda.get_device_properties(dev)
    clk = clocks.summary()
    mhz = clk["sm_mhz"] or 1900.0
    issue_peak = props.multi_processor_count * 128 * mhz * 1e6  # lane-instructions/s
    px_per_s = px_launch / (avg_launch_ms * 1e-3)
    issue = {"sm_count": props.multi_processor_count, "sm_mhz": mhz,
             "peak_lane_inst_per_s": issue_peak,
             "lane_inst_per_px_at_roof": issue_peak / px_per_s}
    ipp = profiled("fused_extract_16384_u16", "lane_inst_per_px")
    if ipp is not None:  # lane-instructions per pixel from the committed ncu summary
        issue.update({"lane_inst_per_px": ipp, "achieved_lane_inst_per_s": px_per_s * ipp,
                      "frac": px_per_s * ipp / issue_peak})

    cpu = None
    if rank == 0 and not args.no_cpu:
        cores = host_cores()
        rows = min(bands_np[0].shape[0], CPU_SAMPLE_ROWS)
        r = oracle_sample(bands_np[0], rows, cores)
        cpu = {"value": r["gpx_s"], "unit": "Gpixel/s", "cores": cores, "kind": "oracle",
               "sample": f"{rows} rows x {args.side} px of band 0 ({r['px']} px, {r['seconds']:.1f} s wall), "
                         f"row chunks of at least 256 rows over {cores} threads"}

    if rank == 0:
        line = {
            "metric": "fused extraction throughput", "value": value, "unit": "Gpixel/s", "n_gpus": world,
            "steps": K, "warmup": max(3, args.warmup), "ms_per_step": elapsed_ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32-exact/int32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "side": args.side, "bands": BANDS, "values": "12-bit",
                       "launch": "fx_extract per band (streaming kernel + integer redo check)",
                       "specialized": specialized,
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (512 MiB per band)"},
            "roofline": roof, "issue_roof": issue, "cpu_baseline": cpu, "e2e": e2e,
            # per band: the streaming kernel and the integer redo check (12-bit data
            # is within the FP32-exact bound, so the redo kernel only reads markers)
            "gpu_launches": K * BANDS * 2, "clocks": clk, "batched": batched, "serving": serving,
            "fp32_log": fp32, "variants": variants, "precompiled_kernel": generic,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def bench_fp32_log(fx, torch, stream, bands, outs_int, warmup, steps):
    """fx_extract in the FP32-LoG mode (non-integer masks, FP32 responses) over
    the same bands: throughput, mean kernel-pair time per band, and the share of
    pixels whose mask differs from the integer-mask mode (different masks, so
    some differ by design)."""
    p32 = fx.make_params(fx.FX_U16, 12, log_mode=fx.FX_LOG_FP32)
    outs = [torch.empty_like(o) for o in outs_int]
    for _ in range(warmup):
        for b, o in zip(bands, outs):
            fx.extract(b, p32, out=o, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps * len(bands))]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        for i, (b, o) in enumerate(zip(bands, outs)):
            ev[k * len(bands) + i][0].record(stream)
            fx.extract(b, p32, out=o, stream=stream)
            ev[k * len(bands) + i][1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    px = sum(b.numel() for b in bands)
    diff = sum(int((a != b).sum()) for a, b in zip(outs, outs_int))
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"gpx_s": px * steps / (e0.elapsed_time(e1) * 1e-3) / 1e9, "kernel_ms": sum(ms) / len(ms),
            "steps": steps, "differs_from_integer_mode": diff / px,
            "launch": "fx_extract per band, log_mode FX_LOG_FP32 (FP32 pass + wide-pass marker check)"}


def bench_variants(fx, torch, stream, band, out, band_np, reps=5):
    """Throughput of fx_extract on one band for the parameter variants (which
    kernel runs them is recorded), on the same band scaled to the full 16-bit
    range (above the FP32-exact bound: the integer pass computes it), and of
    the grayscale hybrid median op."""
    base = dict(sigma=(0.5, 20.0), mask_q=512)
    cases = {
        "median_off": (dict(hmf=()), "streaming"),
        "median_3": (dict(hmf=(3,)), "streaming"),
        "median_5_then_3": (dict(hmf=(5, 3)), "streaming"),
        "median_7": (dict(hmf=(7,)), "streaming"),
        "median_5_then_5": (dict(hmf=(5, 5)), "streaming, wide strips"),
        "median_7_5_3": (dict(hmf=(7, 5, 3)), "streaming, wide strips"),
        "median_7_7_7": (dict(hmf=(7, 7, 7)), "streaming, extra-wide strips"),
        "median_7_7_7_7": (dict(hmf=(7, 7, 7, 7)), "general tile"),
        "stddev_over_crossing_map": (dict(stddev_source=1, t_sd5=(0.2, 0.3), t_sdmax=(0.45, 0.5),
                                          t_sd3=(0.3, 0.4)), "streaming"),
    }
    px = band.numel()
    res = {}
    out = torch.empty_like(out)  # scratch: the caller's masks stay those of the default parameters

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return sorted(ms)[len(ms) // 2]

    for name, (kw, kernel) in cases.items():
        p = fx.make_params(fx.FX_U16, 12, **kw)
        ms = timed(lambda: fx.extract(band, p, out=out, stream=stream))
        res[name] = {"gpx_s": px / ms / 1e6, "ms": ms, "kernel": kernel}
    wide = torch.from_numpy(band_np * np.uint16(16)).to(band.device)  # values up to 65520
    p16 = fx.make_params(fx.FX_U16, 16)
    ms = timed(lambda: fx.extract(wide, p16, out=out, stream=stream))
    res["full_range_16bit"] = {"gpx_s": px / ms / 1e6, "ms": ms,
                               "kernel": "streaming first pass (stops at the first block) + integer pass"}
    del wide
    med = torch.empty_like(band)
    for w in (3, 5, 7):
        ms = timed(lambda: fx.hybrid_median(band, w, out=med, stream=stream))
        res[f"grayscale_median_{w}"] = {"gpx_s": px / ms / 1e6, "ms": ms, "kernel": "median tile",
                                        "gb_s": 4 * px / ms / 1e6}
    res["workload"] = f"one {band.shape[0]}x{band.shape[1]} uint16 12-bit band, median of {reps} timed calls"
    return res


def bench_batched(fx, torch, dev, params, plan_cls):
    from gen import scenes
    batch = scenes.uneven_batch(n=64)
    imgs, outs = [], []
    for view, buf in batch:
        t = torch.from_numpy(buf).to(dev)
        imgs.append(t[:, :view.shape[1]])
        outs.append(torch.empty(view.shape, dtype=torch.uint8, device=dev))
    pairs = list(zip(imgs, outs))
    px = sum(o.numel() for o in outs)
    stream = torch.cuda.current_stream()
    plan = plan_cls(params, max_images=64, device=dev.index or 0)
    tuned = plan.autotune(pairs)

    def time_it(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = 1e30
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    t_batch = time_it(lambda: plan.extract_batch(pairs))
    ref = [o.clone() for o in outs]
    t_plain = time_it(lambda: [fx.extract(i, params, out=o) for i, o in pairs])
    same = all(torch.equal(a, b) for a, b in zip(ref, outs))
    plan.close()
    return {"scenes": 64, "pixels": px, "batched_gpx_s": px / t_batch / 1e6,
            "one_by_one_gpx_s": px / t_plain / 1e6, "speedup": t_plain / t_batch,
            "identical_output": bool(same),
            "tile": {"w": tuned[0], "h": tuned[1] or "automatic", "ctas_per_sm": tuned[2]}}


BURST_RATE_HZ = 4000.0  # well above what the GPU finishes (about 10 requests per ms of copies and kernels)


def bench_serving(fx, torch, dev, params, master16, duration, rate_hz=200.0, check_every=50):
    """Poisson stream (200 req/s by default) of single-band scenes with sides
    log-uniform in [512, 16384] px, uint8/uint16 alternating, cropped from two
    16384^2 masters into a pool of 48 pinned requests; 40 GB HBM budget; masks
    released as soon as they complete.  Every check_every-th served mask is
    compared byte for byte with a lone fx_extract call on the same image.  At
    200 req/s the offered load (about 3.6 Gpx/s) keeps the GPU a few percent
    busy, so most requests find it idle and run alone; at BURST_RATE_HZ
    requests queue up and are batched as they arrive."""
    from gen import scenes
    from paper_1304_3992_gb300.serve import Server, TorchBackend, run_stream
    rng = np.random.default_rng(7)
    side = master16.shape[0]
    master8 = scenes.scene(side, side, seed=8, n_rects=int(40 * side * side / 512 ** 2), noise_sigma=4.0,
                           impulse_frac=0.01, bits=8)
    pool = []
    for i in range(48):
        h, w = (int(round(float(np.exp(rng.uniform(np.log(512), np.log(side)))))) for _ in range(2))
        y0, x0 = int(rng.integers(0, side - h + 1)), int(rng.integers(0, side - w + 1))
        src = master8 if i % 2 == 0 else master16
        pool.append(torch.from_numpy(np.ascontiguousarray(src[y0:y0 + h, x0:x0 + w])).pin_memory().numpy())
    be = TorchBackend(params, slots=2, max_images=64, device=dev.index or 0)
    server = Server(be, budget_bytes=40 * 10**9, max_batch=64)
    checks = {}

    def keep(r):
        if r.rid % check_every == 0:
            checks[r.rid] = (r.image, r.dev["out"].cpu())

    reqs = run_stream(server, pool, rate_hz=rate_hz, duration_s=duration, seed=7, on_done=keep)
    st = server.stats()
    same = all(torch.equal(fx.extract(torch.from_numpy(im).to(dev), params).cpu(), out)
               for im, out in checks.values())
    be.close()
    offered = sum(r.pixels for r in reqs) / duration / 1e9
    st.update({"duration_s": duration, "rate_hz": rate_hz, "offered_gpx_s": offered,
               "budget_gb": 40, "verified_requests": len(checks), "identical_to_alone": bool(same),
               "latency": "arrival to device-side completion of the request's batch"})
    return st


if __name__ == "__main__":
    main()
