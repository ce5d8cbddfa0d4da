"""Throughput benchmark: voxel-view updates per second of the efficient
Bayesian multi-view update on GB300, through the library's C ABI.

Default workload: 256x256x128 volume, 4 views at 0/90/180/270 deg about y,
15x15x41 PSFs (sigma 1.2/4), 3000 ellipsoids, Poisson noise at peak 100
photons, 20 sequential (OSEM-order) iterations of the efficient method.

One step = one deconvolution of that volume: psi reset to the flat estimate,
then 20 iterations x 4 view updates (views and kernel spectra resident in
HBM; the PSFs of a time series are fixed, so kernels are precomputed once).
value = voxels * views * iterations / step time, in Gvoxel-view/s.
e2e = the same metric through the public API from pinned host buffers, for
a time series with fixed PSFs: load the views (H2D) into the context,
iterate, copy the result back (D2H); e2e.cold_value also builds and tears
down the context (create + precompute + destroy) in every step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank deconvolves its own independent volume (another
time point of the same acquisition): weak scaling, no collective on the data
path; barrier + max over ranks around the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gvoxel-view updates/s"
UNIT = "Gvoxel-view/s"
L2_BYTES = 129 * 2 ** 20

# algorithmic bytes per voxel for each update kernel: every input and output
# array it must touch, once (half spectrum = 8 * (X/2+1) * Y * Z bytes)
def _kernel_bytes(X, Y, Z, precise=True):
    M = X * Y * Z
    spec = 8 * (X // 2 + 1) * Y * Z  # FP32 half spectrum; double-float is 2 * spec
    if precise:  # the update reads the double-float spectrum
        return {
            "dd_x_forward": 4 * M + 2 * spec,       # read psi, write S2
            "dd_y": 4 * spec,                       # read S2, write S2
            "dd_z_mul": 6 * spec,                   # read S2 and a double-float kernel spectrum, write S2
            "dd_x_ratio": 4 * spec + 4 * M,         # read S2 and phi, write S2
            "x_update": 2 * spec + 8 * M,           # read S2, read and write psi
        }
    return {
        "x_forward": 4 * M + spec,          # read psi, write S
        "y": 2 * spec,                      # read S, write S
        "z_mul": 3 * spec,                  # read S and the kernel spectrum, write S
        "x_ratio": 2 * spec + 4 * M,        # read S and phi, write S
        "x_update": spec + 8 * M,           # read S and psi, write psi
        "direct_ratio": 12 * M,             # read psi and phi, write r
        "direct_update": 12 * M,            # read r and psi, write psi
    }


# FP32-ALU work model of the double-float kernels (ALU-bound): one op = one FP32
# add, multiply or FMA instruction. A double-float add costs 8 ops (TwoSum and two
# adds), a double-float multiply 7 (product, three FMAs, FastTwoSum), a complex
# double-float multiply 38 (two fused dot products of 19); a complex FFT of
# length N is counted as the radix-2 algorithm's 3 N log2 N real adds and
# 2 N log2 N real multiplies, i.e. 38 N log2 N ops in double-float and 5 N log2 N
# in FP32.
DD_FFT_OPS = 38.0
FP32_FFT_OPS = 5.0
DD_CMUL_OPS = 38.0
FP32_CMUL_OPS = 6.0


def _kernel_alu_ops(X, Y, Z):
    import math

    Xh = X // 2 + 1
    dd = lambda n: DD_FFT_OPS * n * math.log2(n)  # noqa: E731
    f32 = lambda n: FP32_FFT_OPS * n * math.log2(n)  # noqa: E731
    return {
        "dd_x_forward": (Y * Z / 2) * dd(X),                  # two real rows per complex line
        "dd_y": Xh * Z * dd(Y),
        "dd_z_mul": Xh * Y * (2 * dd(Z) + DD_CMUL_OPS * Z),  # forward, times the spectrum, inverse
        "dd_x_ratio": (Y * Z / 2) * (dd(X) + f32(X)),         # inverse in double-float, r - 1 forward in FP32
        "y": Xh * Z * f32(Y),
        "z_mul": Xh * Y * (2 * f32(Z) + FP32_CMUL_OPS * Z),
        "x_update": (Y * Z / 2) * f32(X),
    }


def _alu_peak_tops(sms=152, sm_mhz=2070.0):
    """FP32 instruction peak: 128 FP32 lanes per SM, one instruction per lane per clock."""
    return sms * 128 * sm_mhz * 1e6 / 1e12


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _workload_seed(rank: int) -> int:
    """Each rank deconvolves its own independent volume (weak scaling, no data-path collective)."""
    return 1002 + 1000 * rank


def _workload(rank: int):
    import synth

    return synth.config2(seed=_workload_seed(rank))


def _max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's figure (timings are reported as the maximum over ranks)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput in Gvoxel-view/s: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds / 1e9


def _cpu_baseline(w, eps, steps=1):
    """FP64 oracle on the host cores: one view update of the workload per step."""
    import oracle

    psfs64 = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    K = oracle.compound(psfs64, 0, "efficient")
    psi = np.full(w.truth.shape, float(np.mean([v.mean(dtype=np.float64) for v in w.views])))
    phi = w.views[0].astype(np.float64)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.update(psi, phi, psfs64[0], K, eps)
        times.append(time.perf_counter() - t0)
    return times, oracle.num_threads()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = _workload(0)
    eps = 1e-4 * float(np.mean([v.mean(dtype=np.float64) for v in w.views]))
    _cpu_baseline(w, eps, steps=args.warmup) if args.warmup > 0 else None
    times, cores = _cpu_baseline(w, eps, steps=args.steps)
    total = sum(times)
    value = w.voxels * args.steps / total / 1e9
    sample = (f"one view update (view 0) of the {w.dims[0]}x{w.dims[1]}x{w.dims[2]} 4-view workload per step, "
              f"FP64 direct convolution")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "volume": list(w.dims), "views": w.n_views, "psf_box": [15, 15, 41],
                   "iterations": w.n_iter, "variant": "efficient"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd

    w = _workload(rank)
    X, Y, Z = w.dims
    M = w.voxels
    stream = torch.cuda.Stream()
    upd_per_step = w.n_views * w.n_iter
    units_per_step = M * upd_per_step

    # --- device-resident run (value) ---
    with torch.cuda.stream(stream):
        dviews = [torch.from_numpy(v).to(f"cuda:{local}", non_blocking=False) for v in w.views]
    stream.synchronize()
    d = mvd.Deconvolver(dviews, w.psfs, "efficient", stream=stream, path="fft", device=local)

    def step():
        d.set_estimate(None)
        d.iterate(w.n_iter)

    for _ in range(args.warmup):
        step()
    d.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = mvd.mvd_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        ev1.synchronize()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = mvd.mvd_launch_count() - launches0
    # per-kernel durations: the same K steps again with CUDA events around
    # every launch on the launching stream (kernels launched one by one)
    mvd.mvd_profile_enable(True)
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        step()
    ev3.record(stream)
    ev3.synchronize()
    prof = mvd.mvd_profile_read()
    mvd.mvd_profile_enable(False)
    ms_profiled = ev2.elapsed_time(ev3)
    t_max = _max_over_ranks(ms, dist, f"cuda:{local}")
    psi_dev = d.result()
    d.close()

    if args.quick:  # device-resident timing only (used for profiler captures)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": _job_value(ws, units_per_step * args.steps, t_max * 1e-3),
                              "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": t_max / args.steps, "quick": True,
                              "config": {"workload": w.name}}), flush=True)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # the same steps with every pass in FP32 (MVD_FAST), for comparison
    fast = mvd.Deconvolver(dviews, w.psfs, "efficient", stream=stream, path="fft", device=local, precision="fast")

    def fast_step():
        fast.set_estimate(None)
        fast.iterate(w.n_iter)

    for _ in range(args.warmup):
        fast_step()
    ev4 = torch.cuda.Event(enable_timing=True)
    ev5 = torch.cuda.Event(enable_timing=True)
    ev4.record(stream)
    for _ in range(args.steps):
        fast_step()
    ev5.record(stream)
    ev5.synchronize()
    ms_fast = ev4.elapsed_time(ev5)
    psi_fast = fast.result()
    # per-kernel events of the FP32 passes (HBM-bound): one more step, launched one by one
    mvd.mvd_profile_enable(True)
    fast_step()
    fast.synchronize()
    prof_fast = mvd.mvd_profile_read()
    mvd.mvd_profile_enable(False)
    fast.close()

    # the same steps with the FP32 back-projection (MVD_MIXED), for comparison
    mixed = mvd.Deconvolver(dviews, w.psfs, "efficient", stream=stream, path="fft", device=local, precision="mixed")

    def mixed_step():
        mixed.set_estimate(None)
        mixed.iterate(w.n_iter)

    for _ in range(args.warmup):
        mixed_step()
    ev6 = torch.cuda.Event(enable_timing=True)
    ev7 = torch.cuda.Event(enable_timing=True)
    ev6.record(stream)
    for _ in range(args.steps):
        mixed_step()
    ev7.record(stream)
    ev7.synchronize()
    ms_mixed = ev6.elapsed_time(ev7)
    psi_mixed = mixed.result()
    mixed.close()

    # --- end to end through the public API from pinned host buffers ---
    # A time series with fixed PSFs: one context; every step loads the time
    # point's views from pinned host memory (mvd_set_views: H2D, view mean,
    # flat estimate), runs the 20 iterations and copies the result back.
    # "cold" builds and tears down a whole context per step instead.
    pinned = [torch.from_numpy(v).pin_memory() for v in w.views]
    hviews = [p.numpy() for p in pinned]
    out = torch.empty(w.truth.shape, dtype=torch.float32).pin_memory().numpy()
    series = mvd.Deconvolver(hviews, w.psfs, "efficient", stream=stream, path="fft", device=local)

    def e2e_step():
        series.set_views(hviews)
        series.iterate(w.n_iter)
        series.result(out)

    def cold_step():
        with mvd.Deconvolver(hviews, w.psfs, "efficient", stream=stream, path="fft", device=local) as e:
            e.iterate(w.n_iter)
            e.result(out)

    def timed(step, n):
        step()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            step()
        torch.cuda.synchronize()
        return _max_over_ranks((time.perf_counter() - t0) / n, dist, f"cuda:{local}")

    e2e_s = timed(e2e_step, max(1, args.steps))
    assert np.allclose(out, psi_dev, rtol=1e-6, atol=0), "end-to-end result differs from the device run"
    series.close()
    cold_s = timed(cold_step, max(1, min(args.steps, 5)))
    assert np.allclose(out, psi_dev, rtol=1e-6, atol=0), "end-to-end result differs from the device run"

    if rank == 0:
        peak, peak_kind = _peaks()
        kb = _kernel_bytes(X, Y, Z)
        per_kernel = {}
        for name, (n, tot) in prof.items():
            if n and name in kb:
                per_kernel[name] = {"launches": n, "avg_us": 1e3 * tot / n, "share": tot / max(1e-9, sum(
                    t for (_, t) in prof.values())), "GBps": kb[name] / (tot / n * 1e-3) / 1e9}
        ops = _kernel_alu_ops(X, Y, Z)
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        alu_peak = _alu_peak_tops(sms)
        for name, rec in per_kernel.items():
            if name in ops:
                rec["alu_Tops"] = ops[name] / (rec["avg_us"] * 1e-6) / 1e12
                rec["alu_frac"] = rec["alu_Tops"] / alu_peak
            rec["hbm_frac"] = rec["GBps"] / peak
        dom = max(per_kernel, key=lambda k: prof[k][1])
        traffic = None
        tf = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tf):
            with open(tf) as fh:
                tr = json.load(fh)
            key = f"{dom}@{X}x{Y}x{Z}"
            traffic = tr.get(key)
        if dom.startswith("dd_"):  # issue-bound on the FP32 pipes (see profiles/)
            roofline = {"bound": "alu", "kernel": dom, "achieved": per_kernel[dom]["alu_Tops"], "peak": alu_peak,
                        "unit": "T FP32 ops/s", "frac": per_kernel[dom]["alu_Tops"] / alu_peak,
                        "traffic": traffic, "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2070 MHz",
                        "hbm_frac_same_kernel": per_kernel[dom]["hbm_frac"]}
        else:
            roofline = {"bound": "hbm", "kernel": dom, "achieved": per_kernel[dom]["GBps"], "peak": peak,
                        "unit": "GB/s", "frac": per_kernel[dom]["GBps"] / peak, "traffic": traffic,
                        "peak_source": peak_kind}
        kbf = _kernel_bytes(X, Y, Z, precise=False)
        tot_fast = sum(t for (_, t) in prof_fast.values())
        fast_kernels = {}
        for name, (n, tot) in prof_fast.items():
            if n and name in kbf:
                gbps = kbf[name] / (tot / n * 1e-3) / 1e9
                fast_kernels[name] = {"launches": n, "avg_us": 1e3 * tot / n, "share": tot / max(1e-9, tot_fast),
                                      "GBps": gbps, "hbm_frac": gbps / peak}
        fast_roof = None
        if fast_kernels:
            fd = max(fast_kernels, key=lambda k: prof_fast[k][1])
            fast_roof = {"bound": "hbm", "kernel": fd, "achieved": fast_kernels[fd]["GBps"], "peak": peak,
                         "unit": "GB/s", "frac": fast_kernels[fd]["hbm_frac"], "traffic": None,
                         "peak_source": peak_kind}
        value = _job_value(ws, units_per_step * args.steps, t_max * 1e-3)
        # about 10 s of host work: view updates of the same workload, one after another
        cpu_times, cores = _cpu_baseline(w, 1e-4 * float(np.mean([v.mean(dtype=np.float64) for v in w.views])),
                                         steps=5)
        cpu_value = M * len(cpu_times) / sum(cpu_times) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "volume": [X, Y, Z], "views": w.n_views,
                       "psf_box": [15, 15, 41], "iterations": w.n_iter, "variant": "efficient",
                       "engine": "fft", "l2": "inputs larger than L2 (views + kernel spectra "
                       f"{(4 * M * w.n_views + 16 * (X // 2 + 1) * Y * Z * w.n_views) / 2**20:.0f} MiB > 129 MiB)",
                       "parallelism": f"replicas x{ws}"},
            "e2e": {"value": _job_value(ws, units_per_step, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(v.nbytes for v in w.views)),
                    "d2h_bytes_per_step": int(out.nbytes),
                    "per_step": "time series with fixed PSFs: load the views from pinned host memory "
                                "(mvd_set_views), 20 iterations, result to pinned host memory; kernels "
                                "precomputed once for the series",
                    "cold_value": _job_value(ws, units_per_step, cold_s),
                    "cold_per_step": "create (views H2D) + precompute + iterate + result (D2H) + destroy"},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "update_effective_hbm_frac": (12.0 * units_per_step * args.steps / (ms * 1e-3) / 1e9) / peak,
            "kernels": per_kernel,
            "profiled_ms_per_step": ms_profiled / args.steps,
            "precision": "double-float (pairs of FP32) for the forward blur and the back-projection's y and z passes; FP32 x passes of the back-projection",
            "fast_fp32": {"value": ws * units_per_step * args.steps / (ms_fast * 1e-3) / 1e9, "unit": UNIT,
                          "ms_per_step": ms_fast / args.steps,
                          "kernels": fast_kernels, "roofline": fast_roof,
                          "max_rel_diff_vs_precise": float(np.max(np.abs(psi_fast.astype(np.float64) - psi_dev)
                                                                  / np.maximum(np.abs(psi_dev.astype(np.float64)),
                                                                               1e-3 * np.abs(psi_dev).max())))},
            "mixed": {"value": ws * units_per_step * args.steps / (ms_mixed * 1e-3) / 1e9, "unit": UNIT,
                      "ms_per_step": ms_mixed / args.steps,
                      "precision": "double-float forward blur, FP32 back-projection (not held to 1e-4)",
                      "max_rel_diff_vs_precise": float(np.max(np.abs(psi_mixed.astype(np.float64) - psi_dev)
                                                              / np.maximum(np.abs(psi_dev.astype(np.float64)),
                                                                           1e-3 * np.abs(psi_dev).max())))},
            "clocks": clk.summary(),
            "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(cpu_times)} view updates (view 0) of the {X}x{Y}x{Z} workload, "
                                       f"FP64 direct convolution, {sum(cpu_times):.1f} s"},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """48 volumes of uneven size and view count (15 iterations each): one persistent
    batched launch vs the same volumes deconvolved one after another."""
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd

    t0 = time.perf_counter()
    ws = synth.config4()
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    ds = []
    for w in ws:
        with torch.cuda.stream(stream):
            dv = [torch.from_numpy(v).cuda() for v in w.views]
        stream.synchronize()
        ds.append(mvd.Deconvolver(dv, w.psfs, "efficient", path="fft", stream=stream))
    n_iter = ws[0].n_iter
    units = sum(w.voxels * w.n_views * n_iter for w in ws)

    def reset():
        for d in ds:
            d.set_estimate(None)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # plain: one volume after another (each replays its own per-iteration graph)
    for _ in range(max(1, args.warmup)):
        reset()
        for d in ds:
            d.iterate(n_iter)
    plain_ms = []
    for _ in range(args.steps):
        reset()
        ev0.record(stream)
        for d in ds:
            d.iterate(n_iter)
        ev1.record(stream)
        ev1.synchronize()
        plain_ms.append(ev0.elapsed_time(ev1))
    plain_res = [d.result() for d in ds]

    def time_batch(mode):
        b = mvd.mvd_batch_create(ds, n_iter, mode)
        for _ in range(max(1, args.warmup)):
            reset()
            mvd.mvd_batch_run(b)
            mvd.mvd_batch_wait(b)
        ms = []
        launches0 = mvd.mvd_launch_count()
        with ClockSampler(torch.cuda.current_device()) as clk:
            for _ in range(args.steps):
                reset()
                ev0.record(stream)
                mvd.mvd_batch_run(b)
                ev1.record(stream)
                ev1.synchronize()
                ms.append(ev0.elapsed_time(ev1))
        mvd.mvd_batch_wait(b)
        launches = (mvd.mvd_launch_count() - launches0) / args.steps
        res = [d.result() for d in ds]
        tasks = mvd.mvd_batch_tasks(b)
        mvd.mvd_batch_destroy(b)
        return statistics.median(ms), res, tasks, launches, clk.summary()

    per_ms, per_res, per_tasks, _, _ = time_batch("persistent")
    batch_ms_med, batch_res, tasks, launches, clocks = time_batch("branches")
    for d in ds:
        d.close()
    errs = []
    for p, q, r in zip(plain_res, batch_res, per_res):
        p64 = p.astype(np.float64)
        tau = 1e-3 * np.abs(p64).max()
        errs.append(float(np.max(np.abs(q - p64) / np.maximum(np.abs(p64), tau))))
        errs.append(float(np.max(np.abs(r - p64) / np.maximum(np.abs(p64), tau))))
    pm, bm = statistics.median(plain_ms), batch_ms_med
    line = {
        "metric": METRIC, "value": units / (bm * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": bm, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch of {len(ws)} volumes (48^3 to 320x320x192, 2-6 views, 15 iterations)",
                   "voxels": int(sum(w.voxels for w in ws)), "voxel_view_updates": int(units),
                   "engine": "fft", "batch_mode": "branches", "l2": "inputs larger than L2"},
        "batched_vs_plain": {"batched_ms": bm, "plain_ms": pm, "speedup": pm / bm,
                             "plain_value": units / (pm * 1e-3) / 1e9, "kernels_per_run": tasks,
                             "persistent_ms": per_ms, "persistent_speedup": pm / per_ms,
                             "persistent_tiles_per_run": per_tasks,
                             "max_rel_err_batched_vs_plain": max(errs)},
        "gpu_launches": launches,
        "generation_s": gen_s,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_large(args):
    """The 1024x1024x512 seven-view specimen, 10 iterations, device-resident."""
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd

    t0 = time.perf_counter()
    w = synth.config3()
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dviews = [torch.from_numpy(v).cuda() for v in w.views]
    stream.synchronize()
    d = mvd.Deconvolver(dviews, w.psfs, "efficient", stream=stream, path="fft")
    del dviews
    torch.cuda.empty_cache()
    free_b, total_b = torch.cuda.mem_get_info()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(max(1, args.warmup)):
        d.set_estimate(None)
        d.iterate(1)
    d.synchronize()
    ms = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            d.set_estimate(None)
            ev0.record(stream)
            d.iterate(w.n_iter)
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
    d.close()
    units = w.voxels * w.n_views * w.n_iter
    m = statistics.median(ms)
    print(json.dumps({
        "metric": METRIC, "value": units / (m * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "volume": list(w.dims), "views": w.n_views, "psf_box": [19, 19, 51],
                   "iterations": w.n_iter, "variant": "efficient", "engine": "fft", "precision": "precise",
                   "l2": "inputs larger than L2"},
        "device_used_gib": (total_b - free_b) / 2**30, "generation_s": gen_s, "clocks": clk.summary()}),
        flush=True)
    return 0


def run_grad(args):
    """The PSF-calibration step on the 128x128x96 four-view workload: Gaussian PSFs from
    per-view (sigma_xy, sigma_ax), 8 unrolled iterations, MSE to the truth, backward to
    the sigmas and the views (forward + hand-written adjoint)."""
    import torch

    import __graft_entry__
    import synth
    from synth.workloads import config5_sigmas, rotated_box

    __graft_entry__.build()
    from paper_1308_0730_gb300 import autograd as ag
    from paper_1308_0730_gb300 import mvd

    w = synth.config5()
    box, angles = w.meta["box"], w.meta["angles"]
    views = torch.from_numpy(np.stack(w.views)).cuda()
    truth = torch.from_numpy(w.truth).cuda()
    sig0 = config5_sigmas(w.n_views)
    stream = torch.cuda.current_stream()

    def step():
        sig = [torch.tensor(s_, dtype=torch.float64, requires_grad=True) for s_ in sig0]
        psfs = [ag.gaussian_psf(s_, rotated_box(box, a), a, "z") for s_, a in zip(sig, angles)]
        psi = ag.unrolled_deconvolve(views, psfs, w.n_iter)
        loss = torch.mean((psi.double() - truth.double()) ** 2)
        loss.backward()
        return float(loss.detach()), [s_.grad for s_ in sig]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = mvd.mvd_launch_count()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            loss, grads = step()
        ev1.record(stream)
        ev1.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (mvd.mvd_launch_count() - launches0) / args.steps
    mvd.mvd_profile_enable(True)
    step()
    torch.cuda.synchronize()
    prof = mvd.mvd_profile_read()
    mvd.mvd_profile_enable(False)
    # the forward alone (the same 8 iterations through the single-volume engine)
    psfs32 = [mvd.mvd_gaussian_psf(s_[0], s_[1], rotated_box(box, a), a, "z") for s_, a in zip(sig0, angles)]
    with mvd.Deconvolver([views[v] for v in range(w.n_views)], psfs32, "efficient", stream=stream,
                         path="fft") as d:
        d.iterate(w.n_iter)
        d.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            d.set_estimate(None)
            d.iterate(w.n_iter)
        ev1.record(stream)
        ev1.synchronize()
        fwd_ms = ev0.elapsed_time(ev1) / args.steps
    X, Y, Z = w.dims
    units = w.voxels * w.n_views * w.n_iter
    tot = sum(t for (_, t) in prof.values())
    kernels = {k: {"launches": n, "ms": t, "share": t / tot} for k, (n, t) in prof.items() if n}
    T = max(int(np.prod(p.shape)) for p in psfs32)
    conv_ops = w.voxels * T  # one FMA per voxel and tap
    roof = None
    if "direct_conv" in kernels:
        per = kernels["direct_conv"]["ms"] / kernels["direct_conv"]["launches"]
        ach = conv_ops / (per * 1e-3) / 1e12
        peak = _alu_peak_tops(torch.cuda.get_device_properties(0).multi_processor_count)
        roof = {"bound": "alu", "kernel": "direct_conv", "achieved": ach, "peak": peak, "unit": "T FP32 ops/s",
                "frac": ach / peak, "traffic": None,
                "note": "one FMA per voxel and tap of the largest PSF box"}
    print(json.dumps({
        "metric": "Gvoxel-view updates/s differentiated (forward + backward)", "value": units / (ms * 1e-3) / 1e9,
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "volume": [X, Y, Z], "views": w.n_views, "psf_box": list(box),
                   "unrolled_iterations": w.n_iter, "loss": "mse to truth", "params": "per-view (sigma_xy, sigma_ax)"},
        "forward_only_ms": fwd_ms, "backward_over_forward": (ms - fwd_ms) / fwd_ms, "loss": loss,
        "dsigma": [[float(x) for x in g.tolist()] for g in grads], "gpu_launches": launches,
        "kernels": kernels, "roofline": roof, "clocks": clk.summary()}), flush=True)
    return 0


def _time_steps(args, d, stream, step):
    """W untimed and K timed calls of ``step()`` (one whole deconvolution from the flat start)
    on the context's stream: returns (ms per step, launches per step, clock summary)."""
    import torch

    from paper_1308_0730_gb300 import mvd

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        d.set_estimate(None)
        step()
    d.synchronize()
    launches0 = mvd.mvd_launch_count()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            d.set_estimate(None)
            step()
        ev1.record(stream)
        ev1.synchronize()
    launches = (mvd.mvd_launch_count() - launches0) / args.steps
    return ev0.elapsed_time(ev1) / args.steps, launches, clk.summary()


def _variant_line(args, w, ms, launches, clocks, extra):
    """The JSON line of a variant of the default workload (the same metric, device-resident)."""
    X, Y, Z = w.dims
    units = w.voxels * w.n_views * w.n_iter
    cfg = {"workload": w.name, "volume": [X, Y, Z], "views": w.n_views, "iterations": w.n_iter}
    cfg.update(extra)
    cfg.update({"variant": "efficient", "engine": "fft", "precision": "precise", "l2": "inputs larger than L2"})
    print(json.dumps({
        "metric": METRIC, "value": units / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": cfg, "gpu_launches": launches, "clocks": clocks}), flush=True)
    return 0


def _resident_views(w):
    import torch

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dviews = [torch.from_numpy(v).cuda() for v in w.views]
    stream.synchronize()
    return stream, dviews


def run_combined(args):
    """The combined (simultaneous) update of Eq. 50 / Eq. 220 with the |V|-th root on the
    256x256x128 four-view workload, 20 iterations, device-resident, precise mode."""
    import __graft_entry__

    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd

    w = _workload(0)
    stream, dviews = _resident_views(w)
    with mvd.Deconvolver(dviews, w.psfs, "efficient", stream=stream, path="fft") as d:
        ms, launches, clocks = _time_steps(args, d, stream, lambda: d.iterate_combined(w.n_iter))
    return _variant_line(args, w, ms, launches, clocks, {"update": "combined, geometric mean of the view factors"})


def run_weighted(args):
    """Partially overlapping views on the 256x256x128 four-view workload: each view covers 70 % of
    the volume along x or y with cosine edges, weights normalised to the minimal overlap, 20
    sequential iterations, device-resident, precise mode."""
    import __graft_entry__
    from synth.workloads import blend_weights

    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd

    w = _workload(0)
    X, Y, Z = w.dims
    boxes = [((0, 0, 0), (int(0.7 * X), Y, Z)), ((int(0.3 * X), 0, 0), (X, Y, Z)),
             ((0, 0, 0), (X, int(0.7 * Y), Z)), ((0, int(0.3 * Y), 0), (X, Y, Z))]
    weights = [blend_weights(w.dims, lo, hi, (8, 8, 8)) for lo, hi in boxes]
    stream, dviews = _resident_views(w)
    with mvd.Deconvolver(dviews, w.psfs, "efficient", stream=stream, path="fft") as d:
        T = d.set_weights(weights, "min_overlap")
        ms, launches, clocks = _time_steps(args, d, stream, lambda: d.iterate(w.n_iter))
    return _variant_line(args, w, ms, launches, clocks,
                         {"update": "sequential with view weights (partial overlap)", "weight_norm": "min_overlap",
                          "weight_target": T})


def run_regularized(args):
    """Tikhonov regularisation (Green's one-step-late form, lambda = 0.006, inside the paper's
    0.0006-0.06) on the 256x256x128 four-view workload, 20 sequential iterations,
    device-resident, precise mode."""
    import __graft_entry__

    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd

    w = _workload(0)
    stream, dviews = _resident_views(w)
    with mvd.Deconvolver(dviews, w.psfs, "efficient", stream=stream, path="fft") as d:
        d.set_regularization(0.006)
        ms, launches, clocks = _time_steps(args, d, stream, lambda: d.iterate(w.n_iter))
    return _variant_line(args, w, ms, launches, clocks,
                         {"update": "sequential with Tikhonov regularisation (one-step-late)", "lambda": 0.006})


def run_boundary(args):
    """The 256x256x128 four-view workload with a zero or mirror boundary: the engines run on
    the grid padded by the PSF half-widths h = (20, 7, 20) (zero: by h, 288 x 270 x 150;
    mirror: by 2h, 300 x 270 x 180; {2,3,5}-smooth lengths) with the
    sensitivity-normalised update; the metric counts the user's voxels. 20 sequential
    iterations, device-resident, precise mode."""
    import __graft_entry__

    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd

    w = _workload(0)
    stream, dviews = _resident_views(w)
    with mvd.Deconvolver(dviews, w.psfs, "efficient", stream=stream, path="fft", boundary=args.boundary) as d:
        ms, launches, clocks = _time_steps(args, d, stream, lambda: d.iterate(w.n_iter))
    return _variant_line(args, w, ms, launches, clocks,
                         {"update": f"sequential, {args.boundary} boundary (padded grid, sensitivity-normalised)"})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mvd", choices=["mvd", "reference"])
    ap.add_argument("--quick", action="store_true",
                    help="only the device-resident timing (no FP32 comparison, end-to-end or CPU legs)")
    ap.add_argument("--weighted", action="store_true",
                    help="time the sequential update with partial-overlap view weights instead")
    ap.add_argument("--combined", action="store_true",
                    help="time the combined (simultaneous) update with the geometric mean instead")
    ap.add_argument("--regularized", action="store_true",
                    help="time the sequential update with Tikhonov regularisation (lambda 0.006) instead")
    ap.add_argument("--boundary", choices=["periodic", "zero", "mirror"], default="periodic",
                    help="zero / mirror: time the sequential update with that boundary (padded grid) instead")
    ap.add_argument("--grad", action="store_true",
                    help="time the PSF-calibration step (8 unrolled iterations, forward + adjoint) instead")
    ap.add_argument("--large", action="store_true",
                    help="time the 1024x1024x512 seven-view specimen (10 iterations) instead")
    ap.add_argument("--batched", action="store_true",
                    help="time the 48-volume batched workload against per-volume runs instead")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batched:
        return run_batched(args)
    if args.large:
        return run_large(args)
    if args.grad:
        return run_grad(args)
    if args.combined:
        return run_combined(args)
    if args.weighted:
        return run_weighted(args)
    if args.regularized:
        return run_regularized(args)
    if args.boundary != "periodic":
        return run_boundary(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
