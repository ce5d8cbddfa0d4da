"""Throughput benchmark: voxel-view updates per second of the efficient
Bayesian multi-view update on GB300, through the library's C ABI.

Headline workload: the 1024x1024x512 seven-view specimen (150k ellipsoids,
PSFs sigma 1.5/5 with box 19x19x51 rotated by k*51.43 deg about y, peak 200
photons plus a background of 5, Poisson noise), 10 sequential (OSEM-order)
iterations of the efficient method in precise (double-float) mode. Its inputs
are generated on the device (synth.config3_device); the views are 15 GiB.

One step = one deconvolution of that volume: psi reset to the flat estimate,
then 10 iterations x 7 view updates (views and kernel spectra resident in
HBM). value = voxels * views * iterations / step time, in Gvoxel-view/s.
e2e = the same metric through the public API from pinned host buffers, for a
time series with fixed PSFs: every step loads the seven views (H2D) into the
context (mvd_set_views), iterates and copies the result back (D2H).

The same JSON line also carries
  "mid":      the 256x256x128 four-view workload (20 iterations), with the
              all-FP32 and mixed-precision pipelines beside it;
  "batched":  48 volumes of uneven size and view count (15 iterations each):
              one graph launch over all volumes, one persistent kernel, and the
              48 volumes one after another ("plain"); ratio = plain / batched;
  "roofline", "kernels": per-kernel CUDA-event times of one step and the
              dominant kernel against the measured HBM peak;
  "cpu_baseline": the FP64 oracle on the host cores on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank deconvolves its own independent specimen (another
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
SPECIMEN_DIMS = (1024, 1024, 512)
SPECIMEN_OBJECTS = 150_000
# bounded CPU sample of the specimen (oracle timing): its recipe on a block whose
# axes hold every rotated PSF box (up to 53 x 19 x 53)
CPU_BLOCK = (128, 64, 64)


# algorithmic bytes per launch of each update kernel: every input and output
# array it must touch, once (FP32 half spectrum = 8 * (X/2+1) * Y * Z bytes)
def _kernel_bytes(X, Y, Z, precise=True):
    M = X * Y * Z
    spec = 8 * (X // 2 + 1) * Y * Z  # FP32 half spectrum; double-float is 2 * spec
    if precise:
        # power-of-two x and y lengths: the ratio pass writes the FP32 spectrum of r - 1 and
        # the back-projection's forward y reads it (FP32 in, double-float out), so the four y
        # launches of a view update move 4, 4, 3 and 4 spec, on average 3.75
        return {
            "dd_x_forward": 4 * M + 2 * spec,       # read psi, write S2
            "dd_y": 3.75 * spec,                    # read and write S2 (one launch reads FP32), mean of 4
            "dd_z_mul": 6 * spec,                   # read S2 and a double-float kernel spectrum, write S2
            "dd_x_ratio": 3 * spec + 4 * M,         # read S2 and phi, write the FP32 spectrum
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
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
    return 6800.0, "fallback"


def _workload_seed(rank: int) -> int:
    """Each rank deconvolves its own independent specimen (weak scaling, no data-path collective)."""
    return 1003 + 1000 * rank


WORKLOADS = {
    "specimen": SPECIMEN_DIMS,
    "specimen-half": (512, 512, 256),   # the specimen's recipe at 1/8 of the voxels (profiler captures)
    "specimen-quarter": (256, 256, 128),
    # thin grids with one of the specimen's transform lengths (profiler captures of one pass)
    "specimen-x1024": (1024, 64, 64),
    "specimen-y1024": (64, 1024, 64),
    "specimen-z512": (64, 64, 512),
    # slabs with one of the specimen's transform lengths whose spectra exceed the L2 (per-kernel captures)
    "specimen-1024x256x128": (1024, 256, 128),
    "specimen-256x1024x128": (256, 1024, 128),
    "specimen-256x128x512": (256, 128, 512),
}


def _specimen(rank: int, device: int, name: str = "specimen"):
    """The specimen (or its recipe on a smaller grid), generated on the device."""
    import synth

    dims = WORKLOADS[name]
    n_obj = max(1, round(SPECIMEN_OBJECTS * dims[0] * dims[1] * dims[2] / (SPECIMEN_DIMS[0] * SPECIMEN_DIMS[1]
                                                                              * SPECIMEN_DIMS[2])))
    return synth.config3_device(seed=_workload_seed(rank), dims=dims, n_objects=n_obj, device=f"cuda:{device}")


def _workload(rank: int):
    """The 256x256x128 four-view workload (20 iterations) of the variant benchmarks."""
    import synth

    return synth.config2(seed=1002 + 1000 * rank)


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


# ---------------------------------------------------------------------------
# FP64 oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

class OracleSample:
    """The specimen's recipe (objects, seven rotated PSFs, photon level, background) on the
    block CPU_BLOCK, with the oracle's compound kernels computed once (untimed). One step is
    one iteration: the seven view updates of `oracle.update` (FP64 direct sums) in order.
    The oracle's cost per voxel-view depends on the PSF boxes only, which the block keeps."""

    def __init__(self):
        import oracle
        import synth

        dims = CPU_BLOCK
        n_obj = max(1, round(SPECIMEN_OBJECTS * dims[0] * dims[1] * dims[2] / (SPECIMEN_DIMS[0] * SPECIMEN_DIMS[1]
                                                                                  * SPECIMEN_DIMS[2])))
        self.w = synth.config3(dims=dims, n_objects=n_obj)
        self.pn = [p.astype(np.float64) / p.astype(np.float64).sum() for p in self.w.psfs]
        self.K = [oracle.compound(self.pn, v, "efficient") for v in range(len(self.pn))]
        self.phi = [v.astype(np.float64) for v in self.w.views]
        psi0 = oracle.mean_views(self.w.views)
        self.eps = 1e-4 * psi0
        self.psi = np.full(self.w.truth.shape, psi0)
        self.units = self.w.voxels * len(self.pn)
        self.cores = oracle.num_threads()

    def step(self) -> float:
        import oracle

        t0 = time.perf_counter()
        for v in range(len(self.pn)):
            self.psi = oracle.update(self.psi, self.phi[v], self.pn[v], self.K[v], self.eps)
        return time.perf_counter() - t0

    def describe(self, steps: int, seconds: float) -> str:
        X, Y, Z = CPU_BLOCK
        return (f"{steps} iteration(s) (7 view updates each, FP64 direct sums, compound kernels of Eq. 222) of the "
                f"1024x1024x512 specimen's recipe on a {X}x{Y}x{Z} block, {seconds:.1f} s")


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    s = OracleSample()
    for _ in range(args.warmup):
        s.step()
    times = [s.step() for _ in range(args.steps)]
    total = sum(times)
    value = s.units * args.steps / total / 1e9
    X, Y, Z = SPECIMEN_DIMS
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"ellipsoids-{X}x{Y}x{Z}-7views", "volume": [X, Y, Z], "views": 7,
                   "psf_box": [19, 19, 51], "iterations": 10, "variant": "efficient"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": s.cores, "kind": "oracle",
                         "sample": "per step: " + s.describe(1, total / max(1, args.steps))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# roofline of the dominant kernel
# ---------------------------------------------------------------------------

def _profiled_counters(kernel: str, dims):
    """DRAM bytes and FP32 thread instructions per launch of ``kernel`` on ``dims`` from the
    committed ncu summary (profiles/traffic.json); entries captured on a smaller grid of the
    same recipe carry the voxel ratio they were scaled by."""
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tf):
        return None
    with open(tf) as fh:
        tr = json.load(fh)
    rec = tr.get(f"{kernel}@{dims[0]}x{dims[1]}x{dims[2]}")
    if rec is None:
        return None
    if isinstance(rec, (int, float)):
        return {"dram_bytes": float(rec)}
    return rec


def _kernel_table(prof, kb, peak):
    tot = sum(t for (_, t) in prof.values())
    out = {}
    for name, (n, ms) in prof.items():
        if n and name in kb:
            avg_s = ms / n * 1e-3
            out[name] = {"launches": n, "avg_us": avg_s * 1e6, "share": ms / max(1e-12, tot),
                         "GBps": kb[name] / avg_s / 1e9, "hbm_frac": kb[name] / avg_s / 1e9 / peak}
    return out


def _roofline(prof, kernels, dims, peak, peak_kind, alu_peak, units_per_step, ms_step):
    dom = max(kernels, key=lambda k: prof[k][1])
    rec = kernels[dom]
    roof = {"bound": "hbm", "kernel": dom, "achieved": rec["GBps"], "peak": peak, "unit": "GB/s",
            "frac": rec["GBps"] / peak, "traffic": None, "peak_source": peak_kind,
            "achieved_basis": "algorithmic bytes per launch (every array the kernel must touch, once) / "
                              "CUDA-event launch time"}
    cnt = _profiled_counters(dom, dims)
    if cnt:
        avg_s = rec["avg_us"] * 1e-6
        if "dram_bytes" in cnt:
            roof["traffic"] = int(cnt["dram_bytes"])
            roof["dram_frac"] = cnt["dram_bytes"] / avg_s / 1e9 / peak
        if "fp32_inst" in cnt:
            roof["alu_frac"] = cnt["fp32_inst"] / avg_s / 1e12 / alu_peak
            roof["alu_peak_Tinst"] = alu_peak
        if "source" in cnt:
            roof["counters_source"] = cnt["source"]
    # the whole update against the 12 B per voxel-view it must move (read psi and phi_v, write psi)
    roof["update_effective_frac"] = 12.0 * units_per_step / (ms_step * 1e-3) / 1e9 / peak
    return roof


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def _events_ms(stream, fn, n):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def _profile_step(mvd, d, fn):
    """Per-kernel CUDA-event times of one more step, its kernels launched one by one."""
    mvd.mvd_profile_enable(True)
    fn()
    d.synchronize()
    prof = mvd.mvd_profile_read()
    mvd.mvd_profile_enable(False)
    return prof


def _mid_record(args, mvd, stream, peak):
    """The 256x256x128 four-view workload, 20 iterations, device-resident: precise (the
    parity-held pipeline), all-FP32 and mixed precision."""
    import torch

    w = _workload(0)
    X, Y, Z = w.dims
    units = w.voxels * w.n_views * w.n_iter
    K = max(1, min(args.steps, 10))
    with torch.cuda.stream(stream):
        dviews = [torch.from_numpy(v).cuda() for v in w.views]
    stream.synchronize()
    rec = {"workload": w.name, "volume": [X, Y, Z], "views": w.n_views, "iterations": w.n_iter, "steps": K,
           "warmup": 3}
    results = {}
    for precision in ("precise", "fast", "mixed"):
        with mvd.Deconvolver(dviews, w.psfs, "efficient", stream=stream, path="fft", precision=precision) as d:
            def step():
                d.set_estimate(None)
                d.iterate(w.n_iter)

            for _ in range(3):
                step()
            d.synchronize()
            ms = _events_ms(stream, step, K) / K
            prof = _profile_step(mvd, d, step)
            results[precision] = d.result().astype(np.float64)
        kt = _kernel_table(prof, _kernel_bytes(X, Y, Z, precise=precision != "fast") if precision != "mixed"
                           else {**_kernel_bytes(X, Y, Z, True), **_kernel_bytes(X, Y, Z, False)}, peak)
        entry = {"value": units / (ms * 1e-3) / 1e9, "ms_per_step": ms, "kernels": kt}
        if precision == "precise":
            rec.update(entry)
        else:
            ref = results["precise"]
            tau = 1e-3 * np.abs(ref).max()
            entry["max_rel_diff_vs_precise"] = float(np.max(np.abs(results[precision] - ref)
                                                            / np.maximum(np.abs(ref), tau)))
            entry["precision"] = {"fast": "all FP32 (not held to 1e-4)",
                                  "mixed": "double-float forward blur, FP32 back-projection (not held to 1e-4)"}[
                precision]
            rec["fast_fp32" if precision == "fast" else "mixed"] = entry
    return rec


def _batched_record(args, mvd, stream):
    """The 48-volume batch (sizes 48^3 to 320x320x192, 2-6 views, 15 iterations each): the
    volumes one after another (each its own per-iteration graph), one graph launch with one
    branch per volume, and one persistent kernel over all volumes' FFT tiles."""
    import torch

    import synth

    t0 = time.perf_counter()
    ws = synth.config4(workers=os.cpu_count() or 1)
    gen_s = time.perf_counter() - t0
    ds = []
    for w in ws:
        with torch.cuda.stream(stream):
            dv = [torch.from_numpy(v).cuda() for v in w.views]
        stream.synchronize()
        ds.append(mvd.Deconvolver(dv, w.psfs, "efficient", path="fft", stream=stream))
    n_iter = ws[0].n_iter
    units = sum(w.voxels * w.n_views * n_iter for w in ws)
    K = max(1, min(args.steps, 5))

    def reset():
        for d in ds:
            d.set_estimate(None)

    def plain():
        reset()
        for d in ds:
            d.iterate(n_iter)

    for _ in range(3):
        plain()
    stream.synchronize()
    plain_ms = _events_ms(stream, plain, K) / K
    plain_res = [d.result() for d in ds]
    # each volume alone (its own per-iteration graph): where the plain time goes
    per_volume = []
    for w, d in zip(ws, ds):
        d.set_estimate(None)

        def one(d=d):
            d.iterate(n_iter)

        ms1 = _events_ms(stream, one, 1)
        per_volume.append({"volume": w.name, "voxels": w.voxels, "views": w.n_views, "ms": ms1,
                           "value": w.voxels * w.n_views * n_iter / (ms1 * 1e-3) / 1e9})
    small = [p for p in per_volume if p["voxels"] < 1_000_000]
    small_ms = sum(p["ms"] for p in small)
    tot_ms = sum(p["ms"] for p in per_volume)
    out = {}
    for mode in ("branches", "persistent"):
        b = mvd.mvd_batch_create(ds, n_iter, mode)

        def batched():
            reset()
            mvd.mvd_batch_run(b)

        for _ in range(3):
            batched()
        mvd.mvd_batch_wait(b)
        l0 = mvd.mvd_launch_count()
        ms = _events_ms(stream, batched, K) / K
        mvd.mvd_batch_wait(b)
        launches = (mvd.mvd_launch_count() - l0) / K
        errs = []
        for d, p in zip(ds, plain_res):
            q, p64 = d.result().astype(np.float64), p.astype(np.float64)
            errs.append(float(np.max(np.abs(q - p64) / np.maximum(np.abs(p64), 1e-3 * np.abs(p64).max()))))
        out[mode] = {"ms": ms, "value": units / (ms * 1e-3) / 1e9, "ratio": plain_ms / ms,
                     "launches_per_run": launches, "tasks": mvd.mvd_batch_tasks(b),
                     "max_rel_diff_vs_plain": max(errs)}
        mvd.mvd_batch_destroy(b)
    for d in ds:
        d.close()
    best = max(out, key=lambda m: out[m]["ratio"])
    return {"workload": f"batch of {len(ws)} volumes (48^3 to 320x320x192, 2-6 views, 15 iterations each)",
            "voxels": int(sum(w.voxels for w in ws)), "voxel_view_updates": int(units), "steps": K, "warmup": 3,
            "plain_ms": plain_ms, "plain_value": units / (plain_ms * 1e-3) / 1e9,
            "batched_ms": out[best]["ms"], "value": out[best]["value"], "mode": best,
            "ratio": out[best]["ratio"], "modes": out, "generation_s": gen_s,
            "per_volume": per_volume,
            "volumes_below_1M_voxels": {"count": len(small), "ms": small_ms, "share_of_plain": small_ms / tot_ms,
                                        "ratio_ceiling_if_free": tot_ms / (tot_ms - small_ms)}}


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

    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    w = _specimen(rank, local, args.workload)
    gen_s = time.perf_counter() - t0
    X, Y, Z = w.dims
    M = w.voxels
    units_per_step = M * w.n_views * w.n_iter
    view_bytes = 4 * M * w.n_views
    d = mvd.Deconvolver(w.views, w.psfs, "efficient", stream=stream, path="fft", device=local)
    hviews = None if args.quick else w.host_views(pinned=True)
    w.views = None
    torch.cuda.empty_cache()

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
    with ClockSampler(local) as clk:
        ms = _events_ms(stream, step, args.steps)
    torch.cuda.synchronize()
    launches = mvd.mvd_launch_count() - launches0
    t_max = _max_over_ranks(ms, dist, f"cuda:{local}")
    prof = _profile_step(mvd, d, step)
    value = _job_value(ws, units_per_step * args.steps, t_max * 1e-3)
    peak, peak_kind = _peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = _alu_peak_tops(sms)
    kernels = _kernel_table(prof, _kernel_bytes(X, Y, Z), peak)
    roofline = _roofline(prof, kernels, (X, Y, Z), peak, peak_kind, alu_peak, units_per_step, t_max / args.steps)
    cfg = {"workload": w.name, "volume": [X, Y, Z], "views": w.n_views, "psf_box": [19, 19, 51],
           "iterations": w.n_iter, "variant": "efficient", "engine": "fft", "precision": "precise (double-float)",
           "l2": f"inputs larger than L2 (views {view_bytes / 2**30:.1f} GiB, kernel spectra "
                 f"{32 * (X // 2 + 1) * Y * Z * w.n_views / 2**30:.1f} GiB > 129 MiB)",
           "inputs": "generated on the device (synth.config3_device)", "parallelism": f"replicas x{ws}"}
    if args.quick:
        psi_dev = None
        d.close()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": t_max / args.steps, "quick": True,
                              "config": cfg, "kernels": kernels, "roofline": roofline, "generation_s": gen_s}),
                  flush=True)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # --- end to end through the public API from pinned host buffers ---
    psi_dev = d.result()
    out = torch.empty(psi_dev.shape, dtype=torch.float32).pin_memory().numpy()

    def e2e_step():
        d.set_views(hviews)
        d.iterate(w.n_iter)
        d.result(out)

    e2e_steps = max(1, min(args.steps, 3))
    e2e_step()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, f"cuda:{local}")
    assert np.array_equal(out, psi_dev), "end-to-end result differs from the device-resident run"
    # where an end-to-end step goes (host clock, each part synchronised)
    parts = {}
    for name, fn in (("load_views_h2d", lambda: d.set_views(hviews)), ("iterate", lambda: d.iterate(w.n_iter)),
                     ("result_d2h", lambda: d.result(out))):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        fn()
        d.synchronize()
        parts[name] = 1e3 * (time.perf_counter() - t1)
    d.close()
    del hviews, psi_dev

    mid = batched = cpu = None
    if ws == 1:
        mid = _mid_record(args, mvd, stream, peak)
        batched = _batched_record(args, mvd, stream)
        s = OracleSample()
        times = [s.step() for _ in range(3)]
        cpu = {"value": s.units * len(times) / sum(times) / 1e9, "unit": UNIT, "cores": s.cores, "kind": "oracle",
               "sample": s.describe(len(times), sum(times))}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "e2e": {"value": _job_value(ws, units_per_step, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": int(view_bytes), "d2h_bytes_per_step": int(out.nbytes),
                    "steps": e2e_steps, "breakdown_ms": parts,
                    "per_step": "time series with fixed PSFs: load the 7 views from pinned host memory "
                                "(mvd_set_views), 10 iterations, result to pinned host memory; kernels "
                                "precomputed once for the series"},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "kernels": kernels,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "mid": mid,
            "batched": batched,
            "generation_s": gen_s,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """The 48-volume batch alone (one JSON line)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd

    stream = torch.cuda.Stream()
    with ClockSampler(torch.cuda.current_device()) as clk:
        b = _batched_record(args, mvd, stream)
    print(json.dumps({
        "metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": 1, "steps": b["steps"], "warmup": 3,
        "ms_per_step": b["batched_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": {"workload": b["workload"]}, "batched": b,
        "clocks": clk.summary()}), flush=True)
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
                    help="only the device-resident timing and per-kernel events (no end-to-end, sub-records or CPU legs)")
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="specimen",
                    help="grid of the headline recipe (smaller ones for profiler captures)")
    ap.add_argument("--batched", action="store_true",
                    help="time the 48-volume batched workload against per-volume runs instead")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batched:
        return run_batched(args)
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
