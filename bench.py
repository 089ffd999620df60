"""Benchmark: stationary pmfs per second at N = 2000 bins, each within 1e-6 L1
of the FP64 oracle, learned + batched against plain batched.

Workload (one step): the 256 x 256 pixel array (65536 pixels, N = 2000,
t_r = 100 ns, t_d = 75 ns, tau ~ U[5,95] ns, sigma ~ U[0.2,1] ns,
S, B ~ logU[0.01,5], seed 5).  A step runs the whole path through the C ABI:
the warm-start network's forward pass on the tensor cores, the dead-time
shift (host), FP64 cumulative flux, row sums (O(N) prefix and suffix scans)
and matrix-free power iteration of every pixel to the 1e-6 stop rule in one
persistent launch, every step regenerating all N^2 entries of P~.  The network
is trained first (untimed) on 200k pmfs the plain solver produces.  The plain
arm (uniform start) is timed on the same workload and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  The reference arm times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
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

METRIC = "stationary PDFs/sec at N=2000, 1e-6 L1 vs FP64 oracle (learned+batched vs plain)"
UNIT = "PDFs/s"
TOL = 1e-6
MAX_ITER = 1000
WORKLOAD = "array256: 256x256 pixels, N=2000, t_r=100ns, t_d=75ns, tau~U[5,95], sigma~U[0.2,1], S,B~logU[0.01,5], seed 5"
FP32_LANES = 128           # FP32 FMA lanes per SM (nominal peak, context only)
SM_MAX_MHZ = 2070.0        # maximum SM clock (nominal peak, context only)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_workload(rank: int, pixels: int = 0):
    """The pixels one rank times: an independent seeded 256x256 array per
    rank (weak scaling; pixels are independent, so no collective)."""
    from paper_2509_20500_gb300 import workloads as W
    px = W.array256(seed=5 + rank)
    return px[:pixels] if pixels else px


def max_over_ranks(x: float, device="cpu") -> float:
    """Largest value of x over the ranks of the default process group (the
    step time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = [x for x in sm if smax and x > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def batch_kernel_source_hash() -> str:
    """Hash of the batch kernel's code (spl_kernels.cu up to the end of its
    section, with the pass helpers it uses, plus spl_device.cuh; comments and
    blank space left out), used to tell whether a stored ncu traffic figure still
    describes the kernel being timed."""
    import hashlib
    import re

    def code_only(t: str) -> str:
        # comments and blank space do not change the kernel
        t = re.sub(r"/\*.*?\*/", "", t, flags=re.S)
        t = re.sub(r"//[^\n]*", "", t)
        return "\n".join(line.strip() for line in t.splitlines() if line.strip())

    base = os.path.join(ROOT, "paper_2509_20500_gb300", "csrc")
    txt = open(os.path.join(base, "spl_kernels.cu")).read()
    b = txt.index("// K1 for a single chain: per-bin vectors")
    h = hashlib.sha256(code_only(txt[:b]).encode())      # the batch kernel and every device function before it
    h.update(code_only(open(os.path.join(base, "spl_device.cuh")).read()).encode())
    return h.hexdigest()[:16]


def stored_traffic(arm: str):
    """DRAM bytes per launch of the batch kernel on the 65536-pixel array for
    the given arm ("plain" or "learned") from the last ncu capture
    (profiles/batch_fused_kernel_traffic.json), or None if the kernel source
    changed since."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "batch_fused_kernel_traffic.json")))
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != batch_kernel_source_hash():
        return None
    a = d.get("arms", {}).get(arm)
    if a is None:
        return None
    return float(a["dram_bytes_read_per_launch"]) + float(a["dram_bytes_write_per_launch"])


def stored_structured_pipes():
    """Pipe utilisation of the structured (O(N)) batch kernel from the last
    ncu capture of a 4096-pixel launch (stored beside the traffic figures),
    or None if the kernel source changed since."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "batch_fused_kernel_traffic.json")))
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != batch_kernel_source_hash():
        return None
    return d.get("structured_pipes")


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# ---------------------------------------------------------------- CPU oracle (reference arm, cpu_baseline)

def oracle_rate(px_sample, nthreads):
    import oracle
    pix = [dict(zip(px_sample.dtype.names, (v.item() for v in rec))) for rec in px_sample]
    t0 = time.perf_counter()
    _, _, iters, used = oracle.batch_stationary(pix, tol=1e-12, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return len(pix) / dt, dt, used


def cpu_sample(px, n):
    from paper_2509_20500_gb300 import workloads as W
    idx = W.sample_indices(len(px), n, seed=55)
    return px[idx], idx


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2509_20500_gb300 import workloads as W
    px = W.array256()
    cores = os.cpu_count() or 1
    per_step = args.ref_sample
    sample, _ = cpu_sample(px, per_step * (args.steps + args.warmup))
    times = []
    for s in range(args.warmup + args.steps):
        chunk = sample[s * per_step:(s + 1) * per_step]
        rate, dt, used = oracle_rate(chunk, cores)
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step_sample_pixels": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"{per_step} pixels per step drawn by seed 55 from the 65536-pixel array; "
                                   "sequential FP64 construction + dense power iteration to 1e-12"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm

def flush_l2(buf):
    buf.add_(1.0)       # writes 256 MiB (> 129 MB L2)


def timed_steps(step_fn, steps, flush, stream, kernel_ms_fn=None):
    """Per-step device times (CUDA events on the launching stream, L2 flushed
    between steps outside the events) and, if given, the batch kernel time."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kern = []
    torch.cuda.nvtx.range_push("timed")
    for k in range(steps):
        flush_l2(flush)
        ev[k][0].record(stream)
        step_fn()
        ev[k][1].record(stream)
        if kernel_ms_fn is not None:
            kern.append(kernel_ms_fn())
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], kern


def pdf_wall_ms(ch, reps: int = 20) -> float:
    """Median host wall time of one spl_stationary call (synchronous: build
    excluded, start vector, every step, stop rule and result copy included)."""
    ch.stationary(tol=TOL)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        ch.stationary(tol=TOL)
        ts.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(ts)


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2509_20500_gb300 import build, spl, train as T, workloads as W
    build.build()
    spl.lib()
    peaks = measured_peaks() or {}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # FP32 roofline denominator: the library's FMA-throughput kernel, measured
    # here (launches of about the batch kernel's length, median of five)
    fma = spl.fp32_fma_peak(iters=800_000, reps=5)
    assert fma["sms"] == sms

    # each rank owns an independent 65536-pixel array (weak scaling, no collective)
    px = rank_workload(rank, args.pixels)
    n = len(px)
    off = spl.offsets_of(px)
    total = int(off[-1])
    out = torch.empty(total, dtype=torch.float32, device=dev)
    d_off = torch.from_numpy(off).to(dev)
    c_px = spl.pixels_to_c(px, pinned=True)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # the timed path: dense regenerated power steps (N^2 FFMA per step), the
    # row sums of the normalisation from the O(N) scans of Eq. 6's structure
    head_pass = spl.SPL_PASS_DENSE_ROWSCAN

    def plain_step(time_kernel=False, reports=False):
        return spl.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off, reports=reports,
                                    c_pixels=c_px, time_kernel=time_kernel, pass_kind=head_pass)

    # ---- plain batched arm (uniform start)
    _, _, reps_plain = plain_step(reports=True)
    assert np.all(reps_plain["status"] == 0), "some pixels did not converge"
    for _ in range(args.warmup):
        plain_step()
    torch.cuda.synchronize()
    plain_ms_list, plain_kern = timed_steps(lambda: plain_step(time_kernel=True), args.steps, flush, stream,
                                            spl.batch_kernel_ms)
    plain_ms = sum(plain_ms_list) / len(plain_ms_list)
    # the autotuner's pick for this batch kind, and the fixed heuristic (tune=1) timed beside it
    tcfg = spl.batch_tune_lookup(2000, head_pass)
    spl.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off, reports=False, c_pixels=c_px,
                         pass_kind=head_pass, tune=1)
    _, dflt_kern = timed_steps(lambda: spl.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off,
                                                            reports=False, c_pixels=c_px, pass_kind=head_pass,
                                                            tune=1, time_kernel=True),
                               max(2, args.steps // 2), flush, stream, spl.batch_kernel_ms)

    # ---- learned warm start: trained (untimed) on pmfs the method generates
    learned = not args.no_learned
    if learned:
        t0 = time.perf_counter()
        tpx, ttg = T.make_training_set(args.train_pixels, seed=2)
        net = T.train(tpx, ttg, epochs=args.epochs, batch=4096, lr=3e-3, max_batch=n)
        del ttg
        train_s = time.perf_counter() - t0

        def learned_step(reports=False):
            return net.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off, reports=reports,
                                        c_pixels=c_px, pass_kind=head_pass)

        _, _, reps_l = learned_step(reports=True)
        assert np.all(reps_l["status"] == 0), "some pixels did not converge (learned start)"
        for _ in range(args.warmup):
            learned_step()
        torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    if learned:
        step_ms, kern_ms = timed_steps(lambda: learned_step(), args.steps, flush, stream, spl.batch_kernel_ms)
        reps = reps_l
    else:
        step_ms, kern_ms = timed_steps(lambda: plain_step(time_kernel=True), args.steps, flush, stream,
                                       spl.batch_kernel_ms)
        reps = reps_plain
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(sum(step_ms) / len(step_ms), device=dev)
    value = world * n / (ms / 1e3)

    # roofline of the dominant kernel: the persistent matrix-free batch kernel.
    # Algorithmic work: every pixel runs `iters` dense column passes over its
    # N x N regenerated matrix, one FFMA (2 FLOP) per entry (its row sums are
    # O(N) scans).
    N2 = px["n_bins"].astype(np.float64) ** 2
    flop = float(2.0 * np.sum(N2 * reps["iters"]))
    kms = statistics.median(kern_ms)
    achieved = flop / (kms / 1e3) / 1e12
    peak = fma["tflops_median"]
    peak_nominal = sms * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    arm = "learned" if learned else "plain"
    traffic = stored_traffic(arm) if n == 65536 else None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "batch_fused_kernel", "kernel_ms": kms,
            "algorithmic_bytes": float(total * 4 * (2 if learned else 1) + n * 40),
            "bytes_basis": "pmf write (4 B per bin)" + (" + learned logits read (4 B per bin)" if learned else "")
                           + " + 40 B of parameters per pixel", "arm": arm,
            "work": "2 FLOP x N^2 x iters per pixel (dense power steps, one FFMA per regenerated entry; "
                    "the row sums are O(N) scans)",
            "peak_basis": "of measured: spl_fp32_fma_peak (16 FMA chains per thread, 4 x 256 threads per SM, "
                          "median of 5 launches of ~50 ms) in this run",
            "peak_fp32_best_of_5": fma["tflops_best"], "sms": sms,
            "peak_nominal": peak_nominal,
            "peak_nominal_basis": f"{sms} SMs x 128 FP32 FMA lanes x 2 FLOP x 2070 MHz (max SM clock)"}

    # accuracy audit of the timed outputs: sampled pixels against the FP64 oracle
    line_audit = None
    if not args.no_cpu_baseline and rank == 0:
        import oracle
        idx = W.sample_indices(n, args.audit, seed=91)
        refs, roff, _, _ = oracle.batch_stationary(W.as_dicts(px[idx]), tol=1e-12)
        o = out.cpu().numpy().astype(np.float64)
        dif = [np.abs(o[off[k]:off[k + 1]] - refs[roff[r]:roff[r + 1]]) for r, k in enumerate(idx)]
        errs = [float(d.sum()) for d in dif]
        line_audit = {"sampled_pixels": len(idx), "max_l1": max(errs), "mean_l1": float(np.mean(errs)),
                      "max_abs": max(float(d.max()) for d in dif),
                      "tol": TOL, "of": "the last timed step's output"}

    extra = {}
    if learned:
        # tensor-core roofline of the network's forward pass over the array
        # (device time of the forward kernels alone, logits kept inside the network)
        mlp_ms = net.time_forward(px, reps=10)
        mlp_flop = 2.0 * n * (5 * 512 + 3 * 512 * 512 + 512 * 2000)
        tpeak = float(peaks.get("bf16_tflops", 1900.0))
        extra["learned"] = {"value": value, "ms_per_step": ms, "iters_mean": float(reps_l["iters"].mean()),
                            "iters_max": int(reps_l["iters"].max()), "train_seconds": train_s,
                            "train_pixels": args.train_pixels, "epochs": args.epochs,
                            "mlp_roofline": {"bound": "tensor", "achieved": mlp_flop / (mlp_ms / 1e3) / 1e12,
                                             "peak": tpeak, "unit": "TFLOP/s",
                                             "frac": mlp_flop / (mlp_ms / 1e3) / 1e12 / tpeak,
                                             "ms": mlp_ms, "peak_basis": "MEASURED_PEAKS bf16_tflops (burst), of measured",
                                             "work": "2 x 65536 x (5 x 512 + 3 x 512^2 + 512 x 2000) FLOP (real, unpadded sizes)"}}
    extra["autotune_array256"] = {
        "picked": dict(zip(("threads", "state_level", "blocks_per_sm", "cols"), tcfg)) if tcfg else None,
        "plain_kernel_ms": statistics.median(plain_kern), "default_kernel_ms": statistics.median(dflt_kern),
        "gain_over_default": statistics.median(dflt_kern) / statistics.median(plain_kern),
        "searched": "threads {256, 512} x columns per thread {8, 4} x state level {2, 1, 0} x blocks per SM "
                    "{occupancy limit, one below}, on 48 x SMs pixels of the first batch of the kind, "
                    "each timed twice (minimum); the heuristic's configuration is kept unless another "
                    "is faster by more than 0.5 %"}
    extra["plain"] = {"value": world * n / (plain_ms / 1e3), "ms_per_step": plain_ms,
                      "iters_mean": float(reps_plain["iters"].mean()), "iters_max": int(reps_plain["iters"].max()),
                      "kernel_ms": statistics.median(plain_kern)}

    # the same dense power steps with the row sums from one more dense pass
    # (regenerating every entry of P~ for its row sums): both arms
    if not args.no_rowpass:
        rs = {}
        for arm in (("learned", "plain") if learned else ("plain",)):
            def rs_step(arm=arm, time_kernel=False, reports=False):
                if arm == "learned":
                    return net.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off,
                                                reports=reports, c_pixels=c_px, pass_kind=spl.SPL_PASS_DENSE,
                                                time_kernel=time_kernel)
                return spl.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off, reports=reports,
                                            c_pixels=c_px, time_kernel=time_kernel,
                                            pass_kind=spl.SPL_PASS_DENSE)
            _, _, rr = rs_step(reports=True)
            assert np.all(rr["status"] == 0)
            for _ in range(args.warmup):
                rs_step()
            rms, rkern = timed_steps(lambda: rs_step(time_kernel=True), args.steps, flush, stream,
                                     spl.batch_kernel_ms)
            rk = statistics.median(rkern)
            rflop = float(2.0 * np.sum(N2 * (1 + rr["iters"])))
            item = {"value": world * n / (statistics.mean(rms) / 1e3), "ms_per_step": statistics.mean(rms),
                    "kernel_ms": rk, "iters_mean": float(rr["iters"].mean()),
                    "roofline": {"bound": "alu", "achieved": rflop / (rk / 1e3) / 1e12, "peak": peak,
                                 "unit": "TFLOP/s", "frac": rflop / (rk / 1e3) / 1e12 / peak,
                                 "work": "2 FLOP x N^2 x (1 + iters) per pixel (dense row pass + power steps)"}}
            if arm == "learned" and not args.no_cpu_baseline and rank == 0:
                import oracle
                idx = W.sample_indices(n, args.audit, seed=91)
                refs, roff, _, _ = oracle.batch_stationary(W.as_dicts(px[idx]), tol=1e-12)
                o = out.cpu().numpy().astype(np.float64)
                dif = [np.abs(o[off[k]:off[k + 1]] - refs[roff[r]:roff[r + 1]]) for r, k in enumerate(idx)]
                item["accuracy_vs_oracle"] = {"sampled_pixels": len(idx), "max_l1": max(float(d.sum()) for d in dif),
                                              "max_abs": max(float(d.max()) for d in dif)}
            rs[arm] = item
        rs["note"] = "SPL_PASS_DENSE: the same power steps, row sums by a dense regenerating pass"
        extra["dense_rowpass"] = rs

    # the allocation-free entry point on the same pixels (plain start): what
    # its fixed scratch and default launch shape cost against the plain arm
    if not args.no_noalloc:
        def na_step():
            return spl.batch_stationary_noalloc(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off,
                                                reports=False, c_pixels=c_px)
        for _ in range(args.warmup):
            na_step()
        na_ms, _ = timed_steps(na_step, args.steps, flush, stream)
        na = statistics.mean(na_ms)
        extra["noalloc"] = {"value": world * n / (na / 1e3), "ms_per_step": na,
                            "what": "spl_batch_stationary_noalloc (uniform start, dense row pass and steps), "
                                    "same 65536 pixels"}
        if "dense_rowpass" in extra:
            extra["noalloc"]["vs_spl_batch_stationary_same_pass"] = extra["dense_rowpass"]["plain"]["ms_per_step"] / na

    # the O(N) structured form of the same power step (reported beside the
    # dense path, never as its number): plain and learned starts
    if not args.no_structured:
        st = {}
        def s_plain():
            return spl.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off, reports=False,
                                        c_pixels=c_px, time_kernel=True, pass_kind=spl.SPL_PASS_STRUCTURED)
        _, _, r_sp = spl.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off, reports=True,
                                          c_pixels=c_px, pass_kind=spl.SPL_PASS_STRUCTURED)
        for _ in range(args.warmup):
            s_plain()
        sms, skern = timed_steps(s_plain, args.steps, flush, stream, spl.batch_kernel_ms)
        st["plain"] = {"value": world * n / (statistics.mean(sms) / 1e3), "ms_per_step": statistics.mean(sms),
                       "kernel_ms": statistics.median(skern), "iters_mean": float(r_sp["iters"].mean())}
        if learned:
            def s_learned():
                return net.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off, reports=False,
                                            c_pixels=c_px, pass_kind=spl.SPL_PASS_STRUCTURED)
            _, _, r_sl = net.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off, reports=True,
                                              c_pixels=c_px, pass_kind=spl.SPL_PASS_STRUCTURED)
            for _ in range(args.warmup):
                s_learned()
            lms, lkern = timed_steps(s_learned, args.steps, flush, stream, spl.batch_kernel_ms)
            st["learned"] = {"value": world * n / (statistics.mean(lms) / 1e3), "ms_per_step": statistics.mean(lms),
                             "kernel_ms": statistics.median(lkern), "iters_mean": float(r_sl["iters"].mean())}
        pipes = stored_structured_pipes()
        st["roofline"] = None if pipes is None else {
            "bound": "fp64", "frac": pipes["fp64_pipe_frac"], "unit": "FP64 pipe busy / peak",
            "fma_pipe_frac": pipes["fma_pipe_frac"], "issue_frac": pipes["issue_frac"],
            "basis": "ncu on a 4096-pixel launch of this kernel (" + pipes["capture"] + "); no pipe is saturated: "
                     "the FP64 flux phase keeps the FP64 pipe busiest and the block scans' latency sets the rest"}
        st["note"] = "O(N) scan form of the power step (Eq. 6 triangular structure); same pmfs, not the dense-path number"
        extra["structured"] = st

    # uneven workload: 4096 pixels, N in {500..16000}, one persistent launch;
    # the measured launch configuration against the fixed heuristic (tune=1)
    if not args.no_uneven and rank == 0:
        ux = W.uneven()
        ucp = spl.pixels_to_c(ux)
        uoff = spl.offsets_of(ux)
        uout = torch.empty(int(uoff[-1]), dtype=torch.float32, device=dev)
        udo = torch.from_numpy(uoff).to(dev)
        un = {}
        for name, pk in (("dense", head_pass), ("structured", spl.SPL_PASS_STRUCTURED)):
            _, _, ur = spl.batch_stationary(ux, tol=TOL, max_iter=MAX_ITER, out=uout, offsets=udo, c_pixels=ucp,
                                            pass_kind=pk)
            assert np.all(ur["status"] == 0)
            def fn(pk=pk, tune=0):
                return spl.batch_stationary(ux, tol=TOL, max_iter=MAX_ITER, out=uout, offsets=udo, c_pixels=ucp,
                                            reports=False, time_kernel=True, pass_kind=pk, tune=tune)
            fn()
            ums, ukern = timed_steps(fn, max(2, args.steps // 2), flush, stream, spl.batch_kernel_ms)
            item = {"value": len(ux) / (statistics.mean(ums) / 1e3), "ms_per_step": statistics.mean(ums),
                    "kernel_ms": statistics.median(ukern), "iters_mean": float(ur["iters"].mean()),
                    "iters_max": int(ur["iters"].max())}
            if pk == head_pass:
                uf = float(2.0 * np.sum(ux["n_bins"].astype(np.float64) ** 2 * ur["iters"]))
                ua = uf / (item["kernel_ms"] / 1e3) / 1e12
                item["roofline"] = {"bound": "alu", "achieved": ua, "peak": peak, "unit": "TFLOP/s", "frac": ua / peak,
                                    "work": "2 FLOP x N^2 x iters per pixel"}
                fn(tune=1)
                _, dkern = timed_steps(lambda: fn(tune=1), max(2, args.steps // 2), flush, stream, spl.batch_kernel_ms)
                cfg = spl.batch_tune_lookup(int(ux["n_bins"].max()), head_pass)
                item["autotune"] = {"picked": dict(zip(("threads", "state_level", "blocks_per_sm", "cols"), cfg))
                                    if cfg else None,
                                    "default_kernel_ms": statistics.median(dkern),
                                    "gain_over_default": statistics.median(dkern) / item["kernel_ms"],
                                    "default": "256 threads, 8 columns per thread, largest state level that fits, "
                                               "occupancy-limit blocks per SM"}
            un[name] = item
        un["workload"] = "uneven: 4096 pixels, N~U{500,...,16000}, t_d~U[20,150], tau=30, sigma=0.3, B=0.5, S~U{0.05,0.5,5}, seed 4"
        extra["uneven_4096"] = un
        del uout

    # spectral analysis (Sec. 4, Fig. 4 columns 1-2): |lambda_2| and phase over a
    # 64 x 64 log grid of S, B in [0.01, 10] at t_d = 75 and 95, N = 256
    if not args.no_spectral and rank == 0:
        g = np.exp(np.linspace(np.log(0.01), np.log(10.0), 64))
        grid = np.concatenate([W.pixel(256, t_d, 30.0, 0.5, S, B) for t_d in (75.0, 95.0) for S in g for B in g])
        spl.batch_spectral(grid[:256], subspace_iters=60)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lam2 = spl.batch_spectral(grid, subspace_iters=60).cpu().numpy()
        dt = time.perf_counter() - t0
        m75, m95 = lam2[:4096, 0].reshape(64, 64), lam2[4096:, 0].reshape(64, 64)
        p75, p95 = lam2[:4096, 1].reshape(64, 64), lam2[4096:, 1].reshape(64, 64)
        extra["spectral_grid"] = {
            "pixels": int(len(grid)), "seconds": dt, "per_second": len(grid) / dt,
            "gap_decreases_with_B_fraction": float(np.mean(np.diff(np.concatenate([m75, m95]), axis=1) > 0)),
            "near_zero_phase_fraction": {"t_d=75": float(np.mean(p75 < 0.1)), "t_d=95": float(np.mean(p95 < 0.1))},
            "lambda2_abs_range": [float(lam2[:, 0].min()), float(lam2[:, 0].max())],
            "note": "orthogonal iteration on the deflated O(N) operator, 60 steps, N = 256 (the paper's grid resolution)"}

    # accuracy across (S, B) against the event Monte Carlo (Sec. 5, Fig. 3c):
    # 21 x 21 grid over [0, 10]^2 at 256 bins, 25 runs x 50,000 cycles each
    if not args.no_mc and rank == 0:
        g = W.accuracy_grid()
        runs, cycles, nb = 25, args.mc_cycles, 256
        spl.mc_histograms(g[:4], 2, 1000, seed=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h, _ = spl.mc_histograms(g, runs, cycles, seed=3)
        mc_s = time.perf_counter() - t0
        H = h.cpu().numpy().view(np.uint32).reshape(len(g), runs, nb).sum(axis=1).astype(np.float64)
        nreg = H.sum(axis=1)

        def agreement(flux_kind):
            pig, _, rg = spl.batch_stationary(g, tol=TOL, flux_kind=flux_kind)
            Pg = pig.cpu().numpy().astype(np.float64).reshape(len(g), nb)
            l1 = np.abs(Pg - H / nreg[:, None]).sum(axis=1)
            # L1 distance a multinomial sample of the same size would show from Pg
            noise = np.sqrt(2.0 / np.pi) * np.sqrt(Pg * (1.0 - Pg) / nreg[:, None]).sum(axis=1)
            chi = []
            for k in range(len(g)):
                E = nreg[k] * Pg[k]
                m = E >= 5
                chi.append(float((((H[k][m] - E[m]) ** 2) / E[m]).sum() / max(1, m.sum() - 1)))
            chi = np.array(chi)
            worst = int(np.argmax(l1 / noise))
            return {"l1_median": float(np.median(l1)), "l1_max": float(l1.max()),
                    "mc_noise_l1_median": float(np.median(noise)),
                    "l1_over_noise_median": float(np.median(l1 / noise)),
                    "l1_over_noise_max": float((l1 / noise).max()),
                    "chi2_per_dof_median": float(np.median(chi)), "chi2_per_dof_max": float(chi.max()),
                    "points_within_2x_noise": int(np.sum(l1 < 2 * noise)),
                    "worst_point": {"S": float(g["S"][worst]), "B": float(g["B"][worst])}}

        extra["mc_accuracy_grid"] = {
            "points": int(len(g)), "n_bins": nb, "runs": runs, "cycles_per_run": cycles,
            "mc_seconds": mc_s, "mc_cycles_per_second": len(g) * runs * cycles / mc_s,
            "registrations": float(nreg.sum()),
            "point_flux": agreement(spl.SPL_FLUX_POINT),
            "bin_integrated": agreement(spl.SPL_FLUX_BININT),
            "workload": "S, B on a 21 x 21 grid over [0, 10] without (0, 0), t_d = 75, tau = 30, sigma = 0.5, "
                        "t_r = 100; pmfs from the batch solver (dense step), the paper's point flux and the "
                        "bin-integrated variant"}

    # materialised vs matrix-free power step on one N = 10000 pixel (400 MB P)
    if not args.no_highres and rank == 0:
        hp = W.pixel(10000, 75.0, 30.0, 0.3, 0.5, 0.5)
        hr = {}
        ch = spl.Chain(hp, spl.SPL_MATERIALIZED)
        build_ms = ch.time_build(10)
        bgbs = 4.0 * 1e8 / (build_ms / 1e3) / 1e9
        hr["materialized_build"] = {"bound": "hbm", "achieved": bgbs, "peak": float(peaks.get("hbm_gbs", 6800.0)),
                                    "unit": "GB/s", "frac": bgbs / float(peaks.get("hbm_gbs", 6800.0)),
                                    "ms_per_build": build_ms, "bytes": 4e8,
                                    "peak_basis": "MEASURED_PEAKS hbm_gbs, of measured"}
        gemv_ms = ch.time_pass(100)
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        gbs = 4.0 * 1e8 / (gemv_ms / 1e3) / 1e9
        hr["materialized_gemv"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                                   "ms_per_pass": gemv_ms, "bytes": 4e8,
                                   "peak_basis": "MEASURED_PEAKS hbm_gbs, of measured"}
        mstep_ms = ch.time_step(50)
        mgbs = 4.0 * 1e8 / (mstep_ms / 1e3) / 1e9
        hr["materialized_step"] = {"bound": "hbm", "achieved": mgbs, "peak": hbm, "unit": "GB/s", "frac": mgbs / hbm,
                                   "ms_per_step": mstep_ms,
                                   "what": "GEMV pass + partial reduction + normalisation, statistics and stop rule"}
        _, rep = ch.stationary(tol=TOL)
        hr["materialized_iters"] = int(rep["iters"])
        hr["materialized_ms_per_pdf"] = pdf_wall_ms(ch)
        ch.close()
        ch = spl.Chain(hp, spl.SPL_FUSED)
        fused_ms = ch.time_pass(200)
        tf = 2.0 * 1e8 / (fused_ms / 1e3) / 1e12
        hr["fused_pass"] = {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                            "ms_per_pass": fused_ms}
        fstep_ms = ch.time_step(200)
        tfs = 2.0 * 1e8 / (fstep_ms / 1e3) / 1e12
        hr["fused_step"] = {"bound": "alu", "achieved": tfs, "peak": peak, "unit": "TFLOP/s", "frac": tfs / peak,
                            "ms_per_step": fstep_ms,
                            "what": "regenerating column pass + partial reduction + normalisation, statistics and stop rule"}
        _, rep = ch.stationary(tol=TOL)
        hr["fused_iters"] = int(rep["iters"])
        hr["fused_ms_per_pdf"] = pdf_wall_ms(ch)
        ch.close()
        hr["timing"] = "passes and steps replayed from one captured CUDA graph (no host launch overhead)"
        # the dead-time and signal sweep of the single-pixel workload (12 pixels),
        # each result against the FP64 oracle (L1 and max-abs)
        hx = W.highres()
        hrefs = None
        if not args.no_cpu_baseline:
            import oracle
            ro, rof, _, _ = oracle.batch_stationary(W.as_dicts(hx), tol=1e-12, nthreads=min(6, os.cpu_count() or 1))
            hrefs = [ro[rof[k]:rof[k + 1]] for k in range(len(hx))]
        sweep = []
        for k in range(len(hx)):
            q = hx[k:k + 1]
            row = {"t_d": float(q["t_d"][0]), "S": float(q["S"][0])}
            for mode, key in ((spl.SPL_MATERIALIZED, "materialized"), (spl.SPL_FUSED, "fused")):
                c = spl.Chain(q, mode)
                pq, rr = c.stationary(tol=TOL)
                row[key + "_iters"] = int(rr["iters"])
                row[key + "_status"] = int(rr["status"])
                if hrefs is not None:
                    d = np.abs(pq.cpu().numpy().astype(np.float64) - hrefs[k])
                    row[key + "_l1"] = float(d.sum())
                    row[key + "_max_abs"] = float(d.max())
                row[key + "_wall_ms_per_pdf"] = pdf_wall_ms(c, reps=5)
                c.close()
            sweep.append(row)
        hr["sweep"] = {"pixels": sweep,
                       "fused_wall_ms_per_pdf_median": statistics.median(r["fused_wall_ms_per_pdf"] for r in sweep),
                       "materialized_wall_ms_per_pdf_median":
                           statistics.median(r["materialized_wall_ms_per_pdf"] for r in sweep),
                       "wall_ms": "host wall time of one synchronous spl_stationary call (start vector, every step, "
                                  "stop rule and the report read back), not device time",
                       "workload": "N = 10000, t_d in {10, 40, 75, 130}, tau = 30, sigma = 0.3, S in {0.05, 0.5, 5}, B = 0.5"}
        if hrefs is not None:
            for key in ("materialized", "fused"):
                hr["sweep"][key + "_max_l1"] = max(r[key + "_l1"] for r in sweep)
                hr["sweep"][key + "_max_abs"] = max(r[key + "_max_abs"] for r in sweep)
        # the 12 sweep pixels in one multi-chain launch (one CTA group per
        # chain): device time of the whole call (start kernel, cooperative
        # launch, result copy) by CUDA events, L2 flushed between calls
        cs = spl.ChainSet(hx)
        mo, moff, mreps = cs.stationary(tol=TOL)
        assert np.all(mreps["status"] == 0)
        for _ in range(3):
            cs.stationary(tol=TOL, reports=False)
        mms, _ = timed_steps(lambda: cs.stationary(tol=TOL, out=mo, reports=False), 10, flush, stream)
        m_ms = statistics.median(mms)
        mflop = float(np.sum(2.0 * hx["n_bins"].astype(np.float64) ** 2 * mreps["iters"]))
        mt = mflop / (m_ms / 1e3) / 1e12
        multi = {"value": len(hx) / (m_ms / 1e3), "unit": "PDFs/s", "ms_per_call": m_ms,
                 "iters": mreps["iters"].tolist(),
                 "roofline": {"bound": "alu", "achieved": mt, "peak": peak, "unit": "TFLOP/s", "frac": mt / peak,
                              "work": "2 FLOP x N^2 per power step that the stop rule counts (iters), summed"},
                 "what": "spl_chains_stationary: 12 fused chains in lockstep in one cooperative launch "
                         "(each step's work of the chains still iterating split over all CTAs)"}
        if hrefs is not None:
            mo_h = mo.cpu().numpy().astype(np.float64)
            dd = [np.abs(mo_h[moff[k]:moff[k + 1]] - hrefs[k]) for k in range(len(hx))]
            multi["max_l1"] = max(float(d.sum()) for d in dd)
            multi["max_abs"] = max(float(d.max()) for d in dd)
        cs.close()
        hr["sweep"]["multi_chain_launch"] = multi
        extra["highres_n10000"] = hr

    # end to end through the public API: pixel list from host memory (copied
    # inside the call), every pmf read back to pinned host memory, per step
    # end to end through the host-buffer entry points: the pixel list from
    # pinned host memory, every pmf back into pinned host memory, per call
    # (the library overlaps the copy-back with compute); the pmfs must equal
    # the device path's bit for bit
    e2e_value, e2e_same = None, None
    if not args.no_e2e:
        h_out = torch.empty(total, dtype=torch.float32).pin_memory()
        if learned:
            fn = (lambda: net.batch_stationary_host(px, tol=TOL, max_iter=MAX_ITER, out=h_out, reports=False,
                                                    c_pixels=c_px, pass_kind=head_pass))
        else:
            h_np = h_out.numpy()
            fn = (lambda: spl.batch_stationary_host(px, tol=TOL, max_iter=MAX_ITER, out=h_np, reports=False,
                                                    c_pixels=c_px))
        fn()
        torch.cuda.synchronize()
        e2e_t = []
        for k in range(max(2, min(args.steps, 5))):
            flush_l2(flush)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            e2e_t.append(time.perf_counter() - t0)
        e2e_value = world * n / statistics.median(e2e_t)
        # the device path on the same pixels (out held another section's pmfs)
        if learned:
            learned_step()
        else:
            # the plain host-buffer entry point takes no options: the dense row pass
            spl.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, out=out, offsets=d_off, reports=False,
                                 c_pixels=c_px, pass_kind=spl.SPL_PASS_DENSE)
        torch.cuda.synchronize()
        e2e_same = bool(torch.equal(h_out, out.cpu()))
    h2d = n * 56
    d2h = total * 4

    # per step: pixel_const_kernel + batch_fused_kernel, and for the learned
    # start features_kernel + five GEMMs
    launches = 2 + (6 if learned else 0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pixels_per_gpu": n, "n_bins": 2000, "tol_l1": TOL,
                   "path": ("learned warm start (tcgen05 MLP) + batched matrix-free power iteration" if learned
                            else "plain batched (uniform start), matrix-free dense power step")
                           + "; every step regenerates all N^2 entries, row sums by O(N) scans",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}, pixels sharded, no collective"},
        "iters": {"mean": float(reps["iters"].mean()), "max": int(reps["iters"].max())},
        "gpu_launches": launches * args.steps,
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "host-buffer entry point (one launch; each of eight ranges copied back as soon as the kernel "
                        "has finished it)",
                "same_pmfs_as_device_path": e2e_same},
    }
    line.update(extra)
    if line_audit is not None:
        line["accuracy_vs_oracle"] = line_audit
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample, _ = cpu_sample(px, args.cpu_sample)
        rate, dt, used = oracle_rate(sample, os.cpu_count() or 1)
        rate1, dt1, _ = oracle_rate(sample[:args.cpu_sample_1t], 1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
                                "sample": f"{len(sample)} of the 65536 pixels (seed 55), {dt:.1f} s",
                                "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                                  "sample": f"the first {min(len(sample), args.cpu_sample_1t)} "
                                                            f"of those pixels, {dt1:.1f} s"}}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


PROFILE_CASES = ("batch_dense", "batch_structured", "gemv", "build", "chain_run", "chain_multi", "fma_peak")


def run_profile_case(name: str) -> int:
    """Small, fixed launch sequences for ncu captures (no timing, no JSON
    line): each case launches its kernel twice on the same inputs, so a
    capture with `-k regex:<kernel> -s 1 -c 1` takes a warm, full-size launch.
      batch_dense / batch_structured: 4096 pixels of the array workload (N = 2000),
          fixed launch heuristic (no tuning launches), the timed path's dense steps
          (row sums from scans) or the O(N) step;
      gemv / build / chain_run: one N = 10000 pixel (t_d = 75, S = 0.5), the
          materialised power step, the materialised build, the fused chain;
      chain_multi: the 12 pixels of the N = 10000 dead-time and signal sweep
          in one fused multi-pixel launch;
      fma_peak: the FP32 FMA throughput kernel."""
    import torch
    from paper_2509_20500_gb300 import build, spl, workloads as W
    build.build()
    spl.lib()
    torch.cuda.set_device(0)
    if name in ("batch_dense", "batch_structured"):
        px = W.array256()[:4096]
        pk = spl.SPL_PASS_DENSE_ROWSCAN if name == "batch_dense" else spl.SPL_PASS_STRUCTURED
        for _ in range(2):
            _, _, r = spl.batch_stationary(px, tol=TOL, max_iter=MAX_ITER, pass_kind=pk, tune=1)
            assert np.all(r["status"] == 0)
    elif name in ("gemv", "build", "chain_run"):
        hp = W.pixel(10000, 75.0, 30.0, 0.3, 0.5, 0.5)
        ch = spl.Chain(hp, spl.SPL_FUSED if name == "chain_run" else spl.SPL_MATERIALIZED)
        if name == "build":
            ch.time_build(1)
        else:
            for _ in range(2):
                _, r = ch.stationary(tol=TOL)
                assert r["status"] == 0
        ch.close()
    elif name == "chain_multi":
        hx = W.highres()
        for _ in range(2):
            _, _, r = spl.chains_stationary(hx, tol=TOL)
            assert np.all(r["status"] == 0)
    elif name == "fma_peak":
        spl.fp32_fma_peak(iters=20_000, reps=1)
    torch.cuda.synchronize()
    print(f"profile case {name} done", flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=512)
    ap.add_argument("--ref-sample", type=int, default=128)
    ap.add_argument("--cpu-sample-1t", type=int, default=48, help="pixels of the single-thread oracle timing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--pixels", type=int, default=0, help="use only the first P pixels (profiling)")
    ap.add_argument("--no-learned", action="store_true", help="time the plain batched path only")
    ap.add_argument("--no-highres", action="store_true")
    ap.add_argument("--no-structured", action="store_true")
    ap.add_argument("--no-rowpass", action="store_true")
    ap.add_argument("--no-noalloc", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-spectral", action="store_true")
    ap.add_argument("--no-mc", action="store_true")
    ap.add_argument("--mc-cycles", type=int, default=50000, help="laser cycles per Monte Carlo run")
    ap.add_argument("--audit", type=int, default=512, help="pixels of the timed output checked against the oracle")
    ap.add_argument("--train-pixels", type=int, default=200_000)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--profile-case", choices=PROFILE_CASES, help="run one small launch sequence for ncu and exit")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
