"""Benchmark: tiled Hogbom CLEAN with feedback on one GB300.

One step = one whole deconvolution of the 4096 x 4096 workload (8192^2 PSF,
500 synthetic point sources, 4 x 4 tiles, feedback every K = 50 minor
iterations per tile, gain 0.1, 50000 iterations, threshold 0 so the work is
fixed) through the C ABI: set-up, every round's minor loops and feedback,
the round closes.  Inputs are resident in HBM when the timed region starts.

Prints one JSON line: minor iterations per second (whole job), plus
  roofline      the dominant kernel's algorithmic bytes / CUDA-event time,
                against the L2 -> SM read bandwidth measured in the same run
                (the kernels' hot data is L2-resident)
  cpu_baseline  the CPU oracle on the host cores, on the first round of the
                same workload (a bounded sample)
  e2e           the same metric through clean_deconvolve_host with host
                buffers (host<->device copies inside the timed region)
  clocks        SM clocks and throttle reasons sampled during the timed region

--impl reference times the CPU oracle instead (one round of the same
workload per step) and prints the same kind of line with "impl": "reference".
Multi-GPU (torchrun): every rank deconvolves its own image (replicas, weak
scaling); there is no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "CLEAN minor iterations/s (4096^2, 4x4 tiles, feedback every K)"
UNIT = "iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tiled-4096")
    ap.add_argument("--K", type=int, default=50, help="feedback interval")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fft", action="store_true", help="skip the FFT-feedback comparison run")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-image leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--serve-jobs", type=int, default=60,
                    help="jobs of the serving leg (the sweep runs 500 at three loads)")
    ap.add_argument("--untiled-iters", type=int, default=2000,
                    help="iterations of the untiled whole-GPU comparison run (0: skip)")
    ap.add_argument("--sweep", action="store_true",
                    help="the measurement plan's other configurations: 256^2 untiled and "
                         "1024^2 tiled in full (GPU and CPU oracle), 4096^2 at K = 10..200 "
                         "(exact and FFT feedback); one JSON line, no headline")
    ap.add_argument("--profile", type=int, default=0, metavar="R",
                    help="profiling target: one run of the workload truncated to R rounds "
                         "(no warm-up, no timing, no JSON line)")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="R",
                    help="profiling target: the 64-image batch run for R rounds")
    ap.add_argument("--l2-sweep", action="store_true",
                    help="the L2 read probe over buffers of 8 MiB to 512 MiB (one JSON line)")
    return ap.parse_args()


def run_profile(args):
    """A small, bounded target for ncu captures: plan + one run of R rounds."""
    import torch

    import paper_2501_01461_gb300 as cg
    cg.lib()
    w, data = build_inputs(args)
    d_psf = torch.from_numpy(data["psf"]).cuda()
    d_dirty = torch.from_numpy(data["dirty"]).cuda()
    with cg.Plan(d_psf, w.n, w.n, gain=w.gain, niter=w.niter, threshold=0.0,
                 tiles=w.tiles, feedback_interval=w.feedback_interval) as plan:
        plan.run(d_dirty, max_rounds=args.profile)
        torch.cuda.synchronize()
        print(json.dumps({"profile_rounds": args.profile, "components": plan.n_components()}))


def run_profile_batch(args):
    """A bounded target for ncu captures of the batched kernels: the 64-image
    batch of the batch leg, one run of R rounds."""
    import torch

    import paper_2501_01461_gb300 as cg
    cg.lib()
    jobs = synth.batch_jobs(64)
    psfs = [torch.from_numpy(j["psf"]).cuda() for j in jobs]
    dirties = [torch.from_numpy(j["dirty"]).cuda() for j in jobs]
    spec = [dict(psf=psfs[i], ny=j["n"], nx=j["n"], gain=j["gain"], niter=j["niter"],
                 threshold=0.0, tiles=j["tiles"], feedback_interval=j["K"])
            for i, j in enumerate(jobs)]
    with cg.Batch(spec) as bt:
        bt.run(dirties, max_rounds=args.profile_batch)
        torch.cuda.synchronize()
        print(json.dumps({"profile_batch_rounds": args.profile_batch, **bt.stats()}))


def run_l2_sweep(args):
    """The L2 read probe over buffers of 8 to 512 MiB, every form: the
    bandwidth stays near its L2 value while the buffer fits in L2 and falls
    to the HBM rate beyond."""
    import torch

    import paper_2501_01461_gb300 as cg
    cg.lib()
    out = {}
    for mb in (8, 24, 48, 80, 512):
        buf = torch.ones(mb * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        for name, m, c in (("bulk_copy_1cta", 0, 1), ("bulk_copy_2cta", 0, 2),
                           ("vector_load_2cta", 1, 2), ("vector_load_4cta", 1, 4)):
            best = 0.0
            for _ in range(3):
                nb, ms = cg.probe_l2_read(buf, passes=max(2, 4800 // mb), method=m, ctas_per_sm=c)
                best = max(best, nb / (ms / 1e3) / 1e9)
            out[f"{mb}MiB_{name}"] = round(best, 1)
        del buf
    print(json.dumps({"l2_sweep_GBps": out}))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples (200 ms) taken while the timed region runs."""

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
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_workload(name: str, K: int, rank: int):
    """The workload a rank deconvolves: the same PSF and sizes on every rank,
    its own sky (seed offset by the rank), so the ranks solve independent
    problems.  Rank 0's image is the single-GPU one."""
    import dataclasses
    w = synth.workload(name, feedback_interval=K)
    return dataclasses.replace(w, seed=w.seed + 7919 * rank) if rank else w


def build_inputs(args, rank: int = 0):
    w = rank_workload(args.workload, args.K, rank)
    data = w.build(threshold=0.0)
    return w, data


def aggregate(dist, ms: float, units: float, device=None):
    """Whole-job figures over the ranks: the slowest rank's time (max) and
    the units all ranks processed (sum).  dist is torch.distributed or None
    (one process)."""
    if dist is None:
        return float(ms), float(units)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def minor_bytes_per_run(w) -> int:
    """Algorithmic bytes of all minor iterations of one run: each iteration of
    tile t reads its M_t residual pixels and the M_t-pixel PSF window and
    writes M_t residual pixels (12 M_t bytes)."""
    ty, tx = w.tiles
    T = ty * tx
    M = [((i + 1) * w.n // ty - i * w.n // ty) * ((j + 1) * w.n // tx - j * w.n // tx)
         for i in range(ty) for j in range(tx)]
    per_tile = [w.niter // T + (1 if t < w.niter % T else 0) for t in range(T)]
    return int(sum(12 * m * k for m, k in zip(M, per_tile)))


def feedback_updates_per_run(w) -> int:
    """Pixel-component updates of all feedbacks of one run (threshold 0, every
    tile spends its budget): each component updates every pixel outside its
    own tile once."""
    ty, tx = w.tiles
    T = ty * tx
    N2 = w.n * w.n
    M = [((i + 1) * w.n // ty - i * w.n // ty) * ((j + 1) * w.n // tx - j * w.n // tx)
         for i in range(ty) for j in range(tx)]
    per_tile = [w.niter // T + (1 if t < w.niter % T else 0) for t in range(T)]
    return int(sum((N2 - m) * k for m, k in zip(M, per_tile))) if w.feedback_interval > 0 else 0


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ncu_traffic() -> dict:
    """Per kernel, the committed ncu capture's record (DRAM bytes per launch,
    L2 throughput), kept only while the kernel's source file is unchanged
    since the capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    out = {}
    if not os.path.exists(p):
        return out
    with open(p) as f:
        rec = json.load(f)
    for name, r in rec.items():
        if not isinstance(r, dict) or "source" not in r:
            continue
        src = os.path.join(ROOT, r["source"])
        if os.path.exists(src):
            h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
            if h == r.get("sha256_16"):
                out[name] = r
    return out


def l2_peak(cg, torch, local):
    """L2 -> SM read bandwidth of this GPU, measured by the library's probe
    (clean_probe_l2_read) on a 48 MiB buffer (inside the 126 MB L2): bulk
    copies into shared memory (1 and 2 CTAs per SM) and 16-byte vector loads
    (2 and 4 CTAs per SM), 100 passes each, best of three timed launches.
    The peak is the fastest form; clocks are sampled while it runs."""
    buf = torch.ones(48 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.6)  # the sampler's first readings
    forms = {}
    for name, method, ctas in (("bulk_copy_1cta", 0, 1), ("bulk_copy_2cta", 0, 2),
                               ("vector_load_2cta", 1, 2), ("vector_load_4cta", 1, 4)):
        best = 0.0
        for _ in range(3):
            nb, ms = cg.probe_l2_read(buf, passes=100, method=method, ctas_per_sm=ctas)
            best = max(best, nb / (ms / 1e3) / 1e9)
        forms[name] = round(best, 1)
    clocks = sampler.stop()
    del buf
    top = max(forms, key=forms.get)
    return {"GBps": forms[top], "form": top, "forms_GBps": forms, "buffer_bytes": 48 << 20,
            "clocks": clocks,
            "method": "clean_probe_l2_read: 48 MiB buffer read 100 times over after a warm "
                      "pass, CUDA events, best of 3 per form"}


def batch_leg(cg, torch, stream, n_images=64):
    """64 images of uneven sizes (512..2048, per-channel PSFs): one batch vs
    the same images one at a time, tiled (same results, bit for bit) and
    plain untiled CLEAN on the whole GPU."""
    jobs = synth.batch_jobs(n_images)
    psfs = [torch.from_numpy(j["psf"]).cuda() for j in jobs]
    dirties = [torch.from_numpy(j["dirty"]).cuda() for j in jobs]
    total_iters = sum(j["niter"] for j in jobs)
    spec = [dict(psf=psfs[i], ny=j["n"], nx=j["n"], gain=j["gain"], niter=j["niter"],
                 threshold=0.0, tiles=j["tiles"], feedback_interval=j["K"])
            for i, j in enumerate(jobs)]

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        best = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            best.append(a.elapsed_time(b))
        return sum(best) / len(best)

    with cg.Batch(spec) as bt:
        ms_batch = timed(lambda: bt.run(dirties))
        st0 = bt.stats()
        bt.run(dirties)  # one more run, counted alone
        torch.cuda.synchronize()
        st1 = bt.stats()
    st = {k: st1[k] - st0[k] for k in ("rounds_launched", "kernel_launches")}
    solo = [cg.Plan(psfs[i], j["n"], j["n"], gain=j["gain"], niter=j["niter"], threshold=0.0,
                    tiles=j["tiles"], feedback_interval=j["K"]) for i, j in enumerate(jobs)]
    ms_solo = timed(lambda: [p.run(dirties[i]) for i, p in enumerate(solo)])
    for p in solo:
        p.close()
    plain = [cg.Plan(psfs[i], j["n"], j["n"], gain=j["gain"], niter=j["niter"], threshold=0.0,
                     tiles=(1, 1)) for i, j in enumerate(jobs)]
    ms_plain = timed(lambda: [p.run(dirties[i]) for i, p in enumerate(plain)], reps=1)
    for p in plain:
        p.close()
    sides = [j["n"] for j in jobs]
    # algorithmic bytes of one run: minor loop 12 B per pixel-iteration (of
    # the iteration's tile), feedback 4 B per pixel-component update + 8 N^2
    # per round; the iteration budget is spent in full (threshold 0)
    px_iter = bytes_ = 0.0
    for j in jobs:
        n, (ty, tx), nit, K = j["n"], j["tiles"], j["niter"], j["K"]
        T = ty * tx
        M = n * n / T
        px_iter += nit * M
        bytes_ += 12.0 * nit * M + 4.0 * nit * (n * n - M) + 8.0 * n * n * (-(-nit // (K * T)))
    return {"workload": f"{n_images} images, sides {sorted(set(sides))} (counts "
                        f"{[sides.count(v) for v in sorted(set(sides))]}), PSF 2N, freq scale 1-2, "
                        "2x2 tiles up to 1024 else 4x4, K 50, 2000 iterations each",
            "iters_per_s": total_iters / (ms_batch / 1e3), "ms_per_step": ms_batch,
            "one_at_a_time_tiled_iters_per_s": total_iters / (ms_solo / 1e3),
            "one_at_a_time_plain_iters_per_s": total_iters / (ms_plain / 1e3),
            "vs_one_at_a_time_tiled": ms_solo / ms_batch,
            "vs_one_at_a_time_plain": ms_plain / ms_batch,
            "px_iter_per_s": px_iter / (ms_batch / 1e3),
            "algorithmic_GBps": bytes_ / (ms_batch / 1e3) / 1e9,
            "rounds_per_run": st["rounds_launched"],
            "kernel_launches_per_run": st["kernel_launches"],
            "set_up_launches_per_run": n_images,
            "launches_per_round": (st["kernel_launches"] - n_images) / max(1, st["rounds_launched"]),
            "note": "per run: one set-up kernel per image, then each round one persistent "
                    "minor-loop launch over every image's tiles and one feedback launch"}


def serve_leg(cg, torch, psf_full, n_jobs=60, loads=(0.7,), seed=1004):
    """A Poisson stream of independent deconvolution jobs (sides log-uniform
    over 256 - 4096 rounded to multiples of 64, 10 - 500 sources, 1000 - 20000
    iterations, each its own dirty image) through the continuous-batching
    server, against one-at-a-time plain (untiled) CLEAN on the same arrivals:
    both run the queue in real time.  Arrival rates are `loads` x the
    one-at-a-time server's capacity (1 / its mean service time, measured on
    these jobs), so its queue is stable.  Latency counts from arrival to the
    job's results being done on the device."""
    from paper_2501_01461_gb300 import serve
    t_gen = time.perf_counter()
    specs = synth.serving_stream(psf_full, n_jobs, seed)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    mk = lambda sp, t=0.0: serve.Job(psf=sp["psf"], dirty=sp["dirty"], niter=sp["niter"],
                                     tiles=sp["tiles"], feedback_interval=sp["K"], arrival=t)

    def run_plain(job):  # one-at-a-time plain CLEAN: set-up, run, results ready
        with cg.Plan(job.psf, job.n, job.n, gain=0.1, niter=job.niter, threshold=0.0,
                     tiles=(1, 1)) as p:
            p.run(job.dirty)
            torch.cuda.synchronize()

    # warm-up: every side once each way (kernel attributes, tensor maps)
    seen = {}
    for sp in specs:
        seen.setdefault(sp["n"], sp)
    for sp in seen.values():
        w = dict(sp, niter=min(sp["niter"], 1000))
        run_plain(mk(w))
    serve.serve([mk(dict(sp, niter=min(sp["niter"], 1000))) for sp in seen.values()],
                budget_bytes=150e9, keep_results=False)
    service = []
    for sp in specs:
        t0 = time.perf_counter()
        run_plain(mk(sp))
        service.append(time.perf_counter() - t0)
    capacity = 1.0 / float(np.mean(service))
    gaps = np.random.default_rng(7).exponential(1.0, size=n_jobs)  # unit-rate Poisson
    out = {}
    for ld in loads:
        rate = ld * capacity
        arrivals = np.cumsum(gaps / rate)
        arrivals -= arrivals[0]
        base_jobs = [mk(sp, float(t)) for sp, t in zip(specs, arrivals)]
        base = serve.serve_one_at_a_time(base_jobs, run_plain)
        jobs = [mk(sp, float(t)) for sp, t in zip(specs, arrivals)]
        st = serve.serve(jobs, budget_bytes=150e9, rounds_per_step=2, keep_results=False)
        model = serve.fifo_latencies(arrivals, service)
        out[f"{ld:.1f}"] = {
            "arrival_rate_per_s": rate,
            "p50_s": st["p50_s"], "p99_s": st["p99_s"], "jobs_per_s": st["jobs_per_s"],
            "one_at_a_time_plain_p50_s": base["p50_s"], "one_at_a_time_plain_p99_s": base["p99_s"],
            "one_at_a_time_plain_jobs_per_s": base["jobs_per_s"],
            "modelled_fifo_p50_s": float(np.percentile(model, 50)),
            "modelled_fifo_p99_s": float(np.percentile(model, 99))}
    # saturated: every job waiting at t = 0
    jobs = [mk(sp) for sp in specs]
    sat = serve.serve(jobs, budget_bytes=150e9, rounds_per_step=4, keep_results=False)
    total_iters = sum(sp["niter"] for sp in specs)
    px_iter = sum(sp["niter"] * (sp["n"] ** 2) / (sp["tiles"][0] * sp["tiles"][1]) for sp in specs)
    sides = [sp["n"] for sp in specs]
    return {"workload": f"{n_jobs} jobs, sides log-uniform 256-4096 rounded to multiples of 64 "
                        f"({sum(1 for n in sides if n & (n - 1))} not powers of two), 10-500 "
                        "sources each (own dirty image), 1000-20000 iterations, gain 0.1, K 50, "
                        "tiles 1x1 / 2x2 / 4x4 by side, PSF 2N (crops of the 8192^2 array PSF), "
                        "Poisson arrivals, 150 GB admission budget",
            "loads": out,
            "one_at_a_time_plain_capacity_jobs_per_s": capacity,
            "saturated_jobs_per_s": sat["jobs_per_s"],
            "saturated_iters_per_s": total_iters / sat["makespan_s"],
            "saturated_px_iter_per_s": px_iter / sat["makespan_s"],
            "generation_s": t_gen,
            "note": "both servers run the queue in real time on the same arrivals; "
                    "modelled_fifo_* is the FIFO arithmetic on the measured solo service times, "
                    "for comparison only"}


def cpu_baseline(w, data):
    """The oracle as it stands, single-threaded, on the first round of the
    workload (every tile's first K iterations and that round's feedback)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.clean_f32(data["dirty"], data["psf"], w.gain, w.niter, 0.0, w.tiles,
                         w.feedback_interval, max_rounds=1)
    dt = time.perf_counter() - t0
    return {"value": r.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first round of {w.name}: {r.n} minor iterations + their feedback, "
                      f"{dt:.1f} s single-threaded C (float32, -O2)"}


def cpu_parallel_baseline(w, data):
    """The multi-core CPU baseline (the oracle's arithmetic with the tiles of
    a round on all host cores, OpenMP) on the same first round."""
    import oracle
    oracle.build_parallel()
    cores = oracle.parallel_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    r = oracle.parallel_clean_f32(data["dirty"], data["psf"], w.gain, w.niter, 0.0, w.tiles,
                                  w.feedback_interval, max_rounds=1)
    dt = time.perf_counter() - t0
    return {"value": r.n / dt, "unit": UNIT, "cores": cores, "kind": "oracle_parallel",
            "sample": f"first round of {w.name}: {r.n} minor iterations + their feedback, "
                      f"{dt:.1f} s on {cores} threads (float32, -O2, OpenMP over tiles)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w, data = build_inputs(args)
    import oracle
    oracle.build()
    times, n = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.clean_f32(data["dirty"], data["psf"], w.gain, w.niter, 0.0, w.tiles,
                             w.feedback_interval, max_rounds=1)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            n += r.n
    total = sum(times)
    value = n / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: first round of {w.name} "
                                       f"({n // args.steps} minor iterations + feedback)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """The measurement plan's configurations besides the headline: the 256^2
    untiled workload (whole-GPU grid mode, and the library's automatic group
    choice, a 16-CTA cluster) and the 1024^2 tiled one run in full on the GPU
    and on the CPU oracle (one thread, and the oracle's arithmetic on all host
    cores), and the 4096^2 workload at feedback intervals 10, 20, 50, 100 and
    200 with exact (gather) and FFT feedback, and the serving stream in full
    (500 jobs at 0.5, 0.7 and 0.9 x the one-at-a-time capacity, both servers
    run in real time).  GPU figures are the median of three CUDA-event-timed
    runs after one warm-up, with a 512 MiB write between runs; each run
    deconvolves the whole image."""
    import torch

    import oracle
    import paper_2501_01461_gb300 as cg
    cg.lib()
    oracle.build()
    oracle.build_parallel()
    cores = oracle.parallel_threads(os.cpu_count() or 1)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def gpu(w, data, thr, K, mode=cg.TILED, fb=cg.FB_GATHER, reps=3):
        P = torch.from_numpy(data["psf"]).cuda()
        D = torch.from_numpy(data["dirty"]).cuda()
        with cg.Plan(P, w.n, w.n, gain=w.gain, niter=w.niter, threshold=thr, tiles=w.tiles,
                     feedback_interval=K, mode=mode, feedback_mode=fb) as p:
            p.run(D)
            torch.cuda.synchronize()
            ms = []
            for i in range(reps):
                flush.fill_(float(i))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                p.run(D)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            n = p.n_components()
        med = sorted(ms)[len(ms) // 2]
        return {"iters": n, "ms": med, "iters_per_s": n / (med / 1e3)}

    def cpu(w, data, thr, K, parallel):
        t0 = time.perf_counter()
        if parallel:
            r = oracle.parallel_clean_f32(data["dirty"], data["psf"], w.gain, w.niter, thr,
                                          w.tiles, K)
        else:
            r = oracle.clean_f32(data["dirty"], data["psf"], w.gain, w.niter, thr, w.tiles, K)
        dt = time.perf_counter() - t0
        return {"iters": r.n, "s": dt, "iters_per_s": r.n / dt}

    def cfgd(w, thr):
        c = config_dict(w)
        c.pop("l2", None)
        c["threshold"] = thr
        return c

    out = {"sweep": True, "unit": UNIT, "cpu_cores": cores}
    w0 = synth.workload("untiled-256")
    d0 = w0.build()
    out["untiled-256"] = {
        "config": cfgd(w0, w0.threshold),
        "gpu_untiled_grid": gpu(w0, d0, w0.threshold, 0, mode=cg.UNTILED_GRID),
        "gpu_automatic_group": gpu(w0, d0, w0.threshold, 0),
        "cpu_oracle_1_thread": cpu(w0, d0, w0.threshold, 0, False),
        "cpu_oracle_all_cores": cpu(w0, d0, w0.threshold, 0, True)}
    w1 = synth.workload("tiled-1024")
    d1 = w1.build(threshold=0.0)
    out["tiled-1024"] = {
        "config": cfgd(w1, 0.0),
        "gpu_gather": gpu(w1, d1, 0.0, w1.feedback_interval),
        "gpu_fft": gpu(w1, d1, 0.0, w1.feedback_interval, fb=cg.FB_FFT),
        "cpu_oracle_1_thread": cpu(w1, d1, 0.0, w1.feedback_interval, False),
        "cpu_oracle_all_cores": cpu(w1, d1, 0.0, w1.feedback_interval, True)}
    w2 = synth.workload("tiled-4096")
    d2 = w2.build(threshold=0.0)
    ks = {}
    for K in (10, 20, 50, 100, 200):
        ks[str(K)] = {"gpu_gather": gpu(w2, d2, 0.0, K, reps=2),
                      "gpu_fft": gpu(w2, d2, 0.0, K, fb=cg.FB_FFT, reps=2)}
    out["tiled-4096-K"] = {"config": cfgd(w2, 0.0), "by_K": ks}
    # the serving workload in full: 500 jobs at 0.5, 0.7 and 0.9 x capacity
    out["served-500"] = serve_leg(cg, torch, d2["psf"], n_jobs=500, loads=(0.5, 0.7, 0.9))
    print(json.dumps(out))


def config_dict(w):
    return {"workload": w.name, "image": f"{w.n}x{w.n}", "psf": f"{w.psf_n}x{w.psf_n}",
            "tiles": f"{w.tiles[0]}x{w.tiles[1]}", "feedback_interval": w.feedback_interval,
            "niter": w.niter, "gain": w.gain, "threshold": 0.0, "sources": w.n_sources,
            "l2": "inputs larger than L2 (PSF 256 MiB) and a 512 MiB write between steps"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile > 0:
        run_profile(args)
        return
    if args.profile_batch > 0:
        run_profile_batch(args)
        return
    if args.l2_sweep:
        run_l2_sweep(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    import torch

    import paper_2501_01461_gb300 as cg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cg.lib()

    w, data = build_inputs(args, rank)
    psf, dirty = data["psf"], data["dirty"]
    d_psf = torch.from_numpy(psf).cuda()
    d_dirty = torch.from_numpy(dirty).cuda()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    plan = cg.Plan(d_psf, w.n, w.n, gain=w.gain, niter=w.niter, threshold=0.0,
                   tiles=w.tiles, feedback_interval=w.feedback_interval)
    for _ in range(args.warmup):
        plan.run(d_dirty)
    torch.cuda.synchronize()
    plan.debug_set(cg.DEBUG_TIMING, 1)
    launches0 = plan.stats()["kernel_launches"]

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))           # evicts L2 (outside the timed events)
        ev[i][0].record(stream)
        plan.run(d_dirty)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    st = plan.stats()
    gpu_launches = st["kernel_launches"] - launches0
    n_comp = plan.n_components()
    total_ms, all_comp = aggregate(dist, float(sum(step_ms)), n_comp * args.steps, "cuda")
    value = all_comp / (total_ms / 1e3)

    # ---- roofline of the dominant kernel, at the L2 level ----
    peaks, peak_src = measured_peaks()
    l2 = l2_peak(cg, torch, local)
    l2_gbs = l2["GBps"]
    minor_avg = st["minor_ms"] / max(st["minor_launches"], 1)
    fb_avg = st["feedback_ms"] / max(st["feedback_launches"], 1)
    rounds_per_run = st["minor_launches"] / args.steps
    minor_b = minor_bytes_per_run(w) / rounds_per_run           # per launch
    fb_upd = feedback_updates_per_run(w) / rounds_per_run       # per launch
    fb_b = 8.0 * w.n * w.n + 4.0 * fb_upd                       # per launch
    minor_gbs = minor_b / (minor_avg / 1e3) / 1e9
    fb_gbs = fb_b / (fb_avg / 1e3) / 1e9
    fb_tflops = 2.0 * fb_upd / (fb_avg / 1e3) / 1e12
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = st["sm_count"] * 128 * sm_mhz * 1e6 / 1e12
    rec = ncu_traffic()
    traffic = {k: v["bytes_per_launch"] for k, v in rec.items()}
    minor_name = ("minor_pair_kernel" if st.get("minor_pairs") else "minor_pipe_kernel") \
        if st["minor_pipe"] else "minor_kernel"
    fb_name = "feedback_tma_kernel" if st["feedback_tma"] else "feedback_kernel"
    l2_src = (f"measured in this run: {l2['form']} ({l2['method']}); MEASURED_PEAKS.json "
              f"holds no L2 figure (its HBM copy peak is {peaks['hbm_gbs']:.0f} GB/s, {peak_src})")
    if st["feedback_ms"] >= st["minor_ms"]:
        roof = {"kernel": fb_name, "bound": "l2", "achieved": fb_gbs, "peak": l2_gbs,
                "unit": "GB/s", "frac": fb_gbs / l2_gbs, "traffic": traffic.get(fb_name),
                "peak_source": l2_src, "bytes_per_launch": fb_b,
                "alu": {"achieved_TFLOPs": fb_tflops, "peak_TFLOPs": alu_peak,
                        "frac": fb_tflops / alu_peak,
                        "peak_source": f"derived: {st['sm_count']} SMs x 128 FP32 lanes x "
                                       f"{sm_mhz:.0f} MHz, separately rounded multiply and "
                                       "subtract (no fused multiply-add on this path)"},
                "note": "algorithmic bytes per launch = 8 N^2 (residual in and out) + 4 B of PSF "
                        "per pixel-component update; traffic = DRAM bytes per launch from ncu"}
    else:
        roof = {"kernel": minor_name, "bound": "l2", "achieved": minor_gbs, "peak": l2_gbs,
                "unit": "GB/s", "frac": minor_gbs / l2_gbs, "traffic": traffic.get(minor_name),
                "peak_source": l2_src, "bytes_per_launch": minor_b,
                "note": "12 B per pixel per tile iteration; traffic = DRAM bytes per launch"}
    kernels = {
        "minor": {"kernel": minor_name,
                  "ms_per_step": st["minor_ms"] / args.steps,
                  "launches_per_step": rounds_per_run,
                  "bytes_per_launch": minor_b, "algorithmic_GBps": minor_gbs,
                  "frac_of_l2_peak": minor_gbs / l2_gbs,
                  "traffic": traffic.get(minor_name),
                  "note": "12 B per pixel per tile iteration (read R, read the PSF window, "
                          "write R) over the measured L2 read peak"},
        "feedback": {"kernel": fb_name,
                     "ms_per_step": st["feedback_ms"] / args.steps,
                     "launches_per_step": st["feedback_launches"] / args.steps,
                     "bytes_per_launch": fb_b, "algorithmic_GBps": fb_gbs,
                     "frac_of_l2_peak": fb_gbs / l2_gbs,
                     "updates_per_s": fb_upd / (fb_avg / 1e3), "TFLOPs": fb_tflops,
                     "traffic": traffic.get(fb_name)},
    }

    # ---- end to end through host buffers ----
    e2e = None
    if not args.no_e2e:
        h_dirty = torch.from_numpy(dirty).pin_memory()
        h_psf = torch.from_numpy(psf).pin_memory()
        h_res = torch.empty_like(h_dirty).pin_memory()
        h_mod = torch.empty_like(h_dirty).pin_memory()
        h_comp = torch.empty((w.niter, 4), dtype=torch.int32).pin_memory()
        hp = cg.Plan(None, w.n, w.n, gain=w.gain, niter=w.niter, threshold=0.0,
                     tiles=w.tiles, feedback_interval=w.feedback_interval, psf_shape=psf.shape)

        def host_step():
            import ctypes
            n = ctypes.c_int64(0)
            rc = cg.lib().clean_deconvolve_host(
                hp.handle, ctypes.c_void_p(h_dirty.data_ptr()), ctypes.c_void_p(h_psf.data_ptr()),
                ctypes.c_void_p(h_res.data_ptr()), ctypes.c_void_p(h_mod.data_ptr()),
                ctypes.c_void_p(h_comp.data_ptr()), w.niter, ctypes.byref(n),
                ctypes.c_void_p(stream.cuda_stream))
            if rc:
                raise cg.CleanError(rc, "clean_deconvolve_host")
            return n.value
        for _ in range(max(1, args.warmup)):
            host_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e2e_sampler = ClockSampler(local)
        e2e_sampler.start()
        t0 = time.perf_counter()
        ne = 0
        e2e_steps, phases = [], []
        for _ in range(args.steps):
            ts = time.perf_counter()
            ne += host_step()
            e2e_steps.append((time.perf_counter() - ts) * 1e3)
            phases.append(hp.stats())
        te_ms, ne = aggregate(dist, (time.perf_counter() - t0) * 1e3, ne, "cuda")
        e2e_clocks = e2e_sampler.stop()
        hp.close()
        split = [{"wall_ms": round(wl, 2), "in_ms": round(p["host_in_ms"], 2),
                  "run_ms": round(p["host_run_ms"], 2), "out_ms": round(p["host_out_ms"], 2),
                  "host_ms": round(wl - p["host_in_ms"] - p["host_run_ms"] - p["host_out_ms"], 2)}
                 for wl, p in zip(e2e_steps, phases)]
        e2e = {"value": ne / (te_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(dirty.nbytes + psf.nbytes),
               "d2h_bytes_per_step": int(2 * dirty.nbytes + 16 * w.niter),
               "steps": split,
               "split_note": "per step: wall time of the call; CUDA-event times on its stream "
                             "of the input copies with the PSF check, the run, the output "
                             "copies; host_ms = the rest (host work and gaps)",
               "clocks": e2e_clocks}

    # ---- untiled whole-GPU Hogbom on the same image (rate on a prefix) ----
    untiled = None
    if args.untiled_iters > 0:
        up = cg.Plan(d_psf, w.n, w.n, gain=w.gain, niter=args.untiled_iters, threshold=0.0,
                     tiles=(1, 1))
        up.run(d_dirty)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        up.run(d_dirty)
        b.record(stream)
        torch.cuda.synchronize()
        ums = a.elapsed_time(b)
        untiled = {"iters": args.untiled_iters, "ms": ums,
                   "iters_per_s": args.untiled_iters / (ums / 1e3),
                   "px_iter_per_s": args.untiled_iters * w.n * w.n / (ums / 1e3)}
        up.close()

    # ---- the FFT feedback path on the same workload (tolerance-exact) ----
    fft = None
    if not args.no_fft:
        fp = cg.Plan(d_psf, w.n, w.n, gain=w.gain, niter=w.niter, threshold=0.0,
                     tiles=w.tiles, feedback_interval=w.feedback_interval,
                     feedback_mode=cg.FB_FFT)
        fp.run(d_dirty)
        torch.cuda.synchronize()
        fms = []
        for _ in range(2):
            flush.fill_(0.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fp.run(d_dirty)
            b.record(stream)
            torch.cuda.synchronize()
            fms.append(a.elapsed_time(b))
        fft = {"iters_per_s": w.niter * len(fms) / (sum(fms) / 1e3), "ms_per_step": sum(fms) / len(fms),
               "note": "feedback by FFT convolution with this library's own transforms (sparse "
                       "row DFT fused into pruned radix-16 column FFTs, paired-row inverse); "
                       "residual within 1e-4 Jy of the float64 replay, not bit-exact"}
        fp.close()

    # ---- batched: many uneven images together vs one at a time ----
    batched = None
    if not args.no_batch:
        batched = batch_leg(cg, torch, stream)
        batched["frac_of_l2_peak"] = batched["algorithmic_GBps"] / l2_gbs

    served = None
    if not args.no_serve:
        served = serve_leg(cg, torch, psf, n_jobs=args.serve_jobs)

    cpu = cpu_par = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, data)
        cpu["cores"] = 1
        cpu_par = cpu_parallel_baseline(w, data)

    if rank == 0:
        ty, tx = w.tiles
        px_iter = sum(((i + 1) * w.n // ty - i * w.n // ty) * ((j + 1) * w.n // tx - j * w.n // tx)
                      for i in range(ty) for j in range(tx)) / (ty * tx)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (VLA-like Y array PSF, seeded point-source sky)",
            "config": config_dict(w),
            "px_iter_per_s": value * px_iter,
            "feedback_px_comp_per_s": world * feedback_updates_per_run(w) * args.steps / (total_ms / 1e3),
            "roofline": roof, "kernels": kernels, "l2_probe": l2,
            "cpu_baseline": cpu, "cpu_parallel_baseline": cpu_par,
            "e2e": e2e, "untiled_gpu": untiled,
            "vs_untiled_gpu": (value / untiled["iters_per_s"]) if untiled else None,
            "fft_feedback": fft,
            "batched": batched,
            "served": served,
            "gpu_launches": int(gpu_launches),
            "clocks": clocks, "wall_s_timed": wall,
            "plan": {k: st[k] for k in ("group_ctas", "group_sync", "resident", "sm_count")},
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
