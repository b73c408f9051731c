"""Benchmark of the AGIS hot path on GB300: AL+AC observations per second per AGIS iteration.

One step = one S[ACG] iteration (S pass and 5x5 solves, A pass and segmented banded
Cholesky, C pass and constraint projection, frame rotator) over the whole synthetic
workload, replayed as per-block CUDA graphs.  Inputs are resident in HBM for `value`; `e2e`
repeats the measurement through the C ABI from host buffers (upload, set-up, one
iteration, read-back of the updated sources).  The headline form is FP64 (`--precision
mixed` makes the mixed-precision form the headline); the other form is timed on the same
data and reported beside it, the mixed form over whole refresh cycles.  `--impl reference`
times the FP64 oracle on the host cores on a bounded sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]
For N > 1 (launched with torch.distributed.run) the sources are split over the ranks and
every iteration all-reduces the attitude and calibration normals and the frame sums (NCCL);
every rank then solves the same sums (strong scaling: one problem).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "scale5yr": "1M sources, 5 yr, 30-s knots, 1-day calibration, sigma_AL 100 uas, 1% outliers",
    "small1yr": "10k sources, 1 yr, 1-h knots, 1-day calibration, sigma_AL 100 uas, 1% outliers",
    "uneven5yr": "3M sources, 5 yr, 30-s knots, G ~ U(12, 18) with sigma_AL 50-500 uas, 40-250 transits",
}
# kernels launched by one iteration, (with a full FP64 evaluation, with the linearized pass):
# FP64 form: S (source geometry, observation pass, per-source solve, stats in two stages,
# update-history push), A (accumulate, assemble, solve, apply, rank-defect sum), C
# (accumulate, project, rank-defect sum), frame (normals, solve, apply sources, apply
# attitude) = 18.  Mixed form: the S pass is source geometry + full evaluation, or the one
# linearized-correction kernel; the S solves are scale/round-0 sums, 5 rounds of 5x5 algebra,
# 4 rounds of sums, final pass, per-observation path, stats (two), history push = 15 (default
# 4 reweighting rounds); A, C and frame as above.
KERNELS_PER_STEP = {"fp64": (18, 18), "mixed": (2 + 15 + 12, 1 + 15 + 12)}
# with the excess attitude noise on: x values, per-bucket selection, attitude weights
KERNELS_ATTNOISE = 3
FALLBACK_HBM_GBS = 6800.0
# algorithmic bytes per observation of the linearized observation pass (see time_form)
MIX_PASS_BYTES = 8 + 16 + 4 + 8 + 8
# DRAM bytes per observation (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture
# of 2.47e7 observations, scaled per observation; profiles/k_*_kernels_30k.md): the S block of
# the FP64 form (observation pass + solves) and the mixed form's linearized pass.  None once
# the kernel has changed since its capture.
TRAFFIC_PER_OBS = {"fp64_s_block": 780.0, "mixed_correct": 47.6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="scale5yr", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--n-src", type=int, default=0, help="override the number of sources (testing)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="form timed for the headline value (the other is reported beside it)")
    ap.add_argument("--refresh-every", type=int, default=8, help="mixed form: full FP64 evaluation period")
    ap.add_argument("--single-form", action="store_true", help="time only the --precision form")
    ap.add_argument("--tune-iters", type=int, default=20,
                    help="iterations of the launch-shape autotuner before the warm-up (0: default shapes)")
    ap.add_argument("--knot-dt-s", type=int, default=0, help="override the attitude knot interval (testing)")
    ap.add_argument("--cal-generic", action="store_true",
                    help="the full geometric calibration model (two gates, 30-day long intervals, binned columns)")
    ap.add_argument("--cal-col-bin", type=int, default=16, help="--cal-generic: AC pixel columns per bin")
    ap.add_argument("--no-convergence", action="store_true",
                    help="skip the wall-time-to-1-uas runs that the default line carries")
    ap.add_argument("--convergence", action="store_true",
                    help="wall time to 1 uas RMS of both forms against an FP64 reference solution")
    ap.add_argument("--ref-max-iter", type=int, default=160, help="convergence: cap of the FP64 reference run")
    ap.add_argument("--ref-tol-uas", type=float, default=1e-3, help="convergence: reference stops below this update")
    ap.add_argument("--learned", action="store_true",
                    help="convergence: also the mixed form with the learned proposal, trained first on two "
                         "held-out 100k-source 5-year sets")
    ap.add_argument("--proposal-every", type=int, default=5, help="iterations between learned proposals")
    ap.add_argument("--asi", action="store_true",
                    help="with --convergence: also the accelerated simple iteration (Sect. 4.7) in both forms")
    ap.add_argument("--asi-stride", type=int, default=16, help="ASI: every n-th source enters the lambda estimate")
    ap.add_argument("--orders", action="store_true",
                    help="with --convergence: also the Gauss-Seidel and Jacobi block orders (Sect. 4.6), mixed form")
    ap.add_argument("--asi-lambda-max", type=float, default=0.9, help="ASI: clamp of the lambda estimate")
    ap.add_argument("--attnoise-s", type=float, default=0.0,
                    help="estimate the excess attitude noise on buckets of this many seconds (either form, "
                         "--single-form; 0: off)")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, dist):
    """The largest x over the ranks (the whole job's time is its slowest replica's); x itself
    when there is no process group.  NCCL reduces a device tensor, gloo a host one."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, max clock, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# Algorithmic FP64 flops per observation of the S block (the FP64 form's roofline), counted
# with an FMA as two flops like the peak it is divided by: model and residual ~200, partials
# ~100, the source normal equations 20 FMA = 40 (one accumulation of the 15 + 5 products).
# The peak follows from the unit count and the clock: 152 SMs x 2 FP64 FMA per clock per SM
# x 2 flops x 2.07 GHz = 1.259 TFLOP/s (GB300's nominal 1.25).
S_FLOPS_PER_OBS = 200 + 100 + 40
FP64_PEAK_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _oracle_task(kind, payload):
    """One piece of the oracle's iteration, timed in a worker process: an S block on a batch of
    sources, an A block on one segment, or a C block on one calibration interval."""
    import oracle.blocks as OB
    import oracle.model as OM
    t0 = time.perf_counter()
    if kind == "S":
        sub, st = payload
        P = OM.problem_from_dataset(sub)
        OB.source_update(P, sub.src0, sub.att0, sub.cal0, st)
        n = sub.n_obs
    elif kind == "A":
        sub, st, l_lo, l_hi = payload
        P = OM.problem_from_dataset(sub)
        ev = OM.evaluate(P, sub.src0, sub.att0, sub.cal0)
        W = 1.0 / sub.sigma.astype(np.float64) ** 2
        Nb, b = OB.attitude_normals(P, ev, ev["R"], W, st, l_lo, l_hi)
        from oracle import cholesky as CH
        CH.band_solve(Nb, b)
        n = sub.n_obs
    else:
        sub = payload
        P = OM.problem_from_dataset(sub)
        ev = OM.evaluate(P, sub.src0, sub.att0, sub.cal0, partials=False)
        np.bincount(ev["cal_k"], weights=1.0 / sub.sigma.astype(np.float64) ** 2, minlength=P.n_cal)
        n = sub.n_obs
    return n, time.perf_counter() - t0


def _obs_subset(ds, sel):
    import dataclasses
    take = lambda a: np.ascontiguousarray(a[sel])  # noqa: E731
    return dataclasses.replace(ds, t_ns=take(ds.t_ns), src=take(ds.src), ccd=take(ds.ccd), fov=take(ds.fov),
                               kind=take(ds.kind), sigma=take(ds.sigma), mu=take(ds.mu), noise=take(ds.noise),
                               gate=take(ds.gate))


def _src_range(ds, off, i0, i1):
    """The sources i0..i1-1 (contiguous) with their observations, renumbered from 0 (the
    observations are sorted by source, so this is one slice)."""
    import dataclasses
    sl = slice(int(off[i0]), int(off[i1]))
    take = lambda a: np.ascontiguousarray(a[sl])  # noqa: E731
    return dataclasses.replace(ds, t_ns=take(ds.t_ns), src=(take(ds.src) - i0).astype(np.int32), ccd=take(ds.ccd),
                               fov=take(ds.fov), kind=take(ds.kind), sigma=take(ds.sigma), mu=take(ds.mu),
                               noise=take(ds.noise), gate=take(ds.gate), src_true=ds.src_true[i0:i1].copy(),
                               src_mag=ds.src_mag[i0:i1].copy(), n_transits=ds.n_transits[i0:i1].copy(),
                               src0=ds.src0[i0:i1].copy())


class OracleSampler:
    """The FP64 oracle on the host cores, on bounded samples of the workload, scaled to
    observations/s per iteration.  Pieces of the iteration are independent (sources in the S
    block, segments in the A block, intervals in the C block) and run in a pool of worker
    processes (spawn start, one per core, single-threaded BLAS).  A sample: S on runs of 50
    consecutive sources from random places for a time budget, A on some segments (all
    observations of their time range, spread over the mission), C on some calibration
    intervals.  The iteration time is the observations / throughput of each block; the
    single-core figure comes from the summed task times of the same runs."""

    def __init__(self, ds, workers=None, n_seg=None, n_day=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        import oracle.blocks as OB
        import oracle.model as OM
        self.ds = ds
        self.workers = workers or min(16, os.cpu_count() or 1)
        P = OM.problem_from_dataset(ds)
        self.st = OB.Settings(seg_len=2880 if ds.geometry["knot_dt_ns"] == 30_000_000_000 else 720, seg_overlap=12)
        self.off = ds.src_offsets()
        self.starts = np.random.default_rng(0).permutation(max(1, ds.n_src // 50)) * 50
        self.next_start = 0
        self.segs = OB.segments(P, self.st)
        kn = P.knots()
        self.days = ds.geometry["n_cal_days"]
        n_seg = n_seg or self.workers
        n_day = n_day or self.workers
        pick_a = np.linspace(0, len(self.segs) - 1, min(n_seg, len(self.segs))).astype(int)
        pick_c = np.linspace(0, self.days - 1, min(n_day, self.days)).astype(int)
        t = time.perf_counter()
        self.args_a = [(_obs_subset(ds, np.nonzero((ds.t_ns >= kn[self.segs[k][0]]) &
                                                   (ds.t_ns < kn[self.segs[k][1] + 1]))[0]),
                        self.st, self.segs[k][0], self.segs[k][1]) for k in pick_a]
        day = OM.cal_day(P, ds.t_ns)
        self.args_c = [_obs_subset(ds, np.nonzero(day == d)[0]) for d in pick_c]
        self.t_select = time.perf_counter() - t
        self.env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in self.env_keep:
            os.environ[k] = "1"
        self.ex = cf.ProcessPoolExecutor(max_workers=self.workers, mp_context=mp.get_context("spawn"))
        warm = _src_range(ds, self.off, 0, min(2, ds.n_src))
        list(self.ex.map(_oracle_task, ["S"] * self.workers, [(warm, self.st)] * self.workers))  # start-up

    def close(self):
        self.ex.shutdown()
        for k, v in self.env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

    def step(self, s_seconds, n_seg, n_day):
        import concurrent.futures as cf
        ds, ex, st = self.ds, self.ex, self.st
        t0 = time.perf_counter()
        futs, n_s, t_s_tasks, n_tasks = [], 0, 0.0, 0
        while time.perf_counter() - t0 < s_seconds or n_tasks == 0:
            while len(futs) < 2 * self.workers:
                i0 = int(self.starts[self.next_start % self.starts.size])
                self.next_start += 1
                futs.append(ex.submit(_oracle_task, "S", (_src_range(ds, self.off, i0, min(ds.n_src, i0 + 50)), st)))
            done, pending = cf.wait(futs, return_when=cf.FIRST_COMPLETED)
            for f in done:
                n, dt = f.result()
                n_s, t_s_tasks, n_tasks = n_s + n, t_s_tasks + dt, n_tasks + 1
            futs = list(pending)
        for f in futs:
            n, dt = f.result()
            n_s, t_s_tasks, n_tasks = n_s + n, t_s_tasks + dt, n_tasks + 1
        thr_s = n_s / (time.perf_counter() - t0)
        thr_s1 = n_s / t_s_tasks
        args_a = self.args_a[:n_seg]
        t1 = time.perf_counter()
        res_a = list(ex.map(_oracle_task, ["A"] * len(args_a), args_a))
        thr_a = len(args_a) / (time.perf_counter() - t1)
        thr_a1 = len(args_a) / sum(r[1] for r in res_a)
        args_c = self.args_c[:n_day]
        t2 = time.perf_counter()
        res_c = list(ex.map(_oracle_task, ["C"] * len(args_c), args_c))
        thr_c = len(args_c) / (time.perf_counter() - t2)
        thr_c1 = len(args_c) / sum(r[1] for r in res_c)
        t_iter = ds.n_obs / thr_s + len(self.segs) / thr_a + self.days / thr_c
        t_iter1 = ds.n_obs / thr_s1 + len(self.segs) / thr_a1 + self.days / thr_c1
        distinct = min(n_tasks, self.starts.size)
        again = f", {n_tasks - distinct} of them again (the set has {self.starts.size})" if n_tasks > distinct else ""
        sample = (f"S block on {n_s} obs of {n_tasks} runs of 50 consecutive sources from random places{again}, "
                  f"A block on {len(res_a)} of {len(self.segs)} segments "
                  f"(~{int(np.mean([r[0] for r in res_a]))} obs each), C block on {len(res_c)} of {self.days} "
                  f"intervals, in {self.workers} worker processes; per-iteration time extrapolated to {ds.n_obs} obs "
                  f"= {t_iter:.1f} s ({t_iter1:.1f} s on one core); sample selection {self.t_select:.1f} s, not counted")
        cpu = ""
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            cpu = next((ln.split(":", 1)[1].strip() for ln in out.splitlines() if ln.startswith("Model name")), "")
        except OSError:
            pass
        return {"value": ds.n_obs / t_iter, "unit": "obs/s", "cores": self.workers, "kind": "oracle", "sample": sample,
                "single_core_value": ds.n_obs / t_iter1, "cpu_model": cpu, "host_cores": os.cpu_count()}


def cpu_baseline(ds, seconds=20.0, workers=None):
    """One sample of OracleSampler: S for half the budget, A on one segment and C on one
    interval per worker."""
    smp = OracleSampler(ds, workers)
    try:
        return smp.step(0.5 * seconds, smp.workers, smp.workers)
    finally:
        smp.close()


def make_dataset(args):
    import synth
    over = {}
    if args.n_src:
        over["n_src"] = args.n_src
    if args.knot_dt_s:
        over["knot_dt_s"] = args.knot_dt_s
    if args.cal_generic:
        # the full geometric calibration: two gates, 30-day long intervals, 16-column bins
        over.update(cal_generic=True, n_gate=2, cal_j_per_k=30, cal_col_bin=args.cal_col_bin)
    t = time.perf_counter()
    ds = synth.simulate(synth.config(args.workload, **over))
    return ds, time.perf_counter() - t


def run_reference(args, rank, world):
    if rank != 0:
        return
    ds, _ = make_dataset(args)
    vals = []
    # one pool and sample selection for the run; each step a bounded sample (S for a few
    # seconds, A on a few segments, C on a few intervals), the whole run within a few minutes
    n_steps = max(1, args.warmup + args.steps)
    smp = OracleSampler(ds, n_seg=4, n_day=4)
    try:
        for k in range(n_steps):
            cb = smp.step(max(2.0, 60.0 / n_steps), 4, 4)
            if k >= args.warmup:
                vals.append(cb)
    finally:
        smp.close()
    v = float(np.median([c["value"] for c in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": "AL+AC observations/s per AGIS iteration", "value": v, "unit": "obs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ds.n_obs / v * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n_obs": ds.n_obs,
                       "n_src": ds.n_src}, "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "obs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_form(agis, ds, stream, cfg, steps, warmup, local, dist, tune_iters=0, attnoise_ns=0):
    """Device-resident timing of `steps` iterations after `warmup` untimed ones; before the
    warm-up, up to `tune_iters` iterations of the launch-shape autotuner (untimed).
    attnoise_ns > 0: the excess attitude noise estimated on buckets of that length."""
    import torch
    # the context copies the observations into HBM at set-up; the timed iterations read only
    # device-resident data
    obs_h = agis.obs_from_dataset(ds)
    t = time.perf_counter()
    g = agis.Agis(ds.geometry, cfg, obs_h, np.ascontiguousarray(ds.src0), np.ascontiguousarray(ds.att0),
                  np.ascontiguousarray(ds.cal0), src_ref=np.ascontiguousarray(ds.src_true[:, [0, 1, 3, 4]]),
                  stream=stream.cuda_stream)
    if attnoise_ns > 0:
        g.set_attnoise(attnoise_ns)
    t_init = time.perf_counter() - t
    del obs_h
    tuning = None
    if tune_iters > 0:
        t = time.perf_counter()
        n_t, rep = g.autotune(tune_iters)
        tuning = {"iterations": n_t, "seconds": round(time.perf_counter() - t, 2),
                  "shapes": {k: [v["a"], v["b"]] for k, v in rep.items() if v["n_tried"]},
                  "block_ms_default_vs_kept": {k: [round(v["default_ms"], 3), round(v["best_ms"], 3)]
                                               for k, v in rep.items() if v["n_tried"]}}
    g.iterate(warmup)
    # flush-free timing: the inputs (>= tens of GB) are far larger than the 129 MB L2
    sampler = ClockSampler(local)
    sampler.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    its = g.iterate(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / steps
    if dist is not None:
        ms = max_over_ranks(ms, dist)
    g.close()
    full = [it for it in its if it["s"]["full_eval"]]
    lin = [it for it in its if not it["s"]["full_eval"]]
    med = lambda xs: float(np.median(xs)) if xs else None
    return {"ms": ms, "t_init": t_init, "clocks": clocks, "n_full_eval": len(full), "tuning": tuning,
            "s_ms": med([it["s"]["elapsed_ms"] for it in its]), "a_ms": med([it["a"]["elapsed_ms"] for it in its]),
            "c_ms": med([it["c"]["elapsed_ms"] for it in its]),
            "pass_full_ms": med([it["s"]["pass_ms"] for it in full]),
            "pass_lin_ms": med([it["s"]["pass_ms"] for it in lin]),
            "solve_ms": med([it["s"]["elapsed_ms"] - it["s"]["pass_ms"] for it in its])}


def run_partitioned(args, agis, ds, stream, rank, world, local, dist, t_gen):
    """N > 1: one problem, its sources split into N contiguous parts of about equal observation
    counts, one part per rank (strong scaling).  Per iteration every rank runs its source
    update; the attitude and calibration normals and the frame sums of the parts are added by
    NCCL all-reduces of device buffers, and every rank solves the same sums
    (paper_1112_4139_gb300/partition.py).  value = all observations / the slowest rank's time."""
    import torch
    from paper_1112_4139_gb300 import partition
    b = partition.split_sources(ds.src_offsets(), world)
    part = ds.subset_sources(np.arange(b[rank], b[rank + 1]))
    seg_len = 2880 if ds.geometry["knot_dt_ns"] <= 30_000_000_000 else 720
    cfg = agis.default_config(seg_len=seg_len, use_graph=1, frame_each_iter=1, precision=0)
    obs_h = agis.obs_from_dataset(part)
    t = time.perf_counter()
    g = agis.Agis(part.geometry, cfg, obs_h, np.ascontiguousarray(part.src0), np.ascontiguousarray(part.att0),
                  np.ascontiguousarray(part.cal0), src_ref=np.ascontiguousarray(part.src_true[:, [0, 1, 3, 4]]),
                  stream=stream.cuda_stream)
    t_init = time.perf_counter() - t
    like = torch.zeros(1, dtype=torch.float64, device="cuda")
    bufs = partition.make_buffers([g], like=like)
    red = partition.LocalSum(dist.group.WORLD)
    partition.iterate([g], red, args.warmup, bufs=bufs, sync=torch.cuda.synchronize)
    sampler = ClockSampler(local)
    sampler.start()
    dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    partition.iterate([g], red, args.steps, bufs=bufs, sync=torch.cuda.synchronize)
    ev1.record()
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist)
    g.close()
    n_total = int(max_over_ranks(float(ds.n_obs), dist))
    # end to end: upload of the rank's part from pinned host buffers, one partitioned iteration,
    # read-back of the rank's sources
    import torch as T
    host = {k: T.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in agis.obs_from_dataset(part).items()}
    st0 = [T.from_numpy(np.ascontiguousarray(a)).pin_memory()
           for a in (part.src0, part.att0, part.cal0, part.src_true[:, [0, 1, 3, 4]])]
    out_src = T.empty((part.n_src, 5), dtype=T.float64).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values()) + sum(v.numel() * v.element_size() for v in st0)
    e2e_t = []
    for _ in range(args.e2e_steps):
        dist.barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        ge = agis.Agis(part.geometry, cfg, host, st0[0], st0[1], st0[2], src_ref=st0[3], stream=stream.cuda_stream)
        partition.iterate([ge], red, 1, bufs=bufs, sync=torch.cuda.synchronize)
        ge.sources(out=out_src.numpy())
        torch.cuda.synchronize()
        e2e_t.append(max_over_ranks(time.perf_counter() - t, dist))
        ge.close()
    value = n_total / (ms * 1e-3)
    line = {
        "metric": "AL+AC observations/s per AGIS iteration", "value": value, "unit": "obs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n_obs": n_total,
                   "n_src": ds.n_src, "n_coef": ds.n_coef, "n_cal": ds.n_cal, "precision": "fp64",
                   "l2": "no flush: inputs (tens of GB) exceed the 129 MB L2", "graph": False,
                   "parallelism": f"sources split over {world} GPUs; attitude, calibration and frame sums "
                                  "all-reduced (NCCL)", "t_generate_s": round(t_gen, 1), "t_init_s": round(t_init, 2)},
        "e2e": ({"value": n_total / float(np.median(e2e_t)), "unit": "obs/s", "h2d_bytes_per_step": int(h2d),
                 "d2h_bytes_per_step": int(out_src.numel() * 8)} if e2e_t else None),
        "gpu_launches": (KERNELS_PER_STEP["fp64"][0] + 1) * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def run_convergence(args, agis, ds, stream, rank, emit=True):
    """Wall time to 1 uas RMS (all sources, 5 parameters, uas and uas/yr) of each form against
    x_ref, the FP64 solution iterated until its largest update is below --ref-tol-uas (or
    --ref-max-iter iterations).  Both runs rotate the frame onto the same reference every
    iteration.  Iteration times are device time (CUDA events around each iteration); the
    read-back of the sources for the monitoring is not counted."""
    import synth
    UAS = synth.UAS
    seg_len = 2880 if ds.geometry["knot_dt_ns"] <= 30_000_000_000 else 720
    ref = np.ascontiguousarray(ds.src_true[:, [0, 1, 3, 4]])
    cosd = np.cos(ds.src_true[:, 1])

    def diff_uas(a, b):
        e = a - b
        e[:, 0] = (np.mod(e[:, 0] + np.pi, 2 * np.pi) - np.pi) * cosd
        return e / UAS

    def open_form(prec, order=0):
        cfg = agis.default_config(seg_len=seg_len, use_graph=1, frame_each_iter=1, precision=prec,
                                  refresh_every=args.refresh_every, block_order=order)
        return agis.Agis(ds.geometry, cfg, agis.obs_from_dataset(ds), np.ascontiguousarray(ds.src0),
                         np.ascontiguousarray(ds.att0), np.ascontiguousarray(ds.cal0), src_ref=ref,
                         stream=stream.cuda_stream)

    # FP64 reference trajectory: per-iteration updates kept as FP32 differences in uas
    g = open_form(0)
    prev = g.sources()
    deltas, t64 = [], []
    k = 0
    while k < args.ref_max_iter:
        its = g.iterate(1)
        t64.append(its[0]["elapsed_ms"])
        cur = g.sources()
        dlt = diff_uas(cur, prev)
        deltas.append(dlt.astype(np.float32))
        prev = cur
        k += 1
        if np.max(np.abs(dlt)) < args.ref_tol_uas:
            break
    x_ref = prev
    ref_last_update = float(np.max(np.abs(deltas[-1])))
    g.close()
    # RMS of x_k - x_ref from the stored updates, backwards
    tail = np.zeros_like(deltas[0], dtype=np.float64)
    rms64 = [0.0] * len(deltas)
    for j in range(len(deltas) - 1, -1, -1):
        rms64[j] = float(np.sqrt(np.mean(tail ** 2)))
        tail += deltas[j]
    del deltas

    def first_below(rms, times, thr=1.0):
        # the first iteration from which the RMS stays at or below thr (a proposal can dip
        # below it for one iteration)
        above = [j for j, v in enumerate(rms) if v > thr]
        j = (above[-1] + 1) if above else 0
        if j >= len(rms):
            return None, None
        return j + 1, float(np.sum(times[:j + 1])) * 1e-3

    it64, s64 = first_below(rms64, t64)
    # the other runs against the same reference
    def run_mixed(params=None, extra=3, asi=False, prec=1, order=0):
        g = open_form(prec, order)
        if params is not None:
            g.set_proposal(params, args.proposal_every)
        if asi:
            g.set_asi(args.asi_stride, args.asi_lambda_max)
        rms, tms, props, per_param, below = [], [], [], None, 0
        for k in range(args.ref_max_iter):
            its = g.iterate(1)
            tms.append(its[0]["elapsed_ms"])
            props.append(its[0]["asi_factor"] if asi else its[0]["proposal"])
            e = diff_uas(g.sources(), x_ref)
            rms.append(float(np.sqrt(np.mean(e ** 2))))
            below = below + 1 if rms[-1] <= 1.0 else 0
            if below == 1:
                per_param = np.sqrt(np.mean(e ** 2, axis=0)).tolist()
            if below > extra:   # stays below for a few iterations
                break
        g.close()
        return rms, tms, props, per_param

    rmsm, tm, _, per_param = run_mixed()
    itm, sm = first_below(rmsm, tm)
    learned_line = None
    learned_asi_line = None
    if args.learned:
        import torch
        from paper_1112_4139_gb300 import learned
        t0 = time.perf_counter()
        Xs, Ts = [], []
        for seed in (301, 302):
            tds = synth.simulate(synth.config("scale5yr", n_src=100_000, knot_dt_s=300, seed=seed))
            X, T, _ = learned.collect(tds, 80, 220, first=3, stride=1, seg_len=2880, seg_overlap=12, precision=1,
                                      refresh_every=args.refresh_every)
            Xs.append(X)
            Ts.append(T)
        params, hist = learned.train(torch.cat(Xs), torch.cat(Ts), steps=12000, batch=16384, lr=2e-3,
                                     lr_final=5e-5, log_every=12000)
        del Xs, Ts
        t_train = time.perf_counter() - t0
        rmsl, tl, props, per_l = run_mixed(params)
        itl, sl = first_below(rmsl, tl)
        if args.asi:
            # the proposal with ASI in the iterations that carry none (Sect. 4.7)
            rmsla, tla, propsa, per_la = run_mixed(params, asi=True)
            itla, sla = first_below(rmsla, tla)
            learned_asi_line = {"iterations": itla, "seconds": sla, "ms_per_iter": float(np.median(tla)),
                                "rms_uas": [round(v, 4) for v in rmsla], "per_param_rms_uas_at_1uas": per_la}
        learned_line = {"iterations": itl, "seconds": sl, "ms_per_iter": float(np.median(tl)),
                        "proposal_every": args.proposal_every, "proposals": int(sum(1 for p in props if p == 1)),
                        "rollbacks": int(sum(1 for p in props if p == 2)), "rms_uas": [round(v, 4) for v in rmsl],
                        "per_param_rms_uas_at_1uas": per_l,
                        "training": {"sets": "scale5yr geometry, 100k sources, 300-s knots, seeds 301 and 302, "
                                             "80 plain mixed iterations each, reference after 220",
                                     "adam_steps": 12000,
                                     "final_train_val_loss": hist[-1][1:] if hist else None,
                                     "seconds": round(t_train, 1)},
                        "speedup_vs_mixed": (sm / sl) if (sm and sl) else None,
                        "iterations_saved_vs_mixed": (itm - itl) if (itm and itl) else None}
    asi_lines = {}
    if args.asi:
        # the paper's own accelerator (Sect. 4.7) in both forms
        for name, prec in (("mixed_asi", 1), ("fp64_asi", 0)):
            rmsa, ta, fac, per_a = run_mixed(asi=True, prec=prec)
            ita, sa = first_below(rmsa, ta)
            asi_lines[name] = {"iterations": ita, "seconds": sa, "ms_per_iter": float(np.median(ta)),
                               "stride": args.asi_stride, "lambda_max": args.asi_lambda_max,
                               "factors": [round(v, 3) for v in fac], "rms_uas": [round(v, 4) for v in rmsa],
                               "per_param_rms_uas_at_1uas": per_a}
    order_lines = {}
    if args.orders:
        # the block orders of Sect. 4.6 in the mixed form: Gauss-Seidel SAC and Jacobi [SAC]
        for name, order in (("mixed_gauss_seidel", 1), ("mixed_jacobi", 2)):
            rmso, to, _, per_o = run_mixed(order=order)
            ito, so = first_below(rmso, to)
            order_lines[name] = {"iterations": ito, "seconds": so, "ms_per_iter": float(np.median(to)),
                                 "block_order": order, "rms_uas": [round(v, 4) for v in rmso],
                                 "per_param_rms_uas_at_1uas": per_o}
    line = {"metric": "wall time to 1 uas RMS vs FP64 reference", "unit": "s", "higher_is_better": False,
            "workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n_obs": ds.n_obs, "n_src": ds.n_src,
            "reference": {"form": "fp64", "iterations": len(rms64), "last_max_update_uas": ref_last_update,
                          "tol_uas": args.ref_tol_uas},
            "fp64": {"iterations": it64, "seconds": s64, "ms_per_iter": float(np.median(t64)),
                     "rms_uas": [round(v, 4) for v in rms64[:it64 or len(rms64)]]},
            "mixed": {"iterations": itm, "seconds": sm, "ms_per_iter": float(np.median(tm)),
                      "refresh_every": args.refresh_every, "rms_uas": [round(v, 4) for v in rmsm],
                      "per_param_rms_uas_at_1uas": per_param},
            "speedup": (s64 / sm) if (s64 and sm) else None}
    line.update(asi_lines)
    line.update(order_lines)
    if "fp64_asi" in asi_lines and s64 and asi_lines["fp64_asi"]["seconds"]:
        line["speedup_fp64_asi_vs_fp64"] = s64 / asi_lines["fp64_asi"]["seconds"]
    if "mixed_asi" in asi_lines and s64 and asi_lines["mixed_asi"]["seconds"]:
        line["speedup_mixed_asi_vs_fp64"] = s64 / asi_lines["mixed_asi"]["seconds"]
    if learned_line is not None:
        line["mixed_learned"] = learned_line
        line["speedup_learned_vs_fp64"] = (s64 / learned_line["seconds"]) if (s64 and learned_line["seconds"]) else None
    if learned_asi_line is not None:
        line["mixed_learned_asi"] = learned_asi_line
        if "mixed_asi" in asi_lines and asi_lines["mixed_asi"]["seconds"] and learned_asi_line["seconds"]:
            line["speedup_learned_asi_vs_mixed_asi"] = asi_lines["mixed_asi"]["seconds"] / learned_asi_line["seconds"]
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def convergence_summary(conv):
    """The convergence record without the per-iteration RMS lists (for the throughput line)."""
    out = {"metric": conv["metric"], "unit": conv["unit"], "reference": conv["reference"]}
    for k, v in conv.items():
        if isinstance(v, dict) and "seconds" in v:
            out[k] = {kk: vv for kk, vv in v.items() if kk not in ("rms_uas", "factors")}
        elif k.startswith("speedup"):
            out[k] = v
    return out


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_1112_4139_gb300 as pkg
    pkg.build()
    from paper_1112_4139_gb300 import agis
    ds, t_gen = make_dataset(args)
    stream = torch.cuda.Stream()
    if args.convergence:
        return run_convergence(args, agis, ds, stream, rank)
    if world > 1:
        return run_partitioned(args, agis, ds, stream, rank, world, local, dist, t_gen)
    seg_len = 2880 if ds.geometry["knot_dt_ns"] <= 30_000_000_000 else 720
    forms = {"fp64": dict(precision=0), "mixed": dict(precision=1, refresh_every=args.refresh_every)}
    head = args.precision
    other = "mixed" if head == "fp64" else "fp64"
    an_ns = int(round(args.attnoise_s * 1e9))
    if an_ns > 0 and not args.single_form:
        raise SystemExit("--attnoise-s needs --single-form")
    if args.cal_generic and not (args.single_form and head == "fp64"):
        raise SystemExit("--cal-generic needs --precision fp64 --single-form (the full calibration is FP64 only)")
    calc = agis.calibration_config(ds.geometry)
    cfgs = {k: agis.default_config(seg_len=seg_len, use_graph=1, frame_each_iter=1, **calc, **v)
            for k, v in forms.items()}
    # the mixed form is timed over whole refresh cycles, so its per-iteration time includes
    # the full FP64 evaluation at its share
    cyc = max(1, args.refresh_every)
    steps_of = {"fp64": args.steps, "mixed": cyc * max(1, -(-args.steps // cyc))}
    res = {head: time_form(agis, ds, stream, cfgs[head], steps_of[head], args.warmup, local, dist, args.tune_iters,
                           an_ns)}
    if not args.single_form:
        res[other] = time_form(agis, ds, stream, cfgs[other], steps_of[other], args.warmup, local, dist,
                               args.tune_iters)
    r = res[head]
    value = world * ds.n_obs / (r["ms"] * 1e-3)
    # ---- end to end through the C ABI from pinned host buffers
    import torch as T
    host = {k: T.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in agis.obs_from_dataset(ds).items()}
    src0 = T.from_numpy(np.ascontiguousarray(ds.src0)).pin_memory()
    att0 = T.from_numpy(np.ascontiguousarray(ds.att0)).pin_memory()
    cal0 = T.from_numpy(np.ascontiguousarray(ds.cal0)).pin_memory()
    ref = T.from_numpy(np.ascontiguousarray(ds.src_true[:, [0, 1, 3, 4]])).pin_memory()
    out_src = T.empty((ds.n_src, 5), dtype=T.float64).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values()) + sum(
        v.numel() * v.element_size() for v in (src0, att0, cal0, ref))
    d2h = out_src.numel() * out_src.element_size()
    e2e_times = []
    for k in range(args.e2e_steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        ge = agis.Agis(ds.geometry, cfgs[head], host, src0, att0, cal0, src_ref=ref, stream=stream.cuda_stream)
        if r["tuning"]:
            ge.set_tuning(r["tuning"]["shapes"])
        if an_ns > 0:
            ge.set_attnoise(an_ns)
        ge.iterate(1)
        ge.sources(out=out_src.numpy())
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t)
        ge.close()
    e2e = world * ds.n_obs / float(np.median(e2e_times)) if e2e_times else None
    peaks = load_peaks()
    hbm_peak = peaks.get("hbm_gbs") or FALLBACK_HBM_GBS
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s"

    def fp64_roofline(x):
        # FP64 arithmetic bound of the S block (FP64 pass + FP64 per-source solves): algorithmic
        # flops (FMA = 2) against the FP64 rate measured on the box (FMA = 2)
        achieved = S_FLOPS_PER_OBS * ds.n_obs / (x["s_ms"] * 1e-3) / 1e12
        return {"bound": "alu", "kernel": "k_obs_forward + k_source_solve (S block, FP64)", "achieved": achieved,
                "peak": FP64_PEAK_DERIVED_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_DERIVED_TFLOPS,
                "traffic": (TRAFFIC_PER_OBS["fp64_s_block"] * ds.n_obs
                            if TRAFFIC_PER_OBS["fp64_s_block"] is not None else None),
                "peak_source": "FP64 peak derived from unit counts and clock: 152 SMs x 2 FMA/clk x 2 flops x "
                               "2.07 GHz (of derived)", "flops_per_obs": S_FLOPS_PER_OBS}

    def mixed_roofline(x):
        # HBM bound of the linearized observation pass (k_mix_correct): algorithmic bytes per
        # observation = t (8) + g (16) + calibration index (4) + R read (8) + R written (8)
        if not x["pass_lin_ms"]:
            return None
        achieved = MIX_PASS_BYTES * ds.n_obs / (x["pass_lin_ms"] * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": "k_mix_correct (linearized observation pass)", "achieved": achieved,
                "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": (TRAFFIC_PER_OBS["mixed_correct"] * ds.n_obs
                            if TRAFFIC_PER_OBS["mixed_correct"] is not None else None),
                "peak_source": hbm_src, "bytes_per_obs": MIX_PASS_BYTES}

    def summary(name, x):
        d = {"ms_per_step": x["ms"], "value": world * ds.n_obs / (x["ms"] * 1e-3), "unit": "obs/s",
             "block_ms": {"S": x["s_ms"], "S_pass_full": x["pass_full_ms"], "S_pass_linearized": x["pass_lin_ms"],
                          "S_solve": x["solve_ms"], "A": x["a_ms"], "C": x["c_ms"],
                          "rest": x["ms"] - x["s_ms"] - x["a_ms"] - x["c_ms"]},
             "t_init_s": round(x["t_init"], 2), "clocks": x["clocks"], "autotune": x["tuning"]}
        if name == "mixed":
            d.update({"dtype": "f32+f64", "refresh_every": args.refresh_every, "full_evals_timed": x["n_full_eval"],
                      "roofline": mixed_roofline(x)})
        else:
            d.update({"dtype": "f64", "roofline": fp64_roofline(x)})
        return d

    line = {
        "metric": "AL+AC observations/s per AGIS iteration", "value": value, "unit": "obs/s", "n_gpus": world,
        "steps": steps_of[head], "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if head == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n_obs": ds.n_obs,
                   "n_src": ds.n_src, "n_coef": ds.n_coef, "n_cal": ds.n_cal, "precision": head,
                   "l2": "no flush: inputs (tens of GB) exceed the 129 MB L2", "graph": True,
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "t_generate_s": round(t_gen, 1), "t_init_s": round(r["t_init"], 2),
                   "autotune": r["tuning"], "attnoise_bucket_s": args.attnoise_s or None,
                   "calibration": ({"model": "full (Eq. etazeta)", "n_gate": 2, "j_per_k": 30,
                                    "col_bin": args.cal_col_bin} if args.cal_generic else "r = 0 offsets per day")},
        "e2e": ({"value": e2e, "unit": "obs/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
                if e2e is not None else None),
        "gpu_launches": (KERNELS_PER_STEP[head][0] * r["n_full_eval"] +
                         KERNELS_PER_STEP[head][1] * (steps_of[head] - r["n_full_eval"]) +
                         (KERNELS_ATTNOISE * steps_of[head] if an_ns > 0 else 0)),
        "clocks": r["clocks"],
        "roofline": fp64_roofline(r) if head == "fp64" else mixed_roofline(r),
        "block_ms": summary(head, r)["block_ms"],
    }
    if other in res:
        line[other] = summary(other, res[other])
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(ds)
    if world == 1 and not args.no_convergence and args.workload == "scale5yr":
        # the metric's second half: wall time to 1 uas RMS of the FP64 form, the mixed form, the
        # paper's accelerator (ASI) and the learned proposal (with ASI), on the same data
        cargs = argparse.Namespace(**vars(args))
        cargs.asi, cargs.learned = True, True
        t = time.perf_counter()
        conv = run_convergence(cargs, agis, ds, stream, rank, emit=False)
        line["convergence"] = convergence_summary(conv)
        line["convergence"]["wall_s"] = round(time.perf_counter() - t, 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
