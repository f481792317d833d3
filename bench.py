"""Benchmark: time-to-eps of the adaptive TT cross on one GB300.

A step is one whole adaptive TT cross (every sweep: residual screen of every
bond, candidate merge, pivot updates, and the sampled-error verification) on
the largest workload, the 6D Hilbert tensor X = 1/(1 + i_1 + ... + i_6),
n = 256 per mode (2.8e14 entries, never formed), eps = 1e-10, rank cap 128,
subtensor grid 4^6, error on 10^6 seeded random entries.  The tensor is a
function of its indices, so the inputs are synthetic by construction.

The screen keeps each bond's residual in device memory and carries it
through every pivot's rank-one step (eq. aca_approx_E); ``--residual
recompute`` forms A - T R afresh every sweep instead (Alg. 1).  Two arms are
timed on the same workload: the plain FP64 form (pivots bit-identical to the
oracle) and the mixed form (entries new to a superblock formed in float-float
on the FP32 pipe, the top candidates re-scored in FP64); ``--precision``
picks the arm of the headline value.

One JSON line on rank 0.  ``--impl reference`` times the CPU oracle (plain C,
FP64, OpenMP over the host cores) on the same workload and residual form.
``--workload maxwellian_batch`` times the batch of independent Maxwellians
(one persistent launch vs one launch per instance).  With ``--gpus N``
(under torchrun) every rank runs an independent replica: the path has no
exchange step on one GPU.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-eps TT cross (ms)"
WORKLOAD = "hilbert6d_n256"
SECONDARY = "hilbert6d_n64"
# rank cap of the oracle runs: below it the oracle's decisions are those of
# the workload's cap (its ranks stay under it, as the parity tests assert),
# while its stored residuals need (cap / workload cap)^2 of the host memory
ORACLE_CAP = {"hilbert6d_n256": 32}
# DRAM bytes (read + write) of one k_persistent launch, from one ncu capture of
# the current kernels (dram__bytes_read.sum + dram__bytes_write.sum), keyed by
# (workload, residual form, precision); absent keys report null.  The n = 256
# captures ran with rank capacity 32 (same sweeps: the ranks stay below 24).
DRAM_TRAFFIC = {("hilbert6d_n256", "stored", "fp64"): 6215910144 + 7267844096,
                ("hilbert6d_n256", "stored", "split"): 6212543488 + 7494847744}
THROTTLE_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
                 0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
                 0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
                 0x100: "display_clock_setting"}


def max_over_ranks(value: float, device: str) -> float:
    """The largest of the ranks' values (the replicas' step time is the
    slowest replica's), reduced on ``device`` (a CUDA device under NCCL, the
    CPU under gloo)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples nvidia-smi clocks / throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--id={self.index}",
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 4:
                try:
                    self.samples.append((float(parts[0]), float(parts[1]), parts[2],
                                         int(parts[3], 16) if parts[3].startswith("0x")
                                         else int(parts[3])))
                except ValueError:
                    pass

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [s[0] for s in self.samples]
        mask = 0
        for s in self.samples:
            mask |= s[3]
        reasons = [name for bit, name in THROTTLE_BITS.items() if mask & bit and bit != 0x1]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(s[1] for s in self.samples),
                "reasons": reasons, "samples": len(sm)}


HBM_FALLBACK_GBS = 6800.0


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return None


def cpu_oracle_time(cfg, threads: int, reps: int = 1, residual: str = "stored",
                    workload: str = "", min_s: float = 0.0, max_reps: int = 1):
    """The oracle as it stands, on the host cores: full runs of the workload
    in the same residual form as the GPU line (at least ``reps``; more, up to
    ``max_reps``, until ``min_s`` seconds of runs have been timed)."""
    import oracle
    cap = ORACLE_CAP.get(workload, cfg["max_rank"])
    times = []
    st = None
    while len(times) < reps or (sum(times) < 1e3 * min_s and len(times) < max_reps):
        o = oracle.Oracle(cfg["n"], cfg["gen"], cap, nthreads=threads,
                          stored=residual == "stored")
        t0 = time.perf_counter()
        rc, st = o.run(cfg["eps"], nsamples=cfg["nsamples"])
        times.append((time.perf_counter() - t0) * 1e3)
        st["ranks"] = [int(x) for x in o.ranks()]
        del o
    return times, st


def bench_reference(args, rank, world):
    from paper_2407_11290_gb300 import workloads
    if rank != 0:
        return
    if args.workload == "maxwellian_batch":
        print(json.dumps({"impl": "reference", "unavailable":
                          "the batch reference arm is not built: the oracle runs one tensor at a "
                          "time"}), flush=True)
        return
    cfg = workloads.CONFIGS[args.workload]
    threads = os.cpu_count() or 1
    cpu_oracle_time(cfg, threads, reps=args.warmup, residual=args.residual,
                    workload=args.workload)
    times, st = cpu_oracle_time(cfg, threads, reps=args.steps, residual=args.residual,
                                workload=args.workload)
    ms = sum(times) / len(times)
    cap = ORACLE_CAP.get(args.workload, cfg["max_rank"])
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (analytic tensor)",
        "config": {"workload": args.workload, "d": len(cfg["n"]), "n": cfg["n"][0],
                   "eps": cfg["eps"], "max_rank": cfg["max_rank"], "nsamples": cfg["nsamples"],
                   "residual": args.residual, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} full runs of the workload (oracle rank cap "
                                   f"{cap}; its ranks {st['ranks']} stay below it)"},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "entries_screened": st["entries_screened"], "sweeps": st["sweeps"], "err": st["err"],
    }
    print(json.dumps(line), flush=True)


def _dtype(prec: str) -> str:
    return {"fp64": "f64", "split": "f32x2+f64", "fp32": "f32+f64", "auto": "f32x2+f64"}[prec]


def time_arm(ttcross, cfg, prec, residual, steps, warmup, stream, flush, sampler=None,
             host_loop=False, plans=None):
    """One arm: a TTCross of the workload in the given precision, its tile
    plan from the autotuner's cache (measured on a miss; untimed), ``warmup``
    untimed runs, then ``steps`` timed runs (L2 flushed before each, CUDA
    events on the launching stream around the run)."""
    import torch
    tc = ttcross.TTCross(cfg["n"], cfg["gen"], max_rank=cfg["max_rank"], nsamples=cfg["nsamples"],
                         precision=prec, residual=residual, host_loop=host_loop)
    if not host_loop:
        plan = ttcross.tuned_plan(tc, cfg["eps"], cfg["max_rank"], cfg["grid"], prec, residual,
                                  stream)
        if plans is not None:
            plans[prec] = {"tile_edge": plan[0], "queue_split": plan[1], "source": plan[2]}

    def one_step():
        tc.run(cfg["eps"], subtensor_grid=cfg["grid"], stream=stream)

    for _ in range(warmup):
        one_step()
        tc.sync(allow=(ttcross.OK, ttcross.NOT_CONVERGED))
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    kern_ms = []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))            # L2 flush (512 MB > 129 MB L2), untimed
        ev[i][0].record(stream)
        one_step()
        ev[i][1].record(stream)
        tc.sync(allow=(ttcross.OK, ttcross.NOT_CONVERGED))
        kern_ms.append(tc.stats()["device_ms"])
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler is not None else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    return tc, step_ms, kern_ms, clocks, one_step


def bench_gpu(args, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2407_11290_gb300 import ttcross, workloads

    torch.cuda.set_device(local)
    cfg = dict(workloads.CONFIGS[args.workload])
    if args.max_rank > 0:
        cfg["max_rank"] = args.max_rank
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    plans = {}
    tc, step_ms, kern_ms, clocks, one_step = time_arm(
        ttcross, cfg, args.precision, args.residual, args.steps, args.warmup, stream, flush,
        sampler, host_loop=args.host_loop, plans=plans)
    st = tc.stats()
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        dist.barrier()
        ms = max_over_ranks(ms, "cuda")

    # end to end through the C ABI with host buffers: run + cores to host memory
    e2e = []
    d2h = 0
    for _ in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_step()
        cores = tc.cores()
        e2e.append((time.perf_counter() - t0) * 1e3)
        d2h = sum(c.nbytes for c in cores)

    # the other arm on the same workload (FP64 vs mixed), and both arms on
    # the smaller 6D workload (n = 64)
    arms = {args.precision: {"ms": ms, "median_ms": statistics.median(step_ms),
                             "kernel_ms": statistics.median(kern_ms), "err": st["err"],
                             "status": ttcross.STATUS_NAMES.get(st["status"], st["status"]),
                             "ranks": [int(x) for x in tc.ranks()], "sweeps": st["sweeps"],
                             "phase_ms": st["phase_ms"], "rescored": st["tiles_refined"],
                             "stored_gbs": _stored_gbs(st, kern_ms)}}
    secondary = {}
    if rank == 0 and not args.no_forms:
        other = "split" if args.precision == "fp64" else "fp64"
        a, sm_, km, _, _ = time_arm(ttcross, cfg, other, args.residual, max(3, args.steps // 2),
                                    max(1, args.warmup // 2), stream, flush, plans=plans)
        ast = a.stats()
        arms[other] = {"ms": sum(sm_) / len(sm_), "median_ms": statistics.median(sm_),
                       "kernel_ms": statistics.median(km), "err": ast["err"],
                       "status": ttcross.STATUS_NAMES.get(ast["status"], ast["status"]),
                       "ranks": [int(x) for x in a.ranks()], "sweeps": ast["sweeps"],
                       "phase_ms": ast["phase_ms"], "rescored": ast["tiles_refined"],
                       "stored_gbs": _stored_gbs(ast, km)}
        a.close()
        if args.workload != SECONDARY:
            wc = workloads.CONFIGS[SECONDARY]
            for prec in ("fp64", "split"):
                b, sm_, km, _, _ = time_arm(ttcross, wc, prec, args.residual, 5, 2, stream, flush)
                bs = b.stats()
                secondary[prec] = {"ms": sum(sm_) / len(sm_), "kernel_ms": statistics.median(km),
                                   "err": bs["err"], "ranks": [int(x) for x in b.ranks()]}
                b.close()

    # roofline of the dominant kernel (the persistent cross kernel): its
    # algorithmic FP64 FMAs (screen + error) over its measured duration,
    # against the FP64 pipe measured on this GPU; the stored residuals'
    # algorithmic bytes over the same duration against HBM
    fma64, _ = ttcross.probe_fma_peak(True)
    kms = statistics.median(kern_ms)
    algo_fma = st["screen_fmas"] + st["error_fmas"]
    achieved = 2.0 * algo_fma / (kms * 1e-3) / 1e12
    peak = 2.0 * fma64 / 1e12
    peaks = measured_peaks() or {}
    hbm = peaks.get("hbm_gbs")
    hbm_source = "measured copy bandwidth (MEASURED_PEAKS.json)"
    if not hbm:
        # no measured copy bandwidth on this machine: one earlier GB300 copy
        # measurement stands in, labelled as such
        hbm, hbm_source = HBM_FALLBACK_GBS, "fallback (earlier GB300 copy measurement)"
    stored_gbs = st["stored_bytes"] / (kms * 1e-3) / 1e9
    # each arm's stored-residual bytes against the same HBM peak
    for arm in arms.values():
        arm["hbm_frac"] = arm["stored_gbs"] / hbm if hbm and arm["stored_gbs"] else None
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": _dtype(args.precision),
        "data": "synthetic (analytic tensor, never formed)",
        "config": {"workload": args.workload, "d": len(cfg["n"]), "n": cfg["n"][0],
                   "eps": cfg["eps"], "max_rank": cfg["max_rank"], "grid": cfg["grid"],
                   "nsamples": cfg["nsamples"],
                   "precision": args.precision, "residual": args.residual,
                   "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas x{world}", "plans": plans},
        "min_ms": min(step_ms), "median_ms": statistics.median(step_ms),
        "entries_screened": st["entries_screened"],
        "entries_per_s": st["entries_screened"] * world / (ms * 1e-3),
        # the share of the tensor's entries the cross evaluated (the paper's
        # "% of full tensor size accessed", Sec. 5.1): in the stored form every
        # superblock entry is formed once, plus the error samples
        "accessed_fraction": ((st["entries_fresh"] + cfg["nsamples"]) /
                              float(np.prod([float(v) for v in cfg["n"]]))
                              if args.residual == "stored" else None),
        "sweeps": st["sweeps"], "ranks": [int(x) for x in tc.ranks()], "err": st["err"],
        "phase_ms": st["phase_ms"],
        "status": ttcross.STATUS_NAMES.get(st["status"], st["status"]),
        "e2e": {"value": statistics.median(e2e), "unit": "ms", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": DRAM_TRAFFIC.get((args.workload, args.residual, args.precision)),
                     "peak_source": "measured FP64 FMA loop on this GPU",
                     "kernel": "k_persistent", "kernel_ms": kms,
                     "algorithmic_fma": algo_fma,
                     "stored_bytes": st["stored_bytes"], "stored_gbs": stored_gbs,
                     "hbm_frac": stored_gbs / hbm if hbm else None,
                     "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_source},
        "clocks": clocks,
        "arms": arms,
        "secondary": {"workload": SECONDARY, **secondary} if secondary else None,
    }
    if "split" in arms and "fp64" in arms:
        line["mixed_vs_fp64"] = arms["fp64"]["ms"] / arms["split"]["ms"]
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        times, ost = cpu_oracle_time(cfg, threads, reps=1, residual=args.residual,
                                     workload=args.workload, min_s=10.0, max_reps=8)
        cap = ORACLE_CAP.get(args.workload, cfg["max_rank"])
        line["cpu_baseline"] = {"value": sum(times) / len(times), "unit": "ms", "cores": threads,
                                "kind": "oracle",
                                "sample": f"{len(times)} full runs of the workload, FP64 "
                                          f"{args.residual} form (oracle rank cap {cap}; its "
                                          f"ranks {ost['ranks']} stay below it)",
                                "err": ost["err"]}
        # the same oracle on one thread (one full run), beside the all-core figure
        t1, _ = cpu_oracle_time(cfg, 1, reps=1, residual=args.residual, workload=args.workload)
        line["cpu_baseline"]["single_thread"] = {"value": t1[0], "unit": "ms", "cores": 1,
                                                 "sample": "1 full run of the workload"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    tc.close()


def _stored_gbs(st, kern_ms):
    """The bytes of the stored residual E that the arm's screens read and
    wrote, over its median kernel time, in GB/s; None in the recompute form,
    which stores nothing."""
    if not st["stored_bytes"]:
        return None
    return st["stored_bytes"] / (statistics.median(kern_ms) * 1e-3) / 1e9


def bench_batch(args, rank, world, local):
    """The batch workload: independent Maxwellians of uneven d, n and
    amplitudes (rank cap 64, eps = 1e-6).  A step is the whole batch to eps.
    Arms, all in the stored-residual form: every instance in one persistent
    FP64 launch; one FP64 launch per instance in a loop (the same handles);
    every instance in one persistent launch of the mixed (float-float) form.
    The batched arms are captured once in a CUDA graph (after an ordinary
    batch has sized every buffer) and every step replays it.
    The FP32 / float-float recompute-form batch of these tensors is refused by
    the library, so it is not an arm."""
    import torch
    import torch.distributed as dist

    from paper_2407_11290_gb300 import ttcross, workloads

    torch.cuda.set_device(local)
    ws = workloads.maxwellian_batch(args.batch_count)
    stream = torch.cuda.Stream()
    eps, cap, ns = 1e-6, 64, 10**6
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    allow = (ttcross.OK, ttcross.NOT_CONVERGED)

    tuned = {}

    def make(prec):
        hs = [ttcross.TTCross(w["n"], w["gen"], max_rank=cap, nsamples=ns, precision=prec,
                              residual="stored") for w in ws]
        # the autotuner's plan per shape class (d, n), measured on the class's
        # first instance (cached across runs), applied to every instance
        for w, c in zip(ws, hs):
            key = f"{prec}/d{len(w['n'])}/n{w['n'][0]}"
            if key not in tuned:
                tuned[key] = ttcross.tuned_plan(c, eps, cap, None, prec, "stored", stream)[:2]
            c.set_plan(*tuned[key])
        return hs

    def timed(run):
        # replicas: a barrier on both sides of the timed steps, and the
        # slowest replica's time
        for _ in range(args.warmup):
            run()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        out = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            ev[0].record(stream)
            run()
            ev[1].record(stream)
            torch.cuda.synchronize()
            out.append(ev[0].elapsed_time(ev[1]))
        if world > 1:
            dist.barrier()
            return max_over_ranks(sum(out) / len(out), "cuda")
        return sum(out) / len(out)

    def graphed(hs):
        # an ordinary batch sizes every buffer, then the batch is captured
        ttcross.run_batch(hs, eps, stream=stream)
        for c in hs:
            c.sync(allow=allow)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            ttcross.run_batch(hs, eps, stream=stream)

        def step():
            with torch.cuda.stream(stream):
                g.replay()
            for c in hs:
                c.sync(allow=allow)
        return step, g

    def loop(hs):
        for c in hs:
            c.run(eps, stream=stream)
            c.sync(allow=allow)

    times, summary = {}, {}

    def summarise(name, hs):
        st = [c.stats() for c in hs]
        summary[name] = {"converged": sum(1 for x in st if x["status"] == ttcross.OK),
                         "max_err": max(x["err"] for x in st),
                         "max_err_converged": max([x["err"] for x in st
                                                   if x["status"] == ttcross.OK] or [0.0]),
                         "entries_screened": sum(x["entries_screened"] for x in st)}

    hs = make("fp64")
    step, graph = graphed(hs)
    times["batched_fp64"] = timed(step)
    summarise("batched_fp64", hs)
    del graph
    times["loop_fp64"] = timed(lambda: loop(hs))
    summarise("loop_fp64", hs)
    for c in hs:
        c.close()
    del hs
    hm = make("split")
    step, graph = graphed(hm)
    times["batched_split"] = timed(step)
    summarise("batched_split", hm)
    del graph
    for c in hm:
        c.close()
    best = min(times, key=times.get)
    line = {
        "metric": METRIC, "value": times["batched_split"], "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": times["batched_split"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": _dtype("split"), "data": "synthetic (analytic tensors, never formed)",
        "config": {"workload": f"maxwellian_batch x{args.batch_count}", "eps": eps,
                   "max_rank": cap, "nsamples": ns, "residual": "stored",
                   "launch": "batched arms: one persistent launch captured in a CUDA graph, "
                             "replayed every step",
                   "l2": "working set of the batch exceeds L2"},
        "arms_ms": times, "fastest": best,
        "mixed_batched_vs_fp64_loop": times["loop_fp64"] / times["batched_split"],
        "fp64_batched_vs_loop": times["loop_fp64"] / times["batched_fp64"],
        "arms": summary, "count": len(ws), "plans": tuned,
        # the headline arm's kernels per step (a batch: a control-block
        # kernel per instance, the instance-list kernel per 256 instances,
        # the persistent kernel), over the timed steps
        "gpu_launches": args.steps * (len(ws) + (len(ws) + 255) // 256 + 1),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "split", "auto"])
    ap.add_argument("--residual", default="stored", choices=["recompute", "stored"],
                    help="screen form: the stored residual of eq. aca_approx_E (default), or "
                         "A - T R formed every sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the other arm and the smaller workload")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["hilbert3d_n32", "hilbert6d_n64", "hilbert6d_n256", "maxwellian6d_n64",
                             "maxwellian_batch"])
    ap.add_argument("--max-rank", type=int, default=0,
                    help="rank cap instead of the workload's (0: the workload's); a smaller cap "
                         "shrinks the stored residuals for profiling captures")
    ap.add_argument("--batch-count", type=int, default=256,
                    help="instances of the maxwellian_batch workload")
    ap.add_argument("--host-loop", action="store_true",
                    help="phases as separate launches (per-phase kernels for profiling)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        bench_reference(args, rank, world)
    elif args.workload == "maxwellian_batch":
        bench_batch(args, rank, world, local)
    else:
        bench_gpu(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
