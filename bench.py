#!/usr/bin/env python3
"""Benchmark of the random-phase Trotter path on GB300.

One bench step = one whole job of the hot path: random-phase initialization
(Philox phases), `trotter_steps` second-order Trotter steps (FP64 gate/phase
tables, tile sweeps with the diagonal phase and the fused P/norm reduction).
The default workload is the 2x15 XY ladder (M = 30, 2^30 complex64
amplitudes = 8 GiB, leg 1, rung 0.5, dt 0.05, 200 steps), the largest case,
where the HBM roofline applies; the state (8 GiB) is far larger than L2, so
no flush is needed between steps.

  value   amp-gate updates/s = 2^M * 2B * trotter_steps / device time per job,
          summed over replicas (N > 1 runs one independent job per GPU);
  e2e     the same through the public API with host inputs and the P(t)
          series copied back (system + state creation, init, evolve, read);
  roofline  the tile-sweep kernel: algorithmic bytes per launch = the
          minimal-sweep bytes of a Trotter step (two sweeps, each one read and
          one write of the state) / the plan's sweeps per step, over its mean
          launch time (CUDA events around every launch on the state's stream),
          against the measured HBM copy peak; the kernel's own bandwidth (one
          read and one write of the state per launch) is reported beside it;
  fp64    the complex128 path on the same workload (all Trotter steps), its
          rate and the largest FP32-vs-FP64 |dP(t)| over every recorded step;
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload.

`--impl reference` times the CPU oracle (there is no other implementation of
the paper's method) on the same workload and prints the same JSON line.
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
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "amp·gate updates/s, HBM GB/s FP32 vs FP64; serve p50/p99 latency @|ΔP|≤1e-4"
UNIT = "amp-gate updates/s"


def _peaks():
    try:
        return json.loads((ROOT / "MEASURED_PEAKS.json").read_text()), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload(name: str):
    from paper_0710_3747_gb300 import workloads as W
    if name == "ladder_m30":
        return W.ladder_m30(), "c64", "ladder_2x15_M30_xy_dt0.05_200steps"
    if name == "star_m20":
        return W.star_m20(), "c64", "star_dipolar_M20_dt0.02_1000steps"
    if name == "ladder_m14":
        return W.ladder_m14(), "c64", "ladder_2x7_M14_xy_dt0.05_400steps"
    if name == "ladder_m26":  # profiling case: 512 MiB state, larger than L2
        job = W.ladder_m30()
        job.J = W.ladder(13, 1.0, 0.5)
        job.steps = 10
        return job, "c64", "ladder_2x13_M26_xy_dt0.05_10steps"
    raise SystemExit(f"unknown workload {name}")


def max_over_ranks(x: float, dist=None) -> float:
    """The largest of x over all ranks (x itself without a process group).
    Replicas each time their own job; the job-wide time is the slowest rank's."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput of `world` replicas that each process
    units_per_rank in (the slowest rank's) `seconds`."""
    return world * units_per_rank / seconds


def updates_per_job(M: int, nbonds: int, steps: int) -> float:
    # 2B half-step bond gates per Trotter step, each touching the 2^M-amplitude state
    return float(2 ** M) * 2 * nbonds * steps


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(job, gates: int, threads: int, repeats: int = 1, warmup: int = 0):
    """Time `gates` flip-flop gate applications of the oracle (canonical order,
    tau = dt/2) on the job's random-phase state at full size; the state's
    initialization is set-up, outside the timing."""
    import oracle
    a, b = oracle.couplings(job.J, job.htype)
    bonds = oracle.canonical_bonds(b)
    psi = oracle.init_random_phase(job.M, job.seed, threads=threads)
    times = []
    for r in range(warmup + repeats):
        t0 = time.perf_counter()
        for k in range(gates):
            i, j = bonds[k % len(bonds)]
            oracle.flipflop(psi, i, j, b[i, j], 0.5 * job.dt, threads=threads)
        dt = time.perf_counter() - t0
        if r >= warmup:
            times.append(dt)
    del psi
    return times


def run_reference(args, rank: int):
    if rank != 0:
        return 0
    job, prec, wname = workload(args.workload)
    threads = os.cpu_count() or 1
    gates = args.ref_gates
    times = oracle_sample(job, gates, threads, repeats=args.steps, warmup=args.warmup)
    per = statistics.mean(times)
    value = gates * float(2 ** job.M) / per
    sample = (f"FP64 CPU oracle, {gates} flip-flop gate applications of the M={job.M} "
              f"{job.kind} state per step (2^{job.M} complex128 amplitudes), {threads} threads; "
              f"state initialization untimed")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wname, "M": job.M, "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_batch(args, rank: int, world: int, local_rank: int):
    """Batched dipolar stars (M uniform in 12..22, dt 0.02, `batch_steps`
    Trotter steps): every job of the batch evolved together -- one-tile plans
    (M <= 14) with the whole state resident in shared memory for all steps,
    the others as one sweep launch per plan group with the steady steps
    replayed as one CUDA graph.  One bench step = init + all Trotter steps of
    every job.  Warm-up batches run 20 steps each (every kernel, graph and
    plan exercised once)."""
    import torch

    from paper_0710_3747_gb300 import spinrp
    from paper_0710_3747_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    spinrp.lib()
    jobs = W.star_batch(n=args.batch_jobs, seed=4 + rank, steps=args.batch_steps)
    nsteps = args.batch_steps

    def make_systems():
        out = []
        for j in jobs:
            s_ = spinrp.System(j.J, j.htype)
            if args.regbits:
                s_.set_regbits(args.regbits)
            if args.tile_K:
                s_.set_tile("c64", min(args.tile_K, s_.M))
            out.append(s_)
        return out

    systems = make_systems()
    tuned = None
    if args.autotune:
        tuned = spinrp.autotune_batch(systems, [j.seed for j in jobs])
        args.tile_K, args.regbits = 0, 0  # make_systems() below repeats the tuned setting by hand

        def make_systems():
            out = []
            for j in jobs:
                s_ = spinrp.System(j.J, j.htype)
                if s_.M >= 15:
                    s_.set_tile("c64", tuned["K"])
                    s_.set_regbits(6)
                out.append(s_)
            return out
    b = spinrp.Batch(systems, [j.seed for j in jobs], "c64", series_cap=nsteps + 1)
    b.set_persistent(args.batch_launch == "persistent")
    upd = sum(updates_per_job(j.M, j.M * (j.M - 1) // 2, nsteps) for j in jobs)
    # bytes the plan's sweeps move: per job and step, sweeps_per_step reads and
    # writes of its state; a one-tile plan keeps the state in shared memory and
    # moves it once per evolve call
    plan_bytes = 0.0
    for s_, j in zip(systems, jobs):
        info = s_.plan_info("c64")
        if info["K"] >= j.M:
            plan_bytes += 16.0 * 2 ** j.M
        else:
            plan_bytes += 16.0 * 2 ** j.M * info["sweeps_per_step"] * nsteps

    for _ in range(args.warmup):
        b.init_random_phase()
        b.evolve(0.02, min(nsteps, 20))
    torch.cuda.synchronize()
    n0 = spinrp.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(str(local_rank)) as clk:
        e0.record()
        for _ in range(args.steps):
            b.init_random_phase()
            b.evolve(0.02, nsteps)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    launches = spinrp.launch_count() - n0
    mean, std = b.ensemble()
    info = b.info()
    peaks, peak_src = _peaks()
    achieved = plan_bytes / (ms / 1e3) / 1e9
    out = {"metric": METRIC, "value": world * upd / (ms / 1e3), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"star_batch_{args.batch_jobs}jobs_M12-22_dt0.02_{nsteps}steps",
                      "jobs": args.batch_jobs, "trotter_steps": nsteps, "groups": info["groups"],
                      "launch": args.batch_launch,
                      "autotuned": None if tuned is None else {"K": tuned["K"],
                                                               "ms_per_step": {str(k): v for k, v in tuned["ms_per_step"].items()}},
                      "device_bytes": info["device_bytes"],
                      "l2": "states total far larger than L2; no flush",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                        "kernel": ("pipe_kernel + sweep2_kernel + resident_kernel" if b.pipeline_groups()
                                   else "sweep2_kernel + resident_kernel") + " (all sweep launches of the batch)",
                        "pipelined_groups": b.pipeline_groups(),
                        "algorithmic_bytes": "one read and one write of every state per planned sweep "
                                             "(once per evolve call for states resident in shared memory)",
                        "algorithmic_bytes_per_batch_job": plan_bytes,
                        "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"},
           "gpu_launches": launches, "clocks": clk.summary(),
           "ensemble": {"P_mean_end": float(mean[-1]), "P_spread_end": float(std[-1]),
                        "P_mean_t1": float(mean[len(mean) // 10]),
                        "P_spread_t1": float(std[len(std) // 10]),
                        "chebyshev_scale_M12": 2.0 ** (-(12 - 1) / 2)}}
    b.close()
    # end to end through the public API: host couplings in, every job's P(t)
    # and the ensemble out
    if not args.skip_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sy = make_systems()
        b2 = spinrp.Batch(sy, [j.seed for j in jobs], "c64", series_cap=nsteps + 1)
        b2.set_persistent(args.batch_launch == "persistent")
        b2.init_random_phase().evolve(0.02, nsteps)
        allP = [b2.polarization(k) for k in range(len(jobs))]
        b2.ensemble()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        h2d = sum(j.J.nbytes for j in jobs) + 8 * len(jobs)
        d2h = sum(p.nbytes for p in allP) + 2 * 8 * (nsteps + 1)
        out["e2e"] = {"value": world * upd / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "s_per_step": e2e_s}
        b2.close()
    if rank == 0 and not args.skip_cpu:
        # the oracle on a bounded sample: a few Trotter steps of three jobs
        # (smallest, middle and largest M of the batch)
        import oracle
        threads = os.cpu_count() or 1
        pick = sorted(range(len(jobs)), key=lambda k: jobs[k].M)
        pick = [pick[0], pick[len(pick) // 2], pick[-1]]
        done = 0.0
        t_cpu = 0.0
        for k in pick:
            j = jobs[k]
            a, bb = oracle.couplings(j.J, j.htype)
            psi = oracle.init_random_phase(j.M, j.seed, threads=threads)
            t0 = time.perf_counter()
            oracle.evolve(psi, a, bb, j.dt, args.batch_cpu_steps, threads=threads)
            t_cpu += time.perf_counter() - t0
            done += updates_per_job(j.M, j.M * (j.M - 1) // 2, args.batch_cpu_steps)
        out["cpu_baseline"] = {"value": done / t_cpu, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": (f"FP64 CPU oracle, {args.batch_cpu_steps} Trotter steps of 3 jobs of the "
                                          f"batch (M = {', '.join(str(jobs[k].M) for k in pick)}), {threads} "
                                          f"threads, {t_cpu:.1f} s")}
    if rank == 0:
        print(json.dumps(out))
    return 0


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch

    from paper_0710_3747_gb300 import spinrp

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    spinrp.lib()
    job, prec, wname = workload(args.workload)
    sysm = spinrp.System(job.J, job.htype)
    if args.tile_K:
        sysm.set_tile(prec, args.tile_K)
    if args.regbits:
        sysm.set_regbits(args.regbits)
    tuned = spinrp.autotune(sysm, prec, dt=job.dt) if args.autotune else None
    nb = len(sysm.bonds())
    info = sysm.plan_info(prec)
    st = spinrp.State(sysm, prec, series_cap=job.steps + 1)
    if args.no_pipeline:
        st.set_pipeline(False)
    pipelined = prec == "c64" and st.pipeline()
    if args.sites:
        st.set_sites(True)  # P_{q1}(t) of every spin after every step
    stream = torch.cuda.current_stream()

    def one_job():
        if args.product:
            st.init_product_phase(job.seed + rank)
        else:
            st.init_random_phase(job.seed + rank)
        st.evolve(job.dt, job.steps)

    for _ in range(args.warmup):
        one_job()
    torch.cuda.synchronize()

    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(local_rank).uuid)
        if not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        gpu_id = str(local_rank)

    amp_bytes = 8 if prec == "c64" else 16
    # a state that fits in L2 is flushed out of it (256 MiB write) before every
    # timed job; larger states are streamed from HBM anyway
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if amp_bytes << job.M < (256 << 20) else None

    def timed_jobs(n):
        """Device time per job (ms) of n jobs, each bracketed by CUDA events
        on the state's stream; the L2 flush (if any) runs outside them."""
        evs = []
        for _ in range(n):
            if flush is not None:
                flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            one_job()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / n

    # timed region: the job as a user runs it (steady steps replayed as CUDA graphs)
    n0 = spinrp.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_id) as clk:
        ms = timed_jobs(args.steps)
    if dist:
        dist.barrier()
    launches = spinrp.launch_count() - n0
    ms = max_over_ranks(ms, dist)
    P32 = st.polarization()
    # the same jobs again with every sweep launch bracketed by CUDA events (live
    # launches, no graphs): the sweep kernel's mean launch time for the roofline
    st.profile(True)
    ms_prof = timed_jobs(args.steps)
    st.profile(False)
    sweep_ms, sweep_n = st.profile_read(spinrp.KERNEL_SWEEP)
    init_ms, init_n = st.profile_read(spinrp.KERNEL_INIT)
    upd = updates_per_job(job.M, nb, job.steps)
    value = replica_value(upd, ms / 1e3, world)

    # roofline of the tile-sweep kernel.  Algorithmic bytes are the minimal-sweep
    # bytes of a Trotter step (2 sweeps, each one read and one write of the
    # state) shared over the launches of the step: a launch stands for
    # 1 / sweeps_per_step of a step, so a plan that needs more than 2 sweeps
    # per step pays for them in this fraction.  The kernel's own bandwidth
    # (one read and one write of the state per launch) is reported beside it.
    peaks, peak_src = _peaks()
    state_bytes = amp_bytes * 2 ** job.M
    sweep_bytes = 2 * state_bytes
    min_sweeps = 2 if info["sweeps_per_step"] >= 2 else 1
    alg_bytes_per_launch = min_sweeps * sweep_bytes / info["sweeps_per_step"]
    sweep_avg_s = sweep_ms / max(sweep_n, 1) / 1e3
    achieved = alg_bytes_per_launch / sweep_avg_s / 1e9
    kernel_bw = sweep_bytes / sweep_avg_s / 1e9
    if prec == "c64":
        kname = "pipe_kernel<6, 13>" if pipelined else ("sweep2_kernel" if info["K"] >= 10 else "sweep_kernel<float>")
    else:
        kname = "sweep2d_kernel" if info["K"] >= 10 else "sweep_kernel<double>"
    # DRAM bytes per launch from an ncu capture, used while the kernel and its
    # sources are the ones the capture measured
    traffic = None
    tfile = ROOT / "profiles" / f"traffic_{args.workload}_{prec}.json"
    if tfile.exists():
        try:
            tinfo = json.loads(tfile.read_text())
            import hashlib
            hs = hashlib.sha256()
            for f in tinfo.get("sources", ["kernels.cuh"]):
                hs.update((ROOT / "paper_0710_3747_gb300" / "csrc" / f).read_bytes())
            if tinfo.get("sources_sha256") == hs.hexdigest() and tinfo.get("kernel") == kname:
                traffic = tinfo.get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": kname,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
                "algorithmic_bytes_per_launch": alg_bytes_per_launch,
                "algorithmic_bytes": (f"minimal-sweep bytes of a Trotter step ({min_sweeps} sweeps x 2 x "
                                      f"{amp_bytes} B x 2^{job.M}) / {info['sweeps_per_step']} launches per step"),
                "frac_of_8TBps": achieved / 8000.0,
                "launches": sweep_n, "mean_launch_ms": sweep_avg_s * 1e3,
                "sweep_bandwidth_gbs": kernel_bw, "sweep_bandwidth_frac": kernel_bw / peaks["hbm_gbs"],
                "sweep_share_of_job": sweep_ms / (ms_prof * args.steps),
                "timing": "per-launch CUDA events in a second pass over the same jobs (live launches)"}
    # a state that fits in L2 (129 MB) never streams from HBM: its sweeps are
    # bound inside the SMs, so the roofline is the gate arithmetic's FP32 rate
    # (each gate rotates 2^M / 4 flip-flop pairs at 6 FMAs: 1.5 FMA = 3 FLOP
    # per amplitude update) against the FP32 peak derived from the unit count
    # and the maximum SM clock (128 FP32 FMA lanes per SM), not HBM
    if state_bytes < 126 * 2 ** 20 and prec == "c64":
        sms = torch.cuda.get_device_properties(stream.device).multi_processor_count
        peak32 = sms * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 * 128 * 2 / 1e12
        flop_launch = 3.0 * updates_per_job(job.M, nb, job.steps) / max(sweep_n / args.steps, 1)
        ach32 = flop_launch / sweep_avg_s / 1e12
        roofline = {"bound": "alu", "achieved": ach32, "peak": peak32, "unit": "TFLOP/s",
                    "frac": ach32 / peak32, "traffic": None, "kernel": roofline["kernel"],
                    "peak_source": "derived: SMs x max SM clock x 128 FP32 FMA lanes x 2 FLOP",
                    "flops": "flip-flop gate FMAs of the launch (the step's gate applications / sweeps)",
                    "launches": sweep_n, "mean_launch_ms": sweep_avg_s * 1e3,
                    "l2_resident": True, "hbm_frac_if_streamed": roofline["frac"],
                    "sweep_share_of_job": roofline["sweep_share_of_job"],
                    "timing": roofline["timing"]}
    # the same fraction over whole jobs (graph replays, init included)
    min_bytes_step = min_sweeps * sweep_bytes
    step_roof = {"min_sweeps_per_step": min_sweeps, "sweeps_per_step": info["sweeps_per_step"],
                 "frac_of_measured_peak": (min_bytes_step * job.steps / (ms / 1e3) / 1e9) / peaks["hbm_gbs"],
                 "frac_of_8TBps": (min_bytes_step * job.steps / (ms / 1e3) / 1e9) / 8000.0}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == "c64" else "f64", "data": "synthetic",
        "config": {"workload": wname, "M": job.M, "bonds": nb, "trotter_steps": job.steps,
                   "dt": job.dt, "amplitudes": "complex64" if prec == "c64" else "complex128",
                   "tile_K": info["K"], "sweeps_per_step": info["sweeps_per_step"],
                   "pipelined_sweeps": pipelined,
                   "autotuned": None if tuned is None else {"K": tuned["K"], "rb": tuned["rb"]},
                   "all_site_readout": bool(args.sites),
                   "initial_state": "product" if args.product else "entangled",
                   "state_bytes": amp_bytes * 2 ** job.M,
                   "l2": ("L2 flushed (256 MiB write) before every timed job" if flush is not None
                          else "inputs larger than L2 (state >> 129 MB), no flush"),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline, "hbm_step_roofline": step_roof, "gpu_launches": launches,
        "clocks": clk.summary(),
    }

    # end to end through the public API: host J in, P(t) series out
    if not args.skip_e2e:
        def e2e_job():
            s2 = spinrp.System(job.J, job.htype)
            if args.tile_K:
                s2.set_tile(prec, args.tile_K)
            if args.regbits:
                s2.set_regbits(args.regbits)
            if tuned is not None:
                s2.set_tile(prec, tuned["K"])
                if prec == "c64":
                    s2.set_regbits(tuned["rb"])
            st2 = spinrp.State(s2, prec, series_cap=job.steps + 1)
            st2.init_random_phase(job.seed + rank).evolve(job.dt, job.steps)
            P = st2.polarization()
            N = st2.norm_series()
            h2d, d2h = st2.transfer_bytes()
            st2.close()
            return P, N, h2d + job.J.nbytes, d2h
        e2e_job()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, _, h2d, d2h = e2e_job()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e_s = max_over_ranks(e2e_s, dist)
        out["e2e"] = {"value": world * upd / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "s_per_step": e2e_s}

    # the FP64 (complex128) path on the same workload
    fp64_steps = job.steps if args.fp64_steps < 0 else args.fp64_steps
    if not args.skip_fp64 and fp64_steps > 0:
        st64 = spinrp.State(sysm, "c128", series_cap=fp64_steps + 1)
        st64.init_random_phase(job.seed + rank).evolve(job.dt, 1)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st64.init_random_phase(job.seed + rank)
        f0.record(stream)
        st64.evolve(job.dt, fp64_steps)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        P64 = st64.polarization()
        n = min(len(P64), len(P32))
        upd64 = updates_per_job(job.M, nb, fp64_steps)
        # FP64-pipe roofline: a gate rotates 2^M / 4 flip-flop pairs at 6 FMAs
        # each, 1.5 FMA = 3 FLOP per amplitude update; peak = SMs x max SM
        # clock x 2 FP64 FMA per SM per clock x 2 FLOP
        sms = torch.cuda.get_device_properties(stream.device).multi_processor_count
        peak64 = sms * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 * 2 * 2 / 1e12
        ach64 = 3.0 * upd64 / (ms64 / 1e3) / 1e12
        out["fp64"] = {"value": world * upd64 / (ms64 / 1e3),
                       "unit": UNIT, "trotter_steps": fp64_steps, "ms": ms64,
                       "fp32_vs_fp64_max_dP": float(np.max(np.abs(P32[:n] - P64[:n]))),
                       "fp32_vs_fp64_compared_entries": int(n),
                       "roofline": {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                                    "frac": ach64 / peak64, "traffic": None,
                                    "kernel": ("sweep2d_kernel" if sysm.plan_info("c128")["K"] >= 10
                                               else "sweep_kernel<double>"),
                                    "peak_source": "derived: SMs x max SM clock x 2 FP64 FMA/clk/SM x 2",
                                    "flops": "flip-flop gate FMAs only"}}
        st64.close()

    if rank == 0 and not args.skip_cpu:
        threads = os.cpu_count() or 1
        gates = args.cpu_gates
        t = oracle_sample(job, gates, threads, repeats=1)[0]
        out["cpu_baseline"] = {
            "value": gates * float(2 ** job.M) / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"FP64 CPU oracle, {gates} flip-flop gate applications (canonical order) of the "
                       f"M={job.M} state, {threads} threads, {t:.1f} s; initialization untimed"),
        }
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ladder_m30",
                    choices=["ladder_m30", "star_m20", "ladder_m14", "ladder_m26", "star_batch"])
    ap.add_argument("--batch-jobs", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--batch-cpu-steps", type=int, default=3, help="oracle steps per sampled job (star_batch)")
    ap.add_argument("--batch-launch", choices=["persistent", "per-sweep"], default="per-sweep",
                    help="star_batch: multi-tile groups in one persistent launch, or one launch per sweep")
    ap.add_argument("--fp64-steps", type=int, default=-1,
                    help="Trotter steps of the complex128 run (default: all of the workload's)")
    ap.add_argument("--cpu-gates", type=int, default=43)
    ap.add_argument("--ref-gates", type=int, default=16)
    ap.add_argument("--tile-K", type=int, default=0, help="tile width override (autotuner knob)")
    ap.add_argument("--regbits", type=int, default=0, help="register bits per phase, 5 or 6 (autotuner knob)")
    ap.add_argument("--sites", action="store_true", help="all-site readout P_{q1}(t) of every spin each step")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="one tile per block instead of the pipelined sweep (for comparison)")
    ap.add_argument("--product", action="store_true", help="the paper's product random state instead of the entangled one")
    ap.add_argument("--autotune", action="store_true",
                    help="time tile / register-bit candidates first and run the fastest (spinrp.autotune)")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "star_batch" and args.impl == "ours":
        return run_batch(args, rank, world, local_rank)
    if args.impl == "reference":
        return run_reference(args, rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
