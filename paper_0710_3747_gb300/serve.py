"""Continuous-batching serving loop for spin-dynamics jobs.

Requests (ladder or star jobs of different M and final time) arrive over
time.  The loop keeps every admitted job's state resident on the GPU, each on
its own CUDA stream, and advances all active jobs in chunks of Trotter steps,
so their kernels overlap on the device.  A job is admitted as soon as it has
arrived, a slot is free and its device footprint (amplitudes + workspace, as
spinrp_state_bytes reports) fits in the HBM budget; finished jobs free their
memory and slot at once.  Latency = completion (P(t) copied to the host) -
arrival.  ``run_sequential`` runs the same jobs one at a time for comparison.

All device work goes through the C ABI (``spinrp``); this module only
schedules.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time
from dataclasses import dataclass, field

import numpy as np

from . import spinrp
from . import workloads as W


@dataclass
class Result:
    index: int
    M: int
    kind: str
    steps: int
    arrival: float
    start: float = 0.0
    done: float = 0.0
    P: np.ndarray | None = None
    norm: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Active:
    job: W.Job
    res: Result
    state: spinrp.State
    stream: object
    left: int
    bytes: int
    system: spinrp.System = field(repr=False, default=None)
    events: list = field(default_factory=list)  # CUDA events of the chunks in flight


def footprint(job: W.Job, prec: str) -> int:
    s = spinrp.System(job.J, job.htype)
    p, w = spinrp.state_bytes(s, prec, job.steps + 1)
    return p + w


def job_work(job: W.Job) -> float:
    """Amplitude-gate updates of the whole job (2^M x 2 bonds x steps)."""
    nb = int(np.count_nonzero(np.triu(job.J, 1)))
    return float(2 ** job.M) * 2 * nb * job.steps


# Stream priority of a job by its size: work below 10^10 amplitude-gate
# updates (milliseconds on the GPU) gets the highest priority, below 10^12
# (well under a second) the next, the rest the lowest.  The GPU's block
# scheduler then serves short jobs first when streams compete, so a short job
# arriving behind long ones is not queued behind their sweeps.
def _priority(job: W.Job) -> int:
    w = job_work(job)
    return -2 if w < 1e10 else (-1 if w < 1e12 else 0)


def _start(job: W.Job, prec: str, now: float, tile_K: int | None, priority: int = 0,
           pipeline: bool = True) -> _Active:
    import torch
    stream = torch.cuda.Stream(priority=priority)
    sysm = spinrp.System(job.J, job.htype)
    if tile_K:
        sysm.set_tile(prec, min(tile_K, job.M))
    st = spinrp.State(sysm, prec, series_cap=job.steps + 1, stream=stream.cuda_stream)
    if not pipeline:
        st.set_pipeline(False)
    st.init_random_phase(job.seed)
    p, w = st.psi_bytes, st.work_bytes
    res = Result(job.meta.get("index", -1), job.M, job.kind, job.steps, job.arrival, start=now)
    return _Active(job, res, st, stream, job.steps, p + w, sysm)


def _finish(a: _Active, now_fn) -> Result:
    a.res.P = a.state.polarization()      # synchronizes the job's stream (already done)
    a.res.norm = a.state.norm_series()
    a.res.done = now_fn()
    a.state.close()
    return a.res


def _chunk_done(a: _Active) -> bool:
    """True when the oldest chunk in flight has finished on the device
    (always for host-side fakes, which have no stream)."""
    if not a.events:
        return True
    if a.events[0].query():
        a.events.pop(0)
        return True
    return False


def run_stream(jobs: list[W.Job], prec: str = "c64", max_active: int = 16,
               hbm_budget: int | None = None, chunk: int = 20, tile_K: int | None = None,
               realtime: bool = True, start_fn=None, finish_fn=None, footprint_fn=None,
               trace: list | None = None, depth: int = 2, priorities: bool = True,
               policy: str = "fifo", pipeline: bool = True) -> list[Result]:
    """Serve `jobs` (sorted by arrival) with continuous batching.

    realtime: arrivals follow the wall clock (t = 0 at the call); otherwise all
    jobs are treated as arrived at their arrival offset but admitted as soon
    as resources allow (a saturated queue).  Each admitted job gets its own
    CUDA stream (priority by job size when `priorities`); the loop keeps up to
    `depth` chunks of `chunk` Trotter steps in flight per job, polls their
    completion events without blocking, and retires a job (P(t) to the host,
    memory and slot freed) as soon as its last chunk has finished.  Each job's
    footprint is computed once.  policy "fifo" admits arrived jobs in arrival
    order; "sjf" admits, among the arrived jobs, the one with the least work
    (amplitude-gate updates) first.  pipeline False keeps every job's sweeps
    one tile per block (a pipelined sweep holds every SM for its duration,
    so the other jobs' blocks wait for it).  start_fn / finish_fn / footprint_fn replace
    the device calls (host-side tests); `trace`, when given, receives
    ("admit" | "chunk" | "done", job index, bytes in use)."""
    footprint_fn = footprint_fn or footprint
    start_fn = start_fn or _start
    finish_fn = finish_fn or _finish
    if hbm_budget is None:
        import torch
        free, _ = torch.cuda.mem_get_info()
        hbm_budget = int(0.8 * free)
    pending = sorted(jobs, key=lambda j: j.arrival)
    need = {}
    active: list[_Active] = []
    done: list[Result] = []
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    used = 0
    k = 0
    while k < len(pending) or active:
        progress = False
        # admit arrived jobs while slots and memory allow
        if policy == "sjf" and k < len(pending):
            # order the arrived, not yet admitted jobs by work (least first)
            t_now = now()
            m = k
            while m < len(pending) and (not realtime or pending[m].arrival <= t_now):
                m += 1
            if m - k > 1:
                order = sorted(range(k, m), key=lambda q: (job_work(pending[q]), q))
                moved = [pending[q] for q in order]
                keys = [need.pop(q, None) for q in order]
                pending[k:m] = moved
                for off, v in enumerate(keys):
                    if v is not None:
                        need[k + off] = v
        while k < len(pending) and len(active) < max_active:
            j = pending[k]
            if realtime and j.arrival > now():
                break
            if k not in need:
                need[k] = footprint_fn(j, prec)
                if need[k] > hbm_budget:
                    raise spinrp.SpinrpError(spinrp.ENOMEM,
                                             f"job {k} needs {need[k]} B > budget {hbm_budget} B")
            if used + need[k] > hbm_budget:
                break
            if start_fn is _start:
                a = _start(j, prec, now(), tile_K, _priority(j) if priorities else 0, pipeline)
            else:
                a = start_fn(j, prec, now(), tile_K)
            active.append(a)
            used += a.bytes
            progress = True
            if trace is not None:
                trace.append(("admit", a.res.index, used))
            k += 1
        # keep up to `depth` chunks in flight per job
        for a in active:
            while a.left > 0 and len(a.events) < depth:
                n = min(chunk, a.left)
                a.state.evolve(a.job.dt, n)
                a.left -= n
                if a.stream is not None:
                    import torch
                    ev = torch.cuda.Event()
                    ev.record(a.stream)
                    a.events.append(ev)
                progress = True
                if trace is not None:
                    trace.append(("chunk", a.res.index, used))
        # retire finished chunks and jobs
        still = []
        for a in active:
            while a.events and _chunk_done(a):
                progress = True
            if a.left == 0 and not a.events:
                done.append(finish_fn(a, now))
                used -= a.bytes
                progress = True
                if trace is not None:
                    trace.append(("done", a.res.index, used))
            else:
                still.append(a)
        active = still
        if not progress:
            # idle: wait for the next arrival or completion
            wait = 0.0002
            if not active and k < len(pending):
                wait = max(0.0, min(0.01, pending[k].arrival - now()))
            time.sleep(wait)
    return sorted(done, key=lambda r: r.index)


def run_sequential(jobs: list[W.Job], prec: str = "c64", tile_K: int | None = None,
                   realtime: bool = True, chunk: int | None = None, pipeline: bool = True) -> list[Result]:
    """The same jobs one at a time, each started when it has arrived and the
    previous one is done (in evolve calls of `chunk` steps when given, else
    one call per job)."""
    import torch
    out = []
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    for j in sorted(jobs, key=lambda j: j.arrival):
        if realtime and j.arrival > now():
            time.sleep(j.arrival - now())
        a = _start(j, prec, now(), tile_K, pipeline=pipeline)
        left = j.steps
        while left > 0:
            n = left if not chunk else min(chunk, left)
            a.state.evolve(j.dt, n)
            left -= n
        out.append(_finish(a, now))
    torch.cuda.synchronize()
    return sorted(out, key=lambda r: r.index)


def summary(results: list[Result], wall: float) -> dict:
    lat = np.array([r.latency for r in results])
    return {"jobs": len(results), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "jobs_per_s": len(results) / wall, "wall_s": wall}


def main(argv=None):
    ap = argparse.ArgumentParser(description="serve a Poisson stream of spin-dynamics jobs")
    ap.add_argument("--jobs", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=0.0, help="arrivals per second (0: measure, then 0.7x)")
    ap.add_argument("--m-cap", type=int, default=None)
    ap.add_argument("--max-active", type=int, default=16)
    ap.add_argument("--chunk", type=int, default=20)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--prec", default="c64")
    ap.add_argument("--tile-K", type=int, default=0, help="tile width for every job (0: the library's default)")
    ap.add_argument("--saturated", action="store_true",
                    help="every job arrives at t = 0 (a full queue): throughput is not bound by arrivals")
    ap.add_argument("--no-priorities", action="store_true", help="all job streams at the default priority")
    ap.add_argument("--policy", choices=["fifo", "sjf"], default="fifo",
                    help="admission order among arrived jobs: arrival, or least work first")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="every job's sweeps one tile per block (no pipelined sweeps)")
    ap.add_argument("--mode", choices=["both", "continuous", "sequential"], default="both",
                    help="which modes to run (one per process keeps each run's device state apart)")
    args = ap.parse_args(argv)
    tile_K = args.tile_K or None
    import torch
    spinrp.lib()
    rate = args.rate
    if rate <= 0 and not args.saturated:
        probe = W.serve_stream(n=20, seed=args.seed + 1, rate=1e9, m_cap=args.m_cap)
        t = time.perf_counter()
        run_sequential(probe, args.prec, tile_K=tile_K, realtime=False)
        rate = 0.7 * len(probe) / (time.perf_counter() - t)
    jobs = W.serve_stream(n=args.jobs, seed=args.seed, rate=rate if rate > 0 else 1.0, m_cap=args.m_cap)
    realtime = not args.saturated
    if args.saturated:
        for j in jobs:
            j.arrival = 0.0
    work = sum(job_work(j) for j in jobs)
    Ms = [j.M for j in jobs]
    out = {"jobs": len(jobs), "saturated": args.saturated, "rate_per_s": None if args.saturated else rate,
           "M_range": [min(Ms), max(Ms)], "amp_gate_updates": work, "policy": args.policy,
           "pipelined_sweeps": not args.no_pipeline}
    res = {}
    for mode in ("continuous", "sequential"):
        if args.mode not in ("both", mode):
            continue
        t = time.perf_counter()
        if mode == "continuous":
            r = run_stream(jobs, args.prec, max_active=args.max_active, chunk=args.chunk, tile_K=tile_K,
                           realtime=realtime, priorities=not args.no_priorities, policy=args.policy,
                           pipeline=not args.no_pipeline)
        else:
            r = run_sequential(jobs, args.prec, tile_K=tile_K, realtime=realtime, pipeline=not args.no_pipeline)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t
        res[mode] = r
        out[mode] = summary(r, wall)
        out[mode]["amp_gate_updates_per_s"] = work / wall
    if len(res) == 2:
        out["max_dP_mix_vs_alone"] = max(float(np.max(np.abs(a.P - b.P)))
                                         for a, b in zip(res["continuous"], res["sequential"]))
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
