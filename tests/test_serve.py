"""Serving loop: continuous batching with HBM-footprint admission.

Host-side tests drive the scheduler with fake states (no GPU): admission
respects the slot limit and the memory budget, jobs are admitted in arrival
order as soon as resources free up, and every job gets exactly its number of
Trotter steps.  The GPU test runs a small request stream for real and checks
that each job's P(t) is the same alone and in the mix, and matches the oracle.
"""
import numpy as np
import pytest

from paper_0710_3747_gb300 import serve
from paper_0710_3747_gb300 import workloads as W


class FakeState:
    def __init__(self):
        self.steps = 0

    def evolve(self, dt, n):
        self.steps += n


def _fake_start(job, prec, now, tile_K):
    res = serve.Result(job.meta["index"], job.M, job.kind, job.steps, job.arrival, start=now)
    return serve._Active(job, res, FakeState(), None, job.steps, job.meta["bytes"])


def _fake_finish(a, now_fn):
    a.res.P = np.array([a.state.steps], float)
    a.res.done = now_fn()
    return a.res


def _jobs(n=12, seed=3):
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n):
        M = int(rng.integers(4, 9))
        j = W.Job(W.chain(M), W.XY, seed=k, dt=0.05, steps=int(rng.integers(1, 60)), kind="chain",
                  arrival=0.0, meta={"index": k, "bytes": int(rng.integers(1, 5)) * 100})
        jobs.append(j)
    return jobs


@pytest.mark.parametrize("max_active,budget,chunk", [(1, 10**9, 7), (3, 10**9, 5), (8, 500, 3), (16, 400, 50)])
def test_admission_and_completion(max_active, budget, chunk):
    jobs = _jobs()
    trace = []
    out = serve.run_stream(jobs, max_active=max_active, hbm_budget=budget, chunk=chunk, realtime=False,
                           start_fn=_fake_start, finish_fn=_fake_finish,
                           footprint_fn=lambda j, p: j.meta["bytes"], trace=trace)
    assert [r.index for r in out] == list(range(len(jobs)))
    for r, j in zip(out, jobs):
        assert r.P[0] == j.steps  # every job got exactly its steps
    active, admitted = set(), []
    for ev, idx, used in trace:
        if ev == "admit":
            active.add(idx)
            admitted.append(idx)
        elif ev == "done":
            active.discard(idx)
        assert len(active) <= max_active
        assert used <= budget
        assert used == sum(jobs[i].meta["bytes"] for i in active)
    assert admitted == sorted(admitted)  # arrival order
    # overlap: with more than one slot, several jobs are in flight at once
    if max_active > 1 and budget > 1000:
        assert max(sum(1 for e in trace[:k + 1] if e[0] == "admit") -
                   sum(1 for e in trace[:k + 1] if e[0] == "done") for k in range(len(trace))) > 1


def test_oversized_job_is_rejected():
    jobs = _jobs(3)
    jobs[1].meta["bytes"] = 10**6
    with pytest.raises(Exception):
        serve.run_stream(jobs, max_active=4, hbm_budget=1000, realtime=False, start_fn=_fake_start,
                         finish_fn=_fake_finish, footprint_fn=lambda j, p: j.meta["bytes"])


def test_serve_stream_shapes():
    jobs = W.serve_stream(n=200, seed=1, rate=5.0)
    Ms = np.array([j.M for j in jobs])
    assert Ms.min() >= 10 and Ms.max() <= 28
    assert all(j.M % 2 == 0 for j in jobs if j.kind == "ladder")
    arr = np.array([j.arrival for j in jobs])
    assert np.all(np.diff(arr) > 0)
    assert 0.5 * 200 / 5.0 < arr[-1] < 2.0 * 200 / 5.0
    kinds = [j.kind for j in jobs]
    assert 60 < kinds.count("ladder") < 140


@pytest.mark.gpu
def test_mix_equals_alone_and_oracle():
    import oracle
    from paper_0710_3747_gb300 import spinrp
    spinrp.lib()
    jobs = W.serve_stream(n=10, seed=11, rate=1e6, m_lo=10, m_hi=15, t_lo=1.0, t_hi=3.0)
    mix = serve.run_stream(jobs, "c64", max_active=4, chunk=7, realtime=False)
    # alone, same evolve chunks: bit for bit (concurrency changes nothing)
    alone = serve.run_sequential(jobs, "c64", realtime=False, chunk=7)
    # alone, one evolve call per job: D(dt/2)D(dt/2) at chunk seams instead
    # of D(dt) moves the result by rounding only
    whole = serve.run_sequential(jobs, "c64", realtime=False)
    for a, b, c, j in zip(mix, alone, whole, jobs):
        assert a.P.shape == (j.steps + 1,)
        assert np.array_equal(a.P, b.P)
        assert np.max(np.abs(a.P - c.P)) <= 1e-5
    for r, j in list(zip(mix, jobs))[:4]:
        Pw, _, _ = oracle.run(j.J, j.htype, j.seed, j.dt, j.steps)
        assert np.max(np.abs(r.P - Pw)) <= 1e-4


@pytest.mark.gpu
@pytest.mark.slow
def test_full_stream_sampled_jobs_match_oracle():
    """Twenty jobs with M <= 22 drawn at random from the full 2000-job request
    stream (its seed and distributions: ladders and dipolar stars, M
    log-uniform in 10..28, T in [5, 50]), served together through the
    continuous-batching loop, each P(t) against the FP64 oracle at the FP32
    bar at every step.  Jobs are drawn until the oracle's share of the test
    would exceed about a minute of host time."""
    import os

    import oracle
    from paper_0710_3747_gb300 import spinrp
    spinrp.lib()
    jobs = W.serve_stream(n=2000, seed=5, rate=1.0)
    cand = [j for j in jobs if j.M <= 22]
    rng = np.random.default_rng(7)
    pick, cost = [], 0.0
    for i in rng.permutation(len(cand)):
        j = cand[i]
        c = serve.job_work(j) / 1.0e10  # oracle seconds at about 1e10 updates/s
        if cost + c > 60.0:
            continue
        pick.append(j)
        cost += c
        if len(pick) == 20:
            break
    assert len(pick) == 20
    for j in pick:
        j.arrival = 0.0
    out = serve.run_stream(pick, "c64", max_active=8, chunk=20, realtime=False)
    by_index = {j.meta["index"]: j for j in pick}
    worst = 0.0
    for r in out:
        j = by_index[r.index]
        Pw, _, _ = oracle.run(j.J, j.htype, j.seed, j.dt, j.steps, threads=os.cpu_count() or 1)
        assert r.P.shape == Pw.shape
        err = float(np.max(np.abs(r.P - Pw)))
        worst = max(worst, err)
        assert err <= 1e-4, (j.kind, j.M, j.steps, err)
    print(f"20 sampled jobs (M {min(j.M for j in pick)}..{max(j.M for j in pick)}): max |dP| = {worst:.2e}")


def test_sjf_admits_least_work_first():
    """With every job arrived, policy "sjf" admits in order of work (2^M x
    bonds x steps), least first; each job still gets exactly its steps."""
    jobs = _jobs(10, seed=8)
    trace = []
    out = serve.run_stream(jobs, max_active=1, hbm_budget=10**9, chunk=5, realtime=False,
                           start_fn=_fake_start, finish_fn=_fake_finish,
                           footprint_fn=lambda j, p: j.meta["bytes"], trace=trace, policy="sjf")
    for r, j in zip(out, jobs):
        assert r.P[0] == j.steps
    admitted = [idx for ev, idx, _ in trace if ev == "admit"]
    work = {j.meta["index"]: serve.job_work(j) for j in jobs}
    assert [work[i] for i in admitted] == sorted(work[i] for i in admitted)
