"""Batches: many disorder realizations and phase seeds of uneven M evolved
together (the N_alpha average of the paper's Eq. 4).

Each job of a batch runs the same kernels as a single state of that system;
with the same tile width (the default tile model counts a plan group's jobs,
so large groups may take wider tiles; these small groups do not) it runs the
same plan, so its P(t) equals the single-state result bit for bit; a few jobs
are checked against the FP64 oracle; the device ensemble mean / spread equal
the host reduction of the per-job series.
"""
import os

import numpy as np
import pytest

import oracle
from paper_0710_3747_gb300 import spinrp
from paper_0710_3747_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _jobs(n=18, seed=3):
    jobs = W.star_batch(n=n, seed=seed, m_lo=8, m_hi=14, dt=0.02, steps=40)
    jobs += [W.Job(W.ladder(5, 1.0, 0.5), W.XY, seed=99, dt=0.02, steps=40, kind="ladder")]
    return jobs


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_batch_equals_single_states(prec):
    spinrp.lib()
    jobs = _jobs()
    systems = [spinrp.System(j.J, j.htype) for j in jobs]
    b = spinrp.Batch(systems, [j.seed for j in jobs], prec, series_cap=64)
    assert b.info()["groups"] >= 4
    b.init_random_phase()
    b.evolve(0.02, 25)
    b.evolve(0.02, 15)
    for k, j in enumerate(jobs):
        st = spinrp.State(spinrp.System(j.J, j.htype), prec, series_cap=64)
        st.init_random_phase(j.seed).evolve(0.02, 25).evolve(0.02, 15)
        assert np.array_equal(b.polarization(k), st.polarization()), k
        st.close()
    tol = 1e-10 if prec == "c128" else 1e-4
    for k in (0, 5, len(jobs) - 1):
        j = jobs[k]
        Pw, _, _ = oracle.run(j.J, j.htype, j.seed, 0.02, 40)
        assert np.max(np.abs(b.polarization(k) - Pw)) <= tol
    mean, std = b.ensemble()
    allP = np.array([b.polarization(k) for k in range(len(jobs))])
    np.testing.assert_allclose(mean, allP.mean(axis=0), atol=1e-13)
    np.testing.assert_allclose(std, allP.std(axis=0), atol=1e-13)
    b.close()


def test_batch_spread_shrinks_with_m():
    """Self-averaging across realizations: the spread of P over seeds of one
    system falls with M (paper: Chebyshev bound, max p_i = 2^{-(M-1)})."""
    spinrp.lib()
    spread = {}
    for M in (10, 14):
        J = W.star_dipolar(M, 1)
        systems = [spinrp.System(J, W.DIPOLAR) for _ in range(32)]
        b = spinrp.Batch(systems, list(range(1, 33)), "c64", series_cap=32)
        b.init_random_phase().evolve(0.05, 30)
        mean, std = b.ensemble()
        spread[M] = std[10:].mean()
        b.close()
    assert spread[14] < spread[10] / 2.5


@pytest.mark.slow
def test_full_size_batch_sampled_jobs():
    """The bench's batch at its full size (4096 dipolar stars, M uniform in
    12..22, the bench's seed and launch configuration) for 100 steps, the
    multi-tile groups in one persistent launch and the small stars resident in
    shared memory: sampled jobs (the smallest and largest M and three others)
    against the FP64 oracle at the FP32 bar at every step; the device
    ensemble mean equals the mean of the per-job series."""
    spinrp.lib()
    steps = 100
    jobs = W.star_batch(n=4096, seed=4, steps=steps)
    systems = [spinrp.System(j.J, j.htype) for j in jobs]
    b = spinrp.Batch(systems, [j.seed for j in jobs], "c64", series_cap=steps + 1)
    b.set_persistent(True)
    assert b.info()["groups"] == 11
    b.init_random_phase().evolve(0.02, steps)
    Ms = np.array([j.M for j in jobs])
    picks = [0, 1777, 4095, int(np.argmax(Ms)), int(np.argmin(Ms))]
    for k in picks:
        j = jobs[k]
        Pw, _, _ = oracle.run(j.J, j.htype, j.seed, 0.02, steps, threads=os.cpu_count() or 1)
        assert np.max(np.abs(b.polarization(k) - Pw)) <= 1e-4, (k, j.M)
    mean, _ = b.ensemble()
    allP = np.array([b.polarization(k) for k in range(4096)])
    np.testing.assert_allclose(mean, allP.mean(axis=0), atol=1e-12)
    b.close()


@pytest.mark.parametrize("K", [13, 14])
def test_persistent_launch_equals_per_sweep_launches(K):
    """The batch's multi-tile groups as one persistent launch (blocks pulling
    tiles from a device queue, per-job counters ordering the sweeps) give the
    same P(t) bit for bit as one launch per sweep, over two evolve calls of
    different lengths (a new plan and graph each), for stars and ladders of
    several sizes in one batch; sampled jobs against the oracle."""
    spinrp.lib()
    rng = np.random.default_rng(K)
    jobs = []
    for k in range(40):
        M = int(rng.integers(15, 19))
        if k % 3 == 0:
            J, ht = W.ladder(M // 2, 1.0, float(rng.uniform(0.2, 1.0))), W.XY
        else:
            J, ht = W.star_dipolar(M, 100 + k), W.DIPOLAR
        jobs.append(W.Job(J, ht, seed=1000 + k, dt=0.02, steps=0, kind="x"))

    def run(persistent):
        systems = []
        for j in jobs:
            s = spinrp.System(j.J, j.htype)
            s.set_tile("c64", K)
            s.set_regbits(6)
            systems.append(s)
        b = spinrp.Batch(systems, [j.seed for j in jobs], "c64", series_cap=64)
        b.set_persistent(persistent)
        b.init_random_phase().evolve(0.02, 17).evolve(0.02, 9)
        P = [b.polarization(k) for k in range(len(jobs))]
        mean, std = b.ensemble()
        b.close()
        return P, mean

    Pp, mp = run(True)
    Pl, ml = run(False)
    for k in range(len(jobs)):
        assert np.array_equal(Pp[k], Pl[k]), k
    assert np.array_equal(mp, ml)
    for k in (0, 1, 38):
        j = jobs[k]
        Pw, _, _ = oracle.run(j.J, j.htype, j.seed, 0.02, 26, threads=os.cpu_count() or 1)
        assert np.max(np.abs(Pp[k] - Pw)) <= 1e-4, k


def test_persistent_waits_are_bounded():
    """Failure detection without a GPU fault: a persistent launch whose queue
    starts past the first sweep has every wait run out; the blocks give up
    within the poll limit (about a second), the status reads
    SPINRP_ETIMEOUT, no tile was touched, and the batch then evolves exactly
    as a batch that never saw the failed launch."""
    spinrp.lib()
    jobs = [W.Job(W.star_dipolar(15 + (k % 2), 300 + k), W.DIPOLAR, seed=50 + k, dt=0.02, steps=0)
            for k in range(6)]

    def make():
        systems = []
        for j in jobs:
            s = spinrp.System(j.J, j.htype)
            s.set_tile("c64", 13)
            s.set_regbits(6)
            systems.append(s)
        b = spinrp.Batch(systems, [j.seed for j in jobs], "c64", series_cap=16)
        return b.set_persistent(True)

    b = make()
    b.init_random_phase()
    rc, sec = b.persist_timeout_check(4)
    assert rc == spinrp.ETIMEOUT
    assert 0.0 < sec < 30.0
    b.evolve(0.02, 6)
    ref = make()
    ref.init_random_phase().evolve(0.02, 6)
    for k in range(len(jobs)):
        assert np.array_equal(b.polarization(k), ref.polarization(k)), k
    b.close()
    ref.close()


def test_batch_autotuner_sets_a_measured_width():
    """spinrp.autotune_batch times the whole batch at each candidate tile width
    of its multi-tile systems, keeps the fastest and sets it (six register
    bits) on those systems; the tuned batch still evolves as the oracle does."""
    spinrp.lib()
    jobs = [W.Job(W.star_dipolar(15 + (k % 2), 500 + k), W.DIPOLAR, seed=70 + k, dt=0.02, steps=0)
            for k in range(8)]
    jobs.append(W.Job(W.star_dipolar(12, 599), W.DIPOLAR, seed=99, dt=0.02, steps=0))
    systems = [spinrp.System(j.J, j.htype) for j in jobs]
    r = spinrp.autotune_batch(systems, [j.seed for j in jobs], candidates=(13, 14), probe_steps=4)
    assert set(r["ms_per_step"]) == {13, 14}
    assert r["K"] == min(r["ms_per_step"], key=r["ms_per_step"].get)
    for s in systems[:-1]:
        assert s.plan_info("c64")["K"] == r["K"]
    assert systems[-1].plan_info("c64")["K"] == 12  # below the multi-tile sizes: untouched
    b = spinrp.Batch(systems, [j.seed for j in jobs], "c64", series_cap=11)
    b.init_random_phase().evolve(0.02, 10)
    for k in (0, len(jobs) - 1):
        j = jobs[k]
        Pw, _, _ = oracle.run(j.J, j.htype, j.seed, 0.02, 10, threads=os.cpu_count() or 1)
        assert np.max(np.abs(b.polarization(k) - Pw)) <= 1e-4, k
    b.close()


def test_pipelined_batch_sweeps_equal_one_tile_per_block():
    """Multi-tile groups with enough (job, tile) units run each sweep as one
    pipelined launch over all their jobs' tiles (units job-major, each job's
    partials combined by the block that finishes its last tile); every job's
    P(t) and the ensemble are the same bit for bit as with one tile per block,
    over two evolve calls (a steady-step graph replayed); a small group stays
    one tile per block; sampled jobs against the oracle."""
    spinrp.lib()
    jobs = []
    for k in range(24):
        jobs.append(W.Job(W.star_dipolar(18, 300 + k), W.DIPOLAR, seed=40 + k, dt=0.02, steps=0, kind="s18"))
    for k in range(6):
        jobs.append(W.Job(W.star_dipolar(20, 400 + k), W.DIPOLAR, seed=80 + k, dt=0.02, steps=0, kind="s20"))
    for k in range(8):
        jobs.append(W.Job(W.ladder(8, 1.0, 0.3 + 0.05 * k), W.XY, seed=120 + k, dt=0.02, steps=0, kind="l16"))
    for k in range(3):
        jobs.append(W.Job(W.ladder(11, 1.0, 0.4 + 0.1 * k), W.XY, seed=160 + k, dt=0.02, steps=0, kind="l22"))

    def run(pipe):
        systems = []
        for j in jobs:
            s = spinrp.System(j.J, j.htype)
            s.set_tile("c64", 13)
            s.set_regbits(6)
            systems.append(s)
        b = spinrp.Batch(systems, [j.seed for j in jobs], "c64", series_cap=32)
        b.set_pipeline(pipe)
        groups = b.pipeline_groups()
        b.init_random_phase().evolve(0.02, 17).evolve(0.02, 9)
        P = [b.polarization(k) for k in range(len(jobs))]
        mean, _ = b.ensemble()
        b.close()
        return P, mean, groups

    Pp, mp, gp = run(True)
    Pl, ml, gl = run(False)
    # stars of 18 spins (24 x 32 tiles), of 20 (6 x 128) and ladders of 22
    # (3 x 512) are pipelined; 8 ladders of 16 spins (64 tiles) are not
    assert gp == 3 and gl == 0
    for k in range(len(jobs)):
        assert np.array_equal(Pp[k], Pl[k]), k
    assert np.array_equal(mp, ml)
    for k in (0, 25, 39):
        j = jobs[k]
        Pw, _, _ = oracle.run(j.J, j.htype, j.seed, 0.02, 26, threads=os.cpu_count() or 1)
        assert np.max(np.abs(Pp[k] - Pw)) <= 1e-4, k
