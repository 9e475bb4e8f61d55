"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (stated by the task for P(t)): |dP| <= 1e-10 for the FP64 path and
|dP| <= 1e-4 for the FP32 path, at every recorded step.  Amplitudes of the
FP64 path are compared at 1e-11 (a few hundred gate applications of FP64
rounding); the FP32 initial state at 2e-7 relative (FP32 rounding of the
phase).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_0710_3747_gb300 import spinrp
from paper_0710_3747_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1
TOL_P = {"c128": 1e-10, "c64": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    spinrp.lib()


def _oracle(J, htype, seed, dt, steps, a=None):
    return oracle.run(J, htype, seed, dt, steps, a_generic=a, threads=THREADS)


def _gpu(J, htype, seed, dt, steps, prec, a=None, K=None, chunks=None, rb=None):
    s = spinrp.System(J, htype, a)
    if K:
        s.set_tile(prec, K)
    if rb:
        s.set_regbits(rb)
    st = spinrp.State(s, prec, series_cap=steps + 1)
    st.init_random_phase(seed)
    for n in (chunks or [steps]):
        st.evolve(dt, n)
    return st.polarization(1), st.norm_series(), st


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("M", [2, 3, 5, 14, 20])
def test_initial_state(prec, M):
    J = W.chain(M)
    s = spinrp.System(J, spinrp.XY)
    st = spinrp.State(s, prec, series_cap=1)
    st.init_random_phase(12345 + M)
    got = st.amplitudes()
    want = oracle.init_random_phase(M, 12345 + M, threads=THREADS)
    tol = 1e-15 if prec == "c128" else 2e-7 * 2.0 ** (-(M - 1) / 2)
    assert np.max(np.abs(got - want)) < tol
    P, nrm = st.polarization(1), st.norm_series()
    assert P[0] == pytest.approx(1.0, abs=1e-15)
    assert nrm[0] == pytest.approx(1.0, abs=1e-13 if prec == "c128" else 1e-6)


def _small_systems():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(7, 7))
    A = A + A.T
    return [
        ("pair", np.array([[0, 1.3], [1.3, 0]]), spinrp.DIPOLAR, None),
        ("ladder6", W.ladder(3, 1.0, 0.5), spinrp.XY, None),
        ("chain9", W.chain(9, 0.8), spinrp.XY, None),
        ("star8", W.star_dipolar(8, 3), spinrp.DIPOLAR, None),
        ("iso7", W.star_gaussian(7, 4), spinrp.ISOTROPIC, None),
        ("ising6", W.star_gaussian(6, 5), spinrp.ISING, None),
        ("generic7", W.star_gaussian(7, 6), spinrp.GENERIC, A),
        ("ladder10", W.ladder(5, 1.0, 0.1), spinrp.XY, None),
    ]


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("name,J,htype,a", _small_systems(), ids=lambda v: v if isinstance(v, str) else "")
def test_small_systems_full_state(name, J, htype, a, prec):
    seed, dt, steps = 77, 0.07, 9
    Pw, Nw, psi_w = _oracle(J, htype, seed, dt, steps, a)
    Pg, Ng, st = _gpu(J, htype, seed, dt, steps, prec, a)
    assert np.max(np.abs(Pg - Pw)) <= (1e-12 if prec == "c128" else 1e-5)
    assert np.max(np.abs(Ng - Nw)) <= (1e-12 if prec == "c128" else 1e-5)
    amp = st.amplitudes()
    assert np.max(np.abs(amp - psi_w)) <= (1e-12 if prec == "c128" else 2e-6)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("K", [4, 5, 6, 8, 9])
@pytest.mark.parametrize("kind", ["star12", "ladder12", "generic11"])
def test_multi_tile_plans(kind, K, prec):
    """Narrow tiles force several segments, relabelling sweeps, the diagonal
    phase split across tile/outer bits and the readout spin in outer bits."""
    if kind == "star12":
        J, ht, a = W.star_dipolar(12, 8), spinrp.DIPOLAR, None
    elif kind == "ladder12":
        J, ht, a = W.ladder(6, 1.0, 0.5), spinrp.XY, None
    else:
        rng = np.random.default_rng(2)
        a = rng.normal(size=(11, 11)); a = a + a.T
        J, ht = W.star_gaussian(11, 3), spinrp.GENERIC
    seed, dt, steps = 5, 0.05, 6
    Pw, Nw, psi_w = _oracle(J, ht, seed, dt, steps, a)
    Pg, Ng, st = _gpu(J, ht, seed, dt, steps, prec, a, K=K)
    info = st.system.plan_info(prec)
    assert info["K"] == K
    assert np.max(np.abs(Pg - Pw)) <= (1e-12 if prec == "c128" else 1e-5), info
    amp = st.amplitudes()
    assert np.max(np.abs(amp - psi_w)) <= (1e-12 if prec == "c128" else 2e-6), info


@pytest.mark.parametrize("rb,K", [(5, 10), (5, 11), (5, 12), (5, 13), (6, 11), (6, 12), (6, 13), (6, 14)])
@pytest.mark.parametrize("kind", ["star16", "ladder16", "generic15", "chain18"])
def test_register_blocked_sweeps(kind, rb, K):
    """complex64 tiles of K >= 10 spins run the register-blocked sweep:
    several tiles and segments, relabelling, diagonal phase across tile and
    outer bits."""
    rng = np.random.default_rng(4)
    a = None
    if kind == "star16":
        J, ht = W.star_dipolar(16, 8), spinrp.DIPOLAR
    elif kind == "ladder16":
        J, ht = W.ladder(8, 1.0, 0.5), spinrp.XY
    elif kind == "chain18":
        J, ht = W.chain(18, 0.9), spinrp.XY
    else:
        a = rng.normal(size=(15, 15)); a = a + a.T
        J, ht = W.star_gaussian(15, 3), spinrp.GENERIC
    seed, dt, steps = 11, 0.04, 5
    Pw, Nw, psi_w = _oracle(J, ht, seed, dt, steps, a)
    Pg, Ng, st = _gpu(J, ht, seed, dt, steps, "c64", a, K=K, rb=rb)
    assert st.system.plan_info("c64")["K"] == K
    assert np.max(np.abs(Pg - Pw)) <= 1e-5
    amp = st.amplitudes()
    assert np.max(np.abs(amp - psi_w)) <= 2e-6 * 2.0 ** (-(st.M - 1) / 2) * 64


@pytest.mark.parametrize("K", [10, 11, 12, 13])
@pytest.mark.parametrize("kind", ["star16", "ladder16", "generic15", "chain18"])
def test_register_blocked_sweeps_c128(kind, K):
    """complex128 tiles of K >= 10 spins run the FP64 register-blocked sweep
    (five register bits, 16-byte slots): the FP64 bar on P and on every
    amplitude, over several tiles, segments and relabelling sweeps."""
    rng = np.random.default_rng(4)
    a = None
    if kind == "star16":
        J, ht = W.star_dipolar(16, 8), spinrp.DIPOLAR
    elif kind == "ladder16":
        J, ht = W.ladder(8, 1.0, 0.5), spinrp.XY
    elif kind == "chain18":
        J, ht = W.chain(18, 0.9), spinrp.XY
    else:
        a = rng.normal(size=(15, 15)); a = a + a.T
        J, ht = W.star_gaussian(15, 3), spinrp.GENERIC
    seed, dt, steps = 11, 0.04, 5
    Pw, Nw, psi_w = _oracle(J, ht, seed, dt, steps, a)
    Pg, Ng, st = _gpu(J, ht, seed, dt, steps, "c128", a, K=K)
    assert st.system.plan_info("c128")["K"] == K
    assert np.max(np.abs(Pg - Pw)) <= TOL_P["c128"]
    assert np.max(np.abs(Ng - Nw)) <= 1e-12
    assert np.max(np.abs(st.amplitudes() - psi_w)) <= 1e-12


@pytest.mark.parametrize("steps", [1, 2, 3])
def test_few_steps_and_chunked_evolve(steps):
    J = W.star_dipolar(10, 4)
    Pw, _, psi_w = _oracle(J, spinrp.DIPOLAR, 3, 0.03, 2 * steps)
    # one call, and the same steps in two calls (D(dt/2) D(dt/2) at the seam)
    for chunks in ([2 * steps], [steps, steps]):
        Pg, _, st = _gpu(J, spinrp.DIPOLAR, 3, 0.03, 2 * steps, "c128", K=6, chunks=chunks)
        assert np.max(np.abs(Pg - Pw)) < 1e-12
        assert np.max(np.abs(st.amplitudes() - psi_w)) < 1e-12


def test_time_reversal_on_gpu():
    J = W.star_dipolar(12, 6)
    s = spinrp.System(J, spinrp.DIPOLAR)
    s.set_tile("c128", 7)
    st = spinrp.State(s, "c128", series_cap=41)
    st.init_random_phase(9)
    psi0 = st.amplitudes()
    st.evolve(0.05, 20)
    assert np.max(np.abs(st.amplitudes() - psi0)) > 1e-3
    st.evolve(-0.05, 20)
    assert np.max(np.abs(st.amplitudes() - psi0)) < 1e-12


def test_load_arbitrary_state():
    M = 9
    rng = np.random.default_rng(0)
    psi = rng.normal(size=1 << M) + 1j * rng.normal(size=1 << M)
    psi /= np.linalg.norm(psi)
    J = W.star_dipolar(M, 1)
    a, b = oracle.couplings(J, oracle.DIPOLAR)
    ref = psi.copy()
    P, _ = oracle.evolve(ref, a, b, 0.04, 10)
    s = spinrp.System(J, spinrp.DIPOLAR)
    s.set_tile("c128", 5)
    st = spinrp.State(s, "c128", series_cap=11)
    st.load(psi)
    assert st.polarization()[0] == pytest.approx(oracle.polarization(psi), abs=1e-14)
    st.evolve(0.04, 10)
    assert np.max(np.abs(st.polarization()[1:] - P)) < 1e-12
    assert np.max(np.abs(st.amplitudes() - ref)) < 1e-12


@pytest.mark.parametrize("prec,K", [("c64", 14), ("c64", 10), ("c128", 13), ("c128", 7)])
def test_graph_replay_equals_direct_launches(prec, K):
    """Steady Trotter steps run as replays of a captured CUDA graph unless the
    state is profiling; both give the same bits."""
    J = W.star_dipolar(14, 5)
    out = []
    for profile in (False, True):
        s = spinrp.System(J, spinrp.DIPOLAR)
        s.set_tile(prec, K)
        st = spinrp.State(s, prec, series_cap=60)
        st.profile(profile)
        st.init_random_phase(3)
        st.evolve(0.02, 40)
        st.evolve(0.02, 19)
        out.append((st.polarization(), st.amplitudes()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_deterministic_series():
    J = W.star_dipolar(16, 2)
    out = [_gpu(J, spinrp.DIPOLAR, 4, 0.02, 30, "c64")[0] for _ in range(2)]
    assert np.array_equal(out[0], out[1])


def test_errors_are_reported():
    s = spinrp.System(W.ladder(3), spinrp.XY)
    st = spinrp.State(s, "c64", series_cap=3)
    with pytest.raises(spinrp.SpinrpError) as e:
        st.evolve(0.1, 1)
    assert e.value.code == spinrp.ESTATE
    st.init_random_phase(1)
    with pytest.raises(spinrp.SpinrpError) as e:
        st.evolve(0.1, 5)
    assert e.value.code == spinrp.EINVAL
    with pytest.raises(spinrp.SpinrpError) as e:
        st.evolve(0.1, 1, order=4)
    assert e.value.code == spinrp.EUNSUPPORTED
    with pytest.raises(spinrp.SpinrpError) as e:
        st.polarization(2)  # all-site readout not enabled
    assert e.value.code == spinrp.ESTATE
    with pytest.raises(spinrp.SpinrpError) as e:
        st.polarization(7)
    assert e.value.code == spinrp.EINVAL
    with pytest.raises(spinrp.SpinrpError):
        st.evolve(float("nan"), 1)
    st.evolve(0.1, 2)
    assert st.series_length() == 3


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------
def test_ladder_m14_fp64_and_fp32():
    """2x7 XY ladder (leg 1, rung 0.5), dt 0.05, 400 steps."""
    job = W.ladder_m14()
    Pw, Nw, _ = _oracle(job.J, job.htype, job.seed, job.dt, job.steps)
    for prec in ("c128", "c64"):
        Pg, Ng, _ = _gpu(job.J, job.htype, job.seed, job.dt, job.steps, prec)
        assert Pg.shape == Pw.shape
        assert np.max(np.abs(Pg - Pw)) <= TOL_P[prec], prec
    # smaller tiles: several sweeps per step, same operator
    Pg, _, _ = _gpu(job.J, job.htype, job.seed, job.dt, job.steps, "c128", K=8)
    assert np.max(np.abs(Pg - Pw)) <= 1e-10


def test_star_m20_fp64_and_fp32():
    """Dipolar star M=20 (19 satellites, rms 1), dt 0.02, 1000 steps."""
    job = W.star_m20()
    Pw, Nw, psi_w = _oracle(job.J, job.htype, job.seed, job.dt, job.steps)
    idx = np.random.default_rng(0).integers(0, 1 << 20, size=4096)
    for prec in ("c128", "c64"):
        Pg, Ng, st = _gpu(job.J, job.htype, job.seed, job.dt, job.steps, prec)
        assert np.max(np.abs(Pg - Pw)) <= TOL_P[prec], prec
        assert np.max(np.abs(Ng - 1.0)) <= (1e-10 if prec == "c128" else 1e-4)
        if prec == "c128":
            assert np.max(np.abs(st.read(idx) - psi_w[idx])) < 1e-10


@pytest.mark.slow
def test_ladder_m30_sampled():
    """2x15 ladder at full size (2^30 amplitudes, 8 GiB c64 / 16 GiB c128), in
    the bench's launch configuration: five Trotter steps against the oracle
    (P and norm after every step, 2^14 sampled amplitudes at the end) for both
    precisions -- the first, three steady and the last step's sweeps -- then
    20 more steps as CUDA-graph replays, which must equal the same steps as
    direct launches bit for bit, and the invariants."""
    job = W.ladder_m30()
    steps = 5
    idx = np.random.default_rng(1).integers(0, 1 << 30, size=1 << 14)
    Pw, Nw, psi_w = _oracle(job.J, job.htype, job.seed, job.dt, steps)
    ref = psi_w[idx].copy()
    del psi_w
    for prec in ("c64", "c128"):
        st = spinrp.State(spinrp.System(job.J, job.htype), prec, series_cap=64)
        st.init_random_phase(job.seed)
        st.evolve(job.dt, steps)
        got = st.read(idx)
        Pg, Ng = st.polarization(), st.norm_series()
        assert np.max(np.abs(Pg - Pw)) <= TOL_P[prec], prec
        assert np.max(np.abs(Ng - Nw)) <= (1e-12 if prec == "c128" else 1e-6), prec
        # FP32: ~86 roundings per amplitude and step, max over 2^14 samples
        tol = 1e-12 if prec == "c128" else 1e-5 * 2.0 ** -14.5
        assert np.max(np.abs(got - ref)) < tol, prec
        # 20 steady steps replayed from a graph against the same steps launched
        # directly (profiling turns graphs off) on a copy of the state
        amp_idx = np.random.default_rng(2).integers(0, 1 << 30, size=1 << 12)
        st2 = spinrp.State(spinrp.System(job.J, job.htype), prec, series_cap=64)
        st2.init_random_phase(job.seed)
        st2.evolve(job.dt, steps)
        st.evolve(job.dt, 20)
        st2.profile(True)
        st2.evolve(job.dt, 20)
        st2.profile(False)
        assert np.array_equal(st.polarization(), st2.polarization()), prec
        assert np.array_equal(st.read(amp_idx), st2.read(amp_idx)), prec
        st2.close()
        N = st.norm_series()
        assert np.max(np.abs(N - 1.0)) < (1e-10 if prec == "c128" else 1e-5)
        P = st.polarization()
        assert np.all(np.abs(P) <= 1.0 + 1e-6)
        # total-S^z sector weights: binomial at t = 0, conserved by the flip-flops
        n = st.sector_norms()
        want = np.array([0.0] + [math.comb(29, k - 1) / 2.0 ** 29 for k in range(1, 31)])
        assert np.max(np.abs(n - want)) < (1e-12 if prec == "c128" else 2e-5), prec
        st.close()


@pytest.mark.slow
def test_fp32_against_fp64_over_200_steps_m30():
    """The bench's workload (2x15 ladder, 2^30 amplitudes, dt 0.05, 200
    steps): P(t) of the FP32 path against the FP64 path (held to 1e-10 of the
    oracle over its first steps above) at every one of the 201 entries."""
    job = W.ladder_m30()
    P = {}
    for prec in ("c64", "c128"):
        st = spinrp.State(spinrp.System(job.J, job.htype), prec, series_cap=job.steps + 1)
        st.init_random_phase(job.seed).evolve(job.dt, job.steps)
        P[prec] = st.polarization()
        st.close()
    assert len(P["c64"]) == job.steps + 1
    err = float(np.max(np.abs(P["c64"] - P["c128"])))
    print(f"max |P_fp32 - P_fp64| over {job.steps} steps, M = 30: {err:.3e}")
    assert err <= 1e-5


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_library_built_systems_match_oracle(prec):
    """Systems from spinrp_ladder_create / spinrp_star_dipolar_create evolve
    as the oracle does with the couplings the library reports."""
    for sysm, dt in ((spinrp.System.ladder(6, 1.0, 0.3), 0.05), (spinrp.System.star_dipolar(12, 9), 0.02)):
        a, b = sysm.couplings()
        st = spinrp.State(sysm, prec, series_cap=31)
        st.init_random_phase(4).evolve(dt, 30)
        M = sysm.M
        psi = oracle.init_random_phase(M, 4)
        P, _ = oracle.evolve(psi, a, b, dt, 30)
        tol = 1e-10 if prec == "c128" else 1e-4
        assert np.max(np.abs(st.polarization()[1:] - P)) <= tol
        st.close()


def test_largest_state_m34():
    """2x17 ladder at the largest supported size, 2^34 complex64 amplitudes
    (128 GiB; offsets beyond 32 bits, 2^21 blocks per sweep): the initial
    amplitudes at sampled indices against the oracle's phase draw, then two
    steps forward and two back return every sampled amplitude to its start
    (the step is a palindrome, so U(-dt) U(dt) = 1), with the norm kept."""
    M, seed = 34, 11
    sysm = spinrp.System.ladder(17, 1.0, 0.5)
    st = spinrp.State(sysm, "c64", series_cap=8)
    st.init_random_phase(seed)
    rng = np.random.default_rng(34)
    idx = np.concatenate([rng.integers(0, 1 << M, size=2048), [0, 1, (1 << M) - 1, (1 << M) - 2, (1 << 33) + 1]])
    got0 = st.read(idx)
    amp = 2.0 ** (-(M - 1) / 2)
    want = np.array([amp * np.exp(2j * np.pi * oracle.phase_uniform(seed, int(x) >> 1)) if x & 1 else 0.0
                     for x in idx])
    assert np.max(np.abs(got0 - want)) < 2e-7 * amp
    st.evolve(0.05, 2).evolve(-0.05, 2)
    got1 = st.read(idx)
    assert np.max(np.abs(got1 - got0)) < 1e-5 * amp
    N = st.norm_series()
    assert np.max(np.abs(N - 1.0)) < 1e-5
    assert abs(st.polarization()[-1] - 1.0) < 1e-5
    st.close()


def test_autotune_picks_a_measured_candidate():
    """The autotuner times each (K, rb) candidate, keeps the fastest and sets
    it on the system; the tuned system still evolves as the oracle does."""
    J, ht = W.ladder(8, 1.0, 0.5), spinrp.XY
    s = spinrp.System(J, ht)
    cands = [(11, 5), (12, 5), (12, 6), (13, 6)]
    r = spinrp.autotune(s, "c64", candidates=cands, probe_steps=3, dt=0.05)
    assert set(r["ms_per_step"]) == set(cands)
    assert (r["K"], r["rb"]) == min(r["ms_per_step"], key=r["ms_per_step"].get)
    assert s.plan_info("c64")["K"] == r["K"]
    st = spinrp.State(s, "c64", series_cap=21)
    st.init_random_phase(3).evolve(0.05, 20)
    Pw, _, _ = _oracle(J, ht, 3, 0.05, 20)
    assert np.max(np.abs(st.polarization() - Pw)) <= TOL_P["c64"]
    st.close()
    r = spinrp.autotune(s, "c128", candidates=[8, 12], probe_steps=2, dt=0.05)
    assert r["K"] in (8, 12) and s.plan_info("c128")["K"] == r["K"]


def test_fp32_error_over_200_steps_m26():
    """The FP32 path's P(t) against the FP64 path (itself held to 1e-10 of the
    oracle) over the full 200 steps of the ladder workload's time span, on the
    2x13 ladder (2^26 amplitudes): the FP32 bar holds with a wide margin."""
    J = W.ladder(13, 1.0, 0.5)
    seed, dt, steps = 1, 0.05, 200
    P = {}
    for prec in ("c64", "c128"):
        st = spinrp.State(spinrp.System(J, spinrp.XY), prec, series_cap=steps + 1)
        st.init_random_phase(seed).evolve(dt, steps)
        P[prec] = st.polarization()
        st.close()
    err = float(np.max(np.abs(P["c64"] - P["c128"])))
    print(f"max |P_fp32 - P_fp64| over {steps} steps, M = 26: {err:.3e}")
    assert err <= 1e-5


# ---------------------------------------------------------------------------
# oriented storage (complex64 states of bipartite systems)
def _xy_ising_ladder(L):
    J = W.ladder(L, 1.0, 0.6)
    a = 0.7 * W.ladder(L, 1.0, 0.4) + 0.2 * np.eye(2 * L)[::-1]
    a = 0.5 * (a + a.T)
    np.fill_diagonal(a, 0.0)
    return J, a


def test_orientation_is_used_where_it_applies():
    """With orientation requested, ladders and chains (bipartite flip-flop
    graphs) get oriented complex64 states in the register-blocked kernel;
    stars, complex128 states and systems left at the default (plain storage)
    do not."""
    lad = spinrp.System(W.ladder(8, 1.0, 0.5), spinrp.XY)
    lad.set_tile("c64", 13)
    assert spinrp.State(lad, "c64", series_cap=2).orientation() == 0  # default: plain
    lad.set_orientation(1)
    st = spinrp.State(lad, "c64", series_cap=2)
    black = st.orientation()
    assert black != 0
    # every bond (1-based pairs) joins the two colours
    for i, j in lad.bonds():
        assert ((black >> (i - 1)) & 1) != ((black >> (j - 1)) & 1)
    st.close()
    assert spinrp.State(lad, "c128", series_cap=2).orientation() == 0
    star = spinrp.System(W.star_dipolar(16, 8), spinrp.DIPOLAR)
    star.set_tile("c64", 13)
    star.set_orientation(1)
    assert spinrp.State(star, "c64", series_cap=2).orientation() == 0


@pytest.mark.parametrize("rb,K", [(5, 11), (5, 12), (6, 12), (6, 13), (6, 14)])
@pytest.mark.parametrize("kind", ["ladder18", "chain19", "xy_ising_ladder16"])
def test_oriented_and_plain_storage_match_oracle(kind, rb, K):
    """The oriented and the plain register-blocked programs on the same
    bipartite system, both against the oracle (P every step, every
    amplitude); with S^zS^z terms the oriented diagonal phase is exercised."""
    a = None
    if kind == "ladder18":
        J, ht = W.ladder(9, 1.0, 0.5), spinrp.XY
    elif kind == "chain19":
        J, ht = W.chain(19, 0.8), spinrp.XY
    else:
        J, a = _xy_ising_ladder(8)
        ht = spinrp.GENERIC
    seed, dt, steps = 21, 0.05, 6
    Pw, Nw, psi_w = _oracle(J, ht, seed, dt, steps, a)
    res = {}
    for mode in (1, 0):
        s = spinrp.System(J, ht, a)
        s.set_tile("c64", K)
        s.set_regbits(rb)
        s.set_orientation(mode)
        st = spinrp.State(s, "c64", series_cap=steps + 1)
        assert (st.orientation() != 0) == (mode == 1), (kind, mode)
        st.init_random_phase(seed).evolve(dt, steps)
        P = st.polarization()
        assert np.max(np.abs(P - Pw)) <= 1e-5, (kind, mode)
        assert np.max(np.abs(st.norm_series() - Nw)) <= 1e-5, (kind, mode)
        amp = st.amplitudes()
        assert np.max(np.abs(amp - psi_w)) <= 2e-6 * 2.0 ** (-(st.M - 1) / 2) * 64, (kind, mode)
        res[mode] = P
        st.close()
    assert np.max(np.abs(res[1] - res[0])) <= 1e-6


def test_oriented_buffer_layout():
    """An oriented state's raw buffer holds amplitude x at its physical index
    as (Re, Im) when x has an even number of first-colour spins up and as
    (Im, Re) when odd; spinrp_state_read undoes the swap."""
    J = W.ladder(7, 1.0, 0.5)
    s = spinrp.System(J, spinrp.XY)
    s.set_tile("c64", 12)
    s.set_orientation(1)
    st = spinrp.State(s, "c64", series_cap=4)  # amplitude buffer from PyTorch
    st.init_random_phase(9).evolve(0.05, 3)
    black, lay = st.orientation(), st.layout()
    assert black != 0
    M = st.M
    idx = np.arange(1 << M)
    want = st.read(idx)
    psi_buf = st._bufs[0]
    assert psi_buf.data_ptr() == st.device_ptr()
    w = psi_buf.cpu().numpy().view(np.float32).reshape(-1, 2)
    phys = np.zeros_like(idx)
    for q in range(M):
        phys |= ((idx >> q) & 1) << lay[q]
    odd = np.array([bin(int(x) & black).count("1") & 1 for x in idx], dtype=bool)
    re = np.where(odd, w[phys, 1], w[phys, 0])
    im = np.where(odd, w[phys, 0], w[phys, 1])
    assert np.max(np.abs((re + 1j * im) - want)) < 1e-7
    assert np.any(odd) and np.any(~odd)
    st.close()
