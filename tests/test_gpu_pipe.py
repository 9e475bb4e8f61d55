"""GPU: pipelined sweeps -- one persistent block per SM, a producer warpgroup
gathering tiles into three shared-memory buffers and writing them back, two
compute warpgroups applying the gates -- against the FP64 oracle and, bit for
bit, against the one-tile-per-block sweep.

The pipelined sweep takes complex64 plans with 13-spin tiles and six register
bits, plainly stored, with at least four tiles per SM (M >= 23 on GB300's 152
SMs).  The systems below force that plan (set_tile 13, set_regbits 6).
Tolerances as in test_gpu_parity: |dP| <= 1e-5 at every step (the FP32 bar is
1e-4), amplitudes within 1.3e-4 of the typical amplitude 2^{-(M-1)/2}.
"""
import os

import numpy as np
import pytest

import oracle
from paper_0710_3747_gb300 import spinrp
from paper_0710_3747_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    spinrp.lib()


class _DeviceBuffer:
    """A state's amplitude buffer (2^M complex64) as a CUDA array of floats."""

    def __init__(self, st):
        self.__cuda_array_interface__ = {
            "shape": (2 << st.M,),
            "typestr": "<f4",
            "data": (st.device_ptr(), False),
            "version": 3,
        }


def _raw(st):
    import torch

    torch.cuda.synchronize()
    return torch.as_tensor(_DeviceBuffer(st), device="cuda").clone()


def _xy_ising_ladder(L):
    J = W.ladder(L, 1.0, 0.6)
    a = 0.7 * W.ladder(L, 1.0, 0.4) + 0.2 * np.eye(2 * L)[::-1]
    a = 0.5 * (a + a.T)
    np.fill_diagonal(a, 0.0)
    return J, a


def _system(kind, M):
    if kind == "ladder":
        assert M % 2 == 0
        return W.ladder(M // 2, 1.0, 0.5), spinrp.XY, None
    if kind == "chain":
        return W.chain(M, 0.8), spinrp.XY, None
    if kind == "xy_ising_ladder":
        J, a = _xy_ising_ladder(M // 2)
        return J, spinrp.GENERIC, a
    if kind == "star":
        return W.star_dipolar(M, 5), spinrp.DIPOLAR, None
    raise ValueError(kind)


def _state(J, ht, a, steps, pipe, K=13, rb=6):
    s = spinrp.System(J, ht, a)
    s.set_tile("c64", K)
    s.set_regbits(rb)
    st = spinrp.State(s, "c64", series_cap=steps + 1)
    st.set_pipeline(pipe)
    return st


def test_pipeline_is_used_where_it_applies():
    """Pipelined by default for a 2x12 ladder on 13-spin tiles with six
    register bits; not for complex128, other tile widths or register bits,
    oriented storage, or too few tiles per SM."""
    J = W.ladder(12, 1.0, 0.5)
    st = _state(J, spinrp.XY, None, 1, True)
    assert st.pipeline()
    st.set_pipeline(False)
    assert not st.pipeline()
    st.set_pipeline(True)
    assert st.pipeline()
    st.close()
    s = spinrp.System(J, spinrp.XY)
    s.set_tile("c128", 13)
    assert not spinrp.State(s, "c128", series_cap=2).pipeline()
    for K, rb in ((12, 6), (14, 6), (13, 5)):
        assert not _state(J, spinrp.XY, None, 1, True, K=K, rb=rb).pipeline(), (K, rb)
    s = spinrp.System(J, spinrp.XY)
    s.set_tile("c64", 13)
    s.set_regbits(6)
    s.set_orientation(1)
    o = spinrp.State(s, "c64", series_cap=2)
    assert o.orientation() != 0 and not o.pipeline()
    # 2x10 ladder: 128 tiles of 2^13, fewer than four per SM
    assert not _state(W.ladder(10, 1.0, 0.5), spinrp.XY, None, 1, True).pipeline()


@pytest.mark.parametrize(
    "kind,M,steps,chunks",
    [("ladder", 24, 20, (1, 19)), ("xy_ising_ladder", 24, 6, (2, 4)), ("star", 23, 3, (3,))],
)
def test_pipelined_sweeps_match_oracle(kind, M, steps, chunks):
    """P and the norm at every step and every amplitude at the end against the
    oracle; the ladder's 19-step call replays a captured graph of 16 steady
    steps, the other two run the diagonal phase inside the pipeline."""
    J, ht, a = _system(kind, M)
    seed, dt = 31 + M, 0.05
    Pw, Nw, psi_w = oracle.run(J, ht, seed, dt, steps, a_generic=a, threads=THREADS)
    st = _state(J, ht, a, steps, True)
    assert st.pipeline()
    st.init_random_phase(seed)
    for n in chunks:
        st.evolve(dt, n)
    P, N = st.polarization(), st.norm_series()
    assert P.shape == (steps + 1,)
    assert np.max(np.abs(P - Pw)) <= 1e-5, kind
    assert np.max(np.abs(N - Nw)) <= 1e-5, kind
    amp = st.amplitudes()
    assert np.max(np.abs(amp - psi_w)) <= 1.3e-4 * 2.0 ** (-(M - 1) / 2), kind
    st.close()


@pytest.mark.parametrize(
    "kind,M,steps,chunks",
    [
        ("ladder", 26, 20, (3, 17)),
        ("chain", 23, 5, (1, 4)),
        ("xy_ising_ladder", 24, 4, (4,)),
        ("star", 23, 2, (1, 1)),
    ],
)
def test_pipelined_and_block_sweeps_agree_bit_for_bit(kind, M, steps, chunks):
    """The same plan with the pipelined sweep and with one tile per block:
    identical P and norm series and identical raw amplitude buffers (8192
    tiles over the blocks at M = 26, 1024 at M = 23: blocks with unequal tile
    counts)."""
    J, ht, a = _system(kind, M)
    out = {}
    for pipe in (True, False):
        st = _state(J, ht, a, steps, pipe)
        assert st.pipeline() == pipe
        st.init_random_phase(77)
        for n in chunks:
            st.evolve(0.04, n)
        out[pipe] = (st.polarization(), st.norm_series(), _raw(st))
        st.close()
    import torch

    assert np.array_equal(out[True][0], out[False][0])
    assert np.array_equal(out[True][1], out[False][1])
    assert torch.equal(out[True][2], out[False][2])


def test_pipeline_waits_are_bounded():
    """A pipelined launch whose producer issues no copies: every wait gives
    up after its time limit, the call reports SPINRP_ETIMEOUT, the amplitudes
    and the series are untouched, the error word is cleared, and the state
    evolves on exactly as one that never ran the check."""
    J = W.ladder(12, 1.0, 0.5)
    st = _state(J, spinrp.XY, None, 5, True)
    st.init_random_phase(3).evolve(0.05, 2)
    before = _raw(st)
    n0 = len(st.polarization())
    rc, sec = st.pipeline_timeout_check()
    assert rc == spinrp.ETIMEOUT
    assert 1.5 <= sec <= 15.0, sec
    import torch

    assert torch.equal(_raw(st), before)
    assert len(st.polarization()) == n0
    st.evolve(0.05, 2)
    P = st.polarization()
    assert np.all(np.isfinite(P))
    ref = _state(J, spinrp.XY, None, 5, True)
    ref.init_random_phase(3).evolve(0.05, 2)
    ref.evolve(0.05, 2)
    assert np.array_equal(P, ref.polarization())
    assert torch.equal(_raw(st), _raw(ref))
    st.close()
    ref.close()
    # a state whose plan does not take the pipelined sweep
    small = _state(W.ladder(10, 1.0, 0.5), spinrp.XY, None, 1, True)
    rc, _ = small.pipeline_timeout_check()
    assert rc == spinrp.ESTATE


@pytest.mark.parametrize("kind,M", [("ladder", 24), ("xy_ising_ladder", 24)])
def test_pipelined_all_site_readout(kind, M):
    """All-site readout (P of every spin after every step) from the pipelined
    sweep: against the oracle's all-site series, and bit for bit against the
    one-tile-per-block readout (every site's series and the raw buffer)."""
    J, ht, a = _system(kind, M)
    seed, dt, steps = 17, 0.05, 6
    Pw, _, _ = oracle.run_all_sites(J, ht, seed, dt, steps, a_generic=a, threads=THREADS)
    out = {}
    for pipe in (True, False):
        st = _state(J, ht, a, steps, pipe).set_sites(True)
        assert st.pipeline() == pipe
        st.init_random_phase(seed)
        st.evolve(dt, 2).evolve(dt, 4)
        out[pipe] = (st.site_series(), st.polarization(1), _raw(st))
        st.close()
    got = out[True][0]
    assert got.shape == (steps + 1, M)
    assert np.max(np.abs(got - Pw)) <= 1e-5
    import torch

    assert np.array_equal(out[True][0], out[False][0])
    assert np.array_equal(out[True][1], out[False][1])
    assert torch.equal(out[True][2], out[False][2])
