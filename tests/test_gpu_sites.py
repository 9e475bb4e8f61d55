"""All-site readout P_{q1}(t), q = 1..M (paper's Eq. 2, m = 1) against the
oracle, on both sweep kernels, through graph replay, init and load."""
import numpy as np
import pytest

import oracle
from paper_0710_3747_gb300 import spinrp
from paper_0710_3747_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _system(kind):
    if kind == "ladder12":
        return W.ladder(6, 1.0, 0.5), W.XY, None, 0.05
    if kind == "star11":
        return W.star_dipolar(11, 4), W.DIPOLAR, None, 0.02
    rng = np.random.default_rng(8)
    J = rng.normal(size=(10, 10)); J = J + J.T; np.fill_diagonal(J, 0)
    A = rng.normal(size=(10, 10)); A = A + A.T; np.fill_diagonal(A, 0)
    return J, W.GENERIC, A, 0.03


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("kind", ["ladder12", "star11", "generic10"])
@pytest.mark.parametrize("K", [7, 0])  # plain kernel with narrow tiles; default plan
def test_all_sites_match_oracle(kind, prec, K):
    spinrp.lib()
    J, ht, A, dt = _system(kind)
    M, seed, steps = J.shape[0], 21, 40  # > 16 steady steps: graph replay included
    sysm = spinrp.System(J, ht, A)
    if K:
        sysm.set_tile(prec, K)
    st = spinrp.State(sysm, prec, series_cap=steps + 1).set_sites(True)
    st.init_random_phase(seed).evolve(dt, 17).evolve(dt, steps - 17)
    got = st.site_series()
    P, nrm, _ = oracle.run_all_sites(J, ht, seed, dt, steps, a_generic=A)
    tol = 1e-10 if prec == "c128" else 1e-4
    assert got.shape == (steps + 1, M)
    assert np.max(np.abs(got - P)) <= tol
    # spin 1 of the all-site series and the main series agree; the sum rule
    assert np.max(np.abs(got[:, 0] - st.polarization(1))) <= (1e-12 if prec == "c128" else 1e-6)
    assert np.max(np.abs(got.sum(axis=1) - 1.0)) <= (1e-10 if prec == "c128" else 2e-5)
    for q in (2, M):
        assert np.array_equal(st.polarization(q), got[:, q - 1])
    st.close()


def test_all_sites_product_state_and_load():
    spinrp.lib()
    J, ht, _, dt = _system("ladder12")
    M = J.shape[0]
    st = spinrp.State(spinrp.System(J, ht), "c128", series_cap=32).set_sites(True)
    st.init_product_phase(5).evolve(dt, 20)
    P, _, _ = oracle.run_all_sites(J, ht, 5, dt, 20, product=True)
    assert np.max(np.abs(st.site_series() - P)) <= 1e-10
    # load: an arbitrary state's P(0) for every site
    rng = np.random.default_rng(2)
    psi = rng.normal(size=1 << M) + 1j * rng.normal(size=1 << M)
    st.load(psi)
    x = np.arange(1 << M)
    w = np.abs(psi) ** 2
    want = [np.sum(w * np.where((x >> q) & 1, 1.0, -1.0)) / w.sum() for q in range(M)]
    np.testing.assert_allclose(st.site_series()[0], want, atol=1e-12)
    st.close()


def test_all_sites_large_register_blocked():
    """2x13 ladder (2^26 amplitudes, register-blocked complex64 sweeps): sum
    rule and spin 1 against the main series; a sampled site against the
    weight of a few hundred read-back amplitudes is not meaningful, so the
    check is on invariants."""
    spinrp.lib()
    J = W.ladder(13, 1.0, 0.5)
    st = spinrp.State(spinrp.System(J, W.XY), "c64", series_cap=24).set_sites(True)
    st.init_random_phase(3).evolve(0.05, 20)
    got = st.site_series()
    assert np.max(np.abs(got.sum(axis=1) - 1.0)) < 1e-4
    assert np.max(np.abs(got[:, 0] - st.polarization(1))) < 1e-6
    assert np.max(np.abs(got[0, 1:])) < 1e-6
    # at t = 1 the polarization has spread to the neighbours of spin 1 only
    assert got[-1, 1] > 0.05 and abs(got[-1, 12]) < 1e-3
    st.close()


def test_sites_off_and_errors():
    spinrp.lib()
    J, ht, _, dt = _system("star11")
    st = spinrp.State(spinrp.System(J, ht), "c64", series_cap=8)
    st.init_random_phase(1).evolve(dt, 3)
    with pytest.raises(spinrp.SpinrpError):
        st.polarization(2)
    with pytest.raises(spinrp.SpinrpError):
        st.site_series()
    with pytest.raises(spinrp.SpinrpError):
        st.polarization(12)
    # enabling takes effect at the next init; P_1 is unchanged by the mode
    p_off = st.polarization(1)
    st.set_sites(True).init_random_phase(1).evolve(dt, 3)
    assert np.array_equal(st.polarization(1), p_off)
    assert st.site_series().shape == (4, 11)
    st.set_sites(False).init_random_phase(1).evolve(dt, 3)
    with pytest.raises(spinrp.SpinrpError):
        st.polarization(2)
    st.close()


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_general_initial_spin_by_relabelling(prec):
    """P_{nm}(t) for an initially polarized spin m != 1 (the paper's Eq. 2 in
    general): relabel spin m to spin 1 (spinrp.polarized_at), read every site
    out, map back; against the oracle on the relabelled system (same seed,
    the parity bar) and against exact diagonalization of the original system's
    2^{-M} Tr[sigma^z_n(t) sigma^z_m] (the random-state scale)."""
    from oracle import ed
    spinrp.lib()
    J, m, dt, steps = W.chain(10, 0.9), 4, 0.05, 60
    Jp, _, order = spinrp.polarized_at(J, m)
    assert order[0] == m - 1 and sorted(order) == list(range(10))
    st = spinrp.State(spinrp.System(Jp, W.XY), prec, series_cap=steps + 1).set_sites(True)
    st.init_random_phase(9).evolve(dt, steps)
    got = st.site_series()                                   # columns: relabelled spins
    P, _, _ = oracle.run_all_sites(Jp, W.XY, 9, dt, steps)
    assert np.max(np.abs(got - P)) <= (1e-10 if prec == "c128" else 1e-4)
    a, b = oracle.couplings(J, oracle.XY)
    times = dt * np.arange(steps + 1)
    for n in (m, m + 1, 1, 10):
        ens = ed.ensemble_cross_polarization(a, b, times, n, m=m)
        col = int(np.flatnonzero(order == n - 1)[0])
        assert np.max(np.abs(got[:, col] - ens)) < 6 * 2.0 ** (-9 / 2) + 1e-3, n
    st.close()
