"""Total-S^z sector weights of the device state against the oracle, and their
conservation (every Hamiltonian family here commutes with the total S^z) at
sizes the oracle cannot follow step by step."""
from math import comb

import numpy as np
import pytest

import oracle
from paper_0710_3747_gb300 import spinrp
from paper_0710_3747_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _binomial(M):
    """Sector weights of the random-phase (or product) state: spin 1 up, each
    of the other M - 1 spins up with weight 1/2."""
    return np.array([0.0] + [comb(M - 1, k - 1) / 2.0 ** (M - 1) for k in range(1, M + 1)])


def _system(kind):
    if kind == "ladder12":
        return W.ladder(6, 1.0, 0.5), W.XY, None, 0.05
    if kind == "star11":
        return W.star_dipolar(11, 4), W.DIPOLAR, None, 0.02
    if kind == "m2":
        return W.chain(2, 1.0), W.XY, None, 0.1
    rng = np.random.default_rng(8)
    J = rng.normal(size=(10, 10)); J = J + J.T; np.fill_diagonal(J, 0)
    A = rng.normal(size=(10, 10)); A = A + A.T; np.fill_diagonal(A, 0)
    return J, W.GENERIC, A, 0.03


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("kind", ["ladder12", "star11", "generic10", "m2"])
def test_sector_norms_match_oracle(kind, prec):
    spinrp.lib()
    J, ht, A, dt = _system(kind)
    M, seed, steps = J.shape[0], 13, 30
    st = spinrp.State(spinrp.System(J, ht, A), prec, series_cap=steps + 1)
    st.init_random_phase(seed)
    n0 = st.sector_norms()
    tol = 1e-13 if prec == "c128" else 1e-6
    assert n0.shape == (M + 1,)
    np.testing.assert_allclose(n0, _binomial(M), atol=tol)
    st.evolve(dt, steps)
    _, _, psi = oracle.run(J, ht, seed, dt, steps, a_generic=A)
    want = oracle.sector_norms(psi)
    got = st.sector_norms()
    np.testing.assert_allclose(got, want, atol=1e-12 if prec == "c128" else 2e-6)
    assert np.array_equal(st.sector_norms(), got)  # fixed summation order
    st.close()


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_sector_conservation_large(prec):
    """2x13 ladder (2^26 amplitudes) and a 22-spin dipolar star: the sector
    weights start binomial and stay put under the evolution."""
    spinrp.lib()
    for J, ht, dt in ((W.ladder(13, 1.0, 0.5), W.XY, 0.05), (W.star_dipolar(22, 3), W.DIPOLAR, 0.02)):
        M = J.shape[0]
        st = spinrp.State(spinrp.System(J, ht), prec, series_cap=32)
        st.init_random_phase(5)
        n0 = st.sector_norms()
        np.testing.assert_allclose(n0, _binomial(M), atol=1e-12 if prec == "c128" else 1e-6)
        st.evolve(dt, 20)
        drift = float(np.max(np.abs(st.sector_norms() - n0)))
        assert drift <= (1e-12 if prec == "c128" else 2e-5), drift
        st.close()


def test_sector_norms_product_state_and_errors():
    spinrp.lib()
    J, ht, _, dt = _system("ladder12")
    st = spinrp.State(spinrp.System(J, ht), "c128", series_cap=8)
    with pytest.raises(spinrp.SpinrpError):
        st.sector_norms()  # not initialized
    st.init_product_phase(3)
    np.testing.assert_allclose(st.sector_norms(), _binomial(J.shape[0]), atol=1e-13)
    st.close()
