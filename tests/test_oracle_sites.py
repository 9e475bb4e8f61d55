"""Pins for the oracle's all-site readout P_{n1}(t), n = 1..M (the paper's
local polarization P_{n'n} of Eq. 2 with the initially polarized spin n = 1):

  * exact diagonalization of P_{n1}^ens = 2^{-M} Tr[sigma^z_n(t) sigma^z_1]
    against the free-fermion closed form |[e^{-iht}]_{n1}|^2 of the open XY
    chain, site by site (pins the cross-correlation formula independently);
  * the oracle's Trotter evolution, site by site, against exact e^{-iHt} psi0
    with the second-order rate (halving dt divides the error by 4);
  * total magnetization is conserved by every Hamiltonian of the paper, and
    the entangled random-phase state has <sigma^z_n> = 0 exactly for n != 1,
    so sum_n P_{n1}(t) = 1 at every step;
  * one random state on a free 16-spin chain tracks every site's closed form
    within the self-averaging scale.
"""
import numpy as np
import pytest

import oracle
from oracle import ed
from paper_0710_3747_gb300 import workloads as W


def _hopping(J):
    return 0.5 * J  # b (S^xS^x + S^yS^y) = (b/2)(S^+S^- + h.c.): hopping b/2


@pytest.mark.parametrize("L", [4, 7])
def test_ed_cross_polarization_matches_free_fermions(L):
    J = W.chain(L, 0.8)
    a, b = oracle.couplings(J, oracle.XY)
    t = np.linspace(0.0, 9.0, 19)
    ff = ed.hopping_pn1(_hopping(J), t)
    for n in range(1, L + 1):
        np.testing.assert_allclose(ed.ensemble_cross_polarization(a, b, t, n), ff[:, n - 1], atol=1e-12)


@pytest.mark.parametrize("kind", ["ladder", "star"])
def test_all_sites_trotter_second_order(kind):
    if kind == "ladder":
        J, ht = W.ladder(4, 1.0, 0.5), oracle.XY
    else:
        J, ht = W.star_dipolar(7, 3), oracle.DIPOLAR
    a, b = oracle.couplings(J, ht)
    M, T = a.shape[0], 1.2
    psi0 = oracle.init_random_phase(M, 5)
    ex = ed.ExactSystem(a, b)
    x = np.arange(1 << M)
    w = np.abs(ex.evolve(psi0, T)) ** 2
    exact = np.array([np.sum(w * np.where((x >> q) & 1, 1.0, -1.0)) for q in range(M)]) / w.sum()
    errs = []
    for steps in (12, 24):
        psi = psi0.copy()
        P, _ = oracle.evolve_all_sites(psi, a, b, T / steps, steps)
        errs.append(np.max(np.abs(P[-1] - exact)))
    assert errs[1] < 1e-2
    assert 3.0 < errs[0] / errs[1] < 5.0


@pytest.mark.parametrize("kind", ["ladder", "star", "generic"])
def test_total_magnetization_sum_rule(kind):
    if kind == "ladder":
        J, ht, ag = W.ladder(5, 1.0, 0.3), oracle.XY, None
    elif kind == "star":
        J, ht, ag = W.star_dipolar(9, 1), oracle.DIPOLAR, None
    else:
        rng = np.random.default_rng(3)
        J = rng.normal(size=(8, 8)); J = J + J.T; np.fill_diagonal(J, 0)
        ag = rng.normal(size=(8, 8)); ag = ag + ag.T; np.fill_diagonal(ag, 0)
        ht = oracle.GENERIC
    P, nrm, _ = oracle.run_all_sites(J, ht, seed=11, dt=0.05, steps=30, a_generic=ag)
    np.testing.assert_allclose(P[0, 1:], 0.0, atol=1e-13)
    assert P[0, 0] == pytest.approx(1.0, abs=1e-14)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-12)


def test_random_state_tracks_free_chain_every_site():
    L, dt, steps = 16, 0.05, 40
    J = W.chain(L, 1.0)
    P, _, _ = oracle.run_all_sites(J, oracle.XY, seed=23, dt=dt, steps=steps, threads=4)
    ff = ed.hopping_pn1(_hopping(J), dt * np.arange(steps + 1))
    assert np.max(np.abs(P - ff)) < 6 * 2.0 ** (-(L - 1) / 2) + 1e-3


def test_relabelled_initial_spin_matches_ensemble():
    """General initially polarized spin m: relabelling m to spin 1
    (spinrp.polarized_at, pure host arithmetic) and running the oracle's
    all-site evolution gives P_{nm}(t) of the original system; compared with
    exact diagonalization of 2^{-M} Tr[sigma^z_n(t) sigma^z_m], averaged over
    a few seeds so the random-state error (~2^{-(M-1)/2} per seed) shrinks."""
    from paper_0710_3747_gb300 import spinrp
    J, m, dt, steps = W.ladder(4, 1.0, 0.6), 6, 0.05, 40
    M = J.shape[0]
    Jp, _, order = spinrp.polarized_at(J, m)
    a, b = oracle.couplings(J, oracle.XY)
    times = dt * np.arange(steps + 1)
    runs = [oracle.run_all_sites(Jp, oracle.XY, s, dt, steps)[0] for s in range(1, 9)]
    mean = np.mean(runs, axis=0)
    for n in range(1, M + 1):
        ens = ed.ensemble_cross_polarization(a, b, times, n, m=m)
        col = int(np.flatnonzero(order == n - 1)[0])
        assert np.max(np.abs(mean[:, col] - ens)) < 4 * 2.0 ** (-(M - 1) / 2) / np.sqrt(8) + 5e-3, n
    # and the relabelling is a permutation: the inverse restores J
    inv = np.argsort(order)
    np.testing.assert_array_equal(Jp[np.ix_(inv, inv)], J)
