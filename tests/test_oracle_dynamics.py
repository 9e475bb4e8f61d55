"""Pins for the oracle's Trotter evolution and polarization readout.

Each pin is fixed by the mathematics or the paper, not by the oracle itself:
  * M=2 closed form: one bond, spin 1 up: P(t) = (1 + cos b t)/2 for every
    seed and every S^zS^z coupling (the Trotter step is exact for one bond);
  * second order: against exact e^{-iHt} psi0 from dense exact diagonalization
    (a Kronecker-product construction of H), halving dt divides the error by 4;
  * time reversal: the step is a palindrome, so U(-dt) U(dt) = 1;
  * invariants: norm and every total-S^z sector norm are conserved;
  * ED against the free-fermion closed form of the open XY chain (pins the
    J/2 hopping and S = sigma/2 conventions of the reference itself);
  * short-time expansion P^ens(t) = 1 - (t^2/4) sum_j b_1j^2 + O(t^4);
  * self-averaging (paper: "Ensemble vs. pure entangled state", Chebyshev
    bound with max p_i = 2^{-(M-1)}): the spread of P over seeds is below
    2 * 2^{-(M-1)/2} and shrinks by about 2 when M grows by 2; one random
    state tracks the ensemble within a few times that spread.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import ed
from paper_0710_3747_gb300 import workloads as W


def _system(kind, M, seed=0):
    if kind == "ladder":
        return oracle.couplings(W.ladder(M // 2, 1.0, 0.5), oracle.XY)
    if kind == "star":
        return oracle.couplings(W.star_dipolar(M, seed), oracle.DIPOLAR)
    if kind == "isotropic":
        return oracle.couplings(W.star_gaussian(M, seed), oracle.ISOTROPIC)
    if kind == "generic":
        rng = np.random.default_rng(seed)
        A = rng.normal(size=(M, M)); A = A + A.T; np.fill_diagonal(A, 0)
        return oracle.couplings(W.star_gaussian(M, seed + 1), oracle.GENERIC, A)
    if kind == "ising":
        return oracle.couplings(W.star_gaussian(M, seed), oracle.ISING)
    raise ValueError(kind)


@pytest.mark.parametrize("a12", [0.0, 0.7, -2.4])
@pytest.mark.parametrize("seed", [1, 99])
def test_two_spin_closed_form(a12, seed):
    b12 = 1.3
    a = np.array([[0, a12], [a12, 0]], float)
    b = np.array([[0, b12], [b12, 0]], float)
    psi = oracle.init_random_phase(2, seed)
    dt, steps = 0.11, 60
    P, nrm = oracle.evolve(psi, a, b, dt, steps)
    t = dt * np.arange(1, steps + 1)
    np.testing.assert_allclose(P, 0.5 * (1 + np.cos(b12 * t)), atol=1e-13)
    np.testing.assert_allclose(nrm, 1.0, atol=1e-14)


@pytest.mark.parametrize("kind", ["ladder", "star", "isotropic", "generic", "ising"])
def test_second_order_convergence_to_exact(kind):
    M = 6
    a, b = _system(kind, M, seed=3)
    ex = ed.ExactSystem(a, b)
    psi0 = oracle.init_random_phase(M, 5)
    T = 1.2
    errs = []
    for n in (12, 24, 48):
        psi = psi0.copy()
        oracle.evolve(psi, a, b, T / n, n)
        errs.append(np.linalg.norm(psi - ex.evolve(psi0, T)))
    if kind == "ising":  # all factors commute: the product is exact
        assert max(errs) < 1e-13
        return
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, (errs, r1, r2)
    assert errs[2] < 2e-3


def test_polarization_tracks_exact_state():
    # P read from the Trotter state converges to P of the exact state as dt^2
    M = 8
    a, b = _system("star", M, seed=11)
    ex = ed.ExactSystem(a, b)
    psi0 = oracle.init_random_phase(M, 2)
    T = 2.0
    dev = []
    for n in (40, 80):
        psi = psi0.copy()
        P, _ = oracle.evolve(psi, a, b, T / n, n)
        dev.append(abs(P[-1] - oracle.polarization(ex.evolve(psi0, T))))
    assert dev[1] < 1e-3 and dev[0] / max(dev[1], 1e-300) > 3.0


@pytest.mark.parametrize("kind", ["ladder", "star", "generic"])
def test_time_reversal(kind):
    M = 9
    a, b = _system(kind, M, seed=4)
    psi0 = oracle.init_random_phase(M, 8)
    psi = psi0.copy()
    oracle.evolve(psi, a, b, 0.07, 25)
    assert np.linalg.norm(psi - psi0) > 1e-2
    oracle.evolve(psi, a, b, -0.07, 25)
    assert np.linalg.norm(psi - psi0) < 1e-12


def test_reversed_bond_order_is_not_the_same_product():
    # a fixed order matters at O(dt^2) only: two orders agree to O(dt^2)
    M = 7
    a, b = _system("star", M, seed=6)
    psi0 = oracle.init_random_phase(M, 1)
    bonds = oracle.canonical_bonds(b)
    out = []
    for order in (bonds, bonds[::-1]):
        psi = psi0.copy()
        P, _ = oracle.evolve(psi, a, b, 0.01, 100, bonds=order)
        out.append(P)
    d = np.max(np.abs(out[0] - out[1]))
    assert 1e-12 < d < 1e-4


@pytest.mark.parametrize("kind", ["ladder", "star", "generic"])
def test_norm_and_sector_conservation(kind):
    M = 10
    a, b = _system(kind, M, seed=2)
    psi = oracle.init_random_phase(M, 31)
    n0 = oracle.sector_norms(psi)
    P, nrm = oracle.evolve(psi, a, b, 0.05, 40)
    np.testing.assert_allclose(nrm, 1.0, atol=1e-13)
    np.testing.assert_allclose(oracle.sector_norms(psi), n0, atol=1e-13)
    assert abs(P[0] - 1.0) < 0.05  # short time: still near 1


@pytest.mark.parametrize("L", [3, 6, 8])
def test_ed_matches_free_fermion_chain(L):
    a, b = oracle.couplings(W.chain(L, 0.9), oracle.XY)
    t = np.linspace(0, 12, 25)
    got = ed.ExactSystem(a, b).ensemble_polarization(t)
    np.testing.assert_allclose(got, ed.free_fermion_p11(L, 0.9, t), atol=1e-12)


def test_sector_ed_matches_dense_ed():
    M = 8
    a, b = _system("generic", M, seed=9)
    t = np.linspace(0, 3, 7)
    np.testing.assert_allclose(ed.sector_ensemble_polarization(a, b, t),
                               ed.ExactSystem(a, b).ensemble_polarization(t), atol=1e-12)


def test_ladder_without_rungs_is_the_free_chain():
    # ladder 2x5 with zero rungs: leg 1 is an open XY chain of 5 sites
    a, b = oracle.couplings(W.ladder(5, 1.0, 0.0), oracle.XY)
    t = np.linspace(0, 10, 11)
    np.testing.assert_allclose(ed.sector_ensemble_polarization(a, b, t),
                               ed.free_fermion_p11(5, 1.0, t), atol=1e-12)


def test_short_time_second_moment():
    M = 7
    a, b = _system("star", M, seed=12)
    t = np.array([1e-3, 2e-3])
    P = ed.ExactSystem(a, b).ensemble_polarization(t)
    m2 = 0.25 * np.sum(b[0, 1:] ** 2)
    np.testing.assert_allclose(1 - P, m2 * t**2, rtol=1e-4)


def test_random_state_on_free_chain_large_m():
    # one random-phase state on a 20-spin ladder with zero rungs reproduces the
    # free-fermion ensemble result within statistics + Trotter error
    L, dt, steps = 10, 0.05, 40
    J = W.ladder(L, 1.0, 0.0)
    P, _, _ = oracle.run(J, oracle.XY, seed=17, dt=dt, steps=steps, threads=4)
    exact = ed.free_fermion_p11(L, 1.0, dt * np.arange(steps + 1))
    assert np.max(np.abs(P - exact)) < 6 * 2 * 2.0 ** (-(2 * L - 1) / 2) + 1e-3


def test_self_averaging_spread():
    dt, steps = 0.1, 20
    spread = {}
    for L in (4, 5):
        Ps = [oracle.run(W.ladder(L, 1.0, 0.5), oracle.XY, seed=s, dt=dt, steps=steps)[0]
              for s in range(1, 25)]
        spread[2 * L] = np.std(np.array(Ps)[:, 5:], axis=0).mean()
    for M, s in spread.items():
        assert s < 2 * 2.0 ** (-(M - 1) / 2), (M, s)
    ratio = spread[8] / spread[10]
    assert 1.3 < ratio < 3.0, ratio


def test_single_state_tracks_ensemble_m12():
    # the paper's claim at N_alpha = 1 (Fig. 3a text): ent ~ ens for a ladder
    L, dt, steps = 6, 0.05, 100
    J = W.ladder(L, 1.0, 0.1)   # b_y/b_x = 1/10 as in the paper's Fig. 3a
    a, b = oracle.couplings(J, oracle.XY)
    P, _, _ = oracle.run(J, oracle.XY, seed=21, dt=dt, steps=steps, threads=4)
    ens = ed.sector_ensemble_polarization(a, b, dt * np.arange(0, steps + 1, 10))
    dev = np.abs(P[::10] - ens)
    assert np.max(dev) < 6 * 2 * 2.0 ** (-(2 * L - 1) / 2) + 1e-3, dev
