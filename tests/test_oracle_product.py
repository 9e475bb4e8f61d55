"""Pins for the oracle's product (unentangled) random state, "Testing the
quantum parallelism" section of the paper:

  |Psi_prod> = |up>_1 (x) prod_{l=2..M} (|down>_l + e^{-i phi_l} |up>_l)/sqrt 2.

Each pin comes from outside the oracle's bit-sum formula:
  * a Kronecker-product construction of the same tensor product (checks the
    spin-to-bit order, the sign of the phase and the normalisation);
  * the phase draw is Philox4x32-10 (pinned separately against Triton) at
    counter (l-1, 0, 0, 1);
  * averaged over its phases the state is the paper's infinite-temperature
    ensemble |up><up|_1 (x) (1/2)^{M-1}: every off-diagonal element averages
    to zero, every diagonal element of the spin-1-up block to 2^{-(M-1)};
  * the paper's counting claim: one entangled state (2^{M-1} phases) and an
    average over N ~ 2^{M-1}/(M-1) product states (N (M-1) phases) track the
    ensemble equally well, while a single product state does not (14-spin
    ladder with b_y/b_x = 1/10: 630 x 13 ~ 8192; checked here at M = 10 by
    exact diagonalization).
"""
import numpy as np
import pytest

import oracle
from oracle import ed
from paper_0710_3747_gb300 import workloads as W


def test_product_phase_draw_uses_its_own_counter():
    for seed in (0, 1, 2**40 + 7):
        for q in (1, 2, 13, 33):
            w = oracle.philox4x32_10((q, 0, 0, 1), (seed & 0xFFFFFFFF, seed >> 32))
            bits = ((w[0] << 32) | w[1]) >> 11
            assert oracle.product_uniform(seed, q) == bits * 2.0**-53
            # different counter word 3 from the entangled state's draw of r = q
            assert oracle.product_uniform(seed, q) != oracle.phase_uniform(seed, q)


@pytest.mark.parametrize("M", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("seed", [1, 12345])
def test_product_state_is_the_tensor_product(M, seed):
    up = np.array([0.0, 1.0])  # index 0 = down, 1 = up
    psi = up
    for q in range(1, M):  # spin q+1 = bit q goes to the more significant side
        phi = 2.0 * np.pi * oracle.product_uniform(seed, q)
        f = np.array([1.0, np.exp(-1j * phi)]) / np.sqrt(2.0)
        psi = np.kron(f, psi)
    got = oracle.init_product_phase(M, seed)
    np.testing.assert_allclose(got, psi, rtol=0, atol=1e-14)
    assert abs(np.vdot(got, got).real - 1.0) < 1e-13
    # a product state factorises: psi(x) psi(y) = psi(x & y) psi(x | y)
    rng = np.random.default_rng(M)
    for _ in range(20):
        x, y = (int(v) | 1 for v in rng.integers(0, 1 << M, size=2))
        assert abs(got[x] * got[y] - got[x & y] * got[x | y]) < 1e-14


def test_phase_average_is_the_ensemble():
    M, n = 4, 4000
    rho = np.zeros((1 << M, 1 << M), dtype=complex)
    for s in range(n):
        v = oracle.init_product_phase(M, 1000 + s)
        rho += np.outer(v, v.conj())
    rho /= n
    target = np.diag([(x & 1) * 2.0 ** -(M - 1) for x in range(1 << M)])
    # elements are 2^{-(M-1)} times unit phases: standard error 2^{-(M-1)}/sqrt(n)
    assert np.max(np.abs(rho - target)) < 6 * 2.0 ** -(M - 1) / np.sqrt(n)


def _exact_series(ex, states, times):
    x = np.arange(1 << ex.M)
    sz = np.where(x & 1, 1.0, -1.0)
    C = ex.V.T @ states
    out = []
    for t in times:
        w = np.abs(ex.V @ (np.exp(-1j * ex.E * t)[:, None] * C)) ** 2
        out.append((sz @ w) / w.sum(axis=0))
    return np.array(out)


def test_product_needs_many_realizations_entangled_one():
    L = 5
    M = 2 * L
    a, b = oracle.couplings(W.ladder(L, 1.0, 0.1), oracle.XY)
    ex = ed.ExactSystem(a, b)
    times = np.arange(0.0, 40.01, 0.5)
    Pens = ex.ensemble_polarization(times)
    rms = lambda d: float(np.sqrt(np.mean(d ** 2)))
    ent = np.stack([oracle.init_random_phase(M, s) for s in range(1, 9)], axis=1)
    err_ent = np.mean([rms(c - Pens) for c in _exact_series(ex, ent, times).T])
    nstar = round(2 ** (M - 1) / (M - 1))  # 57 product states ~ one entangled state
    prod = np.stack([oracle.init_product_phase(M, s) for s in range(1, nstar + 1)], axis=1)
    Pprod = _exact_series(ex, prod, times)
    err_prod1 = np.mean([rms(c - Pens) for c in Pprod[:, :8].T])
    err_prodN = rms(Pprod.mean(axis=1) - Pens)
    assert err_prod1 > 2.5 * err_ent
    assert err_prodN < 2.0 * err_ent
    # the entangled state's error is of the order of the Chebyshev scale 2^{-(M-1)/2}
    assert err_ent < 2.0 * 2.0 ** (-(M - 1) / 2)
