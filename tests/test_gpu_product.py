"""Product-state initialization on the GPU against the oracle, and the paper's
N_alpha experiment (Fig. 3a: 14-spin ladder, b_y/b_x = 1/10) run as a batch.
"""
import numpy as np
import pytest

import oracle
from oracle import ed
from paper_0710_3747_gb300 import spinrp
from paper_0710_3747_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("kind", ["ladder12", "star11"])
def test_product_state_matches_oracle(kind, prec):
    spinrp.lib()
    if kind == "ladder12":
        J, ht, dt = W.ladder(6, 1.0, 0.1), W.XY, 0.05
    else:
        J, ht, dt = W.star_dipolar(11, 5), W.DIPOLAR, 0.02
    M, seed, steps = J.shape[0], 77, 60
    sysm = spinrp.System(J, ht)
    st = spinrp.State(sysm, prec, series_cap=steps + 1)
    st.init_product_phase(seed)
    psi0 = oracle.init_product_phase(M, seed)
    amp_tol = 1e-14 if prec == "c128" else 2e-7 * 2.0 ** (-(M - 1) / 2)
    assert np.max(np.abs(st.amplitudes() - psi0)) <= amp_tol
    st.evolve(dt, steps)
    P, nrm, _ = oracle.run_product(J, ht, seed, dt, steps)
    tol = 1e-10 if prec == "c128" else 1e-4
    assert np.max(np.abs(st.polarization() - P)) <= tol
    assert np.max(np.abs(st.norm_series() - nrm)) <= (1e-12 if prec == "c128" else 1e-5)
    st.close()


def test_batch_product_equals_single_states():
    spinrp.lib()
    J = W.ladder(5, 1.0, 0.1)
    seeds = list(range(1, 9))
    systems = [spinrp.System(J, W.XY) for _ in seeds]
    b = spinrp.Batch(systems, seeds, "c64", series_cap=32)
    b.init_product_phase().evolve(0.05, 30)
    for k, s in enumerate(seeds):
        st = spinrp.State(spinrp.System(J, W.XY), "c64", series_cap=32)
        st.init_product_phase(s).evolve(0.05, 30)
        assert np.array_equal(b.polarization(k), st.polarization())
        st.close()
    b.close()


def test_fig3a_product_needs_630_realizations():
    """14-spin ladder, b_y/b_x = 1/10, t up to 40/b_x: <P^ent>_1 and
    <P^prod>_630 follow the exact ensemble dynamics, <P^prod>_1 does not."""
    spinrp.lib()
    L, dt, steps = 7, 0.05, 800
    J = W.ladder(L, 1.0, 0.1)
    a, bb = oracle.couplings(J, oracle.XY)
    times = dt * np.arange(steps + 1)
    Pens = ed.sector_ensemble_polarization(a, bb, times)
    rms = lambda d: float(np.sqrt(np.mean(d ** 2)))
    n = 630
    b = spinrp.Batch([spinrp.System(J, W.XY) for _ in range(n)], list(range(1, n + 1)), "c64",
                     series_cap=steps + 1)
    b.init_product_phase().evolve(dt, steps)
    mean_prod, _ = b.ensemble()
    err_prod1 = np.mean([rms(b.polarization(k) - Pens) for k in range(8)])
    b.close()
    st = spinrp.State(spinrp.System(J, W.XY), "c64", series_cap=steps + 1)
    err_ent = np.mean([rms(st.init_random_phase(s).evolve(dt, steps).polarization() - Pens)
                       for s in range(1, 5)])
    st.close()
    err_prod630 = rms(mean_prod - Pens)
    # Trotter error at dt = 0.05 is ~1e-3, far below the statistical scales here
    scale = 2.0 ** (-(2 * L - 1) / 2)
    assert err_prod1 > 3.0 * err_ent and err_prod1 > 8.0 * scale
    assert err_prod630 < 2.0 * err_ent


def test_fig3b_star_one_state_of_either_kind_suffices():
    """14-spin star with Gaussian dipolar couplings (a/b = -2): both a single
    product state and a single entangled state stay close to the ensemble
    (the paper's Fig. 3b); contrast with the ladder above, where the product
    state fails by a wide margin."""
    spinrp.lib()
    M, dt, steps = 14, 0.02, 500
    J = W.star_gaussian(M, 1)
    a, bb = oracle.couplings(J, oracle.DIPOLAR)
    times = dt * np.arange(steps + 1)
    Pens = ed.sector_ensemble_polarization(a, bb, times)
    rms = lambda d: float(np.sqrt(np.mean(d ** 2)))
    n = 6
    b = spinrp.Batch([spinrp.System(J, W.DIPOLAR) for _ in range(n)], list(range(1, n + 1)), "c64",
                     series_cap=steps + 1)
    b.init_product_phase().evolve(dt, steps)
    err_prod1 = np.mean([rms(b.polarization(k) - Pens) for k in range(n)])
    b.init_random_phase().evolve(dt, steps)
    err_ent = np.mean([rms(b.polarization(k) - Pens) for k in range(n)])
    b.close()
    # "almost indistinguishable": both within a few times the Chebyshev scale
    # 2^{-(M-1)/2} of one entangled state (the ladder's product state misses
    # by more than 8 times that scale, see above)
    scale = 2.0 ** (-(M - 1) / 2)
    assert err_ent < 2.0 * scale
    assert err_prod1 < 4.0 * scale
