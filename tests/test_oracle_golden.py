"""Golden fixtures and planted-mistake checks for the oracle.

* ``golden/paper_counts.json``: the phase counts the paper prints for the
  14-spin ladder (8192 = N_ent 2^{M-1} ~ N_prod (M-1) = 8190).
* ``golden/oracle_series.json``: P(t) written by ``golden/make_golden.py``
  from the oracle alone; a regression guard on the oracle's arithmetic.
* planted mistakes: plausible slips (sign of the flip-flop angle, a dropped
  S^zS^z term, a factor 2 in the coupling, a swapped spin index, reading the
  wrong site) applied on the CPU around the oracle each move the result
  away from exact e^{-iHt} far beyond the Trotter error, so the pins in
  test_oracle_dynamics.py would catch them.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import ed
from paper_0710_3747_gb300 import workloads as W

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_paper_phase_counts():
    d = json.load(open(os.path.join(HERE, "paper_counts.json")))
    M = d["M"]
    assert d["N_alpha_ent"] * 2 ** (M - 1) == d["phases_entangled"]
    assert d["N_alpha_prod"] * (M - 1) == d["phases_product"]


def test_oracle_series_regression():
    d = json.load(open(os.path.join(HERE, "oracle_series.json")))
    assert len(d) >= 4
    for name, c in d.items():
        P, nrm, _ = oracle.run(np.array(c["J"]), c["htype"], c["seed"], c["dt"], c["steps"])
        np.testing.assert_allclose(P, c["P"], atol=1e-13, err_msg=name)
        np.testing.assert_allclose(nrm, c["norm"], atol=1e-13, err_msg=name)


def _err_vs_exact(a, b, a_run=None, b_run=None, bonds=None, dt=0.02, steps=50, site_run=1):
    """Deviation of P (Trotter, possibly with planted slips) from exact P."""
    M = a.shape[0]
    psi0 = oracle.init_random_phase(M, 4)
    ex = ed.ExactSystem(a, b)
    psi = psi0.copy()
    P, _ = oracle.evolve(psi, a if a_run is None else a_run, b if b_run is None else b_run,
                         dt, steps, bonds=bonds, site=site_run)
    t = dt * np.arange(1, steps + 1)
    exact = np.array([oracle.polarization(ex.evolve(psi0, tt)) for tt in t])
    return np.max(np.abs(P - exact))


def test_planted_mistakes_are_caught():
    M = 6
    a, b = oracle.couplings(W.star_dipolar(M, 5), oracle.DIPOLAR)
    base = _err_vs_exact(a, b)
    assert base < 1e-4
    slips = {
        "flip-flop angle sign": dict(b_run=-b),
        "dropped S^zS^z": dict(a_run=np.zeros_like(a)),
        "coupling factor 2": dict(b_run=2 * b),
        "S^zS^z sign": dict(a_run=-a),
        "wrong site read": dict(site_run=2),
    }
    # a swapped spin index in one bond: (i, j) -> (i, j+1)
    bonds = oracle.canonical_bonds(b)
    bad = list(bonds)
    i, j = bad[3]
    bad[3] = (i, (j + 1) % M if (j + 1) % M != i else (j + 2) % M)
    slips["swapped index"] = dict(bonds=bad)
    for name, kw in slips.items():
        e = _err_vs_exact(a, b, **kw)
        assert e > 100 * base and e > 1e-3, (name, e, base)
