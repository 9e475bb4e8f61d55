"""Pins for the oracle's Philox4x32-10 and the random-phase initial state.

The Philox words are checked bit for bit against Triton's Philox4x32 run by
its CPU interpreter (a library routine written from the same published
definition, Salmon et al. SC'11), on counters and keys that exercise every
word.  The initial state is checked against the paper's definition of the
entangled random-phase state ("Testing the quantum parallelism"): spin 1 up,
2^{M-1} components of weight 2^{-(M-1)/2}, phases 2 pi u(seed, r).
"""
import json
import math
import os
import subprocess
import sys
from math import comb

import numpy as np
import pytest

import oracle

_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
from triton.language.random import philox

@triton.jit
def kern(out_ptr, c_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i + 0).to(tl.uint32)
    c1 = tl.load(c_ptr + 4 * i + 1).to(tl.uint32)
    c2 = tl.load(c_ptr + 4 * i + 2).to(tl.uint32)
    c3 = tl.load(c_ptr + 4 * i + 3).to(tl.uint32)
    o0, o1, o2, o3 = philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, o0.to(tl.int64))
    tl.store(out_ptr + 4 * i + 1, o1.to(tl.int64))
    tl.store(out_ptr + 4 * i + 2, o2.to(tl.int64))
    tl.store(out_ptr + 4 * i + 3, o3.to(tl.int64))

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    n = len(ctrs)
    c = torch.tensor([v for ctr in ctrs for v in ctr], dtype=torch.int64)
    out = torch.zeros(4 * n, dtype=torch.int64)
    # the seed is passed as a signed 64-bit integer with the same bits
    s = seed - (1 << 64) if seed >= (1 << 63) else seed
    kern[(1,)](out, c, s, N=n)
    res.append([[int(v) & 0xFFFFFFFF for v in out[4 * k: 4 * k + 4].tolist()] for k in range(n)])
print(json.dumps(res))
"""


def _triton_philox(cases):
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, env=env, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return json.loads(p.stdout)


def _cases():
    rng = np.random.default_rng(1234)
    seeds = [0, 1, 0xFFFFFFFF, 0x100000000, 0xFFFFFFFFFFFFFFFF, 0x243F6A8885A308D3,
             int(rng.integers(0, 2**63)) * 2 + 1]
    ctrs = [[0, 0, 0, 0], [1, 0, 0, 0], [0xFFFFFFFF] * 4, [0, 1, 0, 0], [0, 0, 1, 0],
            [0, 0, 0, 1], [0x13198A2E, 0x03707344, 0xA4093822, 0x299F31D0]]
    ctrs += [[int(v) for v in rng.integers(0, 2**32, size=4)] for _ in range(9)]
    return [[s, ctrs] for s in seeds]


def test_philox_matches_triton_interpreter():
    cases = _cases()
    ref = _triton_philox(cases)
    for (seed, ctrs), outs in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for ctr, want in zip(ctrs, outs):
            got = list(oracle.philox4x32_10(ctr, key))
            assert got == want, (hex(seed), ctr, [hex(v) for v in got], [hex(v) for v in want])


def test_phase_draw_uses_counter_lo_hi_and_top_53_bits():
    # counter (lo r, hi r, 0, 0), key (lo seed, hi seed): words from Triton.
    seed = 0xDEADBEEF12345678
    rs = [0, 1, 2**31, 2**32 + 5, 2**40 - 1, 7, 2**33, 12345678901]  # 8: a power of 2
    ref = _triton_philox([[seed, [[r & 0xFFFFFFFF, r >> 32, 0, 0] for r in rs]]])[0]
    for r, w in zip(rs, ref):
        bits = (w[0] << 32) | w[1]
        assert oracle.phase_uniform(seed, r) == (bits >> 11) / 2.0**53


@pytest.mark.parametrize("M", [1, 2, 5, 9, 12])
def test_initial_state_matches_definition(M):
    seed = 77 + M
    psi = oracle.init_random_phase(M, seed)
    x = np.arange(1 << M)
    amp = 2.0 ** (-(M - 1) / 2)
    assert np.all(psi[(x & 1) == 0] == 0)
    np.testing.assert_allclose(np.abs(psi[(x & 1) == 1]), amp, rtol=1e-15)
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-14
    if M >= 1:
        assert oracle.polarization(psi, 1) == pytest.approx(1.0, abs=1e-15)
    # phases: 2 pi u(seed, r), r = x >> 1
    for xv in [1, 3, (1 << M) - 1]:
        if xv < (1 << M):
            phi = 2 * math.pi * oracle.phase_uniform(seed, xv >> 1)
            assert psi[xv] == pytest.approx(amp * complex(math.cos(phi), math.sin(phi)), abs=1e-15)
    # S^z sectors: spin 1 up, k-1 of the other M-1 up, each component 2^{-(M-1)}
    n = oracle.sector_norms(psi)
    want = [0.0] + [comb(M - 1, k - 1) / 2.0 ** (M - 1) for k in range(1, M + 1)]
    np.testing.assert_allclose(n, want, atol=1e-14)
    # other spins are unpolarized at t=0 (exactly zero: every |r> has equal weight)
    for site in range(2, M + 1):
        assert abs(oracle.polarization(psi, site)) < 1e-13


def test_phases_are_uniform():
    # 2^{M-1} independent uniform phases: |mean e^{i phi}| ~ 2^{-(M-1)/2}
    M = 18
    psi = oracle.init_random_phase(M, 3)
    z = psi[1::2] / np.abs(psi[1::2])
    assert abs(z.mean()) < 5 * 2.0 ** (-(M - 1) / 2)
    assert abs((z**2).mean()) < 5 * 2.0 ** (-(M - 1) / 2)
    # different seeds give unrelated phases
    psi2 = oracle.init_random_phase(M, 4)
    z2 = psi2[1::2] / np.abs(psi2[1::2])
    assert abs(np.vdot(z, z2)) / z.size < 5 * 2.0 ** (-(M - 1) / 2)
