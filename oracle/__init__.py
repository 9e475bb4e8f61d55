"""FP64 CPU oracle for the random-phase pure-state method (arXiv:0710.3747).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
package.  It shares no code with ``paper_0710_3747_gb300`` and imports nothing
from it.

Layers:
  * ``spin_oracle.c`` (plain C, FP64): Philox4x32-10, the random-phase state,
    exact flip-flop and diagonal factors, the symmetric second-order Trotter
    step and the per-step polarization (see that file's header).
  * this module: ctypes bindings, the coupling conventions of the paper's
    Hamiltonian and the canonical bond order.
  * ``ed.py``: exact diagonalization and the free-fermion closed form, used
    only to pin the oracle itself.

Pins (tests/test_oracle_*.py): Philox against Triton's CPU-interpreted
Philox; the M=2 closed form; O(dt^2) convergence to exact e^{-iHt} from ED;
time-reversal of the palindromic step; norm and S^z-sector conservation; ED
against the free-fermion closed form; the self-averaging spread bound.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

import numpy as np

from . import build as _build

# Hamiltonian families of the paper's secular spin-spin Hamiltonian
# ("Spin systems with different coupling networks"):
#   H = sum_{i<j} [a_ij S^z_i S^z_j + 1/2 b_ij (S^+_i S^-_j + S^-_i S^+_j)]
# with b/a = 0 Ising, a/b = 0 XY, a/b = 1 isotropic, a/b = -2 truncated dipolar.
XY, DIPOLAR, ISOTROPIC, ISING, GENERIC = 0, 1, 2, 3, 4

_lib = None


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the C oracle."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(str(path))
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_philox4x32_10.restype = None
        L.oracle_phase_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_phase_uniform.restype = ctypes.c_double
        L.oracle_init_random_phase.argtypes = [ctypes.c_int, ctypes.c_uint64, dp, ctypes.c_int]
        L.oracle_init_random_phase.restype = ctypes.c_int
        L.oracle_flipflop.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.oracle_flipflop.restype = None
        L.oracle_diag.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int]
        L.oracle_diag.restype = None
        L.oracle_diag_energy.argtypes = [ctypes.c_int, dp, ctypes.c_uint64]
        L.oracle_diag_energy.restype = ctypes.c_double
        L.oracle_site_populations.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, dp, ctypes.c_int]
        L.oracle_site_populations.restype = None
        L.oracle_evolve.argtypes = [ctypes.c_int, dp, dp, dp, i32p, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int64, ctypes.c_int, dp, dp, ctypes.c_int]
        L.oracle_evolve.restype = ctypes.c_int
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _threads(threads: int | None) -> int:
    if threads is None:
        return int(os.environ.get("ORACLE_THREADS", "1"))
    return int(threads)


# ---------------------------------------------------------------------------
# Philox4x32-10 and the phase draw
# ---------------------------------------------------------------------------
def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> tuple[int, int, int, int]:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def phase_uniform(seed: int, r: int) -> float:
    """u(seed, r) in [0,1) for basis index r of spins 2..M."""
    return float(lib().oracle_phase_uniform(int(seed) & (2**64 - 1), int(r)))


# ---------------------------------------------------------------------------
# Couplings and bonds
# ---------------------------------------------------------------------------
def couplings(J: np.ndarray, htype: int, a_generic: np.ndarray | None = None):
    """(a, b) matrices of H for coupling matrix J and Hamiltonian family htype.

    XY: a=0, b=J.  Truncated dipolar J[2 S^zS^z - (S^xS^x + S^yS^y)]: a=2J, b=-J
    (a/b = -2).  Isotropic: a=b=J.  Ising: a=J, b=0.  Generic: b=J, a=a_generic.
    """
    J = np.asarray(J, dtype=np.float64)
    if htype == XY:
        a, b = np.zeros_like(J), J.copy()
    elif htype == DIPOLAR:
        a, b = 2.0 * J, -J
    elif htype == ISOTROPIC:
        a, b = J.copy(), J.copy()
    elif htype == ISING:
        a, b = J.copy(), np.zeros_like(J)
    elif htype == GENERIC:
        a, b = np.asarray(a_generic, dtype=np.float64).copy(), J.copy()
    else:
        raise ValueError(f"unknown Hamiltonian type {htype}")
    return np.ascontiguousarray(a), np.ascontiguousarray(b)


def canonical_bonds(b: np.ndarray) -> list[tuple[int, int]]:
    """Flip-flop bonds in canonical order: all pairs i<j (0-based) with b_ij != 0,
    lexicographic in (i, j).  Any fixed order gives a symmetric second-order
    product; this is the one the oracle and the library both default to."""
    M = b.shape[0]
    return [(i, j) for i in range(M) for j in range(i + 1, M) if b[i, j] != 0.0]


# ---------------------------------------------------------------------------
# States and evolution
# ---------------------------------------------------------------------------
def init_random_phase(M: int, seed: int, threads: int | None = None) -> np.ndarray:
    """The entangled random-phase state as a complex128 vector of length 2^M."""
    buf = np.empty(2 * (1 << M), dtype=np.float64)
    rc = lib().oracle_init_random_phase(M, int(seed) & (2**64 - 1), _dptr(buf), _threads(threads))
    if rc != 0:
        raise ValueError("oracle_init_random_phase failed")
    return buf.view(np.complex128)


def _as_buf(psi: np.ndarray) -> np.ndarray:
    assert psi.dtype == np.complex128 and psi.flags["C_CONTIGUOUS"]
    return psi.view(np.float64)


def flipflop(psi: np.ndarray, i: int, j: int, b: float, tau: float, threads: int | None = None):
    """In place: exp(-i tau b (S^x_i S^x_j + S^y_i S^y_j)) on 0-based spins i, j."""
    M = int(np.log2(psi.size))
    lib().oracle_flipflop(M, _dptr(_as_buf(psi)), i, j, float(b), float(tau), _threads(threads))


def diag(psi: np.ndarray, a: np.ndarray, tau: float, threads: int | None = None):
    """In place: exp(-i tau sum_{i<j} a_ij S^z_i S^z_j)."""
    M = int(np.log2(psi.size))
    a = np.ascontiguousarray(a, dtype=np.float64)
    lib().oracle_diag(M, _dptr(_as_buf(psi)), _dptr(a), float(tau), _threads(threads))


def diag_energy(a: np.ndarray, x: int) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return float(lib().oracle_diag_energy(a.shape[0], _dptr(a), int(x)))


def site_populations(psi: np.ndarray, site: int = 1, threads: int | None = None):
    M = int(np.log2(psi.size))
    up, dn = ctypes.c_double(), ctypes.c_double()
    lib().oracle_site_populations(M, _dptr(_as_buf(psi)), site, ctypes.byref(up), ctypes.byref(dn),
                                  _threads(threads))
    return up.value, dn.value


def polarization(psi: np.ndarray, site: int = 1) -> float:
    """P = (N_up - N_dn)/(N_up + N_dn) of spin `site` (= 2<S^z> at unit norm)."""
    up, dn = site_populations(psi, site)
    return (up - dn) / (up + dn)


def sector_norms(psi: np.ndarray) -> np.ndarray:
    """n_k = sum_{popcount(x)=k} |psi_x|^2, k = 0..M (number of up spins)."""
    M = int(np.log2(psi.size))
    x = np.arange(psi.size, dtype=np.uint64)
    pop = np.zeros(psi.size, dtype=np.int64)
    for q in range(M):
        pop += ((x >> np.uint64(q)) & np.uint64(1)).astype(np.int64)
    return np.bincount(pop, weights=np.abs(psi) ** 2, minlength=M + 1)


def evolve(psi: np.ndarray, a: np.ndarray, b: np.ndarray, dt: float, steps: int,
           bonds: Iterable[tuple[int, int]] | None = None, site: int = 1,
           threads: int | None = None):
    """Evolve psi in place by `steps` symmetric second-order Trotter steps.

    Returns (P, norm): arrays of length steps with the polarization of `site`
    and the norm after each step.
    """
    M = int(np.log2(psi.size))
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if bonds is None:
        bonds = canonical_bonds(b)
    bl = np.ascontiguousarray(np.asarray(list(bonds), dtype=np.int32).reshape(-1, 2))
    P = np.empty(steps, dtype=np.float64)
    nrm = np.empty(steps, dtype=np.float64)
    rc = lib().oracle_evolve(M, _dptr(_as_buf(psi)), _dptr(a), _dptr(b),
                             bl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), bl.shape[0],
                             float(dt), int(steps), int(site), _dptr(P), _dptr(nrm),
                             _threads(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_evolve failed ({rc})")
    return P, nrm


def run(J: np.ndarray, htype: int, seed: int, dt: float, steps: int, a_generic=None,
        site: int = 1, threads: int | None = None, bonds=None):
    """Whole job: random-phase state from `seed`, `steps` steps; returns
    (P[0..steps], norm[0..steps], psi_final)."""
    a, b = couplings(J, htype, a_generic)
    M = a.shape[0]
    psi = init_random_phase(M, seed, threads)
    p0 = polarization(psi, site)
    n0 = float(np.vdot(psi, psi).real)
    P, nrm = evolve(psi, a, b, dt, steps, bonds=bonds, site=site, threads=threads)
    return np.concatenate([[p0], P]), np.concatenate([[n0], nrm]), psi


def product_uniform(seed: int, bit: int) -> float:
    """u_l of the product state's phase of the spin at bit index `bit` (>= 1)."""
    L = lib()
    L.oracle_product_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int]
    L.oracle_product_uniform.restype = ctypes.c_double
    return float(L.oracle_product_uniform(int(seed) & (2**64 - 1), int(bit)))


def init_product_phase(M: int, seed: int, threads: int | None = None) -> np.ndarray:
    """The paper's product (unentangled) random state: spin 1 up, each other
    spin l in (|down> + e^{-i phi_l}|up>)/sqrt(2)."""
    L = lib()
    L.oracle_init_product_phase.argtypes = [ctypes.c_int, ctypes.c_uint64,
                                            ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    L.oracle_init_product_phase.restype = ctypes.c_int
    buf = np.empty(2 * (1 << M), dtype=np.float64)
    if L.oracle_init_product_phase(M, int(seed) & (2**64 - 1), _dptr(buf), _threads(threads)) != 0:
        raise ValueError("oracle_init_product_phase failed")
    return buf.view(np.complex128)


def run_product(J: np.ndarray, htype: int, seed: int, dt: float, steps: int, a_generic=None,
                site: int = 1, threads: int | None = None):
    """Whole job from the product state: (P[0..steps], norm[0..steps], psi)."""
    a, b = couplings(J, htype, a_generic)
    M = a.shape[0]
    psi = init_product_phase(M, seed, threads)
    p0 = polarization(psi, site)
    n0 = float(np.vdot(psi, psi).real)
    P, nrm = evolve(psi, a, b, dt, steps, site=site, threads=threads)
    return np.concatenate([[p0], P]), np.concatenate([[n0], nrm]), psi


def evolve_all_sites(psi: np.ndarray, a: np.ndarray, b: np.ndarray, dt: float, steps: int,
                     bonds: Iterable[tuple[int, int]] | None = None, threads: int | None = None):
    """Evolve psi in place; returns (P, norm) with P[n, q-1] the polarization
    of spin q after step n+1 (every site) and norm[n] the norm."""
    L = lib()
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_evolve_all_sites.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int64, dp, dp,
                                          ctypes.c_int]
    L.oracle_evolve_all_sites.restype = ctypes.c_int
    M = int(np.log2(psi.size))
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if bonds is None:
        bonds = canonical_bonds(b)
    bl = np.ascontiguousarray(np.asarray(list(bonds), dtype=np.int32).reshape(-1, 2))
    P = np.empty((steps, M), dtype=np.float64)
    nrm = np.empty(steps, dtype=np.float64)
    rc = L.oracle_evolve_all_sites(M, _dptr(_as_buf(psi)), _dptr(a), _dptr(b),
                                   bl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), bl.shape[0],
                                   float(dt), int(steps), _dptr(P), _dptr(nrm), _threads(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_evolve_all_sites failed ({rc})")
    return P, nrm


def run_all_sites(J: np.ndarray, htype: int, seed: int, dt: float, steps: int, a_generic=None,
                  threads: int | None = None, product: bool = False):
    """Whole job reading out every site: (P[0..steps, 0..M-1], norm[0..steps], psi)."""
    a, b = couplings(J, htype, a_generic)
    M = a.shape[0]
    psi = init_product_phase(M, seed, threads) if product else init_random_phase(M, seed, threads)
    p0 = np.array([polarization(psi, q) for q in range(1, M + 1)])
    n0 = float(np.vdot(psi, psi).real)
    P, nrm = evolve_all_sites(psi, a, b, dt, steps, threads=threads)
    return np.vstack([p0[None, :], P]), np.concatenate([[n0], nrm]), psi
