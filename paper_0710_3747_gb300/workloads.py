"""Seeded synthetic inputs shaped like the paper's test systems.

This module only builds inputs: coupling matrices J_ij, job lists and arrival
streams.  It contains none of the method's arithmetic (no random phases, no
Trotter factors, no observables) and imports nothing else from this package,
so the CPU oracle and the GPU library can both be fed from it.

Systems ("Spin systems with different coupling networks" in the paper):
  * ladder: two legs of L spins, sites 1..L and L+1..2L, leg bonds (n, n+1)
    inside each leg, rung bonds (n, n+L); open ends (no bond closes a leg).
  * star: spin 1 at the origin and M-1 spins uniform in the unit ball (each
    drawn point is redrawn until it is at least rmin from every earlier one),
    all pairs coupled by J_ij = (1 - 3 cos^2 theta_ij) / r_ij^3 with theta_ij
    the angle of r_i - r_j to the field (z) axis, rescaled to unit rms over
    all M(M-1)/2 pairs.  (The paper draws star couplings from a Gaussian;
    ``star_gaussian`` builds that variant.)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

XY, DIPOLAR, ISOTROPIC, ISING, GENERIC = 0, 1, 2, 3, 4


def ladder(L: int, j_leg: float = 1.0, j_rung: float = 0.5) -> np.ndarray:
    """Coupling matrix (2L x 2L, 0-based) of the open two-leg ladder."""
    M = 2 * L
    J = np.zeros((M, M))
    for k in range(L - 1):
        J[k, k + 1] = J[k + 1, k] = j_leg
        J[L + k, L + k + 1] = J[L + k + 1, L + k] = j_leg
    for k in range(L):
        J[k, k + L] = J[k + L, k] = j_rung
    return J


def chain(L: int, j: float = 1.0) -> np.ndarray:
    """Open chain of L spins (nearest neighbours)."""
    J = np.zeros((L, L))
    for k in range(L - 1):
        J[k, k + 1] = J[k + 1, k] = j
    return J


def star_positions(M: int, seed: int, rmin: float = 0.1) -> np.ndarray:
    """Spin 1 at the origin, M-1 points uniform in the unit ball with minimum
    separation rmin (rejection: a point that violates it is drawn again)."""
    rng = np.random.default_rng([0x5EED57A2, int(seed)])
    pos = [np.zeros(3)]
    while len(pos) < M:
        p = rng.uniform(-1.0, 1.0, size=3)
        if p @ p > 1.0:
            continue
        if min(np.linalg.norm(p - q) for q in pos) < rmin:
            continue
        pos.append(p)
    return np.array(pos)


def dipolar_from_positions(pos: np.ndarray) -> np.ndarray:
    """J_ij = (1 - 3 cos^2 theta_ij)/r_ij^3, rescaled to unit rms over pairs."""
    M = pos.shape[0]
    J = np.zeros((M, M))
    for i in range(M):
        for j in range(i + 1, M):
            d = pos[i] - pos[j]
            r = float(np.linalg.norm(d))
            c = d[2] / r
            J[i, j] = J[j, i] = (1.0 - 3.0 * c * c) / r**3
    iu = np.triu_indices(M, 1)
    rms = math.sqrt(float(np.mean(J[iu] ** 2)))
    return J / rms


def star_dipolar(M: int, seed: int, rmin: float = 0.1) -> np.ndarray:
    return dipolar_from_positions(star_positions(M, seed, rmin))


def star_gaussian(M: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """All-to-all couplings drawn from N(0, sigma^2) (the paper's star)."""
    rng = np.random.default_rng([0x6A055, int(seed)])
    J = np.zeros((M, M))
    iu = np.triu_indices(M, 1)
    J[iu] = rng.normal(0.0, sigma, size=iu[0].size)
    return J + J.T


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
@dataclass
class Job:
    """One spin-dynamics job: coupling matrix, Hamiltonian family, phase seed,
    time step and number of steps (plus an arrival time for served jobs)."""
    J: np.ndarray
    htype: int
    seed: int
    dt: float
    steps: int
    kind: str = ""
    arrival: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.J.shape[0])


def ladder_m14() -> Job:
    """2x7 XY ladder, leg 1, rung 0.5, dt 0.05, 400 steps (FP64 case)."""
    return Job(ladder(7, 1.0, 0.5), XY, seed=1, dt=0.05, steps=400, kind="ladder")


def star_m20() -> Job:
    """Dipolar star, M=20, dt 0.02, 1000 steps."""
    return Job(star_dipolar(20, seed=2), DIPOLAR, seed=1, dt=0.02, steps=1000, kind="star")


def ladder_m30() -> Job:
    """2x15 XY ladder, leg 1, rung 0.5, dt 0.05, 200 steps (2^30 amplitudes)."""
    return Job(ladder(15, 1.0, 0.5), XY, seed=1, dt=0.05, steps=200, kind="ladder")


def star_batch(n: int = 4096, seed: int = 4, m_lo: int = 12, m_hi: int = 22,
               dt: float = 0.02, steps: int = 500) -> list[Job]:
    """n dipolar-star disorder realizations, M uniform in m_lo..m_hi, each with
    its own geometry and phase seed."""
    rng = np.random.default_rng([0xBA7C4, int(seed)])
    Ms = rng.integers(m_lo, m_hi + 1, size=n)
    jobs = []
    for k in range(n):
        geom = int(seed) * 1_000_003 + k
        jobs.append(Job(star_dipolar(int(Ms[k]), geom), DIPOLAR, seed=1 + 7919 * k + int(seed),
                        dt=dt, steps=steps, kind="star", meta={"geom_seed": geom, "index": k}))
    return jobs


def serve_stream(n: int = 2000, seed: int = 5, rate: float = 1.0, m_lo: int = 10,
                 m_hi: int = 28, t_lo: float = 5.0, t_hi: float = 50.0, dt: float = 0.05,
                 m_cap: int | None = None) -> list[Job]:
    """Poisson request stream of ladder / star jobs.

    Arrivals have exponential gaps of mean 1/rate seconds.  Each job is an XY
    ladder (rung J uniform in [0.2, 1], leg 1) or a dipolar star with equal
    probability; M = round(exp(U[ln m_lo, ln m_hi])) (ladders rounded down to
    even); final time T uniform in [t_lo, t_hi]; steps = round(T/dt).
    m_cap, when given, clips M (for reduced-size runs)."""
    rng = np.random.default_rng([0x5E12E, int(seed)])
    t = 0.0
    jobs = []
    for k in range(n):
        t += rng.exponential(1.0 / rate)
        M = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        if m_cap is not None:
            M = min(M, m_cap)
        T = float(rng.uniform(t_lo, t_hi))
        steps = max(1, int(round(T / dt)))
        phase_seed = int(rng.integers(1, 2**62))
        if rng.uniform() < 0.5:
            L = max(1, M // 2)
            j_rung = float(rng.uniform(0.2, 1.0))
            J = ladder(L, 1.0, j_rung)
            jobs.append(Job(J, XY, phase_seed, dt, steps, kind="ladder", arrival=t,
                            meta={"j_rung": j_rung, "index": k}))
        else:
            geom = int(rng.integers(1, 2**31))
            jobs.append(Job(star_dipolar(max(M, 2), geom), DIPOLAR, phase_seed, dt, steps,
                            kind="star", arrival=t, meta={"geom_seed": geom, "index": k}))
    return jobs
