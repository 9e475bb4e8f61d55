"""Exact references used to pin the oracle (TEST INFRASTRUCTURE).

* Dense exact diagonalization of the secular Hamiltonian
      H = sum_{i<j} [a_ij S^z_i S^z_j + b_ij (S^x_i S^x_j + S^y_i S^y_j)]
  built from Kronecker products of single-spin matrices (a construction
  independent of the oracle's per-amplitude gates).
* The ensemble polarization of the paper's Eq. 1 with p_i = 1/2^{M-1}
  (infinite temperature, "Spin systems with different coupling networks"):
      P_11^ens(t) = 2 [W_11^ens(t) - 1/2] = 2^{-M} Tr[sigma^z_1(t) sigma^z_1],
  from the projector form W = 2^{-(M-1)} Tr[Pi_up U Pi_up U^dagger] with
  Pi_up = (1 + sigma^z_1)/2.
* The free-fermion closed form for the open XY chain (the exactly solvable
  case the paper says the method reproduces): P_11(t) = |[e^{-i h t}]_11|^2,
  h the L x L nearest-neighbour hopping matrix with entries J/2.

Basis convention as in the oracle: spin n is bit n-1 of the index, set = up.
"""
from __future__ import annotations

import numpy as np

# single-spin matrices in the basis (|down> = 0, |up> = 1)
_SZ = np.array([[-0.5, 0.0], [0.0, 0.5]])
_SP = np.array([[0.0, 0.0], [1.0, 0.0]])  # S^+ |down> = |up>
_SM = _SP.T.copy()
_I2 = np.eye(2)


def _site_op(op: np.ndarray, q: int, M: int) -> np.ndarray:
    """op acting on spin q (0-based, = bit q), identity elsewhere.  numpy's kron
    puts its first factor on the most significant bit, so spin M-1 goes first."""
    out = np.ones((1, 1))
    for k in range(M - 1, -1, -1):
        out = np.kron(out, op if k == q else _I2)
    return out


def hamiltonian(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Dense real-symmetric H for coupling matrices a (S^zS^z) and b (flip-flop)."""
    M = a.shape[0]
    sz = [_site_op(_SZ, q, M) for q in range(M)]
    sp = [_site_op(_SP, q, M) for q in range(M)]
    sm = [_site_op(_SM, q, M) for q in range(M)]
    H = np.zeros((1 << M, 1 << M))
    for i in range(M):
        for j in range(i + 1, M):
            if a[i, j] != 0.0:
                H += a[i, j] * (sz[i] @ sz[j])
            if b[i, j] != 0.0:
                # b (S^x S^x + S^y S^y) = (b/2)(S^+ S^- + S^- S^+)
                H += 0.5 * b[i, j] * (sp[i] @ sm[j] + sm[i] @ sp[j])
    return H


class ExactSystem:
    """Eigendecomposition of H, for exact propagation and ensemble averages."""

    def __init__(self, a: np.ndarray, b: np.ndarray):
        self.M = a.shape[0]
        self.H = hamiltonian(np.asarray(a, float), np.asarray(b, float))
        self.E, self.V = np.linalg.eigh(self.H)

    def evolve(self, psi0: np.ndarray, t: float) -> np.ndarray:
        """e^{-iHt} psi0."""
        c = self.V.T @ psi0
        return self.V @ (np.exp(-1j * self.E * t) * c)

    def ensemble_polarization(self, times, site: int = 1) -> np.ndarray:
        """P^ens(t) = 2^{-M} Tr[sigma^z_site(t) sigma^z_site]."""
        N = 1 << self.M
        x = np.arange(N)
        sz = np.where((x >> (site - 1)) & 1, 1.0, -1.0)
        Z = self.V.T @ (sz[:, None] * self.V)
        W2 = Z * Z
        dE = self.E[:, None] - self.E[None, :]
        return np.array([np.sum(W2 * np.cos(dE * t)) / N for t in np.atleast_1d(times)])


def ensemble_cross_polarization(a: np.ndarray, b: np.ndarray, times, n: int, m: int = 1) -> np.ndarray:
    """P_{nm}(t) = 2^{-M} Tr[sigma^z_n(t) sigma^z_m] by dense exact diagonalization:
    sum_{kl} (Z_n)_{kl} (Z_m)_{kl} cos((E_k - E_l) t) / 2^M in the eigenbasis."""
    ex = ExactSystem(a, b)
    N = 1 << ex.M
    x = np.arange(N)
    zn = ex.V.T @ (np.where((x >> (n - 1)) & 1, 1.0, -1.0)[:, None] * ex.V)
    zm = ex.V.T @ (np.where((x >> (m - 1)) & 1, 1.0, -1.0)[:, None] * ex.V)
    W = zn * zm
    times = np.atleast_1d(np.asarray(times, float))
    u = np.exp(1j * ex.E[:, None] * times[None, :])
    return np.real(np.sum(np.conj(u) * (W @ u), axis=0)) / N


def sector_ensemble_polarization(a: np.ndarray, b: np.ndarray, times, site: int = 1) -> np.ndarray:
    """Same as ExactSystem.ensemble_polarization, by total-S^z blocks (H and
    sigma^z_site both conserve the number of up spins).  Reaches M ~ 14."""
    M = a.shape[0]
    times = np.atleast_1d(np.asarray(times, float))
    x = np.arange(1 << M)
    pop = np.zeros(1 << M, dtype=np.int64)
    for q in range(M):
        pop += (x >> q) & 1
    acc = np.zeros(times.size)
    for k in range(M + 1):
        basis = x[pop == k]
        n = basis.size
        index = {int(v): r for r, v in enumerate(basis)}
        H = np.zeros((n, n))
        bits = ((basis[:, None] >> np.arange(M)[None, :]) & 1).astype(float) - 0.5  # s = +-1/2
        for i in range(M):
            for j in range(i + 1, M):
                if a[i, j] != 0.0:
                    H[np.arange(n), np.arange(n)] += a[i, j] * bits[:, i] * bits[:, j]
                if b[i, j] != 0.0:
                    # |1_i 0_j> <-> |0_i 1_j> with amplitude b/2
                    sel = (((basis >> i) & 1) == 1) & (((basis >> j) & 1) == 0)
                    for r in np.nonzero(sel)[0]:
                        y = int(basis[r]) ^ (1 << i) ^ (1 << j)
                        c = index[y]
                        H[r, c] += 0.5 * b[i, j]
                        H[c, r] += 0.5 * b[i, j]
        E, V = np.linalg.eigh(H)
        sz = np.where((basis >> (site - 1)) & 1, 1.0, -1.0)
        Z = V.T @ (sz[:, None] * V)
        W2 = Z * Z
        # sum_mn W2_mn cos((E_m - E_n) t) = Re sum_m e^{-i E_m t} (W2 u)_m, u_n = e^{i E_n t}
        for t0 in range(0, times.size, 128):
            u = np.exp(1j * E[:, None] * times[None, t0:t0 + 128])
            acc[t0:t0 + 128] += np.real(np.sum(np.conj(u) * (W2 @ u), axis=0))
    return acc / (1 << M)


def free_fermion_p11(L: int, J: float, times) -> np.ndarray:
    """Closed form for the open uniform XY chain of L sites, coupling J
    (hopping J/2, single-particle energies J cos(q pi/(L+1))):
        [e^{-iht}]_11 = 2/(L+1) sum_q sin^2(q pi/(L+1)) e^{-i J cos(q pi/(L+1)) t},
    P_11(t) = |[e^{-iht}]_11|^2."""
    times = np.atleast_1d(np.asarray(times, float))
    q = np.arange(1, L + 1)
    k = q * np.pi / (L + 1)
    w = (2.0 / (L + 1)) * np.sin(k) ** 2
    g = (w[None, :] * np.exp(-1j * J * np.cos(k)[None, :] * times[:, None])).sum(axis=1)
    return np.abs(g) ** 2


def hopping_p11(h: np.ndarray, times) -> np.ndarray:
    """|[e^{-iht}]_11|^2 for a general real-symmetric hopping matrix h."""
    E, V = np.linalg.eigh(h)
    times = np.atleast_1d(np.asarray(times, float))
    g = (V[0, :] ** 2)[None, :] * np.exp(-1j * E[None, :] * times[:, None])
    return np.abs(g.sum(axis=1)) ** 2


def hopping_pn1(h: np.ndarray, times) -> np.ndarray:
    """|[e^{-iht}]_{n1}|^2 for every site n (rows: times, columns: n), the
    free-fermion value of P_{n1}(t) for an XY network with hopping matrix h."""
    E, V = np.linalg.eigh(h)
    times = np.atleast_1d(np.asarray(times, float))
    g = np.einsum("nk,k,tk->tn", V, V[0, :], np.exp(-1j * E[None, :] * times[:, None]))
    return np.abs(g) ** 2
