"""Python binding of the C ABI in ``include/spinrp.h`` (ctypes).

Argument marshalling only: every step of the path runs in ``libspinrp.so``.
Function names mirror the C entry points without their ``spinrp_`` prefix;
``System`` and ``State`` wrap the handles.  Device buffers of a state are
allocated with PyTorch's caching allocator (``torch.empty`` on the current
CUDA device) and handed to the library as plain pointers; the stream is
PyTorch's current stream unless one is given.

There is no fallback: if the library is not built, or cannot run, calls
raise.
"""
from __future__ import annotations

import ctypes
import threading
from pathlib import Path

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, ESTATE = range(7)
KERNEL_SWEEP, KERNEL_INIT, KERNEL_TABLES = range(3)
XY, DIPOLAR, ISOTROPIC, ISING, GENERIC = range(5)
C64, C128 = 0, 1
_PREC = {"c64": C64, "complex64": C64, "fp32": C64, C64: C64,
         "c128": C128, "complex128": C128, "fp64": C128, C128: C128}


class SpinrpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"spinrp error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def library_path() -> Path:
    return _build.LIB


def lib(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libspinrp.so (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not path.exists():
            if build_if_missing:
                _build.build()
            else:
                raise ImportError(f"{path} is not built; run __graft_entry__.build() or "
                                  f"python -m paper_0710_3747_gb300.build")
        L = ctypes.CDLL(str(path))
        vp, i32p, i64p, dp = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double))
        ip, szp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)
        sig = {
            "spinrp_last_error": ([], ctypes.c_char_p),
            "spinrp_version": ([], ctypes.c_char_p),
            "spinrp_system_create": ([ctypes.c_int, dp, ctypes.c_int, dp, ctypes.POINTER(vp)], ctypes.c_int),
            "spinrp_system_destroy": ([vp], None),
            "spinrp_system_num_spins": ([vp], ctypes.c_int),
            "spinrp_system_bonds": ([vp, i32p, ctypes.c_int, ip], ctypes.c_int),
            "spinrp_system_set_tile": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "spinrp_system_set_regbits": ([vp, ctypes.c_int], ctypes.c_int),
            "spinrp_system_set_orientation": ([vp, ctypes.c_int], ctypes.c_int),
            "spinrp_state_orientation": ([vp, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
            "spinrp_state_set_pipeline": ([vp, ctypes.c_int], ctypes.c_int),
            "spinrp_state_pipeline": ([vp, ip], ctypes.c_int),
            "spinrp_state_pipeline_timeout_check": ([vp, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "spinrp_system_orientation": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
            "spinrp_system_plan_info": ([vp, ctypes.c_int, ip, ip, ip], ctypes.c_int),
            "spinrp_system_plan_gates": ([vp, ctypes.c_int, i32p, i32p, ctypes.c_int, ip], ctypes.c_int),
            "spinrp_state_bytes": ([vp, ctypes.c_int, ctypes.c_int64, szp, szp], ctypes.c_int),
            "spinrp_state_create": ([vp, ctypes.c_int, vp, ctypes.c_int64, vp, vp, ctypes.POINTER(vp)],
                                    ctypes.c_int),
            "spinrp_state_destroy": ([vp], None),
            "spinrp_state_init_random_phase": ([vp, ctypes.c_uint64], ctypes.c_int),
            "spinrp_state_init_product_phase": ([vp, ctypes.c_uint64], ctypes.c_int),
            "spinrp_ladder_create": ([ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.POINTER(vp)],
                                     ctypes.c_int),
            "spinrp_star_dipolar_create": ([ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(vp)],
                                           ctypes.c_int),
            "spinrp_system_couplings": ([vp, dp, dp], ctypes.c_int),
            "spinrp_schedule": ([vp, i32p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "spinrp_state_set_sites": ([vp, ctypes.c_int], ctypes.c_int),
            "spinrp_site_series": ([vp, dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
            "spinrp_state_load": ([vp, dp], ctypes.c_int),
            "spinrp_evolve": ([vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int], ctypes.c_int),
            "spinrp_series_length": ([vp], ctypes.c_int64),
            "spinrp_polarization": ([vp, ctypes.c_int, dp, ctypes.c_int64, i64p], ctypes.c_int),
            "spinrp_norm_series": ([vp, dp, ctypes.c_int64, i64p], ctypes.c_int),
            "spinrp_sector_norms": ([vp, dp, ctypes.c_int, ip], ctypes.c_int),
            "spinrp_state_read": ([vp, i64p, ctypes.c_int64, dp], ctypes.c_int),
            "spinrp_state_layout": ([vp, i32p, ctypes.POINTER(vp)], ctypes.c_int),
            "spinrp_profile": ([vp, ctypes.c_int], ctypes.c_int),
            "spinrp_profile_read": ([vp, ctypes.c_int, dp, i64p], ctypes.c_int),
            "spinrp_launch_count": ([], ctypes.c_int64),
            "spinrp_state_transfer_bytes": ([vp, i64p, i64p], ctypes.c_int),
            "spinrp_system_plan_check": ([vp, ctypes.c_int, dp, dp], ctypes.c_int),
            "spinrp_polarization_noalloc": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p,
                                             ctypes.c_int, vp, vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def _check(rc: int):
    if rc != OK:
        raise SpinrpError(rc, lib().spinrp_last_error().decode())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def version() -> str:
    return lib().spinrp_version().decode()


def polarization_noalloc(psi_ptr: int, M: int, prec, site: int, layout, out_ptr: int,
                         stream: int = 0, blocks: int = 0):
    """spinrp_polarization_noalloc: (P, norm) of spin `site` of the device state
    at psi_ptr into the device buffer out_ptr (2 doubles), allocating nothing.
    For callers that may not allocate device memory; see include/spinrp.h."""
    lay = None
    if layout is not None:
        lay = (ctypes.c_int32 * M)(*[int(v) for v in layout])
    _check(lib().spinrp_polarization_noalloc(ctypes.c_void_p(psi_ptr), int(M), _PREC[prec], int(site),
                                             lay, int(blocks), ctypes.c_void_p(out_ptr),
                                             ctypes.c_void_p(stream)))


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().spinrp_launch_count())


# ---------------------------------------------------------------------------
# systems
# ---------------------------------------------------------------------------
def system_create(J, htype: int, a_generic=None) -> ctypes.c_void_p:
    J = np.ascontiguousarray(J, dtype=np.float64)
    M = J.shape[0]
    a = None if a_generic is None else np.ascontiguousarray(a_generic, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib().spinrp_system_create(M, _dp(J), int(htype), None if a is None else _dp(a),
                                      ctypes.byref(h)))
    return h


class System:
    """A spin system (couplings + sweep plan), host side."""

    def __init__(self, J, htype: int, a_generic=None, _handle=None):
        if _handle is None:
            self._h = system_create(J, htype, a_generic)
            self.J = np.array(J, dtype=np.float64)
        else:
            self._h = _handle
            self.J = np.array(J, dtype=np.float64)
        self.htype = int(htype)

    @classmethod
    def ladder(cls, L: int, j_leg: float = 1.0, j_rung: float = 0.5) -> "System":
        """spinrp_ladder_create: the open 2 x L XY ladder."""
        h = ctypes.c_void_p()
        _check(lib().spinrp_ladder_create(int(L), float(j_leg), float(j_rung), ctypes.byref(h)))
        sysm = cls(np.zeros((1, 1)), XY, _handle=h)
        sysm.J = sysm.couplings()[1]
        return sysm

    @classmethod
    def star_dipolar(cls, M: int, geom_seed: int, rmin: float = 0.1) -> "System":
        """spinrp_star_dipolar_create: the truncated dipolar star built in the library."""
        h = ctypes.c_void_p()
        _check(lib().spinrp_star_dipolar_create(int(M), int(geom_seed) & (2**64 - 1), float(rmin),
                                                ctypes.byref(h)))
        sysm = cls(np.zeros((1, 1)), DIPOLAR, _handle=h)
        sysm.J = -sysm.couplings()[1]  # b = -J
        return sysm

    def couplings(self) -> tuple[np.ndarray, np.ndarray]:
        """(a, b): the S^zS^z and flip-flop coupling matrices of H."""
        M = self.M
        a = np.empty((M, M))
        b = np.empty((M, M))
        _check(lib().spinrp_system_couplings(self._h, _dp(a), _dp(b)))
        return a, b

    def schedule(self) -> list[int]:
        """Order of the forward half step's bonds (indices into bonds())."""
        n = ctypes.c_int()
        _check(lib().spinrp_schedule(self._h, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_int32 * max(n.value, 1))()
        _check(lib().spinrp_schedule(self._h, buf, n.value, ctypes.byref(n)))
        return [buf[k] for k in range(n.value)]

    @property
    def handle(self):
        return self._h

    @property
    def M(self) -> int:
        return lib().spinrp_system_num_spins(self._h)

    def bonds(self) -> list[tuple[int, int]]:
        n = ctypes.c_int()
        _check(lib().spinrp_system_bonds(self._h, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_int32 * (2 * max(n.value, 1)))()
        _check(lib().spinrp_system_bonds(self._h, buf, n.value, ctypes.byref(n)))
        return [(buf[2 * k], buf[2 * k + 1]) for k in range(n.value)]

    def set_tile(self, prec, K: int):
        _check(lib().spinrp_system_set_tile(self._h, _PREC[prec], int(K)))

    def set_regbits(self, rb: int):
        """Register bits per phase of the complex64 kernel (5 or 6; 0 = default)."""
        _check(lib().spinrp_system_set_regbits(self._h, int(rb)))

    def set_orientation(self, mode: int):
        """1: complex64 states of a bipartite system are stored oriented (see
        include/spinrp.h); 0 (default): always plainly."""
        _check(lib().spinrp_system_set_orientation(self._h, int(mode)))

    def orientation(self, prec="c64") -> int:
        """First-colour mask a state of this precision would be oriented with
        (0: stored plainly); host only."""
        m = ctypes.c_uint64()
        _check(lib().spinrp_system_orientation(self._h, _PREC[prec], ctypes.byref(m)))
        return int(m.value)

    def plan_info(self, prec="c64") -> dict:
        s, w, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().spinrp_system_plan_info(self._h, _PREC[prec], ctypes.byref(s), ctypes.byref(w),
                                             ctypes.byref(k)))
        return {"segments": s.value, "sweeps_per_step": w.value, "K": k.value}

    def plan_gates(self, prec="c64"):
        n = ctypes.c_int()
        _check(lib().spinrp_system_plan_gates(self._h, _PREC[prec], None, None, 0, ctypes.byref(n)))
        m = max(n.value, 1)
        pairs, seg = (ctypes.c_int32 * (2 * m))(), (ctypes.c_int32 * m)()
        _check(lib().spinrp_system_plan_gates(self._h, _PREC[prec], pairs, seg, n.value, ctypes.byref(n)))
        return [((pairs[2 * k], pairs[2 * k + 1]), seg[k]) for k in range(n.value)]

    def plan_check(self, prec="c64") -> dict:
        """Host self-check of the device program; raises on a mismatch."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().spinrp_system_plan_check(self._h, _PREC[prec], ctypes.byref(a), ctypes.byref(b)))
        return {"phases_per_sweep": a.value, "gates_per_phase": b.value}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.spinrp_system_destroy(h)
            self._h = None


def state_bytes(system: System, prec, series_cap: int) -> tuple[int, int]:
    p, w = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().spinrp_state_bytes(system.handle, _PREC[prec], int(series_cap), ctypes.byref(p),
                                    ctypes.byref(w)))
    return p.value, w.value


class State:
    """One device-resident state and its FP64 P(t)/norm series.

    Device memory comes from PyTorch (``alloc="torch"``, default) or from the
    library's own cudaMalloc (``alloc="library"``)."""

    def __init__(self, system: System, prec="c64", series_cap: int = 1024, stream=None,
                 alloc: str = "torch"):
        self.system = system
        self.prec = _PREC[prec]
        self.M = system.M
        psi_b, work_b = state_bytes(system, self.prec, series_cap)
        self._bufs = []
        psi_ptr = work_ptr = None
        if stream is None or alloc == "torch":
            import torch
            if not torch.cuda.is_available():
                raise SpinrpError(ECUDA, "no CUDA device available")
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
            if alloc == "torch":
                psi = torch.empty(psi_b, dtype=torch.uint8, device="cuda")
                work = torch.empty(work_b, dtype=torch.uint8, device="cuda")
                self._bufs = [psi, work]
                psi_ptr, work_ptr = psi.data_ptr(), work.data_ptr()
        self.stream = int(stream) if stream is not None else 0
        h = ctypes.c_void_p()
        _check(lib().spinrp_state_create(system.handle, self.prec, ctypes.c_void_p(self.stream),
                                         int(series_cap), ctypes.c_void_p(psi_ptr),
                                         ctypes.c_void_p(work_ptr), ctypes.byref(h)))
        self._h = h
        self.psi_bytes, self.work_bytes = psi_b, work_b

    @property
    def handle(self):
        return self._h

    def init_random_phase(self, seed: int):
        _check(lib().spinrp_state_init_random_phase(self._h, int(seed) & (2**64 - 1)))
        return self

    def init_product_phase(self, seed: int):
        """The paper's product (unentangled) random state: M-1 phases."""
        _check(lib().spinrp_state_init_product_phase(self._h, int(seed) & (2**64 - 1)))
        return self

    def load(self, amps: np.ndarray):
        a = np.ascontiguousarray(np.asarray(amps, dtype=np.complex128)).view(np.float64)
        assert a.size == 2 << self.M
        _check(lib().spinrp_state_load(self._h, _dp(a)))
        return self

    def evolve(self, dt: float, steps: int, order: int = 2):
        _check(lib().spinrp_evolve(self._h, float(dt), int(steps), int(order)))
        return self

    def series_length(self) -> int:
        return int(lib().spinrp_series_length(self._h))

    def set_sites(self, all_sites: bool = True):
        """All-site readout from the next init / load on."""
        _check(lib().spinrp_state_set_sites(self._h, 1 if all_sites else 0))
        return self

    def site_series(self) -> np.ndarray:
        """(len, M) array: P_{q1}(t_k) of every spin q."""
        n = self.series_length()
        out = np.empty((max(n, 1), self.M), dtype=np.float64)
        got = ctypes.c_int64()
        _check(lib().spinrp_site_series(self._h, _dp(out), n, ctypes.byref(got)))
        return out[:got.value]

    def polarization(self, site: int = 1) -> np.ndarray:
        n = self.series_length()
        out = np.empty(max(n, 1), dtype=np.float64)
        got = ctypes.c_int64()
        _check(lib().spinrp_polarization(self._h, int(site), _dp(out), n, ctypes.byref(got)))
        return out[:got.value]

    def sector_norms(self) -> np.ndarray:
        """Weights of the total-S^z sectors, k = 0..M spins up (FP64)."""
        out = np.zeros(self.M + 1)
        n = ctypes.c_int()
        _check(lib().spinrp_sector_norms(self._h, _dp(out), self.M + 1, ctypes.byref(n)))
        return out

    def norm_series(self) -> np.ndarray:
        n = self.series_length()
        out = np.empty(max(n, 1), dtype=np.float64)
        got = ctypes.c_int64()
        _check(lib().spinrp_norm_series(self._h, _dp(out), n, ctypes.byref(got)))
        return out[:got.value]

    def read(self, idx) -> np.ndarray:
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        out = np.empty(2 * idx.size, dtype=np.float64)
        _check(lib().spinrp_state_read(self._h, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       idx.size, _dp(out)))
        return out.view(np.complex128)

    def amplitudes(self) -> np.ndarray:
        """All 2^M amplitudes in logical order (complex128)."""
        return self.read(np.arange(1 << self.M, dtype=np.int64))

    def layout(self) -> list[int]:
        lay = (ctypes.c_int32 * self.M)()
        p = ctypes.c_void_p()
        _check(lib().spinrp_state_layout(self._h, lay, ctypes.byref(p)))
        return list(lay)

    def orientation(self) -> int:
        """Mask of first-colour spins (bit q-1 = spin q) of an oriented state,
        whose amplitudes with an odd number of them up are stored (Im, Re);
        0 for a plainly stored state."""
        m = ctypes.c_uint64()
        _check(lib().spinrp_state_orientation(self._h, ctypes.byref(m)))
        return int(m.value)

    def set_pipeline(self, on: bool = True):
        """Pipelined sweeps (one persistent launch per sweep, producer and
        compute warpgroups) where the plan takes them (True, the default), or
        one tile per block (False); the results are the same bit for bit."""
        _check(lib().spinrp_state_set_pipeline(self._h, int(bool(on))))
        return self

    def pipeline(self) -> bool:
        """True when the state's sweeps run pipelined."""
        on = ctypes.c_int()
        _check(lib().spinrp_state_pipeline(self._h, ctypes.byref(on)))
        return bool(on.value)

    def pipeline_timeout_check(self) -> tuple[int, float]:
        """Diagnostic: a pipelined launch whose waits all run out (see
        include/spinrp.h); returns (status code, launch seconds)."""
        sec = ctypes.c_double()
        rc = lib().spinrp_state_pipeline_timeout_check(self._h, ctypes.byref(sec))
        return rc, sec.value

    def device_ptr(self) -> int:
        """Device address of the amplitude buffer."""
        p = ctypes.c_void_p()
        _check(lib().spinrp_state_layout(self._h, None, ctypes.byref(p)))
        return int(p.value)

    def profile(self, enable: bool = True):
        _check(lib().spinrp_profile(self._h, int(bool(enable))))

    def profile_read(self, kind: int = KERNEL_SWEEP) -> tuple[float, int]:
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib().spinrp_profile_read(self._h, int(kind), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def transfer_bytes(self) -> tuple[int, int]:
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().spinrp_state_transfer_bytes(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.spinrp_state_destroy(h)
        self._h = None
        self._bufs = []

    def __del__(self):
        self.close()


def run_job(J, htype: int, seed: int, dt: float, steps: int, prec="c64", a_generic=None,
            tile_K: int | None = None):
    """Whole job through the C ABI: returns (P[0..steps], norm[0..steps], state)."""
    sysm = System(J, htype, a_generic)
    if tile_K:
        sysm.set_tile(prec, tile_K)
    st = State(sysm, prec, series_cap=steps + 1)
    st.init_random_phase(seed).evolve(dt, steps)
    return st.polarization(1), st.norm_series(), st


def polarized_at(J, m: int, a_generic=None):
    """Couplings relabelled so that spin m (1-based) becomes spin 1, the spin
    the random-phase state polarizes: returns (J', a', order) with
    J'[i, j] = J[order[i], order[j]], order[0] = m - 1 and the other spins in
    their original order.  A state of the relabelled system gives the paper's
    W_{m'm} / P_{m'm}(t) (Eq. 2) for a general initially polarized spin m:
    its spin q is original spin order[q - 1] + 1."""
    J = np.asarray(J, dtype=np.float64)
    M = J.shape[0]
    if not 1 <= m <= M:
        raise SpinrpError(EINVAL, f"polarized_at: m={m} outside 1..{M}")
    order = np.array([m - 1] + [q for q in range(M) if q != m - 1])
    A = None if a_generic is None else np.asarray(a_generic, dtype=np.float64)[np.ix_(order, order)]
    return J[np.ix_(order, order)], A, order


def autotune(system: System, prec="c64", candidates=None, probe_steps: int = 4, dt: float = 0.02,
             seed: int = 1, repeats: int = 2) -> dict:
    """Pick the tile width K (and, for complex64, the register bits rb) for
    `system` by timing `probe_steps` Trotter steps of each candidate on the
    device (CUDA events, best of `repeats`), then set the winner with
    spinrp_system_set_tile / spinrp_system_set_regbits.  `candidates` is a
    list of K or of (K, rb) pairs (rb 0 = the library's default for K).
    Returns {"K": best K, "rb": best rb, "ms_per_step": {(K, rb): ms}}."""
    import torch
    p = _PREC[prec]
    M = system.M
    if candidates is None:
        kmax = 14 if p == C64 else 13
        ks = [k for k in range(max(2, min(M, kmax) - 4), min(M, kmax) + 1)]
        candidates = [(k, rb) for k in ks for rb in ((5, 6) if p == C64 and k >= 11 else (0,))]
    cands = [c if isinstance(c, tuple) else (int(c), 0) for c in candidates]
    timings = {}
    for K, rb in cands:
        system.set_tile(p, K)
        if p == C64:
            system.set_regbits(rb)
        st = State(system, p, series_cap=1 + (repeats + 1) * probe_steps)
        st.init_random_phase(seed)
        st.evolve(dt, probe_steps)  # warm-up
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st.evolve(dt, probe_steps)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / probe_steps)
        timings[(K, rb)] = best
        st.close()
    K_best, rb_best = min(timings, key=timings.get)
    system.set_tile(p, K_best)
    if p == C64:
        system.set_regbits(rb_best)
    return {"K": K_best, "rb": rb_best, "ms_per_step": timings}


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------
_BATCH_SIG = {
    "spinrp_batch_create": ([ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_uint64),
                             ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
                            ctypes.c_int),
    "spinrp_batch_destroy": ([ctypes.c_void_p], None),
    "spinrp_batch_info": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)],
                          ctypes.c_int),
    "spinrp_batch_init_random_phase": ([ctypes.c_void_p], ctypes.c_int),
    "spinrp_batch_init_product_phase": ([ctypes.c_void_p], ctypes.c_int),
    "spinrp_batch_evolve": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int], ctypes.c_int),
    "spinrp_batch_set_persistent": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "spinrp_batch_set_pipeline": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "spinrp_batch_pipeline": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "spinrp_batch_persist_timeout_check": ([ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)],
                                           ctypes.c_int),
    "spinrp_batch_polarization": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "spinrp_batch_ensemble": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
}


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_sig", False):
        for name, (args, res) in _BATCH_SIG.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        L._batch_sig = True
    return L


class Batch:
    """Many independent jobs (systems + phase seeds) evolved together; the
    N_alpha realizations of the paper's Eq. 4.  Device memory is allocated by
    the library."""

    def __init__(self, systems: list, seeds, prec="c64", series_cap: int = 1024, stream=None):
        L = _batch_lib()
        n = len(systems)
        self.systems = list(systems)  # keep the handles alive while creating
        hs = (ctypes.c_void_p * n)(*[s.handle.value for s in systems])
        sd = (ctypes.c_uint64 * n)(*[int(x) & (2**64 - 1) for x in seeds])
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        _check(L.spinrp_batch_create(n, hs, sd, _PREC[prec], int(series_cap), ctypes.c_void_p(int(stream)),
                                     ctypes.byref(h)))
        self._h = h
        self.n = n

    def info(self) -> dict:
        bts, g = ctypes.c_size_t(), ctypes.c_int()
        _check(_batch_lib().spinrp_batch_info(self._h, ctypes.byref(bts), ctypes.byref(g)))
        return {"device_bytes": bts.value, "groups": g.value}

    def set_persistent(self, on: bool = True):
        """Multi-tile groups in one persistent launch per evolve call (True)
        or one launch per sweep (False, the default)."""
        _check(_batch_lib().spinrp_batch_set_persistent(self._h, int(bool(on))))
        return self

    def set_pipeline(self, on: bool = True):
        """Pipelined sweeps for the multi-tile groups that take them (True,
        the default) or one tile per block (False); same results bit for bit."""
        _check(_batch_lib().spinrp_batch_set_pipeline(self._h, int(bool(on))))
        return self

    def pipeline_groups(self) -> int:
        """Number of plan groups whose sweeps run pipelined."""
        n = ctypes.c_int()
        _check(_batch_lib().spinrp_batch_pipeline(self._h, ctypes.byref(n)))
        return n.value

    def persist_timeout_check(self, steps: int = 4) -> tuple[int, float]:
        """Diagnostic: a persistent launch whose waits all run out (see
        include/spinrp.h); returns (status code, launch seconds)."""
        sec = ctypes.c_double()
        rc = _batch_lib().spinrp_batch_persist_timeout_check(self._h, int(steps), ctypes.byref(sec))
        return rc, sec.value

    def init_random_phase(self):
        _check(_batch_lib().spinrp_batch_init_random_phase(self._h))
        return self

    def init_product_phase(self):
        _check(_batch_lib().spinrp_batch_init_product_phase(self._h))
        return self

    def evolve(self, dt: float, steps: int, order: int = 2):
        _check(_batch_lib().spinrp_batch_evolve(self._h, float(dt), int(steps), int(order)))
        return self

    def polarization(self, job: int) -> np.ndarray:
        n = ctypes.c_int64()
        _check(_batch_lib().spinrp_batch_polarization(self._h, int(job), None, 0, ctypes.byref(n)))
        out = np.empty(max(n.value, 1), dtype=np.float64)
        _check(_batch_lib().spinrp_batch_polarization(self._h, int(job), _dp(out), n.value, ctypes.byref(n)))
        return out[:n.value]

    def ensemble(self) -> tuple[np.ndarray, np.ndarray]:
        """(mean, standard deviation) over jobs of P(t_k), reduced on the device."""
        n = ctypes.c_int64()
        _check(_batch_lib().spinrp_batch_ensemble(self._h, None, None, 0, ctypes.byref(n)))
        mean = np.empty(max(n.value, 1))
        std = np.empty(max(n.value, 1))
        _check(_batch_lib().spinrp_batch_ensemble(self._h, _dp(mean), _dp(std), n.value, ctypes.byref(n)))
        return mean[:n.value], std[:n.value]

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.spinrp_batch_destroy(h)
        self._h = None

    def __del__(self):
        self.close()


def autotune_batch(systems: list, seeds, candidates=(13, 14), probe_steps: int = 20, dt: float = 0.02,
                   min_M: int = 15, repeats: int = 1) -> dict:
    """Pick the common tile width of a batch's multi-tile groups (systems of
    at least min_M spins, six register bits: the persistent launch's tiles)
    by timing `probe_steps` Trotter steps of the whole batch per candidate on
    the device (CUDA events, after a warm-up call of the same length that
    also plans and captures), then set the winner on those systems.  Returns
    {"K": best K, "ms_per_step": {K: ms}}."""
    import torch
    big = [s for s in systems if s.M >= min_M]
    timings = {}
    for K in candidates:
        for s in big:
            s.set_tile(C64, min(K, s.M))
            s.set_regbits(6)
        b = Batch(systems, seeds, "c64", series_cap=1 + (repeats + 1) * probe_steps)
        b.init_random_phase().evolve(dt, probe_steps)
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.evolve(dt, probe_steps)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / probe_steps)
        timings[K] = best
        b.close()
    K_best = min(timings, key=timings.get)
    for s in big:
        s.set_tile(C64, min(K_best, s.M))
        s.set_regbits(6)
    return {"K": K_best, "ms_per_step": timings}

