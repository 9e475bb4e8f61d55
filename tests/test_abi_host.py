"""Host-side tests of the C-ABI library (no GPU needed).

* the library loads and exports every entry point that include/spinrp.h declares;
* spin systems: Hamiltonian families, canonical bond order (checked against
  the oracle's definition), argument validation;
* the sweep plan: the device gate order is the canonical one up to exchanges
  of gates on disjoint spins (per-spin gate sequences identical), every gate
  appears exactly once, and the sweep counts are as designed.
"""
import re
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_0710_3747_gb300 import build, spinrp
from paper_0710_3747_gb300 import workloads as W

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _declared_symbols():
    text = (ROOT / "include" / "spinrp.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spinrp_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = spinrp.lib()
    syms = _declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(L, s), s
    assert "sm_103a" in spinrp.version()


def _systems():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(9, 9))
    A = A + A.T
    return [
        ("ladder14", W.ladder(7, 1.0, 0.5), spinrp.XY, None),
        ("ladder30", W.ladder(15, 1.0, 0.5), spinrp.XY, None),
        ("star20", W.star_dipolar(20, 2), spinrp.DIPOLAR, None),
        ("star22", W.star_dipolar(22, 9), spinrp.DIPOLAR, None),
        ("iso9", W.star_gaussian(9, 1), spinrp.ISOTROPIC, None),
        ("generic9", W.star_gaussian(9, 2), spinrp.GENERIC, A),
        ("chain24", W.chain(24, 1.0), spinrp.XY, None),
    ]


@pytest.mark.parametrize("name,J,htype,a", _systems(), ids=lambda v: v if isinstance(v, str) else "")
def test_bonds_are_canonical(name, J, htype, a):
    s = spinrp.System(J, htype, a)
    _, b = oracle.couplings(J, htype, a)
    want = [(i + 1, j + 1) for i, j in oracle.canonical_bonds(b)]
    assert s.bonds() == want


def _chains(gates, M):
    ch = [[] for _ in range(M + 1)]
    for i, j in gates:
        ch[i].append((i, j))
        ch[j].append((i, j))
    return ch


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("name,J,htype,a", _systems(), ids=lambda v: v if isinstance(v, str) else "")
def test_plan_is_canonical_up_to_disjoint_exchanges(name, J, htype, a, prec):
    s = spinrp.System(J, htype, a)
    M = s.M
    canon = s.bonds()
    plan = s.plan_gates(prec)
    gates = [g for g, _ in plan]
    segs = [k for _, k in plan]
    assert sorted(gates) == sorted(canon)           # each gate exactly once
    assert _chains(gates, M) == _chains(canon, M)   # same order on every spin
    assert segs == sorted(segs)                     # segments in sweep order
    info = s.plan_info(prec)
    assert info["segments"] == max(segs) + 1
    if M <= info["K"]:
        assert info["segments"] == 1 and info["sweeps_per_step"] == 1


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("K", list(range(2, 14)))
@pytest.mark.parametrize("kind", ["star16", "ladder12", "chain13", "generic11"])
def test_plan_every_tile_width(kind, K, prec):
    rng = np.random.default_rng(7)
    J, ht = {"star16": (W.star_dipolar(16, 5), spinrp.DIPOLAR),
             "ladder12": (W.ladder(6, 1.0, 0.5), spinrp.XY),
             "chain13": (W.chain(13), spinrp.XY),
             "generic11": (W.star_gaussian(11, 3), spinrp.ISOTROPIC)}[kind]
    s = spinrp.System(J, ht)
    s.set_tile(prec, K)
    info = s.plan_info(prec)
    assert info["K"] == min(K, s.M)
    gates = [g for g, _ in s.plan_gates(prec)]
    assert sorted(gates) == sorted(s.bonds())
    assert _chains(gates, s.M) == _chains(s.bonds(), s.M)
    spinrp.state_bytes(s, prec, 4)  # the sweep descriptors validate too


@pytest.mark.parametrize("K", [10, 11, 12, 13, 14])
@pytest.mark.parametrize("name,J,htype,a", _systems(), ids=lambda v: v if isinstance(v, str) else "")
def test_register_phase_programs(name, J, htype, a, K):
    """Every sweep's register-blocked program, run on a random host tile,
    equals the sweep's plain op list (gates, diagonal phase, reduction)."""
    s = spinrp.System(J, htype, a)
    s.set_tile("c64", K)
    st = s.plan_check("c64")
    if s.M >= 10:
        assert st["phases_per_sweep"] >= 1.0
        if s.bonds():
            assert 1.0 <= st["gates_per_phase"] <= 10.0


@pytest.mark.parametrize("K", [10, 11, 12, 13])
@pytest.mark.parametrize("name,J,htype,a", _systems(), ids=lambda v: v if isinstance(v, str) else "")
def test_register_phase_programs_c128(name, J, htype, a, K):
    """The complex128 register-blocked programs (five register bits, 16-byte
    slots): every index the kernel forms, replayed on the host, and every
    program against its sweep's plain op list."""
    s = spinrp.System(J, htype, a)
    s.set_tile("c128", K)
    st = s.plan_check("c128")
    if s.M >= 10:
        assert st["phases_per_sweep"] >= 1.0
        if s.bonds():
            assert 1.0 <= st["gates_per_phase"] <= 10.0
    else:
        assert st["phases_per_sweep"] == 0.0  # tiles below 10 bits run the plain kernel


def test_plan_sweep_counts():
    # 2x15 ladder, 13-spin tiles (the default for 2^30 complex64 amplitudes)
    # sharing 4 low bits: three segments -> four sweeps per step; the same at 14
    s = spinrp.System(W.ladder(15, 1.0, 0.5), spinrp.XY)
    assert s.plan_info("c64") == {"segments": 3, "sweeps_per_step": 4, "K": 13}
    s.set_tile("c64", 14)
    assert s.plan_info("c64") == {"segments": 3, "sweeps_per_step": 4, "K": 14}
    # M=20 dipolar star, 14-spin tiles: three segments
    s = spinrp.System(W.star_dipolar(20, 2), spinrp.DIPOLAR)
    s.set_tile("c64", 14)
    assert s.plan_info("c64")["segments"] <= 3


def test_default_tile_model():
    """Default complex64 tile width: sweeps per step x max(2^K, 2^M / 152),
    least cost among 14, 13, 12 spins, ties to 13 then 12 (values from the
    plan's own sweep counts), the 13-spin cost weighted by 0.5 where that plan
    runs as the pipelined sweep (at least 4 x 152 tiles: M >= 23); complex128:
    the widest K <= 12 leaving at least 128 tiles, at least 8."""
    def pick(J, ht):
        M = J.shape[0]
        if M <= 12:
            return M
        costs = {}
        for K in (13, 12, 14):
            if K > M:
                continue
            s = spinrp.System(J, ht)
            s.set_tile("c64", K)
            costs[K] = s.plan_info("c64")["sweeps_per_step"] * max(2.0 ** K, 2.0 ** M / 152)
            if K == 13 and 2.0 ** (M - 13) >= 4 * 152:
                costs[K] *= 0.5
        best = min(costs.values())
        return next(K for K in (13, 12, 14) if K in costs and costs[K] == best)
    cases = [(W.ladder(5), spinrp.XY, 10), (W.ladder(7), spinrp.XY, 12), (W.ladder(9), spinrp.XY, 12),
             (W.ladder(11), spinrp.XY, 13), (W.ladder(12), spinrp.XY, 13), (W.ladder(15), spinrp.XY, 13),
             (W.star_dipolar(16, 3), spinrp.DIPOLAR, 12), (W.star_dipolar(20, 2), spinrp.DIPOLAR, 12),
             (W.star_dipolar(22, 3), spinrp.DIPOLAR, 13), (W.star_dipolar(23, 3), spinrp.DIPOLAR, 13),
             (W.star_dipolar(24, 3), spinrp.DIPOLAR, 13), (W.star_dipolar(26, 3), spinrp.DIPOLAR, 13),
             (W.ladder(13), spinrp.XY, 13), (W.ladder(14), spinrp.XY, 13)]
    for J, ht, want in cases:
        s = spinrp.System(J, ht)
        assert s.plan_info("c64")["K"] == want == pick(J, ht)
        M = J.shape[0]
        assert s.plan_info("c128")["K"] == next((K for K in range(12, 7, -1) if M - K >= 7), min(8, M))


def test_tile_model_weights_only_pipelined_plans():
    """The 0.5 weight applies only where the 13-spin plan runs as the
    pipelined sweep: six register bits and enough tiles.  With five register
    bits forced, a 24-spin star and the 2x12 ladder go back to 14-spin tiles
    (fewer sweeps per step); a 22-spin star (512 tiles, fewer than 4 x 152)
    is not weighted either."""
    for J, ht, sweeps13 in ((W.star_dipolar(24, 3), spinrp.DIPOLAR, 12), (W.ladder(12), spinrp.XY, 4)):
        s = spinrp.System(J, ht)
        assert s.plan_info("c64") == {"segments": (sweeps13 + 2) // 2, "sweeps_per_step": sweeps13, "K": 13}
        s.set_regbits(5)
        assert s.plan_info("c64")["K"] == 14
    s = spinrp.System(W.star_dipolar(22, 3), spinrp.DIPOLAR)
    costs = {}
    for K in (13, 12, 14):
        t = spinrp.System(W.star_dipolar(22, 3), spinrp.DIPOLAR)
        t.set_tile("c64", K)
        costs[K] = t.plan_info("c64")["sweeps_per_step"] * max(2.0 ** K, 2.0 ** 22 / 152)
    best = min(costs.values())
    assert s.plan_info("c64")["K"] == next(K for K in (13, 12, 14) if costs[K] == best)


def test_plan_cache_keys():
    """Plans are cached by bond list, S^zS^z presence, precision and tile /
    register settings: systems with equal keys share a plan (schedule and
    sizes), and every key change gives the plan of its own settings."""
    a = spinrp.System(W.star_dipolar(16, 3), spinrp.DIPOLAR)
    b = spinrp.System(W.star_dipolar(16, 4), spinrp.DIPOLAR)  # other couplings, same bonds
    assert a.schedule() == b.schedule()
    assert spinrp.state_bytes(a, "c64", 100) == spinrp.state_bytes(b, "c64", 100)
    assert a.plan_check("c64") == b.plan_check("c64")
    # the XY form of the same couplings has no S^zS^z term: no diagonal phases
    c = spinrp.System(W.star_dipolar(16, 3), spinrp.XY)
    assert c.plan_check("c64")["phases_per_sweep"] < a.plan_check("c64")["phases_per_sweep"]
    for K in (11, 12, 13, 14):
        a.set_tile("c64", K)
        assert a.plan_info("c64")["K"] == K
        a.plan_check("c64")
    a.set_regbits(6)
    a.set_tile("c64", 12)
    r6 = a.plan_check("c64")
    a.set_regbits(5)
    assert a.plan_check("c64") != r6


def test_plan_cache_concurrent_threads():
    """Plans built and looked up from several host threads at once (the
    binding releases the GIL during library calls): sparse random graphs whose
    bond lists no other test uses, so the first lookups race to build; every
    thread must see the same plans, equal to a serial rebuild of the same
    systems."""
    import threading
    rng = np.random.default_rng(0xCAC4E)
    systems = []
    for M in (12, 13, 14, 15, 16, 17):
        J = rng.normal(size=(M, M)) * (rng.random((M, M)) < 0.3)
        J = np.triu(J, 1)
        J = J + J.T
        J[0, 1] = J[1, 0] = 1.0
        systems.append((J, spinrp.XY))
    results = [dict() for _ in range(6)]
    errors = []

    def worker(k):
        order = np.random.default_rng(k).permutation(len(systems))
        try:
            for i in order:
                J, ht = systems[i]
                s = spinrp.System(J, ht)
                results[k][i] = (spinrp.state_bytes(s, "c64", 50), s.plan_check("c64"),
                                 spinrp.state_bytes(s, "c128", 50))
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(6)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors[:3]
    for i, (J, ht) in enumerate(systems):
        s = spinrp.System(J, ht)
        want = (spinrp.state_bytes(s, "c64", 50), s.plan_check("c64"), spinrp.state_bytes(s, "c128", 50))
        assert all(r[i] == want for r in results), i


def test_state_bytes():
    s = spinrp.System(W.ladder(7, 1.0, 0.5), spinrp.XY)
    p64, w64 = spinrp.state_bytes(s, "c64", 401)
    p128, _ = spinrp.state_bytes(s, "c128", 401)
    assert p64 == 8 << 14 and p128 == 16 << 14
    assert w64 >= 16 * 401


@pytest.mark.parametrize("bad", [
    dict(J=np.zeros((1, 1)), htype=spinrp.XY),
    dict(J=np.zeros((35, 35)), htype=spinrp.XY),
    dict(J=np.zeros((4, 4)), htype=9),
    dict(J=np.zeros((4, 4)), htype=spinrp.GENERIC),
    dict(J=np.full((4, 4), np.nan), htype=spinrp.XY),
])
def test_system_create_rejects(bad):
    with pytest.raises(spinrp.SpinrpError) as e:
        spinrp.System(bad["J"], bad["htype"])
    assert e.value.code == spinrp.EINVAL


def test_set_tile_rejects():
    s = spinrp.System(W.ladder(3), spinrp.XY)
    with pytest.raises(spinrp.SpinrpError):
        s.set_tile("c64", 15)
    with pytest.raises(spinrp.SpinrpError):
        s.set_tile("c128", 14)


def test_hamiltonian_families_match_oracle_convention():
    # the library's (a, b) for each family reproduces the oracle's through the
    # bond list (b != 0 pattern) -- dipolar b = -J keeps every pair
    J = W.star_dipolar(6, 1)
    for ht in (spinrp.XY, spinrp.DIPOLAR, spinrp.ISOTROPIC):
        assert len(spinrp.System(J, ht).bonds()) == 15
    assert spinrp.System(J, spinrp.ISING).bonds() == []


@pytest.mark.parametrize("seed", range(12))
def test_register_programs_random_graphs(seed):
    """Random coupling graphs (sparse to dense, with and without S^zS^z
    terms), tile widths and register widths: the host replay of every index
    the register-blocked kernel forms and of every register program against
    its sweep's op list must pass (plan_check raises otherwise)."""
    rng = np.random.default_rng([0xF022, seed])
    M = int(rng.integers(11, 23))
    density = float(rng.uniform(0.1, 1.0))
    J = rng.normal(size=(M, M)) * (rng.random((M, M)) < density)
    J = np.triu(J, 1)
    J = J + J.T
    J[0, 1] = J[1, 0] = 1.0  # spin 1 always coupled
    htype = [spinrp.XY, spinrp.DIPOLAR, spinrp.ISOTROPIC][seed % 3]
    s = spinrp.System(J, htype)
    for K in sorted({int(rng.integers(10, min(M, 14) + 1)), min(M, 14)}):
        for rb in (5, 6):
            if K < 5 + rb:
                continue
            s.set_tile("c64", K)
            s.set_regbits(rb)
            st = s.plan_check("c64")
            assert st["phases_per_sweep"] >= 1.0
        if K <= 13:
            s.set_tile("c128", K)
            assert s.plan_check("c128")["phases_per_sweep"] >= 1.0


def test_ladder_constructor_matches_definition():
    for L, jl, jr in ((1, 1.0, 0.3), (4, 0.7, 0.2), (15, 1.0, 0.5)):
        s = spinrp.System.ladder(L, jl, jr)
        a, b = s.couplings()
        assert np.array_equal(b, W.ladder(L, jl, jr)) and not a.any()
        assert s.schedule() == list(range(len(s.bonds())))


def _star_from_recipe(M, seed, rmin):
    """The documented geometry recipe, replayed with the (separately pinned)
    Philox4x32-10 of the test oracle."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    u = lambda hi, lo: (((hi << 32) | lo) >> 11) * 2.0 ** -53
    pos = [np.zeros(3)]
    n = 0
    while len(pos) < M:
        a = oracle.philox4x32_10((n, 0, 0, 2), key)
        b = oracle.philox4x32_10((n, 1, 0, 2), key)
        n += 1
        p = np.array([2 * u(a[0], a[1]) - 1, 2 * u(a[2], a[3]) - 1, 2 * u(b[0], b[1]) - 1])
        if p @ p > 1.0 or min(np.linalg.norm(p - q) for q in pos) < rmin:
            continue
        pos.append(p)
    J = W.dipolar_from_positions(np.array(pos))
    return J


@pytest.mark.parametrize("M,seed,rmin", [(2, 1, 0.1), (9, 2**40 + 3, 0.1), (14, 7, 0.15)])
def test_star_constructor_matches_recipe(M, seed, rmin):
    s = spinrp.System.star_dipolar(M, seed, rmin)
    a, b = s.couplings()
    J = _star_from_recipe(M, seed, rmin)
    np.testing.assert_allclose(-b, J, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a, 2 * J, rtol=1e-12, atol=1e-12)
    iu = np.triu_indices(M, 1)
    assert abs(np.sqrt(np.mean(b[iu] ** 2)) - 1.0) < 1e-12
    if M > 2:  # two spins: J_12 = +-1 after the rms scaling for any geometry
        assert not np.array_equal(b, spinrp.System.star_dipolar(M, seed + 1, rmin).couplings()[1])


def test_constructors_reject_bad_arguments():
    for call in (lambda: spinrp.System.ladder(0), lambda: spinrp.System.ladder(18),
                 lambda: spinrp.System.star_dipolar(1, 1), lambda: spinrp.System.star_dipolar(40, 1),
                 lambda: spinrp.System.star_dipolar(8, 1, rmin=0.9)):
        with pytest.raises(spinrp.SpinrpError):
            call()


@pytest.mark.parametrize("name,J,htype,a,K,rb", [
    ("ladder30_K13", W.ladder(15, 1.0, 0.5), W.XY, None, 13, 6),
    ("ladder16_K12", W.ladder(8, 1.0, 0.5), W.XY, None, 12, 5),
    ("ladder16_K14", W.ladder(8, 1.0, 0.5), W.XY, None, 14, 6),
    ("ladder12_one_tile", W.ladder(6, 1.0, 0.3), W.XY, None, 12, 6),
    ("chain19_K11", W.chain(19, 0.8), W.XY, None, 11, 5),
    ("xy_ising_ladder16", W.ladder(8, 1.0, 0.6), W.GENERIC, 0.4 * W.ladder(8, 1.0, 1.0), 13, 6),
])
def test_oriented_register_programs(name, J, htype, a, K, rb):
    """Oriented programs (bipartite couplings, orientation requested): every
    phase holds its first-colour register bits first in an allowed count,
    every gate joins the two colours, and the packed arithmetic of the
    oriented kernel -- emulated in FP64 thread by thread and word by word,
    (Re, Im) / (Im, Re) words, sign pattern and conjugated diagonal phases --
    reproduces the plain program on a random tile for both orientations of
    the outer bits (spinrp_system_plan_check)."""
    s = spinrp.System(J, htype, a)
    s.set_tile("c64", K)
    s.set_regbits(rb)
    s.set_orientation(1)
    black = s.orientation("c64")
    assert black != 0
    for i, j in s.bonds():  # 1-based pairs: every bond joins the two colours
        assert ((black >> (i - 1)) & 1) != ((black >> (j - 1)) & 1)
    assert s.orientation("c128") == 0
    r = s.plan_check("c64")
    assert r["phases_per_sweep"] > 0
    # the same system with plain storage plans the same number of phases
    s.set_orientation(0)
    assert abs(s.plan_check("c64")["phases_per_sweep"] - r["phases_per_sweep"]) < 1.0


def test_orientation_setting_is_validated():
    s = spinrp.System(W.ladder(7), W.XY)
    with pytest.raises(spinrp.SpinrpError):
        s.set_orientation(2)
    assert s.orientation() == 0  # default: plain storage
    s.set_orientation(1)
    assert s.orientation() != 0
    star = spinrp.System(W.star_dipolar(14, 2), W.DIPOLAR)
    star.set_orientation(1)
    assert star.orientation() == 0  # not bipartite
