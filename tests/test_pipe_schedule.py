"""Host model of the pipelined sweep's hand-over protocol (no GPU).

pipe_kernel gives block b the units b, b + G, b + 2G, ... (local unit i in
tile buffer i mod 3, computed by group i mod 2).  The producer, at its step
i, waits for done[i mod 3] of unit i - 3 (parity ((i - 3) / 3) & 1), writes
that unit back, then gathers unit i and arrives on full[i mod 3]; group g
waits on full[i mod 3] with parity (i / 3) & 1 for each of its units i and
arrives on done[i mod 3] when finished.  An mbarrier wait on parity p
returns once the phase of that parity has completed, i.e. while the number
of completed phases c satisfies c mod 2 != p -- so a waiter two phases
behind would be released by the wrong phase.

This model runs the three agents of one block in random interleavings and
checks, at every wait that returns, that the completed-phase count is
exactly the one the waiter means (no aliasing), that every unit is gathered,
computed and written back exactly once and in that order, that a buffer is
never refilled before its previous unit was written back, and that the
agents always finish (no deadlock).
"""
import random

import pytest


def _units(b, G, nunits):
    return list(range(b, nunits, G))


class _Barrier:
    def __init__(self):
        self.completed = 0  # phases completed

    def ready(self, parity):
        return self.completed % 2 != parity


def _run_block(nloc, rng):
    full = [_Barrier() for _ in range(3)]
    done = [_Barrier() for _ in range(3)]
    log = []  # (event, local unit)
    buf_owner = [None] * 3  # local unit whose data is in the buffer
    state = {"p": 0, "g": [0, 1]}

    def producer_step():
        i = state["p"]
        if i >= nloc + 3:
            return None
        b = i % 3
        if i >= 3:
            j = i - 3
            par = (j // 3) & 1
            if not done[b].ready(par):
                return False
            # the wait returned: exactly j // 3 + 1 phases of done[b] completed
            assert done[b].completed == j // 3 + 1, ("done aliasing", i, done[b].completed)
            assert buf_owner[b] == j
            log.append(("store", j))
            buf_owner[b] = None
        if i < nloc:
            assert buf_owner[b] is None, ("refill before write-back", i)
            buf_owner[b] = i
            log.append(("load", i))
            full[b].completed += 1
        state["p"] = i + 1
        return True

    def group_step(g):
        i = state["g"][g]
        if i >= nloc:
            return None
        b = i % 3
        par = (i // 3) & 1
        if not full[b].ready(par):
            return False
        assert full[b].completed == i // 3 + 1, ("full aliasing", g, i, full[b].completed)
        assert buf_owner[b] == i
        log.append(("compute", i))
        done[b].completed += 1
        state["g"][g] = i + 2
        return True

    agents = [producer_step, lambda: group_step(0), lambda: group_step(1)]
    for _ in range(100 * (nloc + 3) + 100):
        live = [a for a in agents]
        rng.shuffle(live)
        progressed = False
        finished = 0
        for a in live:
            r = a()
            if r is None:
                finished += 1
            elif r:
                progressed = True
                break
        if finished == len(agents):
            return log
        assert progressed, "deadlock: no agent can move"
    raise AssertionError("did not finish")


@pytest.mark.parametrize("nunits,G", [(1024, 152), (8192, 152), (608, 152), (131072, 152), (41 * 512, 152),
                                      (7, 2), (3, 1), (4, 1), (5, 3)])
def test_pipe_schedule_covers_units_once_and_never_aliases(nunits, G):
    rng = random.Random(nunits * 131 + G)
    seen = {"load": [], "compute": [], "store": []}
    blocks = range(G) if G <= 8 else rng.sample(range(G), 6)
    for b in blocks:
        units = _units(b, G, nunits)
        if len(units) > 300:  # the protocol repeats with period 6 in i; a prefix covers every residue
            units = units[:300]
        log = _run_block(len(units), rng)
        per = {"load": [], "compute": [], "store": []}
        for ev, i in log:
            per[ev].append(i)
        n = len(units)
        assert sorted(per["load"]) == list(range(n))
        assert sorted(per["compute"]) == list(range(n))
        assert sorted(per["store"]) == list(range(n))
        # each unit: gathered, then computed, then written back
        pos = {(ev, i): k for k, (ev, i) in enumerate(log)}
        for i in range(n):
            assert pos[("load", i)] < pos[("compute", i)] < pos[("store", i)]
        # group g computes units i = g mod 2, in order
        comp = [i for ev, i in log if ev == "compute"]
        for g in (0, 1):
            mine = [i for i in comp if i % 2 == g]
            assert mine == sorted(mine)
        for ev in seen:
            seen[ev] += [units[i] for i in per[ev]]
    if G <= 8:
        # every unit of the sweep exactly once over all blocks
        assert sorted(seen["compute"]) == list(range(nunits))


def test_pipe_schedule_units_partition_the_sweep():
    """Blocks' unit sets b, b + G, ... partition 0..nunits-1 (tiles of one job,
    or (job, tile) pairs job-major), with per-block counts as the kernel
    computes them: (nunits - 1 - b) // G + 1."""
    for nunits, G in ((1024, 152), (131072, 152), (608, 152), (41 * 512, 152), (2048 * 3, 152)):
        allu = []
        for b in range(G):
            u = _units(b, G, nunits)
            assert len(u) == ((nunits - 1 - b) // G + 1 if b < nunits else 0)
            allu += u
        assert sorted(allu) == list(range(nunits))
