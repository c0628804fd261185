"""Host-side model of the row-barrier protocol of the two tile marches.

Both marches (the plain march for P <= 4 and the long-split march for MHD-GLM)
hand the x neighbours' f*_1 / f*_2 of a row to each other through three
shared-memory row buffers, ordered by one mbarrier with a thread count of the
block: a thread arrives once per row iteration and waits on the previous
iteration's phase only where it next reads the other threads' values.  A race
or a lost phase there shows on the GPU only by chance (or as a bounded wait
giving up), so this test runs the protocol itself under many random thread
schedules, with the mbarrier's semantics as PTX defines them: an arrival
decrements the pending count, the phase completes when it reaches zero, and
`try_wait.parity(p)` succeeds iff the current phase's parity differs from p
(it cannot tell phase k from k - 2).

Every read of a neighbour's buffer slot must see the row the reader expects
(so no writer overwrote it early and no reader ran before the write), and every
schedule must finish (no thread waits on a phase that has aliased).  Two
variants are negative controls, which the model must find schedules to break:
the long-split march also arriving after the ring row behind the tile (two
arrivals before the first wait), and the plain march with the wait skipped by
threads without a column.
"""
import random

import pytest


class MBarrier:
    def __init__(self, count):
        self.count = count
        self.pending = count
        self.phase = 0

    def arrive(self):
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def try_wait_parity(self, parity):
        return (self.phase & 1) != parity


def plain_march(tx, act, h, wait_if_active_only=False):
    """Ops of one thread of the plain march (rows 0 .. h-1): iteration r waits
    for phase r - 1 (r > 0), reads row r from buffer r mod 3, writes row r + 1
    into buffer (r + 1) mod 3, then arrives.  Row 0 is written in the prologue,
    published by a block barrier.  ``wait_if_active_only``: threads without a
    column skip the wait but still arrive (the form with the wait inside the
    column's branch)."""
    ops = []
    if act:
        ops.append(("write", 0, 0))
    ops.append(("sync",))
    for r in range(h):
        if r > 0 and (act or not wait_if_active_only):
            ops.append(("wait", (r - 1) & 1))
        if act:
            ops.append(("read", r % 3, r))
            if r + 1 < h:
                ops.append(("write", (r + 1) % 3, r + 1))
        ops.append(("arrive",))
    return ops


def long_split_march(tx, act, h, buggy=False):
    """Ops of one thread of the long-split march (rows -1 .. h, the ring rows
    behind and ahead included): iteration r writes row r (0 <= r < h) into
    buffer r mod 3 after its split, then for r >= 1 waits for the phase of
    iteration r - 1 and reads row r - 1 from buffer (r - 1) mod 3, then
    arrives (from iteration 0 on).  ``buggy``: arrives from iteration -1 on and
    waits on phase r (parity r & 1), the form that let a thread run two phases
    ahead."""
    ops = [("sync",)]   # after the barrier's initialisation and the x ring
    for r in range(-1, h + 1):
        if act and 0 <= r < h:
            ops.append(("write", r % 3, r))
        if r >= 1:
            ops.append(("wait", (r & 1) if buggy else ((r - 1) & 1)))
            if act:
                ops.append(("read", (r - 1) % 3, r - 1))
        if buggy or r >= 0:
            ops.append(("arrive",))
    return ops


def run(programs, nthreads, nact, rng, bias):
    """Runs the threads' ops under a random schedule; returns None, or the first
    violation ("stale read ...", "deadlock")."""
    buf = [[None] * nthreads for _ in range(3)]
    bar = MBarrier(nthreads)
    pc = [0] * nthreads
    at_sync = set()
    weights = [bias ** rng.random() for _ in range(nthreads)]   # per-thread speed
    while True:
        live = [t for t in range(nthreads) if pc[t] < len(programs[t])]
        if not live:
            return None
        runnable = []
        for t in live:
            op = programs[t][pc[t]]
            if op[0] == "wait" and not bar.try_wait_parity(op[1]):
                continue
            if op[0] == "sync" and t in at_sync:
                continue
            runnable.append(t)
        if not runnable:
            return "deadlock"
        t = rng.choices(runnable, weights=[weights[u] for u in runnable])[0]
        op = programs[t][pc[t]]
        kind = op[0]
        if kind == "write":
            buf[op[1]][t] = op[2]
        elif kind == "read":
            for u in (t - 1, t + 1):
                if 0 <= u < nact and buf[op[1]][u] != op[2]:
                    return f"stale read: thread {t} wanted row {op[2]} of thread {u}, saw {buf[op[1]][u]}"
        elif kind == "arrive":
            bar.arrive()
        elif kind == "sync":
            at_sync.add(t)
            if len(at_sync) == nthreads:
                # everyone at the block barrier: all move past it
                for u in range(nthreads):
                    pc[u] += 1
                at_sync.clear()
            continue
        pc[t] += 1


def cases(seed0, n):
    rng = random.Random(seed0)
    for i in range(n):
        nthreads = rng.randint(2, 6)
        nact = rng.randint(1, nthreads)   # columns of a ragged tile
        h = rng.randint(1, 6)
        bias = rng.choice([1.0, 10.0, 1000.0])
        yield nthreads, nact, h, bias, random.Random(seed0 * 100003 + i)


@pytest.mark.parametrize("march", ["plain", "long_split"])
def test_row_barrier_protocol_has_no_race_or_lost_phase(march):
    for nthreads, nact, h, bias, rng in cases(7 if march == "plain" else 11, 3000):
        if march == "plain":
            progs = [plain_march(t, t < nact, h) for t in range(nthreads)]
        else:
            progs = [long_split_march(t, t < nact, h) for t in range(nthreads)]
        err = run(progs, nthreads, nact, rng, bias)
        assert err is None, f"{march}: {err} (threads {nthreads}, active {nact}, rows {h})"


def test_model_catches_two_arrivals_before_the_first_wait():
    """Negative control: the long-split march arriving after the ring row
    behind the tile too (and waiting on phase r) loses a phase or reads stale
    rows under some schedules; threads without a column, which skip the split,
    are the ones that race ahead."""
    found = []
    for nthreads, nact, h, bias, rng in cases(13, 3000):
        progs = [long_split_march(t, t < nact, h, buggy=True) for t in range(nthreads)]
        err = run(progs, nthreads, nact, rng, bias)
        if err is not None:
            found.append(err)
    assert found, "the model found no failure of the two-arrival form"


def test_model_catches_a_wait_skipped_by_threads_without_a_column():
    """Negative control: in the plain march, threads without a column that
    arrive without waiting can arrive twice in one phase."""
    found = []
    for nthreads, nact, h, bias, rng in cases(17, 3000):
        progs = [plain_march(t, t < nact, h, wait_if_active_only=True) for t in range(nthreads)]
        err = run(progs, nthreads, nact, rng, bias)
        if err is not None:
            found.append(err)
    assert found, "the model found no failure of the skipped wait"
