"""CPU model of the column-inverse kernel's mbarrier protocol (no GPU).

k_col_inverse hands data between warps with mbarriers and parity waits:
producers (units go round two issuing threads at FP32 storage, four at 16 bit)
stream units into a ring of S stages (full/empty barriers), a loader fills
two r slots, a manager prepares r and reduces partial sums, and C consumers
(8 at FP32, 12 at 16 bit) walk units g = warp, warp+C, ...  A parity wait is only exact
when the waiter is at most one phase ahead of the barrier.  This model runs
the same protocol under random timings and checks that every successful wait
is for data that has landed, that no copy is issued into a busy stage, that
every unit is processed exactly once and that nothing deadlocks.  It also
shows that assigning units by their index within a column (instead of across
columns) breaks the invariant.
"""
import random

import pytest


class Bar:
    """mbarrier: arrival count + transaction bytes; a phase completes when both reach 0."""

    def __init__(self, count):
        self.count = count
        self.pending = count
        self.phase = 0
        self.tx = 0

    def arrive(self):
        self.pending -= 1
        self._maybe()

    def expect_tx(self, b):
        self.tx += b
        self.arrive()

    def complete_tx(self, b):
        self.tx -= b
        assert self.tx >= 0, "transaction count underflow"
        self._maybe()

    def _maybe(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def try_wait(self, parity):
        return (self.phase & 1) != parity


def simulate(S, nunits, ncols, seed, W=8, per_column_mapping=False, producers=1):
    rnd = random.Random(seed)
    full = [Bar(1) for _ in range(S)]
    empty = [Bar(1) for _ in range(S)]
    landed, busy, inflight, processed = set(), [None] * S, [], set()
    rfull, rempty = [Bar(1), Bar(1)], [Bar(1), Bar(1)]
    rv_full, yc_empty, col_done = [Bar(1), Bar(1)], [Bar(1), Bar(1)], [Bar(W), Bar(W)]
    rinfl = []

    def consumer(w):
        u, st, ph = w, w, 0
        for n in range(ncols):
            bb = n & 1
            while not rv_full[bb].try_wait((n >> 1) & 1):
                yield
            if n >= 2:
                while not yc_empty[bb].try_wait(((n >> 1) - 1) & 1):
                    yield
            if per_column_mapping:          # the faulty assignment: unit index within the column
                for uu in range(w, nunits, W):
                    g = n * nunits + uu
                    while not full[g % S].try_wait((g // S) & 1):
                        yield
                    assert g in landed, f"wait passed for unit {g} before it landed"
                    processed.add(g)
                    busy[g % S] = None
                    empty[g % S].arrive()
            else:
                while u < nunits:
                    g = n * nunits + u
                    assert st == g % S and ph == (g // S) & 1
                    while not full[st].try_wait(ph):
                        yield
                    assert g in landed, f"wait passed for unit {g} before it landed"
                    processed.add(g)
                    for _ in range(rnd.randint(0, 3)):
                        yield
                    busy[st] = None
                    empty[st].arrive()
                    u += W
                    st += W
                    if st >= S:
                        st -= S
                        ph ^= 1
                u -= nunits
            col_done[bb].arrive()

    def producer(p):
        # producer p issues units g = p, p + P, ... into stage g mod S
        st, wraps = p, 0
        for g in range(p, ncols * nunits, producers):
            if wraps > 0:
                while not empty[st].try_wait((wraps - 1) & 1):
                    yield
            assert busy[st] is None, "copy issued into a stage still in use"
            assert g == wraps * S + st
            busy[st] = g
            full[st].expect_tx(1)
            inflight.append([rnd.randint(1, 30), st, g])
            st += producers
            if st >= S:
                st, wraps = st - S, wraps + 1
            yield

    def loader():
        for n in range(ncols):
            sl = n % 2
            if n >= 2:
                while not rempty[sl].try_wait(((n // 2) - 1) & 1):
                    yield
            rfull[sl].expect_tx(1)
            rinfl.append([rnd.randint(1, 20), sl])
            yield

    def manager():
        def prepare(n):
            while not rfull[n % 2].try_wait((n // 2) & 1):
                yield
            rempty[n % 2].arrive()
            rv_full[n & 1].arrive()
        for n in range(min(2, ncols)):
            yield from prepare(n)
        for n in range(ncols):
            while not col_done[n & 1].try_wait((n >> 1) & 1):
                yield
            for _ in range(rnd.randint(0, 5)):
                yield
            yc_empty[n & 1].arrive()
            if n + 2 < ncols:
                yield from prepare(n + 2)

    alive = [consumer(w) for w in range(W)] + [producer(p) for p in range(producers)] + [loader(), manager()]
    steps = 0
    while alive:
        steps += 1
        assert steps < 2_000_000, "no progress (deadlock)"
        for c in inflight[:]:
            c[0] -= 1
            if c[0] <= 0:
                inflight.remove(c)
                landed.add(c[2])
                full[c[1]].complete_tx(1)
        for c in rinfl[:]:
            c[0] -= 1
            if c[0] <= 0:
                rinfl.remove(c)
                rfull[c[1]].complete_tx(1)
        rnd.shuffle(alive)
        for gen in alive[:]:
            try:
                next(gen)
            except StopIteration:
                alive.remove(gen)
    assert processed == set(range(ncols * nunits))


@pytest.mark.parametrize("producers", [1, 2, 4])
@pytest.mark.parametrize("S", [8, 16, 24, 32])
@pytest.mark.parametrize("nunits", [1, 2, 3, 13, 32, 36])
def test_protocol_holds_for_ring_depths_multiple_of_8(S, nunits, producers):
    """FP32 storage: 8 consumer warps, two producers (units go round them)."""
    for ncols in (1, 2, 5):
        for seed in range(3):
            simulate(S, nunits, ncols, seed, producers=producers)


@pytest.mark.parametrize("S", [12, 24, 36])
@pytest.mark.parametrize("nunits", [1, 5, 13, 36, 78])
def test_protocol_holds_with_twelve_consumers(S, nunits):
    """16-bit storage: 12 consumer warps, four producers, S a multiple of 12."""
    for ncols in (1, 2, 5):
        for seed in range(3):
            simulate(S, nunits, ncols, seed, W=12, producers=4)


def test_per_column_unit_mapping_breaks_parity_waits():
    with pytest.raises(AssertionError, match="before it landed"):
        for seed in range(20):
            simulate(16, 13, 5, seed, per_column_mapping=True)
