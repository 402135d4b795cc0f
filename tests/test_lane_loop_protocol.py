"""A CPU model of the persistent lane loop's ring protocol, checked over random lane mixes
and random interleavings of the CTAs.

The model follows the seed kernel, the loop kernel and the host relaunch loop step by step
in their counts and order: the seeded slots per lane (tile groups or row blocks, the larger
count with symmetric storage; skips for unused slots and finished lanes), the sequence-tagged
ring of capacity 2 (items + grid) rounded up to a power of two, one atomic reservation of the
tail before each batch of pushes, the per-lane tile and block counters, the lane's budget per
launch, and one poison entry per CTA pushed by the last lane to stop.  Each model CTA pops,
waits for its slot, and pushes its entries one write at a time, with the CTAs interleaved at
random.

Checked: no CTA waits forever (every launch ends), no slot is written before the entry it
held has been read, every lane runs exactly its steps, and every launch ends with all CTAs
at a poison entry.  The old seeding rule (one slot per tile group, which leaves an
evaluation step short of row-block entries once groups are fewer than row blocks) is shown
to deadlock in the model at four tiles per entry, and a ring below the bound is shown to
overrun, so both checks are live.

This is a model of the protocol, not the kernel: a change to the counts or order in
csrc/lane_loop.cu or to the slot count in csrc/engine.cu belongs here as well.
"""
import random

import pytest

FLAG, SKIP, POISON = 0x8000, 0xFFFE, 0xFFFF


class Lane:
    def __init__(self, nb, kinds, sym, group):
        self.nb = nb                   # row blocks (128 rows each in symmetric mode)
        self.kinds = kinds             # step kinds: "T" multiplies by Q_off, "E" evaluates
        self.step = 0
        self.ntiles = nb * (nb + 1) // 2
        self.ngroups = (self.ntiles + group - 1) // group
        self.sym = sym
        self.c1 = 0                    # first-stage entries counted this step
        self.c2 = 0                    # row-block entries counted this step
        self.budget = 0

    @property
    def done(self):
        return self.step >= len(self.kinds)

    @property
    def kind(self):
        return None if self.done else self.kinds[self.step]

    def slots(self, old_rule):
        if not self.sym:
            return self.nb
        return self.ngroups if old_rule else max(self.ngroups, self.nb)


class Deadlock(Exception):
    pass


class Loop:
    def __init__(self, lanes, grid, budget, old_rule, rng, cap_factor=2, pop_ahead=False,
                 ahead_on_poison=False):
        self.lanes, self.G, self.B, self.rng = lanes, grid, budget, rng
        self.pop_ahead = pop_ahead     # reserve the next position before processing an entry
        self.ahead_on_poison = ahead_on_poison
        self.items = [(l, b) for l, L in enumerate(lanes) for b in range(L.slots(old_rule))]
        cap = 1
        while cap < cap_factor * (len(self.items) + grid):
            cap *= 2
        self.cap = cap
        self.slot = [None] * cap       # (position, entry, read?)
        self.head = self.tail = 0
        self.launches = 0

    # ---- ring
    def write(self, pos, entry):
        old = self.slot[pos % self.cap]
        assert old is None or (old[0] == pos - self.cap and old[2]), \
            f"slot of position {pos} overwritten before position {old and old[0]} was read"
        self.slot[pos % self.cap] = [pos, entry, False]

    def reserve(self, entries):
        base = self.tail
        self.tail += len(entries)
        return [(base + i, e) for i, e in enumerate(entries)]

    # ---- one launch: the seed, then the CTAs until all have left
    def launch(self):
        self.launches += 1
        active = 0
        for L in self.lanes:
            L.budget = self.B if not L.done else 0
            active += not L.done
        pending = []
        for (l, b) in self.items:
            L = self.lanes[l]
            act, blk = not L.done, b
            if L.sym and act:
                act = b < (L.nb if L.kind == "E" else L.ngroups)
                if L.kind == "E":
                    blk |= FLAG
            pending.append((l, blk) if act else (SKIP, 0))
        if active == 0:
            pending += [(POISON, 0)] * self.G
        for pos, e in self.reserve(pending):
            self.write(pos, e)
        self.running = active
        self.active_after = 0
        ctas = [{"state": "pop", "pos": None, "out": []} for _ in range(self.G)]
        while True:
            live = [c for c in ctas if c["state"] != "exit"]
            if not live:
                assert self.head == self.tail, "a launch ended with reserved but unwritten positions"
                return
            ready = [c for c in live if c["out"] or c["state"] == "pop" or self.readable(c["pos"])]
            if not ready:
                raise Deadlock(f"launch {self.launches}: {len(live)} CTAs wait on unwritten slots")
            self.advance(self.rng.choice(ready))

    def readable(self, pos):
        s = self.slot[pos % self.cap]
        return s is not None and s[0] == pos

    def advance(self, c):
        if c["out"]:                                   # one pending write
            pos, e = c["out"].pop(self.rng.randrange(len(c["out"])))
            self.write(pos, e)
            return
        if c["state"] == "pop":
            c["pos"], self.head = self.head, self.head + 1
            c["state"] = "wait"
            return
        s = self.slot[c["pos"] % self.cap]
        s[2] = True
        lane, blk = s[1]
        c["state"] = "pop"
        if lane == POISON:
            c["state"] = "exit"
            if self.pop_ahead and self.ahead_on_poison:
                self.head += 1                         # a reservation nobody will read
            return
        if self.pop_ahead:                             # the next position, before the work
            c["pos"], self.head = self.head, self.head + 1
            c["state"] = "wait"
        if lane != SKIP:
            c["out"] = self.process(lane, blk)

    def process(self, l, blk):
        L = self.lanes[l]
        if L.sym and not blk & FLAG:                   # first stage: a group of tiles
            assert L.kind == "T" and blk < L.ngroups
            L.c1 += 1
            if L.c1 == L.ngroups:
                L.c1 = 0
                return self.reserve([(l, FLAG | t) for t in range(L.nb)])
            return []
        b = blk & ~FLAG
        assert b < L.nb
        L.c2 += 1
        if L.c2 < L.nb:
            return []
        L.c2 = 0                                       # the step is complete: the update
        L.step += 1
        L.budget -= 1
        if not L.done and L.budget > 0:
            tiles = L.sym and L.kind != "E"
            cnt = L.ngroups if tiles else L.nb
            flag = FLAG if (L.sym and not tiles) else 0
            return self.reserve([(l, flag | t) for t in range(cnt)])
        if not L.done:
            self.active_after += 1
        self.running -= 1
        return self.reserve([(POISON, 0)] * self.G) if self.running == 0 else []

    def run(self, max_launches=10000):
        while not all(L.done for L in self.lanes):
            self.launch()
            assert self.launches <= max_launches
        self.launch()                                  # a launch with nothing left ends at once


def _random_lanes(rng, sym, group):
    lanes = []
    for _ in range(rng.randint(1, 10)):
        nb = rng.randint(1, 9)
        steps = rng.randint(1, 12)
        kinds = ["E" if rng.random() < 0.3 else "T" for _ in range(steps)]
        lanes.append(Lane(nb, kinds, sym, group))
    return lanes


@pytest.mark.parametrize("pop_ahead", [False, True], ids=["pop", "pop_ahead"])
@pytest.mark.parametrize("sym,group", [(False, 2), (True, 2), (True, 4), (True, 1)])
def test_random_lane_mixes_never_deadlock_or_overrun(sym, group, pop_ahead):
    """pop_ahead: a CTA reserves its next position right after reading a (non-poison) entry
    and before processing it, so that the reservation's latency overlaps the work."""
    rng = random.Random(1000 * group + sym + 7 * pop_ahead)
    for trial in range(150):
        lanes = _random_lanes(rng, sym, group)
        loop = Loop(lanes, grid=rng.randint(1, 8), budget=rng.choice([1, 2, 3, 5, 1024]), old_rule=False, rng=rng,
                    pop_ahead=pop_ahead)
        loop.run()
        assert all(L.step == len(L.kinds) for L in lanes)
        assert all(L.c1 == 0 and L.c2 == 0 for L in lanes)
        assert loop.head == loop.tail                  # every written entry was popped


def test_old_seeding_rule_deadlocks_at_four_tiles_per_entry():
    """One slot per tile group: a lane of 2 row blocks has one group, so an evaluation step
    seeded at a relaunch gets one of its two row-block entries and never completes."""
    rng = random.Random(7)
    lanes = [Lane(2, ["T", "E", "T"], True, 4)]
    with pytest.raises(Deadlock):
        Loop(lanes, grid=2, budget=1, old_rule=True, rng=rng).run()
    lanes = [Lane(2, ["T", "E", "T"], True, 4)]
    Loop(lanes, grid=2, budget=1, old_rule=False, rng=rng).run()
    assert lanes[0].done


def test_a_ring_below_the_bound_is_caught_overrunning():
    """The overrun check is live: a ring of half of (items + grid) loses entries."""
    rng = random.Random(5)
    lanes = [Lane(rng.randint(3, 9), ["T", "E"] * 4, True, 2) for _ in range(6)]
    with pytest.raises(AssertionError, match="overwritten"):
        Loop(lanes, grid=4, budget=3, old_rule=False, rng=rng, cap_factor=0.5).run()


def test_pop_ahead_must_not_reserve_past_its_poison():
    """A CTA that also reserved ahead on its poison entry would leave a reserved position
    with no reader, and the next launch's entry there would never be popped."""
    rng = random.Random(9)
    lanes = [Lane(3, ["T", "E", "T", "T"], True, 2), Lane(5, ["E", "T"], True, 2)]
    with pytest.raises(AssertionError, match="reserved but unwritten"):
        Loop(lanes, grid=3, budget=2, old_rule=False, rng=rng, pop_ahead=True, ahead_on_poison=True).run()
