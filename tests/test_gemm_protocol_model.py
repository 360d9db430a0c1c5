"""CPU model of the barrier protocol of the persistent closure GEMM (k_gemm_nt_pers):
a copy warp, an MMA warp and eight epilogue warps over a ring of operand stages and two
TMEM accumulators, with copies and MMA completions landing asynchronously and the warps
scheduled at random.  The model follows the kernel's waits and arrivals (barrier counts,
phase parities) and checks that it never deadlocks, that an MMA reads the stage the
copies filled for its K step, and that no accumulator is overwritten before its eight
epilogue warps have read it; removing one of the kernel's waits makes it fail."""
import random

import pytest


class MBar:
    """An mbarrier: `count` arrivals and the expected transaction bytes end a phase."""

    def __init__(self, count):
        self.count, self.pending, self.phase, self.tx = count, count, 0, 0

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0, "more arrivals than the barrier counts"
        self._advance()

    def expect(self, nbytes):
        self.tx += nbytes
        self.arrive()

    def complete(self, nbytes):
        self.tx -= nbytes
        self._advance()

    def _advance(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def done(self, parity):
        # try_wait.parity: the phase of this parity has completed
        return (self.phase & 1) != parity


def run(ntiles, nk, stages, epi_warps, seed, skip_acc_wait=False):
    rnd = random.Random(seed)
    full = [MBar(1) for _ in range(stages)]
    empty = [MBar(1) for _ in range(stages)]
    accf = [MBar(1) for _ in range(2)]
    acce = [MBar(epi_warps) for _ in range(2)]
    stage_holds = [None] * stages       # (tile, k step) the copies put in the stage
    mma_reads = [None] * stages
    acc_holds = [None, None]            # tile whose sums are in the accumulator
    reads = [0, 0]
    events = []

    def copies():
        g = 0
        for t in range(ntiles):
            for kt in range(nk):
                st, use = g % stages, g // stages
                if g >= stages:
                    while not empty[st].done((use - 1) & 1):
                        yield
                assert mma_reads[st] is None, "stage refilled while the MMAs read it"
                full[st].expect(1)
                events.append(("copy", st, (t, kt)))
                g += 1
                yield

    def mmas():
        g = 0
        for i in range(ntiles):
            b = i & 1
            if i >= 2 and not skip_acc_wait:
                while not acce[b].done(((i >> 1) - 1) & 1):
                    yield
            assert acc_holds[b] is None, "accumulator overwritten before it was read"
            for kt in range(nk):
                st = g % stages
                while not full[st].done((g // stages) & 1):
                    yield
                assert stage_holds[st] == (i, kt)
                mma_reads[st] = (i, kt)
                events.append(("mma", st, None))
                g += 1
                yield
            events.append(("acc", b, i))

    def epilogue():
        for i in range(ntiles):
            b = i & 1
            while not accf[b].done((i >> 1) & 1):
                yield
            assert acc_holds[b] == i
            yield
            reads[b] += 1
            if reads[b] == epi_warps:
                acc_holds[b], reads[b] = None, 0
            acce[b].arrive()
            yield

    warps = [copies(), mmas()] + [epilogue() for _ in range(epi_warps)]
    alive = set(range(len(warps)))
    for _ in range(2_000_000):
        if not alive and not events:
            return
        if events and (not alive or rnd.random() < 0.3):
            # copies land in any order; the MMAs complete in issue order
            k = rnd.randrange(len(events))
            if events[k][0] != "copy":
                k = next(q for q, ev in enumerate(events) if ev[0] != "copy")
            kind, a, val = events.pop(k)
            if kind == "copy":
                stage_holds[a] = val
                full[a].complete(1)
            elif kind == "mma":
                mma_reads[a] = None
                empty[a].arrive()
            else:
                acc_holds[a] = val
                accf[a].arrive()
            continue
        if alive:
            w = rnd.choice(sorted(alive))
            try:
                next(warps[w])
            except StopIteration:
                alive.discard(w)
    raise AssertionError("deadlock")


@pytest.mark.parametrize("stages", [2, 5])
def test_persistent_gemm_protocol(stages):
    for seed in range(150):
        r = random.Random(seed)
        run(r.randint(1, 7), r.randint(1, 6), stages, 8, seed)


def test_the_model_catches_a_missing_accumulator_wait():
    with pytest.raises(AssertionError):
        for seed in range(150):
            r = random.Random(seed)
            run(r.randint(3, 7), r.randint(1, 6), 2, 8, seed, skip_acc_wait=True)
