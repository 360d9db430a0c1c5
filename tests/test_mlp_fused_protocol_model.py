"""CPU model of the barrier protocol of the fused closure network (k_mlp_fused): a copy
warp streaming the K-blocks of every layer (and the first layer's features) through a
ring of stages, an MMA warp running the four layers of each tile into one TMEM
accumulator, and eight epilogue warps that drain it and write the next layer's input into
the shared activation tile.  Copies and MMA completions land asynchronously and the warps
are scheduled at random.  The model follows the kernel's waits and arrivals and checks:
no deadlock; an MMA reads the K-block the copies filled for it; a layer's MMAs read the
activation tile only after all eight epilogue warps wrote the previous layer into it; the
epilogue never writes the tile while MMAs still read it, nor overwrites an accumulator
before it was drained.  Removing the MMA warp's wait on the epilogue makes it fail."""
import random

import pytest

from tests.test_gemm_protocol_model import MBar

LAYERS = 4


def run(ntiles, nkb, stages, epi_warps, seed, skip_epilogue_wait=False):
    rnd = random.Random(seed)
    full = [MBar(1) for _ in range(stages)]
    empty = [MBar(1) for _ in range(stages)]
    accf, acce = MBar(1), MBar(epi_warps)
    stage_holds = [None] * stages        # (tile, layer, K-block) the copies put there
    mma_reads = [None] * stages
    state = dict(acc=None, drained=0, act=None, act_parts=0, act_reads=0)
    events = []

    def copies():
        g = 0
        for t in range(ntiles):
            for l in range(LAYERS):
                for kb in range(nkb[l]):
                    st, use = g % stages, g // stages
                    if g >= stages:
                        while not empty[st].done((use - 1) & 1):
                            yield
                    assert mma_reads[st] is None, "stage refilled while the MMAs read it"
                    full[st].expect(1)
                    events.append(("copy", st, (t, l, kb)))
                    g += 1
                    yield

    def mmas():
        g = u = 0
        for t in range(ntiles):
            for l in range(LAYERS):
                if u >= 1 and not skip_epilogue_wait:
                    while not acce.done((u - 1) & 1):
                        yield
                assert state["acc"] is None, "accumulator overwritten before it was drained"
                if l > 0:
                    assert state["act"] == (t, l - 1) and state["act_parts"] == epi_warps, \
                        "layer input read before the epilogue wrote it"
                for kb in range(nkb[l]):
                    st = g % stages
                    while not full[st].done((g // stages) & 1):
                        yield
                    assert stage_holds[st] == (t, l, kb)
                    mma_reads[st] = (t, l, kb)
                    if l > 0:
                        state["act_reads"] += 1
                    events.append(("mma", st, l > 0))
                    g += 1
                    yield
                events.append(("acc", None, (t, l)))
                u += 1

    def epilogue():
        u = 0
        for t in range(ntiles):
            for l in range(LAYERS):
                while not accf.done(u & 1):
                    yield
                assert state["acc"] == (t, l)
                yield
                if l < LAYERS - 1:   # this warp's part of the next layer's input
                    assert state["act_reads"] == 0, "activation tile written while MMAs read it"
                    if state["act"] != (t, l):
                        state["act"], state["act_parts"] = (t, l), 0
                    state["act_parts"] += 1
                state["drained"] += 1
                if state["drained"] == epi_warps:
                    state["acc"], state["drained"] = None, 0
                acce.arrive()
                u += 1
                yield

    warps = [copies(), mmas()] + [epilogue() for _ in range(epi_warps)]
    alive = set(range(len(warps)))
    for _ in range(3_000_000):
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
                if val:
                    state["act_reads"] -= 1
                empty[a].arrive()
            else:
                state["acc"] = val
                accf.arrive()
            continue
        if alive:
            w = rnd.choice(sorted(alive))
            try:
                next(warps[w])
            except StopIteration:
                alive.discard(w)
    raise AssertionError("deadlock")


@pytest.mark.parametrize("stages", [2, 3])
def test_fused_network_protocol(stages):
    for seed in range(120):
        r = random.Random(seed)
        nkb = [r.randint(1, 5)] + [r.randint(1, 4)] * 3
        run(r.randint(1, 4), nkb, stages, 8, seed)


def test_the_model_catches_a_missing_epilogue_wait():
    with pytest.raises(AssertionError):
        for seed in range(120):
            r = random.Random(seed)
            nkb = [r.randint(1, 5)] + [r.randint(1, 4)] * 3
            run(r.randint(2, 4), nkb, 3, 8, seed, skip_epilogue_wait=True)
