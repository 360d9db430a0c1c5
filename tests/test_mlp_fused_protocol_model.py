"""CPU model of the barrier protocol of the fused closure network (k_mlp_fused).

The kernel's roles:
- a copy warp streams the K-blocks of every layer's weights through a ring of stages,
  and another the tiles' feature K-blocks (the first layer's input) through a ring of
  their own;
- an MMA warp runs use u = 4 n + l (tile n, layer l) into TMEM accumulator u mod 2;
- sixteen epilogue warps drain an accumulator into registers, 32 columns at a time,
  release it, and write the next layer's input into the shared activation tile; eight
  warps write each K-block, announced on its own barrier, so that the next layer's MMAs
  start on K-blocks 0 and 1 while the epilogue still writes the others.

Copies and MMA completions land asynchronously and the warps are scheduled at random. The
model follows the kernel's waits and arrivals (barrier counts, phase parities) and
checks:
- it never deadlocks;
- an MMA reads the weight and feature K-blocks the copies filled for it, and the
  activation K-block of the layer before, once the eight epilogue warps that write it
  did;
- the epilogue never writes an activation K-block while MMAs still read it;
- no accumulator is overwritten before it was drained.
Removing any one of the MMA warp's waits makes it fail."""
import random

import pytest

from tests.test_gemm_protocol_model import MBar

LAYERS = 4


def run(ntiles, nkb, stages, epi_warps, seed, skip=None, xstages=3):
    """nkb[l]: K-blocks of layer l; layers 1..3 read the hidden width, nkb[1] K-blocks
    of the activation tile."""
    rnd = random.Random(seed)
    full = [MBar(1) for _ in range(stages)]
    empty = [MBar(1) for _ in range(stages)]
    accf = [MBar(1) for _ in range(2)]
    acce = [MBar(epi_warps) for _ in range(2)]
    nact = nkb[1]
    actf = [MBar(epi_warps // 2) for _ in range(nact)]
    fullx = [MBar(1) for _ in range(xstages)]
    emptyx = [MBar(1) for _ in range(xstages)]
    stage_holds = [None] * stages        # (tile, layer, K-block) the copies put there
    mma_reads = [None] * stages
    xstage_holds = [None] * xstages      # (tile, K-block) of the features
    xmma_reads = [None] * xstages
    acc = [None, None]                   # (tile, layer) whose sums the accumulator holds
    acc_busy = [False, False]            # MMAs in flight into it
    drained = [0, 0]
    act = [None] * nact                  # (tile, layer) whose output the K-block holds
    act_parts = [0] * nact
    act_reads = [0] * nact
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

    def xcopies():
        g = 0
        for t in range(ntiles):
            for kb in range(nkb[0]):
                st, use = g % xstages, g // xstages
                if g >= xstages:
                    while not emptyx[st].done((use - 1) & 1):
                        yield
                assert xmma_reads[st] is None, "feature stage refilled while the MMAs read it"
                fullx[st].expect(1)
                events.append(("xcopy", st, (t, kb)))
                g += 1
                yield

    def mmas():
        g = gx = 0
        for t in range(ntiles):
            for l in range(LAYERS):
                u = 4 * t + l
                b = u & 1
                if u >= 2 and skip != "acce":
                    while not acce[b].done(((u >> 1) - 1) & 1):
                        yield
                assert acc[b] is None and not acc_busy[b], \
                    "accumulator overwritten before it was drained"
                acc_busy[b] = True
                for kb in range(nkb[l]):
                    st = g % stages
                    while not full[st].done((g // stages) & 1):
                        yield
                    assert stage_holds[st] == (t, l, kb)
                    sx = gx % xstages
                    if l == 0:
                        if skip != "fullx":
                            while not fullx[sx].done((gx // xstages) & 1):
                                yield
                        assert xstage_holds[sx] == (t, kb), "features read before they landed"
                        xmma_reads[sx] = (t, kb)
                    if l > 0:
                        if skip != "actf":
                            while not actf[kb].done((3 * t + l - 1) & 1):
                                yield
                        assert act[kb] == (t, l - 1) and act_parts[kb] == epi_warps // 2, \
                            "layer input read before the epilogue wrote it"
                        act_reads[kb] += 1
                    mma_reads[st] = (t, l, kb)
                    events.append(("mma", st, kb if l > 0 else None, sx if l == 0 else None))
                    g += 1
                    if l == 0:
                        gx += 1
                    yield
                events.append(("acc", b, (t, l)))

    def epilogue(e):
        # warp group e // 4 writes its chunks' K-blocks e // 8 and e // 8 + 2, the first
        # before it reads its second chunk out of the accumulator
        kbs = [e // 8, e // 8 + 2]
        for t in range(ntiles):
            for l in range(LAYERS):
                u = 4 * t + l
                b = u & 1
                while not accf[b].done((u >> 1) & 1):
                    yield
                assert acc[b] == (t, l)
                for h in range(2):
                    yield                 # one chunk of the accumulator into registers
                    assert acc[b] == (t, l), "accumulator overwritten while being read"
                    if h == 1:
                        drained[b] += 1
                        if drained[b] == epi_warps:
                            acc[b], drained[b] = None, 0
                        acce[b].arrive()
                    kb = kbs[h]
                    if l < LAYERS - 1 and kb < nact:   # the next layer's input
                        yield
                        assert act_reads[kb] == 0, "activation K-block written while MMAs read it"
                        if act[kb] != (t, l):
                            assert act_parts[kb] in (0, epi_warps // 2)
                            act[kb], act_parts[kb] = (t, l), 0
                        act_parts[kb] += 1
                        actf[kb].arrive()
                yield

    warps = [copies(), xcopies(), mmas()] + [epilogue(e) for e in range(epi_warps)]
    alive = set(range(len(warps)))
    for _ in range(5_000_000):
        if not alive and not events:
            return
        if events and (not alive or rnd.random() < 0.3):
            # copies land in any order; MMA completions in issue order
            k = rnd.randrange(len(events))
            if events[k][0] not in ("copy", "xcopy"):
                k = next(q for q, ev in enumerate(events) if ev[0] not in ("copy", "xcopy"))
            kind, a, val, *rest = events.pop(k)
            if kind == "copy":
                stage_holds[a] = val
                full[a].complete(1)
            elif kind == "xcopy":
                xstage_holds[a] = val
                fullx[a].complete(1)
            elif kind == "mma":
                mma_reads[a] = None
                if val is not None:
                    act_reads[val] -= 1
                empty[a].arrive()
                if rest[0] is not None:
                    xmma_reads[rest[0]] = None
                    emptyx[rest[0]].arrive()
            else:
                acc[a], acc_busy[a] = val, False
                accf[a].arrive()
            continue
        if alive:
            w = rnd.choice(sorted(alive))
            try:
                next(warps[w])
            except StopIteration:
                alive.discard(w)
    raise AssertionError("deadlock")


def _shapes(r):
    h = r.randint(1, 4)
    return [r.randint(1, 5), h, h, h]


@pytest.mark.parametrize("stages,xstages", [(2, 2), (3, 3), (3, 2)])
def test_fused_network_protocol(stages, xstages):
    for seed in range(150):
        r = random.Random(seed)
        run(r.randint(1, 4), _shapes(r), stages, 16, seed, xstages=xstages)


@pytest.mark.parametrize("skip", ["acce", "actf", "fullx"])
def test_the_model_catches_a_missing_wait(skip):
    with pytest.raises(AssertionError):
        for seed in range(150):
            r = random.Random(seed)
            run(r.randint(2, 4), _shapes(r), 3, 16, seed, skip=skip)
