"""The synchronisation protocol of the grid S'v product (k_sr_grid), checked on the CPU by a randomised
interleaving model with the constants read from the CUDA source.

The kernel's CTAs and warp roles hand data to one another through rings: two copy rings (HBM, then L2)
guarded by full / empty mbarriers, a ring of per-warp partials (compute warps -> publisher), a ring of
published-block barriers (publisher -> exchange warps), the exchange slots in global memory (tagged words,
reused every kGPB blocks) and the t slots (exchange warps -> compute warps).  The model runs every role of
several CTAs as a coroutine, picks the next runnable one at random, lands bulk copies at random times, and
gives each mbarrier wait the hardware's parity rule (a wait for parity p passes while the barrier's
completed-phase count has the other parity), so a waiter two phases behind would deadlock here as on the
device.  At every hand-off it asserts that the consumer sees the block it expects and that no producer
overwrites a stage, slot or word that some consumer may still read.  A change of the ring sizes, the
lookahead or the role order that breaks the protocol fails here before it reaches a GPU."""
import os
import random
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2502_20723_gb300", "csrc", "k_sr.cu")


def constants():
    text = open(SRC).read()
    out = {}
    for name in ("kGR", "kGLook", "kGExch", "kGAhead", "kGPB", "kGTB", "kGRB"):
        m = re.search(rf"\b{name} = (\d+)", text)
        assert m, name
        out[name] = int(m.group(1))
    return out


class Bar:
    """An mbarrier: expected arrivals per phase, pending transaction bytes, completed phases."""

    def __init__(self, expected):
        self.exp, self.pend, self.tx, self.done = expected, expected, 0, 0

    def arrive(self, tx=0):
        self.tx += tx
        self.pend -= 1
        assert self.pend >= 0, "more arrivals than a phase expects"
        self._complete()

    def complete_tx(self, n):
        self.tx -= n
        assert self.tx >= 0
        self._complete()

    def _complete(self):
        if self.pend == 0 and self.tx == 0:
            self.done += 1
            self.pend = self.exp

    def passed(self, parity):
        return (self.done & 1) != parity


def run_model(c, G, nb, ns1, ns2, nw, seed):
    R, LOOK, NE, AHEAD, PB, TB, RB = (c[k] for k in ("kGR", "kGLook", "kGExch", "kGAhead", "kGPB", "kGTB", "kGRB"))
    rnd = random.Random(seed)
    words = [[-1] * G for _ in range(PB)]    # block whose words sit in exchange slot / CTA (-1: cleared)
    read = [set() for _ in range(G)]          # blocks whose words each CTA has finished reading
    pending, actors, ctas = [], [], []
    for q in range(G):
        s = dict(tf=[Bar(1) for _ in range(ns1)], te=[Bar(nw) for _ in range(ns1)],
                 wf=[Bar(1) for _ in range(ns2)], we=[Bar(nw) for _ in range(ns2)],
                 xf=[Bar(1) for _ in range(TB)], xe=[Bar(nw) for _ in range(TB)],
                 pf=[Bar(nw) for _ in range(RB)], pe=[Bar(1) for _ in range(RB)], pb=[Bar(1) for _ in range(TB)],
                 tst=[None] * ns1, wst=[None] * ns2, tb=[None] * TB, red=[[None] * nw for _ in range(RB)],
                 tdone=[-1] * nw, wdone=[-1] * nw, published=[-1])
        ctas.append(s)

        def copier(kind, q=q, s=s):
            ns = ns1 if kind == "t" else ns2
            full, empty = (s["tf"], s["te"]) if kind == "t" else (s["wf"], s["we"])
            for b in range(nb):
                st, m = b % ns, b // ns
                if m > 0:
                    yield lambda: empty[st].passed((m - 1) & 1)
                full[st].arrive(tx=1)
                pending.append((q, st, b, kind))

        def publisher(q=q, s=s):
            for b in range(nb):
                rs = b % RB
                yield lambda: s["pf"][rs].passed((b // RB) & 1)
                assert all(x == b for x in s["red"][rs]), "publisher sums partials of another block"
                if b - PB >= 0:
                    for x in range(G):
                        assert b - PB in read[x], "exchange slot reused before every CTA read it"
                words[b % PB][q] = b
                s["published"][0] = b
                s["pe"][rs].arrive()
                s["pb"][b % TB].arrive()

        def exchange(e, q=q, s=s):
            for b in range(e, nb, NE):
                j, m, slot = b % TB, b // TB, b % PB
                if m > 0:
                    yield lambda: s["xe"][j].passed((m - 1) & 1)
                cb = min(b + AHEAD, nb - 1)
                yield lambda: s["pb"][cb % TB].passed((cb // TB) & 1)
                yield lambda: all(words[slot][g] == b for g in range(G))
                read[q].add(b)
                assert all(wd >= b - TB for wd in s["wdone"]), "t slot overwritten while in use"
                s["tb"][j] = b
                s["xf"][j].arrive()

        def compute(w, s=s):
            for b in range(nb + LOOK):
                if b < nb:
                    st = b % ns1
                    yield lambda: s["tf"][st].passed((b // ns1) & 1)
                    assert s["tst"][st] == b, "t stage holds another block"
                    s["tdone"][w] = b
                    s["te"][st].arrive()
                    rs = b % RB
                    if b >= RB:
                        yield lambda: s["pe"][rs].passed((b // RB - 1) & 1)
                    assert s["published"][0] >= b - RB, "partial slot overwritten before it was published"
                    s["red"][rs][w] = b
                    s["pf"][rs].arrive()
                bw = b - LOOK
                if bw >= 0:
                    st, j = bw % ns2, bw % TB
                    yield lambda: s["xf"][j].passed((bw // TB) & 1)
                    yield lambda: s["wf"][st].passed((bw // ns2) & 1)
                    assert s["tb"][j] == bw and s["wst"][st] == bw, "w-part sees another block"
                    s["wdone"][w] = bw
                    s["we"][st].arrive()
                    s["xe"][j].arrive()

        actors += [copier("t"), copier("w"), publisher()]
        actors += [exchange(e) for e in range(NE)]
        actors += [compute(w) for w in range(nw)]
    conds = [None] * len(actors)

    def step(i):
        try:
            conds[i] = next(actors[i])
        except StopIteration:
            conds[i] = "done"

    for i in range(len(actors)):
        step(i)
    while True:
        runnable = [i for i, cd in enumerate(conds) if cd != "done" and cd()]
        choices = runnable + (["copy"] * min(3, len(pending)) if pending else [])
        if not choices:
            assert all(cd == "done" for cd in conds), "deadlock"
            return
        ch = rnd.choice(choices)
        if ch != "copy":
            step(ch)
            continue
        q, st, b, kind = pending.pop(rnd.randrange(len(pending)))
        s = ctas[q]
        if kind == "t":
            assert all(td >= b - ns1 for td in s["tdone"]), "copy lands on a t stage still being read"
            s["tst"][st] = b
            s["tf"][st].complete_tx(1)
        else:
            assert all(wd >= b - ns2 for wd in s["wdone"]), "copy lands on a w stage still being read"
            s["wst"][st] = b
            s["wf"][st].complete_tx(1)


def test_constants_satisfy_the_ring_rules():
    c = constants()
    assert c["kGPB"] >= 2 * c["kGLook"] + 2     # exchange slots outlive every reader
    assert c["kGTB"] >= c["kGLook"] + c["kGExch"]
    assert 32 % (2 * c["kGR"]) == 0             # the lane reduction's value count divides the warp


@pytest.mark.parametrize("seed", range(40))
def test_random_interleavings_deliver_every_block_once(seed):
    c = constants()
    rnd = random.Random(1000 + seed)
    G = rnd.choice([1, 2, 3, 5])
    nb = rnd.choice([1, 2, 3, 5, 9, 17, 40, 70])
    ns1, ns2, nw = rnd.choice([2, 3, 4]), rnd.choice([2, 3]), rnd.choice([1, 2, 3])
    run_model(c, G, nb, ns1, ns2, nw, seed)


def test_a_too_small_exchange_ring_is_caught():
    """The model is sharp: with exchange slots reused after 2 blocks a fast CTA overwrites words that a
    slow CTA has not read yet, in some interleaving."""
    c = dict(constants(), kGPB=2)
    failures = 0
    for seed in range(60):
        try:
            run_model(c, 3, 40, 3, 2, 2, seed)
        except AssertionError:
            failures += 1
    assert failures > 0
