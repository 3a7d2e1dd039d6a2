"""The chunk-ticket protocol of the batched dataflow PCG, modelled on the CPU.

Each problem's solve is a chain of epochs.  A 64-bit ticket (epoch << 32 |
next chunk) hands out the open epoch's chunks: a CTA reads the ticket, and if
it shows an open chunk, atomically adds its grab size m and owns chunks
[c, min(c + m, n_e)) of the epoch e that the add returned (which may be newer
than the one it read).  A CTA that finishes chunks adds their count to the
epoch's done counter; the one that brings it to n_e resets the counter and
publishes epoch e + 1 by storing (e + 1) << 32 into the ticket.  No CTA waits
for another.

This model runs many CTAs as interleaved steps (one atomic operation per
step, random order, random grab sizes) and checks what the device code
relies on: every chunk of every epoch is processed exactly once, by a CTA
that knew which epoch it belonged to, and only after the previous epoch had
finished; each epoch is closed exactly once; the problems finish."""
import random

import pytest


class Problem:
    def __init__(self, chunks_per_epoch, epochs):
        self.n = chunks_per_epoch           # chunks of epoch e: n[e % len(n)]
        self.epochs = epochs
        self.ticket = 0                     # epoch << 32 | count
        self.done = 0
        self.finished = False
        self.closed = []                    # epochs closed, in order
        self.work = {}                      # (epoch, chunk) -> times processed

    def chunks(self, e):
        return self.n[e % len(self.n)]


def cta(problems, rng, log):
    """One CTA as a generator: yields after every atomic step."""
    while True:
        live = [k for k, P in enumerate(problems) if not P.finished]
        if not live:
            return
        k = rng.choice(live)
        P = problems[k]
        t = P.ticket                         # volatile read
        yield
        e0, c0 = t >> 32, t & 0xFFFFFFFF
        if c0 >= P.chunks(e0):
            yield
            continue
        m = rng.randint(1, 4)
        t2 = P.ticket                        # atomicAdd returns the old value
        P.ticket = t2 + m
        yield
        e, c = t2 >> 32, t2 & 0xFFFFFFFF
        if c >= P.chunks(e):
            continue                         # a late grab past the epoch's end: nothing taken
        cnt = min(m, P.chunks(e) - c)
        for cc in range(c, c + cnt):
            # the previous epoch must be complete before any chunk of this one runs
            assert P.closed == list(range(e)), (k, e, P.closed)
            P.work[(e, cc)] = P.work.get((e, cc), 0) + 1
            yield
        d = P.done                           # atomicAdd(done, cnt)
        P.done = d + cnt
        yield
        if d + cnt == P.chunks(e):           # the last finisher closes the epoch
            P.closed.append(e)
            P.done = 0
            if e + 1 == P.epochs:
                P.finished = True
            else:
                P.ticket = (e + 1) << 32
            log.append((k, e))
            yield


@pytest.mark.parametrize("seed", range(12))
def test_every_chunk_once_epochs_in_order(seed):
    rng = random.Random(seed)
    problems = [Problem([rng.randint(1, 9), rng.randint(1, 5)], rng.randint(1, 40)) for _ in range(rng.randint(1, 6))]
    log = []
    ctas = [cta(problems, random.Random(seed * 100 + i), log) for i in range(rng.randint(1, 12))]
    steps = 0
    while ctas:
        g = rng.choice(ctas)
        try:
            next(g)
        except StopIteration:
            ctas.remove(g)
        steps += 1
        assert steps < 10_000_000
    for P in problems:
        assert P.finished
        assert P.closed == list(range(P.epochs))
        expect = {(e, c) for e in range(P.epochs) for c in range(P.chunks(e))}
        assert set(P.work) == expect
        assert all(v == 1 for v in P.work.values())
    assert len(log) == sum(P.epochs for P in problems)
