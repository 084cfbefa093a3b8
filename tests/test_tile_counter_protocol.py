"""Host-side model of the persistent, pipelined TMA collide kernel's protocol
(csrc/collide2d_tma.cu, launch-shape variant 7): resident CTAs take tiles from
a per-handle counter (atomicAdd), each with two shared-memory stages whose
copies complete on one mbarrier per stage; a CTA claims and starts the next
tile's copies before it waits for and computes the current one, and the last
CTA to finish resets the counter for the next launch.

The model runs the CTAs as coroutines in random interleavings (the claims,
the copies' completions and the computations interleave arbitrarily) and
checks what the kernel relies on: every tile is computed exactly once per
launch, a stage is refilled only after its previous tile was computed, each
wait with parity (k >> 1) & 1 on stage k & 1 is satisfied by exactly the copy
of the tile the CTA is about to compute (never by an older or a newer phase),
and the counter and the finished-CTA count are back at zero after every
launch, so that repeated launches all see every tile."""
import random


class Bar:
    """mbarrier with one arrival per phase (the expect_tx arrival; the copy's
    bytes complete the phase)."""

    def __init__(self):
        self.phase = 0  # completed phases

    def done(self, parity):
        # try_wait.parity(P) succeeds once the phase with parity P completed
        # and the next one has not: the model flags anything else as stale
        return self.phase > 0 and ((self.phase - 1) & 1) == parity


def launch(ntiles, nctas, sched, rng):
    computed = []
    inflight = []  # (cta, stage, tile): copies issued, not yet landed
    events = []

    def cta(c):
        bars = [Bar(), Bar()]
        stile = [None, None]
        stage_busy = [False, False]  # a computed-but-unconsumed tile sits in the stage
        issued = [[], []]  # tiles issued into each stage, in order

        def issue(tile, st):
            assert not stage_busy[st], "stage refilled before its tile was computed"
            stage_busy[st] = True
            issued[st].append(tile)
            inflight.append((c, st, tile, bars[st]))

        # prologue: claim the first tile
        t0 = sched[0]
        sched[0] += 1
        yield
        stile[0] = t0
        if t0 < ntiles:
            issue(t0, 0)
        k = 0
        while True:
            st = k & 1
            tile = stile[st]
            if tile >= ntiles:
                break
            tn = sched[0]  # claim the next tile and start its copies
            sched[0] += 1
            yield
            stile[st ^ 1] = tn
            if tn < ntiles:
                issue(tn, st ^ 1)
            parity = (k >> 1) & 1
            while not bars[st].done(parity):
                yield  # bounded in the kernel by %globaltimer; here by the scheduler
            # the completed phase is the copy of exactly this tile
            assert bars[st].phase == (k >> 1) + 1
            assert issued[st][k >> 1] == tile
            yield
            computed.append(tile)
            stage_busy[st] = False  # __syncthreads at the end of the iteration
            k += 1
        # count out; the last CTA resets both counters
        d = sched[1]
        sched[1] += 1
        yield
        if d == nctas - 1:
            sched[0] = 0
            sched[1] = 0
        events.append(("exit", c))

    gens = {c: cta(c) for c in range(nctas)}
    live = list(gens)
    steps = 0
    while live or inflight:
        steps += 1
        assert steps < 200000, "deadlock"
        if inflight and (not live or rng.random() < 0.3):
            i = rng.randrange(len(inflight))  # copies land in any order
            _, _, _, bar = inflight.pop(i)
            bar.phase += 1
            continue
        c = rng.choice(live)
        try:
            next(gens[c])
        except StopIteration:
            live.remove(c)
    return computed


def test_every_tile_exactly_once_and_counter_reset():
    rng = random.Random(1)
    for trial in range(300):
        ntiles = rng.randint(1, 40)
        nctas = rng.randint(1, 12)
        sched = [0, 0]
        for _ in range(3):  # repeated launches reuse the reset counter
            computed = launch(ntiles, nctas, sched, rng)
            assert sorted(computed) == list(range(ntiles)), (trial, ntiles, nctas)
            assert sched == [0, 0]


def test_more_ctas_than_tiles():
    rng = random.Random(2)
    sched = [0, 0]
    for _ in range(50):
        computed = launch(3, 10, sched, rng)
        assert sorted(computed) == [0, 1, 2]
        assert sched == [0, 0]
