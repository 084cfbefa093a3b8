"""Host-side model of the tcgen05 convolution's barrier protocol
(csrc/conv_tcgen05.cu): a loader, an MMA issuer and the epilogue meet only on
mbarriers (loaded[slot], sfree[slot] per staged-row slot; full[acc],
aempty[acc] per tensor-memory accumulator).  The model runs the three roles
as coroutines in random interleavings against barrier objects with the
parity semantics of mbarrier.test_wait.parity and checks what the kernel
relies on: a copy never lands in a slot that an unfinished MMA reads, every
MMA finds its three operand rows, no parity wait ever falls two phases behind
(which would make it wait for a phase that already passed), and the protocol
never deadlocks.  The schedule constants are the kernel's: SLOTS = 4,
NACC = 2, the loader announcing rows DEPTH = 2 behind its requests and
flushing before it blocks."""
import random

SLOTS, NACC, DEPTH = 4, 2, 2


class Bar:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0

    def arrive(self):
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def done(self, parity):
        return self.phase > 0 and ((self.phase - 1) & 1) == parity


def run(items, rng):
    full = [Bar(1) for _ in range(NACC)]
    aempty = [Bar(4) for _ in range(NACC)]
    loaded = [Bar(1) for _ in range(SLOTS)]
    sfree = [Bar(1) for _ in range(SLOTS)]
    slot_row = [None] * SLOTS
    copies, mma_q, reading = [], [], []

    def wait(bar, k):  # wait for completed phase number k (0-based)
        while not bar.done(k & 1):
            assert bar.phase <= k, "a parity wait fell two phases behind"
            yield
        assert bar.phase == k + 1

    def loader():
        q = 0
        pending = []

        def announce(keep):
            while len(pending) > keep:
                sl, qq = pending[0]
                while (sl, qq) in copies:
                    yield
                pending.pop(0)
                assert slot_row[sl] == qq
                loaded[sl].arrive()

        for rows in items:
            for _ in range(rows + 2):
                sl = q % SLOTS
                if q >= SLOTS and not sfree[sl].done((q // SLOTS - 1) & 1):
                    yield from announce(0)
                    yield from wait(sfree[sl], q // SLOTS - 1)
                assert all(sl not in r for r in reading), "copy into a slot an MMA reads"
                slot_row[sl] = None
                copies.append((sl, q))
                pending.append((sl, q))
                q += 1
                if len(pending) > DEPTH:
                    yield from announce(DEPTH)
                yield
        yield from announce(0)

    def issuer():
        g = qbase = 0
        for rows in items:
            for t in range(rows):
                q0 = qbase + t
                if g >= NACC:
                    yield from wait(aempty[g % NACC], g // NACC - 1)
                for d in range(3):
                    yield from wait(loaded[(q0 + d) % SLOTS], (q0 + d) // SLOTS)
                    assert slot_row[(q0 + d) % SLOTS] == q0 + d, "operand row missing"
                rd = [(q0 + d) % SLOTS for d in range(3)]
                reading.append(rd)
                commits = [("full", g % NACC), ("sfree", q0 % SLOTS)]
                if t == rows - 1:
                    commits += [("sfree", (q0 + 1) % SLOTS), ("sfree", (q0 + 2) % SLOTS)]
                mma_q.append((rd, commits))
                g += 1
                yield
            qbase += rows + 2

    def engines():  # copies land in any order; MMAs complete in issue order
        while True:
            if copies and rng.random() < 0.5:
                sl, q = copies.pop(rng.randrange(len(copies)))
                slot_row[sl] = q
            if mma_q and rng.random() < 0.4:
                rd, commits = mma_q.pop(0)
                reading.remove(rd)
                for kind, k in commits:
                    (full if kind == "full" else sfree)[k].arrive()
            yield

    def epilogue():
        g = 0
        for rows in items:
            for _ in range(rows):
                yield from wait(full[g % NACC], g // NACC)
                for _ in range(4):
                    aempty[g % NACC].arrive()
                g += 1
                yield

    roles = {"loader": loader(), "issuer": issuer(), "epilogue": epilogue()}
    eng = engines()
    steps = 0
    while roles:
        steps += 1
        assert steps < 200000, "deadlock"
        name = rng.choice(list(roles) + ["engines", "engines"])
        try:
            next(eng if name == "engines" else roles[name])
        except StopIteration:
            del roles[name]


def test_protocol_random_interleavings():
    rng = random.Random(5)
    for _ in range(600):
        run([rng.randint(1, 20) for _ in range(rng.randint(1, 4))], rng)


def test_protocol_single_tile_runs():
    rng = random.Random(6)
    for _ in range(200):
        run([1] * rng.randint(1, 6), rng)
