"""Model check of the tensor-core tile kernel's pipeline protocol on the CPU.

The distance-tile kernel coordinates a TMA producer, one or two MMA-issuing threads
and the epilogue warps through mbarriers waited on by phase parity.  This test restates
that protocol (the same loops, barrier counts and parities as the kernel) over a small
simulated machine with random interleavings:

* copies (TMA) complete after a random delay and then arrive on their barrier;
* the tensor pipe executes each issuer's MMAs in that issuer's order, interleaving the
  two issuers arbitrarily; a commit arrives once every earlier MMA of its own issuer has
  executed.

Each run asserts that no MMA reads a query stage or point tile before its copy landed or
after the stage was refilled, that no MMA writes an accumulator the epilogue is reading,
that the epilogue reads only completed tiles, that no copy overwrites data an MMA still
needs, and that the run ends without deadlock.  Configurations cover 2-8 query stages,
one or two point-tile buffers, one-stage and multi-stage query tiles, single and dual
issue, and ragged work items."""
import random

import pytest


class Bar:
    """mbarrier: `count` arrivals complete a phase; a parity wait passes once the phase
    of that parity has completed (current phase parity differs)."""

    def __init__(self, count):
        self.count, self.pending, self.phase = count, 0, 0

    def arrive(self):
        self.pending += 1
        assert self.pending <= self.count
        if self.pending == self.count:
            self.pending = 0
            self.phase += 1

    def passed(self, parity):
        return (self.phase & 1) != parity


def run(astg, bbuf, nstage, dual, items, seed, mutant=None):
    rnd = random.Random(seed)
    skip_stage_wait = mutant == "skip_stage_wait"
    b_full = [Bar(1) for _ in range(bbuf)]
    b_empty = [Bar(2 if dual and mutant != "b_empty_count1" else 1) for _ in range(bbuf)]
    a_full = [Bar(1) for _ in range(astg)]
    a_empty = [Bar(1) for _ in range(astg)]
    t_full = [Bar(1) for _ in range(2)]
    t_empty = [Bar(1) for _ in range(2)]        # the epilogue warps modelled as one arrival
    tiles = [(i, t) for i, n in enumerate(items) for t in range(n)]   # (item, tile in item)
    T = len(tiles)

    a_content = [None] * astg                    # (tile, stage) whose copy has landed
    b_content = [None] * bbuf                    # item whose point tile has landed
    acc_progress = [None] * 2                    # (tile, stages accumulated)
    acc_reader = [None] * 2
    inflight = []                                # copies: (delay, kind, index, payload, barrier)
    need_a = [0] * astg                          # issued MMAs not yet executed, per stage
    need_b = [0] * bbuf
    queues = {0: [], 1: []}                      # per issuer: ("mma", ...) / ("commit", bar)
    violations = []

    def check(cond, msg):
        if not cond:
            violations.append(msg)

    # ---------------------------------------------------------------- agents (generators)
    def producer():
        a_st = a_ph = b_buf = b_ph = 0
        k = 0
        for it, n in enumerate(items):
            while not b_empty[b_buf].passed(b_ph ^ 1):
                yield
            check(need_b[b_buf] == 0, "point tile %d refilled while MMAs need it" % b_buf)
            inflight.append([rnd.randint(0, 3), "b", b_buf, it, b_full[b_buf]])
            b_buf += 1
            if b_buf == bbuf:
                b_buf, b_ph = 0, b_ph ^ 1
            for _ in range(n):
                for q in range(nstage):
                    while not a_empty[a_st].passed(a_ph ^ 1):
                        yield
                    check(need_a[a_st] == 0, "query stage %d refilled while MMAs need it" % a_st)
                    inflight.append([rnd.randint(0, 3), "a", a_st, (k, q), a_full[a_st]])
                    a_st += 1
                    if a_st == astg:
                        a_st, a_ph = 0, a_ph ^ 1
                k += 1
                yield
        return

    def issue(me, k, st, b_buf, q, acc):
        need_a[st] += 1
        need_b[b_buf] += 1
        queues[me].append(("mma", k, q, st, b_buf, acc))

    def issuer_single():
        a_st = a_ph = b_buf = b_ph = t_buf = t_ph = 0
        k = 0
        for it, n in enumerate(items):
            while not b_full[b_buf].passed(b_ph):
                yield
            for _ in range(n):
                while not t_empty[t_buf].passed(t_ph ^ 1):
                    yield
                for q in range(nstage):
                    while not (skip_stage_wait or a_full[a_st].passed(a_ph)):
                        yield
                    issue(0, k, a_st, b_buf, q, t_buf)
                    queues[0].append(("commit", a_empty[a_st]))
                    a_st += 1
                    if a_st == astg:
                        a_st, a_ph = 0, a_ph ^ 1
                queues[0].append(("commit", t_full[t_buf]))
                t_buf += 1
                if t_buf == 2:
                    t_buf, t_ph = 0, t_ph ^ 1
                k += 1
                yield
            queues[0].append(("commit", b_empty[b_buf]))
            b_buf += 1
            if b_buf == bbuf:
                b_buf, b_ph = 0, b_ph ^ 1

    def issuer_dual(me):
        b_buf = b_ph = 0
        t_seq = 0
        for it, n in enumerate(items):
            while not b_full[b_buf].passed(b_ph):
                yield
            i = (me ^ t_seq) & 1
            while i < n:
                tt = t_seq + i
                st, sph, tph = tt % astg, (tt // astg) & 1, (tt >> 1) & 1
                if mutant == "acc_parity":
                    tph ^= 1
                while not (t_empty[me].passed(tph ^ 1) and (skip_stage_wait or a_full[st].passed(sph))):
                    yield
                issue(me, tt, st, b_buf, 0, me)
                queues[me].append(("commit", a_empty[st]))
                queues[me].append(("commit", t_full[me]))
                i += 2
                yield
            t_seq += n
            queues[me].append(("commit", b_empty[b_buf]))
            b_buf += 1
            if b_buf == bbuf:
                b_buf, b_ph = 0, b_ph ^ 1

    def epilogue():
        t_buf = t_ph = 0
        for k in range(T):
            while not t_full[t_buf].passed(t_ph):
                yield
            check(acc_progress[t_buf] == (k, nstage), "tile %d read before its MMAs completed" % k)
            acc_reader[t_buf] = k
            yield
            yield
            acc_reader[t_buf] = None
            t_empty[t_buf].arrive()
            t_buf += 1
            if t_buf == 2:
                t_buf, t_ph = 0, t_ph ^ 1

    agents = [producer(), epilogue()] + ([issuer_dual(0), issuer_dual(1)] if dual else [issuer_single()])
    live = list(agents)

    def pipe_step():
        heads = [m for m in (0, 1) if queues[m]]
        if not heads:
            return False
        me = rnd.choice(heads)
        op = queues[me].pop(0)
        if op[0] == "commit":          # all earlier MMAs of this issuer have executed
            op[1].arrive()
            return True
        _, k, q, st, b, acc = op
        item = tiles[k][0]
        check(a_content[st] == (k, q), "MMA of tile %d stage %d read stage %d holding %r" % (k, q, st, a_content[st]))
        check(b_content[b] == item, "MMA of tile %d read point tile %d holding item %r" % (k, b, b_content[b]))
        check(acc_reader[acc] is None, "MMA of tile %d wrote accumulator %d during its read" % (k, acc))
        prev = acc_progress[acc]
        check(q == 0 or prev == (k, q), "MMA of tile %d stage %d out of order on accumulator %d" % (k, q, acc))
        acc_progress[acc] = (k, q + 1)
        need_a[st] -= 1
        need_b[b] -= 1
        return True

    def copy_step():
        ready = [c for c in inflight if c[0] == 0]
        for c in inflight:
            c[0] = max(0, c[0] - 1)
        if not ready:
            return bool(inflight)
        c = rnd.choice(ready)
        inflight.remove(c)
        _, kind, idx, payload, bar = c
        if kind == "a":
            a_content[idx] = payload
        else:
            b_content[idx] = payload
        bar.arrive()
        return True

    steps = 0
    while live or inflight or queues[0] or queues[1]:
        steps += 1
        assert steps < 200000, "no progress (deadlock)"
        choice = rnd.random()
        if choice < 0.3 and pipe_step():
            continue
        if choice < 0.55 and copy_step():
            continue
        if live:
            g = rnd.choice(live)
            try:
                next(g)
            except StopIteration:
                live.remove(g)
        elif not pipe_step():
            copy_step()
    assert not violations, violations[:5]
    assert acc_progress[(T - 1) & 1] == (T - 1, nstage) if T else True


CONFIGS = [(astg, bbuf, nstage, dual)
           for astg in (2, 3, 5, 8) for bbuf in (1, 2) for nstage in (1, 3, 5) for dual in (False, True)
           if not (dual and nstage != 1) and astg <= 16]


@pytest.mark.parametrize("astg,bbuf,nstage,dual", CONFIGS)
def test_tile_pipeline_protocol(astg, bbuf, nstage, dual):
    rnd = random.Random(astg * 1000 + bbuf * 100 + nstage * 10 + dual)
    for seed in range(12):
        items = [rnd.randint(1, 7) for _ in range(rnd.randint(1, 5))]
        run(astg, bbuf, nstage, dual, items, seed)


@pytest.mark.parametrize("mutant,dual,expect", [
    ("skip_stage_wait", False, "read stage"),
    ("skip_stage_wait", True, "read stage"),
    ("b_empty_count1", True, "point tile"),
    ("acc_parity", True, "no progress"),     # waits for a release that never comes
])
def test_model_detects_a_broken_protocol(mutant, dual, expect):
    """The checker is not vacuous: each planted protocol mistake (an issuer that does not
    wait for its query stage; one release instead of two for a point tile read by two
    issuers; the accumulator wait one phase off, which deadlocks) is caught as the
    violation it causes."""
    msgs = []
    for seed in range(30):
        try:
            run(3, 1, 1, dual, [4, 3, 5, 2], seed, mutant=mutant)
        except AssertionError as e:
            msgs.append(str(e))
    assert any(expect in m for m in msgs), msgs[:3]
