"""A CPU model of the barrier protocol of the tensor-memory RowSel kernel
(rowsel_tmem.cu), single-CTA and SM-pair forms, run under random
interleavings.

The model restates the kernel's rules with exact mbarrier semantics (arrival
count, transaction bytes, phase parity; no code shared with the CUDA source):
  - the producer of each CTA claims units one ahead (the pair's odd CTA
    receives them through a mailbox); for its i-th k-chunk it copies the ring
    tile into ring slot i % RS after rempty[slot] (arrive.expect_tx on
    rfull[slot]) and the B part into B stage i % NS after empty[stage]
    (expect_tx on full[stage]; RS, NS even; the copies land asynchronously,
    in any order), and ends with a sentinel in two consecutive k-chunks, one
    per converter set, the B stage's tag written before the slot's arrive;
    the pair's producers then wait for the commits of their other stages;
  - k-chunk i goes into part i % KPB of A buffer (i // KPB) % NBUF (KPB = 1:
    four buffers of one k-chunk; KPB = 2: two buffers of two); converter set
    c (two sets of four warps) takes k-chunks i = c, c + 2, ...: it waits
    rfull[slot], stops at a sentinel (after waiting aempty of its buffer, the
    buffer's previous k-chunks read by their MMAs, and arriving on afull),
    else reads the ring tile, arrives on rempty[slot], waits aempty and
    full[stage] (the MMAs read the B part too), writes its part and arrives
    on afull (count
    4 KPB; in the pair, both CTAs' sets arrive on the even CTA's afull, count
    8 KPB);
  - the (even CTA's) MMA thread waits afull at the first part of a buffer
    only, issues each k-chunk's MMAs, which read both CTAs' stage and A
    buffer part and accumulate into both CTAs' tensor memory, commits to
    empty[stage] after each k-chunk and to aempty[buffer] after the last
    part (both CTAs in the pair); after each 512-row group it commits to
    acc_full (both CTAs) and arrives on its own; in the pair a relay warp of
    the even CTA then copies the group's tag into the odd CTA and arrives on
    the odd CTA's acc_full, so that this release arrive does not hold up the
    MMA thread;
  - the epilogues drain the accumulators (acc_full / acc_empty, double
    buffered); the odd CTA also arrives on the even CTA's acc_empty.
Checked: no deadlock; every MMA reads, in both CTAs, the stage and A buffer of
its own unit and k-chunk; no A buffer or stage is overwritten before the MMAs
that read it have run; each epilogue sees every group of every unit once.
"""

import random

import pytest

EPI = 8


class Bar:
    def __init__(self, count):
        self.count = count
        self.pending = count
        self.tx = 0
        self.phase = 0

    def _check(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def arrive(self, n=1, tx=0):
        self.tx += tx
        self.pending -= n
        assert self.pending >= 0, "too many arrivals in one phase"
        self._check()

    def complete_tx(self, b):
        self.tx -= b
        self._check()

    def done(self, parity):
        return (self.phase & 1) != parity


class Cta:
    def __init__(self, ns, rs, nbuf, afull_count, acc_empty_count):
        self.full = [Bar(1) for _ in range(ns)]
        self.empty = [Bar(1) for _ in range(ns)]
        self.rfull = [Bar(1) for _ in range(rs)]
        self.rempty = [Bar(4) for _ in range(rs)]
        self.slot = [None] * rs             # ring tile in the slot: (unit, kc) once landed
        self.slot_unit = [None] * rs
        self.afull = [Bar(afull_count) for _ in range(nbuf)]
        self.aempty = [Bar(1) for _ in range(nbuf)]
        self.acc_full = [Bar(2) for _ in range(2)]
        self.acc_empty = [Bar(acc_empty_count) for _ in range(2)]
        self.hand_full = [Bar(1) for _ in range(2)]
        self.stage = [None] * ns            # B part in the stage: (unit, kc) once landed
        self.stage_unit = [None] * ns
        self.abuf = [[None, None] for _ in range(nbuf)]  # (unit, kc) converted into each part
        self.acc_unit = [None] * 2
        self.acc = [None] * 2               # (unit, group) accumulated
        self.seen = []                      # epilogue log


def run_model(pair, ns, n_units, kch, kgroup, seed, skip_aempty=False, kpb=1, afull_sets=None,
              relay_early=False, rs=None, early_release=False, skip_b_wait=False):
    rng = random.Random(seed)
    nbuf = 4 // kpb
    rs = ns if rs is None else rs
    sets = kpb if afull_sets is None else afull_sets
    if pair:
        ctas = [Cta(ns, rs, nbuf, 8 * sets, 2 * EPI), Cta(ns, rs, nbuf, 4 * sets, EPI)]
    else:
        ctas = [Cta(ns, rs, nbuf, 4 * sets, EPI)]
    mail, mail_full, mail_empty = [None] * 4, [Bar(1) for _ in range(4)], [Bar(1) for _ in range(4)]
    claims = [0]
    copies = []
    engine = []
    kgroups = (kch + kgroup - 1) // kgroup

    def wait(bar, parity):
        while not bar.done(parity):
            yield "blocked"

    def producer(r):
        cta = ctas[r]
        st = ph = 0
        sl = sph = 0
        mi = [0]

        def claim():
            if not pair:
                u = claims[0] if claims[0] < n_units else None
                claims[0] += 1
                return u
                yield
            ms, mph = mi[0] % 4, (mi[0] // 4) & 1
            mi[0] += 1
            if r == 0:
                u = claims[0] if claims[0] < n_units else None
                claims[0] += 1
                yield from wait(mail_empty[ms], mph ^ 1)
                mail[ms] = u
                mail_full[ms].arrive()
            else:
                yield from wait(mail_full[ms], mph)
                u = mail[ms]
                mail_empty[ms].arrive()
            return u

        def get():
            return (yield from claim())

        u = yield from get()
        un = (yield from get()) if u is not None else None
        while u is not None:
            for kc in range(kch):
                yield from wait(cta.rempty[sl], sph ^ 1)
                cta.slot_unit[sl] = (u, kc)
                cta.slot[sl] = None
                cta.rfull[sl].arrive(tx=1)
                copies.append((cta, "slot", sl, (u, kc)))
                sl, sph = (sl + 1) % rs, sph ^ (sl + 1 == rs)
                yield from wait(cta.empty[st], ph ^ 1)
                cta.stage_unit[st] = (u, kc)
                cta.stage[st] = None
                cta.full[st].arrive(tx=1)
                copies.append((cta, "stage", st, (u, kc)))
                st, ph = (st + 1) % ns, ph ^ (st + 1 == ns)
            u, un = un, None
            if u is not None:
                un = yield from get()
        for _ in range(2):
            yield from wait(cta.empty[st], ph ^ 1)
            cta.stage_unit[st] = "end"
            st, ph = (st + 1) % ns, ph ^ (st + 1 == ns)
            yield from wait(cta.rempty[sl], sph ^ 1)
            cta.slot_unit[sl] = "end"
            cta.rfull[sl].arrive()
            sl, sph = (sl + 1) % rs, sph ^ (sl + 1 == rs)
        if pair:
            for _ in range(2, ns):
                yield from wait(cta.empty[st], ph ^ 1)
                st, ph = (st + 1) % ns, ph ^ (st + 1 == ns)

    def converter(r, cs):
        cta = ctas[r]
        target = ctas[0]          # the pair's odd CTA arrives on the even CTA's afull
        it = 0
        while True:
            i = 2 * it + cs
            st, ph = i % ns, (i // ns) & 1
            sl, sph = i % rs, (i // rs) & 1
            bi = i // kpb
            ab, aph, part = bi % nbuf, (bi // nbuf) & 1, i % kpb
            yield from wait(cta.rfull[sl], sph)
            tag = cta.slot_unit[sl]
            # the A buffer's previous pair of k-chunks must have been read by
            # its MMAs, also before a sentinel: an early sentinel arrival would
            # complete the afull phase of that previous pair without the other
            # set's (or, in the pair, the other CTA's) arrivals
            if not (skip_aempty and tag == "end"):
                yield from wait(cta.aempty[ab], aph ^ 1)
            if tag == "end":
                target.afull[ab].arrive(4)
                return
            if early_release:
                cta.rempty[sl].arrive(4)
                yield "step"
            assert cta.slot[sl] == tag, "converter read a ring slot that has not landed or was refilled"
            if not early_release:
                cta.rempty[sl].arrive(4)
            if not skip_b_wait:
                yield from wait(cta.full[st], ph)
            cta.abuf[ab][part] = tag
            target.afull[ab].arrive(4)
            it += 1

    def mma():
        me = ctas[0]
        st = ph = buf = 0
        ci = [0]                  # k-chunk sequence number

        def wait_a():
            i = ci[0]
            if i % kpb == 0:
                bi = i // kpb
                yield from wait(me.afull[bi % nbuf], (bi // nbuf) & 1)

        aph = [0, 0]
        while True:
            yield from wait_a()
            tag = me.stage_unit[st]
            if tag == "end":
                yield from wait(me.acc_empty[buf], aph[buf] ^ 1)
                me.acc_unit[buf] = "end"
                if pair:
                    me.hand_full[buf].arrive()
                me.acc_full[buf].arrive(2)
                return
            u = tag[0]
            first = True
            for gi in range(kgroups):
                yield from wait(me.acc_empty[buf], aph[buf] ^ 1)
                for kc in range(gi * kgroup, min(kch, (gi + 1) * kgroup)):
                    if not first:
                        yield from wait_a()
                    first = False
                    i = ci[0]
                    ab, half = (i // kpb) % nbuf, i % kpb
                    engine.append(("mma", st, (ab, half), (u, kc), buf, gi))
                    engine.append(("commit", [c.empty[st] for c in ctas]))
                    if half == kpb - 1:
                        engine.append(("commit", [c.aempty[ab] for c in ctas]))
                    st, ph = (st + 1) % ns, ph ^ (st + 1 == ns)
                    ci[0] += 1
                me.acc_unit[buf] = (u, gi)
                engine.append(("commit", [c.acc_full[buf] for c in ctas]))
                if pair:
                    me.hand_full[buf].arrive()    # to the relay
                me.acc_full[buf].arrive()         # the issuing thread's own arrive
                aph[buf] ^= 1
                buf ^= 1

    def relay():
        me, odd = ctas[0], ctas[1]
        hb = 0
        hph = [0, 0]
        while True:
            yield from wait(me.hand_full[hb], hph[hb])
            tag = me.acc_unit[hb]
            if relay_early:
                odd.acc_full[hb].arrive()
                yield "step"
                odd.acc_unit[hb] = tag
            else:
                odd.acc_unit[hb] = tag        # remote store, ordered by the release arrive
                odd.acc_full[hb].arrive()
            if tag == "end":
                odd.acc_full[hb].arrive()
                return
            hph[hb] ^= 1
            hb ^= 1

    def epilogue(r):
        cta = ctas[r]
        buf = 0
        aph = [0, 0]
        while True:
            yield from wait(cta.acc_full[buf], aph[buf])
            tag = cta.acc_unit[buf]
            if tag == "end":
                return
            assert cta.acc[buf] == tag, "epilogue read an incomplete accumulator"
            cta.seen.append(tag)
            cta.acc[buf] = None
            cta.acc_empty[buf].arrive(EPI)
            if pair and r == 1:
                ctas[0].acc_empty[buf].arrive(EPI)
            aph[buf] ^= 1
            buf ^= 1

    def run_engine(op):
        if op[0] == "mma":
            _, st, (ab, half), want, buf, gi = op
            for c in ctas:
                assert c.stage[st] == want, "MMA read a stale B stage"
                assert c.abuf[ab][half] == want, "MMA read a stale A buffer"
                prev = c.acc[buf]
                c.acc[buf] = (want[0], gi)
                assert prev in (None, (want[0], gi)), "accumulator overwritten before it was read"
        else:
            for b in op[1]:
                b.arrive()

    actors = []
    for r in range(len(ctas)):
        actors += [producer(r), converter(r, 0), converter(r, 1), epilogue(r)]
    actors.append(mma())
    if pair:
        actors.append(relay())
    alive = list(actors)
    idle = 0
    while alive or copies or engine:
        kinds = ["actor"] * len(alive) + (["copy"] if copies else []) + (["engine"] if engine else [])
        k = rng.randrange(len(kinds))
        if kinds[k] == "copy":
            cta, kind, k, tag = copies.pop(rng.randrange(len(copies)))
            if kind == "slot":
                cta.slot[k] = tag
                cta.rfull[k].complete_tx(1)
            else:
                cta.stage[k] = tag
                cta.full[k].complete_tx(1)
            idle = 0
        elif kinds[k] == "engine":
            run_engine(engine.pop(0))
            idle = 0
        else:
            a = alive[k]
            try:
                if next(a) == "blocked":
                    idle += 1
                else:
                    idle = 0
            except StopIteration:
                alive.remove(a)
                idle = 0
        if not copies and not engine and alive and idle > 200 * len(alive):
            raise AssertionError("deadlock: %d actors blocked with nothing in flight" % len(alive))
    for c in ctas:
        want = [(u, gi) for u in range(n_units) for gi in range(kgroups)] if not pair else None
        if want is not None:
            assert sorted(c.seen) == want
    if pair:
        per = [(u, gi) for u in range(n_units) for gi in range(kgroups)]
        assert sorted(ctas[0].seen) == per and sorted(ctas[1].seen) == per
    return True


@pytest.mark.parametrize("pair,ns,rs", [(False, 5, 4), (False, 4, 6), (True, 8, 6), (True, 4, 6), (False, 6, 4), (True, 6, 10)])
@pytest.mark.parametrize("n_units,kch", [(0, 3), (1, 3), (5, 3), (3, 16), (7, 9)])
@pytest.mark.parametrize("kpb", [1, 2])
def test_protocol_random_interleavings(pair, ns, rs, n_units, kch, kpb):
    for seed in range(30):
        run_model(pair, ns, n_units, kch, 8, seed, kpb=kpb, rs=rs)


def test_sentinel_without_buffer_wait_is_caught():
    """Sensitivity: letting the sentinel skip its A-buffer wait (the mistake a
    GPU parity run exposed as an expired bounded wait) breaks the pair form
    with more stages than A buffers."""
    bad = 0
    for seed in range(60):
        try:
            run_model(True, 6, 1, 3, 8, seed, skip_aempty=True, kpb=1)
        except AssertionError:
            bad += 1
    assert bad > 0


@pytest.mark.parametrize("pair", [False, True])
@pytest.mark.parametrize("kpb", [1, 2])
def test_odd_b_stage_count_is_safe(pair, kpb):
    """A converter waits for its A buffer's previous use (the MMAs of k-chunk
    i - 4 and earlier) before the B stage of k-chunk i, so the stage's
    previous use i - NS has landed for any NS >= 4, odd or even."""
    for seed in range(30):
        run_model(pair, 5, 5, 9, 8, seed, kpb=kpb, rs=4)


@pytest.mark.parametrize("pair", [False, True])
@pytest.mark.parametrize("kpb", [1, 2])
@pytest.mark.parametrize("odd", ["slots"])
def test_odd_stage_count_is_caught(pair, kpb, odd):
    """Sensitivity: with an odd number of ring slots, k-chunk i - RS belongs
    to the other converter set, so a set can reach chunk i before the slot's
    previous copy has landed and pass its parity wait on the earlier phase
    (why the kernel requires an even count)."""
    bad = 0
    for seed in range(60):
        try:
            run_model(pair, 4, 5, 9, 8, seed, kpb=kpb, rs=5)
        except AssertionError:
            bad += 1
    assert bad > 0


@pytest.mark.parametrize("pair", [False, True])
def test_buffer_count_of_one_set_is_caught(pair):
    """Sensitivity: with two k-chunks per A buffer, an afull count that covers
    one converter set only (the count of one-k-chunk buffers) lets the MMA
    thread read the second part of a buffer before the other set has written
    it."""
    bad = 0
    for seed in range(40):
        try:
            run_model(pair, 4 if not pair else 6, 3, 5, 8, seed, kpb=2, afull_sets=1)
        except AssertionError:
            bad += 1
    assert bad > 0


def test_relay_arriving_before_the_tag_is_caught():
    """Sensitivity: a relay whose arrive on the odd CTA's acc_full is not
    ordered after the tag store (a relaxed arrive) lets the odd epilogue read
    the previous group's tag."""
    bad = 0
    for seed in range(60):
        try:
            run_model(True, 6, 3, 9, 2, seed, kpb=2, relay_early=True)
        except AssertionError:
            bad += 1
    assert bad > 0


@pytest.mark.parametrize("pair", [False, True])
def test_ring_slot_released_before_its_read_is_caught(pair):
    """Sensitivity: releasing a ring slot before the converters have read it
    lets the producer refill it under them."""
    bad = 0
    for seed in range(40):
        try:
            run_model(pair, 4, 3, 9, 8, seed, rs=2, early_release=True)
        except AssertionError:
            bad += 1
    assert bad > 0


@pytest.mark.parametrize("pair", [False, True])
def test_converter_skipping_the_b_stage_wait_is_caught(pair):
    """Sensitivity: signalling an A buffer without waiting for the k-chunk's B
    stage lets the MMAs read a B part still in flight."""
    bad = 0
    for seed in range(40):
        try:
            run_model(pair, 4, 3, 5, 8, seed, rs=6, skip_b_wait=True)
        except AssertionError:
            bad += 1
    assert bad > 0


def _kernel_cfg():
    """(NS, RS, KPB) of both forms, read from the kernel source's TmemCfg."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2604_04696_gb300", "csrc", "rowsel_tmem.cu"), encoding="utf-8").read()

    def value(name, pair):
        m = re.search(r"static constexpr int %s = ([^;]+);" % name, src)
        assert m, name
        e = m.group(1).strip()
        t = re.fullmatch(r"PAIR \? (\d+) : (\d+)", e)
        return int(t.group(1) if pair else t.group(2)) if t else int(e)

    return {pair: (value("NS", pair), value("RS", pair), value("KPB", pair)) for pair in (False, True)}


@pytest.mark.parametrize("pair", [False, True])
@pytest.mark.parametrize("n_units,kch", [(1, 1), (6, 3), (4, 16), (9, 5)])
def test_protocol_with_the_kernels_own_configuration(pair, n_units, kch):
    """The stage, ring-slot and A-buffer counts the kernel is compiled with
    (read from its source) run the protocol without deadlock or stale reads."""
    ns, rs, kpb = _kernel_cfg()[pair]
    assert rs % 2 == 0 and ns >= 4
    for seed in range(20):
        run_model(pair, ns, n_units, kch, 8, seed, kpb=kpb, rs=rs)
