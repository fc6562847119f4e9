"""A CPU model of the stage-level protocol of the SM-pair form of the fused
tensor-core RowSel kernel (two CTAs, cta_group::2 MMAs issued by the even
CTA), run under random interleavings.

The model restates the kernel's rules with exact mbarrier semantics (arrival
count, transaction bytes, phase parity; no code is shared with the CUDA
source):
  - the even CTA's producer claims units and passes each to the odd CTA's
    producer through a mailbox of P_MAIL slots (mail_full / mail_empty);
  - each producer fills its own stage st for every k-chunk after empty[st]
    (arrive.expect_tx on its full[st]; the copies complete asynchronously);
  - the odd CTA's warp 1 waits full[st] and arrives on the even CTA's
    pfull[st]; per accumulator group it also waits its own acc_empty (count 8),
    writes its acc_unit and arrives once on its acc_full;
  - the even CTA's MMA thread waits full[st] and pfull[st], issues the MMAs
    (read both CTAs' stage st, accumulate into both CTAs' tensor memory) and
    commits: the commits arrive on empty[st] and acc_full[b] of both CTAs once
    the MMAs before them have executed, in order;
  - each epilogue waits acc_full[b] (count 2: commit + own warp-1 arrive),
    reads its tensor memory and arrives on its acc_empty[b] (8 warps); the odd
    epilogue also arrives on the even CTA's acc_empty[b] (count 16 there);
  - the end of work is a sentinel stage in each CTA.
Checked: no deadlock; every MMA reads the stage data of its own unit and
k-chunk in both CTAs; no accumulator is overwritten before both epilogues
have read it; every epilogue reads a complete group of its unit.
"""

import random

import pytest

NST = 4
EPI = 8


class Bar:
    def __init__(self, count):
        self.count = count
        self.pending = count
        self.tx = 0
        self.phase = 0          # completed phases

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
    def __init__(self, even, even_acc_empty=2 * EPI):
        self.full = [Bar(1) for _ in range(NST)]
        self.empty = [Bar(1) for _ in range(NST)]
        self.pfull = [Bar(1) for _ in range(NST)]
        self.acc_full = [Bar(2) for _ in range(2)]
        self.acc_empty = [Bar(even_acc_empty if even else EPI) for _ in range(2)]
        self.stage = [None] * NST          # (unit, k-chunk) held by stage st
        self.stage_unit = [None] * NST
        self.acc_unit = [None] * 2
        self.tmem = [None] * 2             # [unit, group, chunks so far, read-by-epilogue]


def run_model(n_units, kch, kgroup, p_mail, seed, even_acc_empty=2 * EPI, wait_relay=True, release_mail=True):
    """even_acc_empty / wait_relay / release_mail: switches for the sensitivity
    tests (the kernel's rules are the defaults)."""
    rng = random.Random(seed)
    E, O = Cta(True, even_acc_empty), Cta(False)
    mail = [None] * p_mail
    mail_full = [Bar(1) for _ in range(p_mail)]
    mail_empty = [Bar(1) for _ in range(p_mail)]
    claims = [0]
    copies = []            # in-flight copies: (cta, st, bytes)
    engine = []            # issued MMA-side operations, executed in order
    kgroups = (kch + kgroup - 1) // kgroup
    seen = {"E": [], "O": []}

    def wait(bar, parity):
        while not bar.done(parity):
            yield

    def producer(cta, even):
        st = ph = mi = 0
        while True:
            ms, mph = mi % p_mail, (mi // p_mail) & 1
            mi += 1
            if even:
                u = claims[0] if claims[0] < n_units else None
                claims[0] += 1
                yield from wait(mail_empty[ms], mph ^ 1)
                mail[ms] = u
                mail_full[ms].arrive()
            else:
                yield from wait(mail_full[ms], mph)
                u = mail[ms]
                if release_mail:
                    mail_empty[ms].arrive()
            if u is None:
                break
            for kc in range(kch):
                yield from wait(cta.empty[st], ph ^ 1)
                cta.stage_unit[st] = u
                cta.stage[st] = None                  # being refilled
                cta.full[st].arrive(tx=2)
                copies.append((cta, st, (u, kc)))
                st, ph = (st + 1) % NST, ph ^ (st + 1 == NST)
        # sentinel stage, then drain the commits that target this CTA
        yield from wait(cta.empty[st], ph ^ 1)
        cta.stage_unit[st] = None
        cta.full[st].arrive()
        for _ in range(1, NST):
            st, ph = (st + 1) % NST, ph ^ (st + 1 == NST)
            yield from wait(cta.empty[st], ph ^ 1)

    def mma_or_relay(cta, even):
        st = ph = buf = 0
        aph = [0, 0]
        while True:
            yield from wait(cta.full[st], ph)
            u = cta.stage_unit[st]
            if u is None:
                yield from wait(cta.acc_empty[buf], aph[buf] ^ 1)
                cta.acc_unit[buf] = None
                cta.acc_full[buf].arrive(2)
                return
            first = True
            for gi in range(kgroups):
                yield from wait(cta.acc_empty[buf], aph[buf] ^ 1)
                c0, c1 = gi * kgroup, min(kch, gi * kgroup + kgroup)
                for kc in range(c0, c1):
                    if not first:
                        yield from wait(cta.full[st], ph)
                    first = False
                    if not even:
                        E.pfull[st].arrive()
                    else:
                        if wait_relay:
                            yield from wait(E.pfull[st], ph)
                        engine.append(("mma", st, u, kc, buf, kc == c0, gi))
                        engine.append(("commit_empty", st))
                    st, ph = (st + 1) % NST, ph ^ (st + 1 == NST)
                cta.acc_unit[buf] = (u, gi, gi + 1 == kgroups)
                if even:
                    engine.append(("commit_acc", buf))
                cta.acc_full[buf].arrive()
                aph[buf] ^= 1
                buf ^= 1

    def epilogue(cta, even, name):
        buf = 0
        aph = [0, 0]
        while True:
            yield from wait(cta.acc_full[buf], aph[buf])
            tag = cta.acc_unit[buf]
            if tag is None:
                return
            u, gi, _last = tag
            t = cta.tmem[buf]
            c0, c1 = gi * kgroup, min(kch, gi * kgroup + kgroup)
            assert t is not None and t[0] == u and t[1] == gi and t[2] == list(range(c0, c1)), (name, tag, t)
            t[3].add(name)
            seen[name].append((u, gi))
            cta.acc_empty[buf].arrive(EPI)
            if not even:
                E.acc_empty[buf].arrive(EPI)
            aph[buf] ^= 1
            buf ^= 1

    agents = [producer(E, True), producer(O, False), mma_or_relay(E, True), mma_or_relay(O, False),
              epilogue(E, True, "E"), epilogue(O, False, "O")]
    alive = list(agents)
    steps = 0
    while alive or copies or engine:
        steps += 1
        assert steps < 500000
        choices = [("agent", a) for a in alive] + [("copy", i) for i in range(len(copies))]
        if engine:
            choices.append(("engine", 0))
        kind, x = rng.choice(choices)
        if kind == "copy":
            cta, st, data = copies.pop(x)
            cta.stage[st] = data
            cta.full[st].complete_tx(2)
        elif kind == "engine":
            op = engine.pop(0)
            if op[0] == "mma":
                _, st, u, kc, buf, first, gi = op
                for cta in (E, O):
                    assert cta.stage[st] == (u, kc), "MMA read stale stage data"
                    if first:
                        old = cta.tmem[buf]
                        assert old is None or ("E" if cta is E else "O") in old[3], \
                            "accumulator overwritten before its epilogue read it"
                        cta.tmem[buf] = [u, gi, [kc], set()]
                    else:
                        assert cta.tmem[buf][0] == u
                        cta.tmem[buf][2].append(kc)
            elif op[0] == "commit_empty":
                E.empty[op[1]].arrive()
                O.empty[op[1]].arrive()
            else:
                E.acc_full[op[1]].arrive()
                O.acc_full[op[1]].arrive()
        else:
            try:
                next(x)
            except StopIteration:
                alive.remove(x)
        # deadlock: every live agent blocked and nothing asynchronous pending
        if not copies and not engine and alive:
            if all(_blocked(a) for a in alive):
                raise AssertionError("deadlock")
    groups = [(u, g) for u in range(n_units) for g in range(kgroups)]
    assert seen["E"] == groups and seen["O"] == groups


def _blocked(gen):
    """True if the generator sits in a wait whose condition is false (peeked
    through the frame of the innermost wait)."""
    f = gen.gi_frame
    sub = gen.gi_yieldfrom
    while sub is not None and getattr(sub, "gi_yieldfrom", None) is not None:
        sub = sub.gi_yieldfrom
    if sub is None or sub.gi_frame is None:
        return False
    loc = sub.gi_frame.f_locals
    if "bar" in loc and "parity" in loc:
        return not loc["bar"].done(loc["parity"])
    return False


CASES = [
    # n_units, kch, kgroup, p_mail
    (3, 4, 2, 4),
    (5, 1, 1, 4),        # one chunk per unit: the sentinel follows at once
    (4, 5, 2, 2),        # ragged last group, a small mailbox
    (6, 3, 8, 1),        # one group per unit, a one-slot mailbox
    (1, 9, 4, 4),
    (0, 4, 2, 4),        # no work: both sentinels only
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "u%d_kch%d_kg%d_mail%d" % c)
def test_pair_protocol(case):
    for seed in range(60):
        run_model(*case, seed=seed)


def _fails(case, **kw):
    for seed in range(300):
        try:
            run_model(*case, seed=seed, **kw)
        except AssertionError as e:
            return str(e)
    return None


def test_even_acc_empty_must_count_both_epilogues():
    """With a count of 8 on the even CTA's acc_empty the 16 arrivals of one use
    complete two phases: the pair MMAs either overwrite an accumulator an
    epilogue has not read yet or lose the phase and stall. Either is caught."""
    msg = _fails((4, 2, 1, 4), even_acc_empty=EPI)
    assert msg is not None and ("overwritten" in msg or "deadlock" in msg)


def test_mma_must_wait_for_the_relay():
    """Without the wait on pfull the MMAs can read the odd CTA's stage before
    its copies have landed."""
    msg = _fails((4, 4, 2, 4), wait_relay=False)
    assert msg is not None and "stale" in msg


def test_mailbox_slots_must_be_released():
    """If the odd producer never frees mailbox slots, the even producer stalls
    once the mailbox is full: the model reports a deadlock."""
    msg = _fails((6, 1, 1, 2), release_mail=False)
    assert msg is not None and "deadlock" in msg
