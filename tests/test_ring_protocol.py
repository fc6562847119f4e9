"""A CPU model of the flow control of the fused tensor-core RowSel kernel (the
digit ring between the ingest warps and the GEMM warps), in both its
single-CTA and SM-pair forms, run under random interleavings.

It restates the kernel's rules (no code is shared with the CUDA source):
  - ingest tasks (entry E, k-chunk) are claimed in increasing order from one
    counter; a task may write ring slot E % R only once the previous occupant
    E - R is fully consumed (consumed[E % R] >= (E / R) * upe) and, with a
    lookahead of `la` entries, once the unit claims reach
    ((E - la) >> s) * upe (s = 1 in the pair form, where a claimed unit covers
    two entries); a finished task counts into ready[E % R];
  - units are claimed in increasing order (in the pair form by the even CTA,
    which hands each claim to the odd CTA); a unit waits until ready shows
    every k-chunk of its entry (of both entries in the pair form), and
    releases the entry (consumed[E % R] += 1) when its epilogue finishes;
  - a CTA's producer claims its next unit only after issuing the current one,
    and at most `depth` issued units wait for their epilogues.
The checks: no state without an enabled step while work remains (no deadlock
for any residency), and every unit reads exactly the ring contents of its own
entry (no overwrite before consumption, no read before the data is complete).
"""

import random

import pytest


def run_model(n_entries, R, kch, upe, la, n_cta, pair, depth, seed, wait_consumed=True, shift=None):
    """wait_consumed / shift: switches for the sensitivity tests (the kernel's
    rules are the defaults)."""
    rng = random.Random(seed)
    if shift is None:
        shift = 1 if pair else 0
    n_units = (n_entries // 2 if pair else n_entries) * upe
    n_tasks = n_entries * kch
    ctr_units = 0
    ctr_tasks = 0
    ready = [0] * R
    consumed = [0] * R
    ring = [[None] * kch for _ in range(R)]      # which entry each ring slot's k-chunk holds
    ingest = [None] * n_cta                      # claimed task waiting for its conditions
    producer = [None] * (n_cta // 2 if pair else n_cta)   # claimed unit waiting for ready
    pending = [[] for _ in producer]             # issued units waiting for the epilogue
    done_units = 0

    def entries_of(u):
        E2 = u // upe
        return [2 * E2, 2 * E2 + 1] if pair else [E2]

    def task_may_write(c):
        E = c // kch
        near = la == 0 or E < la or ctr_units >= ((E - la) >> shift) * upe
        free = not wait_consumed or E < R or consumed[E % R] >= (E // R) * upe
        return near and free

    def unit_ready(u):
        return all(ready[E % R] >= (E // R + 1) * kch for E in entries_of(u))

    steps = 0
    while done_units < n_units or ctr_tasks < n_tasks or any(t is not None for t in ingest):
        steps += 1
        assert steps < 200000
        actions = []
        for i in range(n_cta):
            if ingest[i] is None and ctr_tasks < n_tasks:
                actions.append(("claim_task", i))
            elif ingest[i] is not None and task_may_write(ingest[i]):
                actions.append(("ingest", i))
        for p in range(len(producer)):
            if producer[p] is None and ctr_units < n_units and len(pending[p]) < depth:
                actions.append(("claim_unit", p))
            elif producer[p] is not None and unit_ready(producer[p]):
                actions.append(("issue", p))
            if pending[p]:
                actions.append(("epilogue", p))
        assert actions, "deadlock: no enabled step with work remaining"
        kind, i = rng.choice(actions)
        if kind == "claim_task":
            ingest[i] = ctr_tasks
            ctr_tasks += 1
        elif kind == "ingest":
            c = ingest[i]
            E, kc = divmod(c, kch)
            slot = ring[E % R]
            assert slot[kc] is None or slot[kc] == E - R      # previous occupant, fully consumed
            slot[kc] = E
            ready[E % R] += 1
            ingest[i] = None
        elif kind == "claim_unit":
            producer[i] = ctr_units
            ctr_units += 1
        elif kind == "issue":
            u = producer[i]
            for E in entries_of(u):
                assert ring[E % R] == [E] * kch               # complete, and still this entry's data
            pending[i].append(u)
            producer[i] = None
        else:   # the oldest issued unit's epilogue finishes
            u = pending[i].pop(0)
            for E in entries_of(u):
                assert ring[E % R] == [E] * kch
                consumed[E % R] += 1
            done_units += 1
    assert ctr_units == n_units and ctr_tasks == n_tasks
    assert sum(consumed) == n_units * (2 if pair else 1)


CASES = [
    # n_entries, R, kch, upe, la, n_cta, pair, depth
    (12, 3, 2, 2, 0, 3, False, 2),
    (12, 3, 2, 2, 2, 3, False, 2),
    (20, 5, 3, 4, 3, 4, False, 2),
    (9, 2, 1, 3, 2, 1, False, 1),       # one CTA, the smallest ring
    (16, 16, 2, 2, 4, 5, False, 3),     # ring holds everything
    (12, 4, 2, 2, 0, 4, True, 2),       # pairs: two entries per unit
    (12, 4, 2, 2, 2, 4, True, 2),
    (20, 2, 2, 3, 2, 2, True, 1),       # one pair, the smallest ring
    (24, 6, 3, 2, 4, 6, True, 2),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "E%d_R%d_kch%d_upe%d_la%d_cta%d_%s" % (
    c[0], c[1], c[2], c[3], c[4], c[5], "pair" if c[6] else "single"))
def test_ring_protocol_progresses_and_reads_its_own_entry(case):
    for seed in range(40):
        run_model(*case, seed=seed)


def _fails(case, **kw):
    for seed in range(200):
        try:
            run_model(*case, seed=seed, **kw)
        except AssertionError as e:
            return str(e)
    return None


def test_model_catches_a_missing_consumption_wait():
    """Sensitivity: without the consumed[] condition an ingest task overwrites a
    ring slot that a unit still has to read, and the model notices."""
    assert _fails((12, 2, 2, 3, 0, 3, False, 2), wait_consumed=False) is not None


def test_pair_lookahead_needs_its_shift():
    """Sensitivity: in the pair form a claimed unit covers two entries; comparing
    entries with claims without the shift makes an ingest task wait for claims
    that need its own entry, and the model deadlocks."""
    msg = _fails((12, 4, 2, 2, 2, 4, True, 2), shift=0)
    assert msg is not None and "deadlock" in msg
