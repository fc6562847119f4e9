"""A CPU model of the ring flow control of the tensor-memory RowSel kernel
(rowsel_tmem.cu) with several jobs in one launch, run under random
interleavings.

It restates the kernel's rules (no code is shared with the CUDA source):
  - jobs are numbered one after the other: job j has n_entries_j entries,
    kch_j k-chunks per entry and upe_j units per entry (pair form: a unit
    covers two consecutive entries of its job); entries, units and ingest
    tasks (entry, k-chunk) have one global index space each;
  - the ring has R slots of kch_max chunks; entry E lives in slot E % R;
  - one ready and one consumed counter per entry: a finished ingest task adds
    one to ready[E]; a unit adds one to consumed[E] (for each of its entries)
    once its last k-chunk of E has been copied out of the ring;
  - an ingest group claims tasks in increasing order and claims its next task
    while the current one is still being written, but runs a task's checks
    only at its start, after the previous task is published: the slot's
    previous entry E - R consumed by all its upe units, and (lookahead la) the
    unit claims past the first unit of entry E - la;
  - a producer claims units in increasing order, one ahead; it copies a
    unit's k-chunks one at a time once ready[E] = kch (each copy reads the
    ring), with at most `depth` copies waiting for the MMAs.
Checked: no state without an enabled step while work remains (no deadlock
for any residency), every copy reads its own entry's data, and every slot is
overwritten only after its previous entry was consumed.
"""

import random

import pytest


def run_model(jobs, R, la, n_ing, n_prod, pair, depth, seed, cumulative=False, early_release=False,
              check_before_publish=False):
    """jobs: [(n_entries, kch, upe)]. Switches for the sensitivity tests:
    cumulative: the counters of the base-256 kernel (one per ring slot,
    compared with (E / R) * upe of the entry's own job); early_release: a unit
    releases its entry after its first k-chunk; check_before_publish: the ingest
    runs its next task's ring check before publishing the current one."""
    rng = random.Random(seed)
    e0, u0, t0 = [], [], []
    ne = nu = nt = 0
    for n_e, kch, upe in jobs:
        e0.append(ne)
        u0.append(nu)
        t0.append(nt)
        ne += n_e
        nu += (n_e // 2 if pair else n_e) * upe
        nt += n_e * kch
    kch_max = max(j[1] for j in jobs)

    def job_of(base, x):
        j = 0
        while j + 1 < len(base) and x >= base[j + 1]:
            j += 1
        return j

    def entries_of(u):
        j = job_of(u0, u)
        ul = (u - u0[j]) // jobs[j][2]
        return j, ([e0[j] + 2 * ul, e0[j] + 2 * ul + 1] if pair else [e0[j] + ul])

    def first_unit_of(E):
        j = job_of(e0, E)
        return u0[j] + ((E - e0[j]) >> (1 if pair else 0)) * jobs[j][2]

    def task_entry(c):
        j = job_of(t0, c)
        tl = c - t0[j]
        return j, e0[j] + tl // jobs[j][1], tl % jobs[j][1]

    ready = [0] * (ne if not cumulative else R)
    consumed = [0] * (ne if not cumulative else R)
    ring = [[None] * kch_max for _ in range(R)]
    units_done_on = [0] * ne          # ground truth: units that finished copying each entry
    ctr_units = ctr_tasks = 0

    def may_write(E):
        j = job_of(e0, E)
        near = la == 0 or E < la or ctr_units >= first_unit_of(E - la)
        if E < R:
            return near
        if cumulative:
            return near and consumed[E % R] >= (E // R) * jobs[j][2]
        return near and consumed[E - R] >= jobs[job_of(e0, E - R)][2]

    def entry_ready(E):
        j = job_of(e0, E)
        if cumulative:
            return ready[E % R] >= (E // R + 1) * jobs[j][1]
        return ready[E] >= jobs[j][1]

    # ingest group: current task (checked or not, chunk written?) and next task
    ing = [{"cur": None, "ok": False, "next": None} for _ in range(n_ing)]
    # producer: claimed units (current first), next k-chunk of the current one
    prod = [{"units": [], "kc": 0, "inflight": 0} for _ in range(n_prod)]
    done = 0
    steps = 0
    while done < nu or ctr_tasks < nt or any(g["cur"] is not None for g in ing):
        steps += 1
        assert steps < 400000
        acts = []
        for i, g in enumerate(ing):
            if g["cur"] is None and g["next"] is None and ctr_tasks < nt:
                acts.append(("claim_task", i))
            if g["cur"] is not None and g["next"] is None and ctr_tasks < nt:
                acts.append(("claim_next", i))            # while the current task is in progress
            if g["cur"] is not None and not g["ok"] and may_write(task_entry(g["cur"])[1]):
                acts.append(("check", i))
            # the mistake: the next task's ring check blocks before the current
            # task is published (its claim comes first, while tasks remain)
            blocked = check_before_publish and g["cur"] is not None and (
                (g["next"] is None and ctr_tasks < nt) or (g["next"] is not None and not g.get("next_ok")))
            if g["cur"] is not None and g["ok"] and not blocked:
                acts.append(("write", i))
            if g["cur"] is None and g["next"] is not None:
                acts.append(("advance", i))
            if check_before_publish and g["cur"] is not None and g["ok"] and g["next"] is not None \
                    and not g.get("next_ok") and may_write(task_entry(g["next"])[1]):
                acts.append(("check_next", i))
        for i, p in enumerate(prod):
            if len(p["units"]) < 2 and ctr_units < nu:
                acts.append(("claim_unit", i))
            if p["units"] and p["inflight"] < depth:
                j, es = entries_of(p["units"][0])
                if all(entry_ready(E) for E in es):
                    acts.append(("copy", i))
            if p["inflight"]:
                acts.append(("mma", i))
        assert acts, "deadlock: no enabled step with work remaining"
        kind, i = rng.choice(acts)
        if kind == "claim_task":
            ing[i]["cur"], ing[i]["ok"] = ctr_tasks, False
            ctr_tasks += 1
        elif kind == "claim_next":
            ing[i]["next"] = ctr_tasks
            ctr_tasks += 1
        elif kind == "check":
            ing[i]["ok"] = True
        elif kind == "check_next":
            ing[i]["next_ok"] = True
        elif kind == "write":
            j, E, kc = task_entry(ing[i]["cur"])
            slot = ring[E % R]
            old = slot[kc]   # an earlier entry of this slot (a job with fewer k-chunks may leave older ones)
            assert old is None or (old < E and old % R == E % R and
                                   units_done_on[old] == jobs[job_of(e0, old)][2]), \
                "ring slot overwritten before its entry was consumed"
            slot[kc] = E
            if cumulative:
                ready[E % R] += 1
            else:
                ready[E] += 1
            ing[i]["cur"] = None
        elif kind == "advance":
            g = ing[i]
            g["cur"], g["next"] = g["next"], None
            g["ok"] = bool(g.pop("next_ok", False)) if check_before_publish else False
        elif kind == "claim_unit":
            prod[i]["units"].append(ctr_units)
            ctr_units += 1
        elif kind == "copy":
            p = prod[i]
            u = p["units"][0]
            j, es = entries_of(u)
            kc = p["kc"]
            for E in es:
                assert ring[E % R][kc] == E, "a copy read another entry's ring data"
            p["inflight"] += 1
            last = kc + 1 == jobs[j][1]
            if last:
                for E in es:
                    units_done_on[E] += 1
            if last or (early_release and kc == 0):
                for E in es:
                    if cumulative:
                        consumed[E % R] += 1
                    else:
                        consumed[E] += 1
            if last:
                p["units"].pop(0)
                p["kc"] = 0
                done += 1
            else:
                p["kc"] += 1
        else:
            prod[i]["inflight"] -= 1
    assert ctr_units == nu and ctr_tasks == nt


CASES = [
    # jobs [(entries, kch, upe)], R, la, ingest groups, producers, pair, depth
    ([(12, 2, 2)], 3, 0, 3, 3, False, 2),
    ([(12, 3, 2), (6, 1, 3), (10, 2, 1)], 4, 2, 3, 3, False, 2),
    ([(8, 4, 1), (9, 1, 4), (5, 3, 2), (7, 2, 3)], 3, 0, 2, 4, False, 3),
    ([(6, 2, 2), (4, 5, 1)], 2, 1, 1, 1, False, 1),                 # one CTA, the smallest ring
    ([(10, 2, 3), (10, 3, 2)], 20, 4, 4, 2, False, 2),              # ring holds everything
    ([(12, 2, 2)], 4, 2, 4, 2, True, 2),                            # pairs: two entries per unit
    ([(20, 2, 3)], 2, 2, 2, 1, True, 1),                            # one pair, the smallest ring
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "jobs%d_R%d_la%d_%s" % (
    len(c[0]), c[1], c[2], "pair" if c[5] else "single"))
def test_flow_control_progresses_and_reads_its_own_entry(case):
    for seed in range(40):
        run_model(*case, seed=seed)


def _fails(case, **kw):
    for seed in range(300):
        try:
            run_model(*case, seed=seed, **kw)
        except AssertionError as e:
            return str(e)
    return None


def test_cumulative_slot_counters_break_with_uneven_jobs():
    """Sensitivity: counters per ring slot compared with (E / R) * upe of the
    entry's own job (the single-job scheme) miscount once entries of jobs with
    different unit or k-chunk counts share a slot."""
    assert _fails(([(3, 2, 3), (6, 1, 1), (3, 3, 2)], 2, 0, 2, 2, False, 2), cumulative=True) is not None


def test_release_before_the_last_chunk_is_caught():
    """Sensitivity: releasing an entry when the unit's first k-chunk is copied
    lets the ingest overwrite chunks a copy still has to read."""
    msg = _fails(([(8, 4, 1), (4, 3, 1)], 2, 0, 3, 2, False, 2), early_release=True)
    assert msg is not None and "ring" in msg


def test_ring_check_before_publishing_deadlocks():
    """Sensitivity: running the next task's ring check before the current task
    is published (the next task's slot may be waiting for the current task's
    own entry) deadlocks once other groups claim in between."""
    msg = _fails(([(12, 1, 1)], 2, 0, 3, 2, False, 2), check_before_publish=True)
    assert msg is not None and "deadlock" in msg
