"""Binomial checkpoint schedule of the gradient pass (host logic, no GPU).

Every schedule is replayed here: each reversal must find the state of its
segment current, segments must be reversed last to first, slots must stay
within the budget, and the number of segment advances must equal the
minimum found by brute force over all recursive split points."""
from functools import lru_cache

import pytest


@pytest.fixture(scope="module")
def fw():
    from paper_1609_03361_gb300 import build, fdwave
    build.build()
    return fdwave


ADVANCE, TAKESHOT, RESTORE, REVERSE = 1, 2, 3, 4


@lru_cache(None)
def best_advances(l, c):
    """Fewest segment advances to reverse l segments from a held start state
    with c free slots: advance j, store, reverse the right part with c - 1
    slots, then the left part with c; without slots, re-advance from the start
    for every segment."""
    if l == 1:
        return 0
    if c == 0:
        return l * (l - 1) // 2
    return min(j + best_advances(l - j, c - 1) + best_advances(j, c) for j in range(1, l))


def replay(actions, nseg, nslots):
    cur, slots, advances, order, used = 0, {}, 0, [], 0
    for op, arg in actions:
        if op == ADVANCE:
            assert arg > cur
            advances += arg - cur
            cur = arg
        elif op == TAKESHOT:
            assert 0 <= arg < nslots
            slots[arg] = cur
            used = max(used, len(slots))
        elif op == RESTORE:
            cur = 0 if arg == -1 else slots[arg]
        elif op == REVERSE:
            assert arg == cur, "reversal without its start state"
            order.append(arg)
        else:
            raise AssertionError(op)
    assert order == list(range(nseg - 1, -1, -1))
    return advances, used


@pytest.mark.parametrize("nslots", [0, 1, 2, 3, 5])
def test_schedule_is_valid_and_optimal(fw, nslots):
    for nseg in range(1, 41):
        acts = fw.fdw_checkpoint_schedule(nseg, nslots)
        adv, used = replay(acts, nseg, nslots)
        assert used <= nslots
        assert adv == best_advances(nseg, nslots), (nseg, nslots)


def test_first_sweep_ends_at_last_segment(fw):
    # the forward call performs every action before the first reversal: it
    # must only advance and store, and end at the start of the last segment
    for nseg, nslots in [(9, 2), (30, 3), (200, 10), (17, 1)]:
        acts = fw.fdw_checkpoint_schedule(nseg, nslots)
        first = next(i for i, a in enumerate(acts) if a[0] == REVERSE)
        assert all(op in (ADVANCE, TAKESHOT) for op, _ in acts[:first])
        assert acts[first] == (REVERSE, nseg - 1)
        cur = max([arg for op, arg in acts[:first] if op == ADVANCE], default=0)
        assert cur == nseg - 1


def test_enough_slots_means_no_recomputation(fw):
    for nseg in (2, 5, 12):
        adv, _ = replay(fw.fdw_checkpoint_schedule(nseg, nseg - 1), nseg, nseg - 1)
        assert adv == nseg - 1      # the forward sweep only


def test_large_schedule_cost(fw):
    # 200 segments (2000 steps, 10 per segment) with 10 pairs: the extra
    # advances of the reverse sweep stay below two more forward passes
    acts = fw.fdw_checkpoint_schedule(200, 10)
    adv, used = replay(acts, 200, 10)
    assert used <= 10 and adv - 199 < 2 * 200


def test_bad_arguments(fw):
    L = fw.lib()
    assert L.fdw_checkpoint_schedule(0, 1, None, 0) == -1
    assert L.fdw_checkpoint_schedule(3, -1, None, 0) == -1
    assert L.fdw_checkpoint_schedule(5, 1, None, 0) > 0   # size query writes nothing
