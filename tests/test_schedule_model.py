"""The time-sliced planner's queue protocol, checked as a model on random interleavings (CPU).

The kernel's persistent CTAs share one queue of problems (a ring of n slots with lap
markers): a ticket below n starts a problem; a later ticket takes the problem pushed as
number ticket - n, whose slot is s = u % n in lap L = u // n. A pusher waits until the slot
reads 2L (its previous occupant taken), stores the problem and marks 2L + 1; a taker waits
for 2L + 1, reads the problem and marks 2L + 2. A CTA takes a ticket only while a problem
waits for one (compare-and-swap on the head), and ends when none waits. After a slice a CTA
keeps its problem when nothing waits or when the problem is slow; otherwise it pushes it and
takes the next ticket. Every CTA step below is one atomic step of the model (the decision
to push and the tail ticket are separate steps, as in the kernel, and so are the queue
check and the head's compare-and-swap); the scheduler picks the next CTA at random.

Checked: every problem runs all its rounds, in order, exactly once and ends; no CTA waits
forever; and a slot is never overwritten before it was read."""
import random

import pytest


def run_model(n, grid, need, first, sl, seed, keep_prob):
    rng = random.Random(seed)
    head = tail = 0
    seq = [0] * n
    ring = [-1] * n
    done_rounds = [0] * n
    finished = set()
    ctas = {c: ("pick", None) for c in range(grid)}
    exited = set()
    holder = {}  # problem -> CTA currently holding it
    steps = 0
    while len(exited) < grid:
        steps += 1
        if steps > 2_000_000:
            return None  # livelock or deadlock
        c = rng.choice([k for k in ctas if k not in exited])
        phase, data = ctas[c]
        if phase == "pick":  # data: a problem kept from the last slice, or None
            if data is not None:
                ctas[c] = ("run", data)
                continue
            h, tl = head, tail
            if h >= n and h - n >= tl:
                exited.add(c)
                continue
            ctas[c] = ("cas", (h, tl))
        elif phase == "cas":
            h, _ = data
            if head != h:  # another CTA took the ticket: look again
                ctas[c] = ("pick", None)
                continue
            head = h + 1
            if h < n:
                ctas[c] = ("run", h)
            else:
                ctas[c] = ("take", h - n)
        elif phase == "take":
            u = data
            s, lap = u % n, u // n
            if seq[s] == 2 * lap + 1:
                p = ring[s]
                seq[s] = 2 * lap + 2
                ctas[c] = ("run", p)
        elif phase == "run":
            p = data
            assert p not in finished, "a finished problem ran again"
            assert holder.get(p, c) == c, "two CTAs hold one problem"
            holder[p] = c
            r0 = done_rounds[p]
            done_rounds[p] = min(need[p], r0 + (first if r0 == 0 else sl))
            if done_rounds[p] >= need[p]:
                finished.add(p)
                del holder[p]
                ctas[c] = ("pick", None)
                continue
            waiting = head < n or tail > head - n
            if waiting and rng.random() >= keep_prob:
                del holder[p]
                ctas[c] = ("ticket", p)
            else:
                ctas[c] = ("pick", p)
        elif phase == "ticket":
            u = tail
            tail += 1
            ctas[c] = ("push", (u, data))
        elif phase == "push":
            u, p = data
            s, lap = u % n, u // n
            if seq[s] == 2 * lap:
                ring[s] = p
                seq[s] = 2 * lap + 1
                ctas[c] = ("pick", None)
    assert finished == set(range(n))
    assert done_rounds == need
    return steps


@pytest.mark.parametrize("keep_prob", [0.0, 0.3])
def test_queue_protocol_finishes_every_problem_exactly_once(keep_prob):
    for seed in range(400):
        rng = random.Random(seed)
        n, grid = rng.randint(1, 48), rng.randint(1, 32)
        need = [rng.randint(1, 24) for _ in range(n)]
        steps = run_model(n, grid, need, rng.randint(1, 8), rng.randint(1, 4), seed, keep_prob)
        assert steps is not None, (seed, n, grid)
