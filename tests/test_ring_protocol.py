"""A randomised model of the binary64 kernel's copy protocol (no GPU).

Thread 0 of every CTA issues the copies of its share of each k-stage into a
ring of STAGES slots: after each stage's release it refills the slots that
every receiving CTA has released, without waiting (refill(g + 1, g + 1 +
STAGES, block=False)), and before each stage it waits only when that stage is
not issued yet (refill(g, g + STAGES, block=True)).  A slot's "empty" barrier
completes one phase per stage when every CTA has released it, and the copy
tests it by parity, as mbarrier.try_wait.parity does.  The model runs the CTAs
of one cluster (each delivering to all the others, the worst case) in random
interleavings and checks that nothing deadlocks, that a copy only fills a slot
every receiver has released, and that the parity test is never ambiguous (the
barrier is never more than one phase behind the copy's expectation)."""
import random

import pytest

STAGES = 4


def run(ncta, total, seed):
    rnd = random.Random(seed)
    released = [[False] * total for _ in range(ncta)]
    issued = [0] * ncta
    gst = [0] * ncta
    at_top = [True] * ncta

    def completed(slot):
        # completed phases of the slot's empty barrier (every CTA released)
        k = 0
        while slot + k * STAGES < total and all(r[slot + k * STAGES] for r in released):
            k += 1
        return k

    def try_issue(c):
        i = issued[c]
        slot, need = i % STAGES, i // STAGES
        done = completed(slot)
        assert need - 1 <= done <= need, (c, i, done, need)    # within one phase
        parity_says = (done & 1) != ((need & 1) ^ 1)
        assert parity_says == (done >= need)                   # parity decides right
        return done >= need

    steps = 0
    while min(gst) < total:
        steps += 1
        assert steps < 10 ** 6, "deadlock"
        c = rnd.randrange(ncta)
        g = gst[c]
        if g >= total:
            continue
        if at_top[c]:
            while issued[c] < min(total, g + STAGES) and issued[c] <= g and try_issue(c):
                issued[c] += 1
            if issued[c] <= g or not all(issued[x] > g for x in range(ncta)):
                continue                       # waiting for a slot or for the stage's bytes
            at_top[c] = False
        else:
            for x in range(ncta):              # the copies of stage g have all landed
                assert issued[x] > g
            released[c][g] = True
            while issued[c] < min(total, g + 1 + STAGES) and try_issue(c):
                issued[c] += 1
            gst[c] += 1
            at_top[c] = True


@pytest.mark.parametrize("ncta", [1, 2, 4])
@pytest.mark.parametrize("total", [1, 3, 4, 5, 9, 40])
def test_ring_protocol(ncta, total):
    for seed in range(60):
        run(ncta, total, seed)
