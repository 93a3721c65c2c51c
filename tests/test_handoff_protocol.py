"""CPU model of the named-barrier hand-off between the recursion warps and the
output warps of the warp-specialised generation kernel (mtgp_device.cuh,
run_item_split).  The kernel's schedule is restated here as two operation
lists; a random-interleaving simulator checks, for many round counts, buffer
sizes and ring depths K, that

  * the schedule never deadlocks;
  * no party arrives twice at a barrier instance before it completes (that
    would complete the barrier early on hardware);
  * every barrier is idle (no pending arrivals) when the work item ends, so
    the next work item starts from clean barriers;
  * the output warps read a round only after the recursion warps published it
    and the recursion warps compact the buffer only after the output warps
    have consumed every earlier round.
"""
import random

import pytest


def schedule(rounds: int, K: int, compact_every: int):
    """Operation lists (recursion, output) for one work item.

    Recursion warps, round r: if r is a compaction round, drain (sync EMPTY of
    every round not yet drained) and compact; else if r - K >= drained, sync
    EMPTY of round r - K; compute round r; arrive FULL[r % K].  After the last
    round, drain the rest.  Output warps, round r: sync FULL[r % K]; read;
    arrive EMPTY[r % K].
    """
    rec, out = [], []
    drained = 0
    for r in range(rounds):
        if r > 0 and r % compact_every == 0:
            for j in range(max(drained, r - K), r):
                rec.append(("sync", ("E", j % K), j))
            drained = r
            rec.append(("compact", r))
        elif r - K >= drained:
            rec.append(("sync", ("E", (r - K) % K), r - K))
        rec.append(("compute", r))
        rec.append(("arrive", ("F", r % K), r))
        out.append(("sync", ("F", r % K), r))
        out.append(("read", r))
        out.append(("arrive", ("E", r % K), r))
    for j in range(max(drained, rounds - K), rounds):
        rec.append(("sync", ("E", j % K), j))
    return rec, out


def simulate(rec, out, seed):
    rnd = random.Random(seed)
    ops = {"R": rec, "O": out}
    pc = {"R": 0, "O": 0}
    pending = {}              # barrier -> {party: tag}
    waiting = {}              # party -> barrier it is blocked on
    published, consumed = set(), set()
    compacted_at = []
    steps = 0
    while pc["R"] < len(rec) or pc["O"] < len(out) or waiting:
        steps += 1
        assert steps < 10 ** 6
        runnable = [p for p in ("R", "O") if p not in waiting and pc[p] < len(ops[p])]
        if not runnable:
            raise AssertionError(f"deadlock: waiting={waiting} pending={pending}")
        p = rnd.choice(runnable)
        op = ops[p][pc[p]]
        pc[p] += 1
        if op[0] in ("arrive", "sync"):
            b, tag = op[1], op[2]
            arrived = pending.setdefault(b, {})
            assert p not in arrived, f"{p} arrives twice at {b} (tags {arrived[p]}, {tag})"
            arrived[p] = tag
            if op[0] == "sync":
                waiting[p] = b
            if len(arrived) == 2:                  # both groups arrived: complete
                tags = set(arrived.values())
                assert len(tags) == 1, f"barrier {b} mixes rounds {tags}"
                del pending[b]
                for q in [q for q, wb in waiting.items() if wb == b]:
                    del waiting[q]
        elif op[0] == "compute":
            published.add(op[1])
        elif op[0] == "read":
            assert op[1] in published
            consumed.add(op[1])
        elif op[0] == "compact":
            assert all(j in consumed for j in range(op[1])), "compaction before consumption"
            compacted_at.append(op[1])
    assert not pending, f"barriers left with pending arrivals: {pending}"
    assert consumed == set(range(len([o for o in out if o[0] == 'read'])))


@pytest.mark.parametrize("K", [1, 2, 3, 4])
@pytest.mark.parametrize("rounds", [0, 1, 2, 3, 4, 5, 7, 8, 9, 31, 64])
@pytest.mark.parametrize("compact_every", [1, 2, 3, 5, 1000])
def test_handoff_schedule(K, rounds, compact_every):
    rec, out = schedule(rounds, K, compact_every)
    for seed in range(30):
        simulate(rec, out, seed)


def test_model_catches_a_broken_schedule():
    # dropping the final drain leaves EMPTY arrivals pending: the model must flag it
    rec, out = schedule(9, 3, 1000)
    rec = [op for op in rec if not (op[0] == "sync" and op[2] >= 6)]
    with pytest.raises(AssertionError):
        simulate(rec, out, 0)
    # dropping the EMPTY syncs of early rounds lets the recursion warps run more
    # than K rounds ahead: a FULL barrier then collects two of their arrivals
    rec, out = schedule(12, 2, 1000)
    bad = [op for op in rec if not (op[0] == "sync" and op[1][0] == "E" and op[2] < 8)]
    with pytest.raises(AssertionError):
        for seed in range(50):
            simulate(bad, out, seed)
