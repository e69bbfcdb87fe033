"""The thread kernel's hand-off between warps, as a protocol model on the CPU.

The kernel's steps are replayed one atomic operation at a time by Python
generators under random interleavings (many seeds).  Counters as in the
kernel: `avail` (registrations of waiting warps not yet claimed), `head`
(states taken), `tail` (states claimed for writing), `multi` (warps that may
still hand off: every warp from its start until it runs at most one
trajectory), one sequence word per slot.  A producer warp hands off only
after taking one registration; a waiting warp leaves only by taking back an
unclaimed registration, once `multi` is zero or after an idle limit.  Each
schedule must end with every trajectory finished exactly once, every warp
gone and no state left in the ring; at every step the warps still waiting
are at least the states claimed and not yet taken (the invariant that
leaves no state without a taker: waiting = unclaimed registrations + claimed
and untaken states)."""
import random

import pytest


class Pool:
    def __init__(self):
        self.avail = 0
        self.head = 0
        self.tail = 0
        self.multi = 0
        self.seq = {}        # slot index -> trajectory written there
        self.claims = 0      # registrations claimed by producers (for the invariant)
        self.waiting = 0     # warps between registering and taking a state or leaving


def take_one(pool):
    """CAS loop on avail: take one unit if positive (one atomic step per try)."""
    if pool.avail > 0:
        pool.avail -= 1
        return True
    return False


def warp(pool, name, trajs, finished, rng, idle_limit):
    """One warp: its own trajectories (cooperative mode with hand-off), then
    waiting for handed-off ones.  Yields after every atomic operation."""
    live = list(trajs)
    pool.multi += 1                     # counted from its start
    yield
    in_multi = True
    while live:
        if in_multi and len(live) < 2:
            pool.multi -= 1             # at most one trajectory left
            in_multi = False
            yield
        # a batch of its trajectories
        if rng.random() < 0.3:
            finished.append(live.pop(rng.randrange(len(live))))
            yield
            continue
        if in_multi and len(live) >= 2 and pool.avail > 0:   # avail seen at the batch start
            yield
            if take_one(pool):          # claim one waiting warp
                pool.claims += 1
                yield
                idx = pool.tail         # atomicAdd(tail, 1)
                pool.tail += 1
                yield
                t = live.pop()          # write the state, then its sequence word
                yield
                pool.seq[idx] = t
                yield
                continue
        yield
    if in_multi:
        pool.multi -= 1
        yield
    # waiting for handed-off trajectories
    while True:
        pool.avail += 1                 # register
        pool.waiting += 1
        yield
        idle = 0
        got = None
        while True:
            if pool.head < pool.tail:
                idx = pool.head         # CAS(head, h, h + 1)
                pool.head += 1
                got = idx
                yield
                break
            if pool.multi == 0 or idle >= idle_limit:
                if take_one(pool):      # take back an unclaimed registration
                    pool.waiting -= 1
                    yield
                    return
            idle += 1
            yield
        while got not in pool.seq:      # the producer is still writing
            yield
        t = pool.seq.pop(got)
        pool.waiting -= 1
        pool.claims -= 1
        yield
        finished.append(t)              # runs it alone (no hand-off with one trajectory)
        yield


def run_schedule(seed, n_warps, max_traj, idle_limit):
    rng = random.Random(seed)
    pool = Pool()
    finished = []
    all_traj = []
    actors = []
    nxt = 0
    for w in range(n_warps):
        k = rng.randint(0, max_traj)    # some warps start without a trajectory
        trajs = list(range(nxt, nxt + k))
        nxt += k
        all_traj += trajs
        actors.append(warp(pool, w, trajs, finished, random.Random(rng.random()), idle_limit))
    steps = 0
    while actors:
        a = rng.choice(actors)
        try:
            next(a)
        except StopIteration:
            actors.remove(a)
        steps += 1
        # invariant: the warps still waiting are the unclaimed registrations
        # plus the states claimed and not yet taken, so never fewer than those
        assert pool.waiting == pool.avail + pool.claims, (seed, steps)
        assert pool.avail >= 0 and pool.claims >= 0
        assert steps < 2_000_000, f"schedule {seed} did not end"
    return pool, sorted(finished), sorted(all_traj)


@pytest.mark.parametrize("seed", range(60))
def test_handoff_protocol_finishes_every_trajectory_once(seed):
    n_warps = 2 + seed % 9
    pool, finished, all_traj = run_schedule(seed, n_warps, max_traj=6, idle_limit=50 + 13 * (seed % 5))
    assert finished == all_traj, seed        # every trajectory ends exactly once
    assert pool.head == pool.tail and not pool.seq
    assert pool.multi == 0 and pool.waiting == 0 and pool.claims == 0
