"""Writes tests/golden/batch_networks.txt: the network seeds of the batched
workload (random networks, species in [4, 64], reactions in [8, 512],
trajectory counts log-uniform in [1024, 65536], t_end = 10, 501-point grids),
keeping a drawn network only when a 16-trajectory pilot of the oracle (FP32
propensities, W32 summation, seed 1) stays below 20,000 events per
trajectory and every count below 2^24.  Draws that fail are rejected and
counted.  Calls the oracle only.

Usage: python tests/golden/make_batch_networks.py [n_networks] [first_seed]
"""
import os
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

PILOT_TRAJ = 16
PILOT_MAX_EVENTS = 20000
STATE_LIMIT = 1 << 24


def pilot(seed: int):
    w = W.batch_network(seed)
    r = oracle.run(w.net, PILOT_TRAJ, w.t_end, 11, 1, max_events=PILOT_MAX_EVENTS, schedule=oracle.SCHEDULE_W32,
                   precision=oracle.PRECISION_FP32)
    return seed, r.truncated == 0 and r.overflowed == 0 and r.max_x < STATE_LIMIT


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 256
    first = int(sys.argv[2]) if len(sys.argv) > 2 else 1000
    accepted, rejected = [], []
    seed = first
    with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        while len(accepted) < n:
            batch = list(range(seed, seed + (n - len(accepted)) + 8))
            seed += len(batch)
            for s, ok in ex.map(pilot, batch):
                if len(accepted) >= n:
                    break
                (accepted if ok else rejected).append(s)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_networks.txt")
    with open(out, "w") as f:
        f.write(f"# batched workload: {n} accepted network seeds from {first}; pilot {PILOT_TRAJ} trajectories, "
                f"max_events {PILOT_MAX_EVENTS}, counts < 2^24 (oracle, FP32 propensities, W32)\n")
        f.write(f"# rejected {len(rejected)}: {' '.join(map(str, rejected))}\n")
        for s in accepted:
            f.write(f"{s}\n")
    print(f"accepted {len(accepted)}, rejected {len(rejected)}")


if __name__ == "__main__":
    main()
