"""Writes tests/golden/hiv_target_v.txt: the ensemble mean of V on the
3001-point grid of [0, 30] for the HIV-shaped model at seeded perturbed rates
(workloads.hiv_target_rates(2)), 65,536 trajectories, seed 2, FP64 exact
mode, schedule L -- the fixed target of the rate-gradient workload.  Calls the
oracle only.

Usage: python tests/golden/make_hiv_target.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    net = W.hiv_shaped().with_rates(W.hiv_target_rates(2))
    N, T, G = 65536, 30.0, 3001
    r = oracle.run(net, N, T, G, 2, threads=os.cpu_count() or 4)
    mean, _ = oracle.finalize(N, r.S1, r.S2)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hiv_target_v.txt")
    with open(out, "w") as f:
        f.write("# mean V(g_k), k = 0..3000, g_k = 30 k / 3000; HIV-shaped model at rates "
                "workloads.hiv_target_rates(2), 65536 trajectories, seed 2, FP64, oracle\n")
        for k in range(G):
            f.write(f"{float(mean[k, 2]).hex()}  {float(mean[k, 2]):.12g}\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
