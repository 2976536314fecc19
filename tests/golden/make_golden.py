"""Writes the stored expected values under tests/golden/ from the oracle alone.

    python tests/golden/make_golden.py

c0_ida_md.json: the twenty 8-puzzle starts of the plain-form workload (60-move seeded
walks), each with its IDA* cost under Manhattan distance, the per-iteration
(bound, expanded, generated) counts in complete-final-iteration mode, and its BFS distance.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    dist, _, _ = oracle.stp3_bfs()
    rows = []
    for i in range(20):
        dirs = W.stp_walk(3, 60, W.seed_for(W.TAG_C0, i))
        s = oracle.stp_apply_walk(3, dirs)
        r = oracle.ida_star(oracle.DOM_STP3, s, oracle.Heur(oracle.H_MD), complete=True)
        cells = [(s >> (4 * p)) & 15 for p in range(9)]
        rows.append(dict(index=i, state=s, cost=r["cost"], bfs=int(dist[oracle.perm_rank(cells)]),
                         iters=[list(t) for t in r["iters"]]))
    with open(os.path.join(HERE, "c0_ida_md.json"), "w") as f:
        json.dump(dict(source="oracle.ida_star, Manhattan distance, complete final iteration",
                       instances=rows), f, indent=1)


if __name__ == "__main__":
    main()
