"""Writes the stored expected values under tests/golden/ from the oracle alone.

    python tests/golden/make_golden.py

c0_ida_md.json: the twenty 8-puzzle starts of the plain-form workload (60-move seeded
walks), each with its IDA* cost under Manhattan distance, the per-iteration
(bound, expanded, generated) counts in complete-final-iteration mode, and its BFS distance.

rc_corner_pdb.json: the oracle's full 8-corner table of the cube (88,179,840 entries, about
four minutes): the number of entries at each distance, and 2,000 entries at seeded indices.

    python tests/golden/make_golden.py rc_corner      # only the corner table file
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def rc_corner():
    import numpy as np
    t = oracle.rc_corner_pdb()
    hist = np.bincount(t, minlength=256)
    idx = (W.splitmix64_array(W.seed_for(0xC2, 77), 2000) % np.uint64(oracle.RC_CORNER_ENTRIES)).astype(np.int64)
    with open(os.path.join(HERE, "rc_corner_pdb.json"), "w") as f:
        json.dump(dict(source="oracle.rc_corner_pdb (breadth-first search over corner configurations)",
                       entries=int(len(t)), histogram=[int(x) for x in hist[:int(t.max()) + 1]],
                       sample_index=[int(i) for i in idx], sample_value=[int(t[i]) for i in idx]), f)


def main():
    if sys.argv[1:] == ["rc_corner"]:
        rc_corner()
        return
    rc_corner()
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
