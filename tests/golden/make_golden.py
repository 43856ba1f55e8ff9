"""Write brute_random.json: induced 4-motif counts of seeded random tiny graphs.

Calls only the oracle's brute force (the definition of an induced occurrence, Section II, over all
4-subsets) and the seeded generators; no value comes from the CUDA path.
Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen  # noqa: E402
import oracle  # noqa: E402


def cases():
    out = []
    for seed in range(24):
        n = 6 + seed % 13
        k = 1.0 + (seed * 7) % 9
        g = graphgen.er(n, k, 5000 + seed) if seed % 3 else graphgen.rgg(n, k, 5000 + seed)
        out.append((g.name, n, g.src.tolist(), g.dst.tolist()))
    for seed in range(6):
        g = graphgen.ba(30 + 5 * seed, 2 + seed % 3, 7000 + seed)
        out.append((g.name, g.n, g.src.tolist(), g.dst.tolist()))
    return out


def main():
    rows = []
    for name, n, s, d in cases():
        c = oracle.count4_brute(n, np.array(s, np.int32), np.array(d, np.int32))
        rows.append({"name": name, "n": n, "src": s, "dst": d, "counts": [int(x) for x in c]})
    with open(os.path.join(HERE, "brute_random.json"), "w") as f:
        json.dump({"order": list(oracle.MOTIFS), "source": "oracle.count4_brute", "graphs": rows}, f)
        f.write("\n")


if __name__ == "__main__":
    main()
