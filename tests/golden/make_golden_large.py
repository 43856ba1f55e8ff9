"""Write rmat20_oracle.json: oracle counts for the R-MAT scale-20 workload (edge factor 16,
a=0.57, b=0.19, c=0.19, seed 1).  Calls only the seeded generator and oracle.count4_combo /
oracle.noninduced (plain non-induced counts + containment inversion); nothing from the CUDA path.
Takes about a minute on 8 cores.  Run: python tests/golden/make_golden_large.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen  # noqa: E402
import oracle  # noqa: E402


def main():
    g = graphgen.rmat_scale20()
    t = time.time()
    stats = oracle.noninduced(g.n, g.src, g.dst)
    counts = oracle.induced_from_noninduced(stats)
    m, maxdeg = oracle.graph_summary(g.n, g.src, g.dst)
    with open(os.path.join(HERE, "rmat20_oracle.json"), "w") as f:
        json.dump({"graph": g.name, "n": g.n, "m_in": g.m_in, "m": m, "max_degree": maxdeg,
                   "order": list(oracle.MOTIFS), "counts": [int(x) for x in counts],
                   "stats_order": list(oracle.STATS), "stats": [int(x) for x in stats],
                   "source": "oracle.noninduced + oracle.induced_from_noninduced",
                   "oracle_seconds_here": round(time.time() - t, 1)}, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
