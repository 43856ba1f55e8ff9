"""Write rmat_literal_oracle.json: the counts of oracle.count4_literal (the closure equations of
Section III-F taken literally: per-triangle X_j, per-edge A_e x B_e pairs, per-vertex H_u stars) on
the R-MAT graphs of scales 14, 15 and 16 (edge factor 16, a=0.57, b=0.19, c=0.19, seed 1), beside
oracle.count4_combo's counts of the same graphs.  Calls only the seeded generator and oracle/;
nothing from the CUDA path.  The literal oracle's pair scan is slow (about 100 s at scale 14 and
500 s at scale 15 on 8 cores), which is why its counts are stored rather than computed by the
tests.  Run: python tests/golden/make_golden_literal.py [scales...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "rmat_literal_oracle.json")


def main(scales):
    rec = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            rec = json.load(f)
    for scale in scales:
        g = graphgen.rmat(scale, 16, 0.57, 0.19, 0.19, seed=1)
        t = time.time()
        lit = oracle.count4_literal(g.n, g.src, g.dst)
        t_lit = time.time() - t
        combo = oracle.count4_combo(g.n, g.src, g.dst)
        m, maxdeg = oracle.graph_summary(g.n, g.src, g.dst)
        rec[str(scale)] = {"graph": g.name, "n": g.n, "m": m, "max_degree": maxdeg, "order": list(oracle.MOTIFS),
                           "literal": [int(x) for x in lit], "combo": [int(x) for x in combo],
                           "source": "oracle.count4_literal (and oracle.count4_combo)",
                           "literal_seconds_here": round(t_lit, 1)}
        with open(OUT, "w") as f:
            json.dump(rec, f, indent=1)
            f.write("\n")
        print(scale, round(t_lit, 1), flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [14, 15, 16])
