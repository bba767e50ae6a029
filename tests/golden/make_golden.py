"""Write tests/golden/oracle_k.json: converged k-eff of named workloads from
the FP64 oracle (power iteration to |dk| < 1e-10 and fission-source residual
< 1e-9).  Every value in that file comes from this script and the oracle only.

    python tests/golden/make_golden.py [workload ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "oracle_k.json")


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        p = synth.workload(name)
        o = oracle.Oracle(p, n_threads=os.cpu_count())
        t0 = time.time()
        r = o.solve(tol_k=1e-10, tol_src=1e-9, max_iter=20000)
        data[name] = {"k": r["k"], "iterations": r["iterations"], "residual": r["residual"],
                      "converged": r["converged"], "production": r["production"],
                      "absorption": r["absorption"], "leakage": r["leakage"],
                      "seconds": round(time.time() - t0, 1), "tol_k": 1e-10, "tol_src": 1e-9,
                      "source": "FP64 oracle, tests/golden/make_golden.py"}
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(name, data[name], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["pin_cell", "lattice17_small", "lattice5", "lattice17"])
