"""Write the stored expected values of the GPU parity tests, from the FP64
oracle only:

* tests/golden/oracle_k.json: converged k-eff of named workloads (power
  iteration to |dk| < 1e-10 and fission-source residual < 1e-9);
* tests/golden/oracle_flux_<name>.npz: the converged, normalised scalar flux
  phi[fsr, g] of the same solve (float64), with its k, for the workloads
  whose converged flux the tests compare element by element.

Every value in those files comes from this script and the oracle only.

    python tests/golden/make_golden.py [workload ...]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "oracle_k.json")
# converged fluxes are stored for these (the bench workload and a small one)
FLUX = ("lattice17", "lattice17_small", "lattice5", "lattice5_rings", "asm1_absorber")


def flux_path(name):
    return os.path.join(HERE, f"oracle_flux_{name}.npz")


def main(names):
    for name in names:
        p = synth.workload(name)
        o = oracle.Oracle(p, n_threads=os.cpu_count())
        t0 = time.time()
        r = o.solve(tol_k=1e-10, tol_src=1e-9, max_iter=20000)
        # re-read so that concurrent runs for other workloads are kept
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[name] = {"k": r["k"], "iterations": r["iterations"], "residual": r["residual"],
                      "converged": r["converged"], "production": r["production"],
                      "absorption": r["absorption"], "leakage": r["leakage"],
                      "seconds": round(time.time() - t0, 1), "tol_k": 1e-10, "tol_src": 1e-9,
                      "source": "FP64 oracle, tests/golden/make_golden.py"}
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        if name in FLUX:
            np.savez_compressed(flux_path(name), phi=o.flux(), k=np.float64(r["k"]),
                                iterations=np.int64(r["iterations"]))
        print(name, data[name], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["pin_cell", "lattice17_small", "lattice5", "lattice17"])
