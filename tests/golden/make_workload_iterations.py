"""Write workload_iterations.json: how many ADM iterations the FP64 oracle needs
to reach the 1e-4 relative-objective stop on the benchmark's paper-shaped
workload (512 x 512, 60 views, 736 bins, head phantoms, I0 = 2e5; mu = 4,
rho = 256, beta = (1, 0.6), exact-step rule).

Calls only the oracle and the input generator.  The benchmark's CPU
reference arm times a few oracle iterations and scales them by this count.

    python tests/golden/make_workload_iterations.py [n_slices]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    count = int(sys.argv[1]) if len(sys.argv) > 1 else 2
    g = synth.paper_geometry()
    t = oracle.table(g)
    out = []
    for i in range(count):
        seed = 1000 + i  # the benchmark's first slices
        m = synth.make_slice(g, seed, kind="head", i0=2e5).m.astype(np.float32).astype(np.float64)
        for e in range(2):
            beta = (1.0, 0.6)[e]
            prm = oracle.AdmParams(mu=4.0, rho=256.0, step_rule=oracle.CAUCHY, max_iter=2000, tol=1e-4)
            t0 = time.time()
            f, k, phi, alpha = oracle.adm_channel(t, beta * m[e], prm)
            out.append({"seed": seed, "energy": e, "iterations": k, "phi": phi[-1],
                        "seconds": time.time() - t0})
            print(out[-1], flush=True)
    res = {"workload": "512x512/0.5mm, 60 views, 736 bins x 0.6mm, SOD 500, SDD 1000, head phantom, I0=2e5",
           "params": {"mu": 4.0, "rho": 256.0, "beta": [1.0, 0.6], "rule": "exact step", "tol": 1e-4},
           "channels": out, "mean_iterations": float(np.mean([c["iterations"] for c in out]))}
    with open(os.path.join(HERE, "workload_iterations.json"), "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
