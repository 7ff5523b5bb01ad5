"""Write workload_iterations.json: how many ADM iterations the FP64 oracle needs
to reach the 1e-4 relative-objective stop on the benchmark's paper-shaped
workload (512 x 512, 60 views, 736 bins, head phantoms, I0 = 2e5; mu = 4,
rho = 256, beta = (1, 0.6), exact-step rule), and the objective Phi of
Eq. (4) at every iteration from 5 before to 5 after that stop.

Calls only the oracle and the input generator.  The benchmark's CPU
reference arm scales its timed oracle sample by the mean count; the GPU
parity test of the benchmark's run to the stop compares the GPU's stop
iteration and its reported objective with these values.

Each channel runs a fixed 1200 iterations (more than any stop on this
workload) and the stop is read off the objective trajectory with the rule
of the oracle's own loop: the first k >= 1 with
|Phi_k - Phi_{k-1}| / Phi_{k-1} < tol.  The channels run in threads (the
oracle's C calls release the interpreter lock).

    python tests/golden/make_workload_iterations.py [n_slices]
"""
import concurrent.futures as cf
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

TOL = 1e-4
RUN = 1200
WINDOW = 5


def stop_iteration(phi, tol):
    for k in range(1, len(phi)):
        if phi[k - 1] > 0 and abs(phi[k] - phi[k - 1]) / phi[k - 1] < tol:
            return k
    return None


def main():
    count = int(sys.argv[1]) if len(sys.argv) > 1 else 2
    g = synth.paper_geometry()
    t = oracle.table(g)
    jobs = []
    for i in range(count):
        seed = 1000 + i  # the benchmark's first slices
        m = synth.make_slice(g, seed, kind="head", i0=2e5).m.astype(np.float32).astype(np.float64)
        for e in range(2):
            jobs.append((seed, e, (1.0, 0.6)[e] * m[e]))

    def one(job):
        seed, e, gdata = job
        prm = oracle.AdmParams(mu=4.0, rho=256.0, step_rule=oracle.CAUCHY, max_iter=RUN, tol=0.0)
        t0 = time.time()
        f, k, phi, alpha = oracle.adm_channel(t, gdata, prm)
        ks = stop_iteration(phi, TOL)
        assert ks is not None and ks + WINDOW <= RUN
        rec = {"seed": seed, "energy": e, "iterations": ks, "phi": float(phi[ks]),
               "phi_window_first": ks - WINDOW,
               "phi_window": [float(v) for v in phi[ks - WINDOW: ks + WINDOW + 1]],
               "seconds_per_iteration": (time.time() - t0) / RUN}
        print(rec, flush=True)
        return rec

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        out = list(ex.map(one, jobs))
    res = {"workload": "512x512/0.5mm, 60 views, 736 bins x 0.6mm, SOD 500, SDD 1000, head phantom, I0=2e5",
           "params": {"mu": 4.0, "rho": 256.0, "beta": [1.0, 0.6], "rule": "exact step", "tol": TOL},
           "channels": out, "mean_iterations": float(np.mean([c["iterations"] for c in out]))}
    with open(os.path.join(HERE, "workload_iterations.json"), "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
