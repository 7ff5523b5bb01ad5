"""ADM-TV parity at the length and in the launch configuration the benchmark
runs (Eq. (3)-(10); 512^2 / 60 views / 736 bins, head phantoms, I0 = 2e5,
mu = 4, rho = 256, beta = (1, 0.6), exact step), through the C ABI.

- 200 fixed iterations, the paper-shaped configuration's count: the images
  of two slices of a 32-slice call (64 interleaved channels) against the
  FP64 oracle at 1e-4 relative L2.
- The benchmark's run to the 1e-4 relative-objective stop (about 1000
  iterations): each stop iteration of the benchmark's first two slices
  within 2 of the oracle's, and the reported objective against the oracle's
  objective at the GPU's own stop iteration
  (tests/golden/workload_iterations.json, written by an oracle-only script).
- The residual r that the GPU carries by r <- r - alpha A G over the whole
  run against A f - g recomputed from the result (every channel), and the
  reported objective against the oracle's objective of the GPU's image.
"""
import concurrent.futures as cf
import json
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_01650_gb300 as dect  # noqa: E402

MU, RHO, BETA = 4.0, 256.0, (1.0, 0.6)
S = 32
HERE = os.path.dirname(os.path.abspath(__file__))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def workload():
    g = synth.paper_geometry()
    m = np.stack([synth.make_slice(g, seed=1000 + i, kind="head", i0=2e5).m for i in range(S)]).astype(np.float32)
    return g, dect.Plan(g), oracle.table(g), m


def oracle_channels(t, m, jobs, K):
    """Oracle ADM of (slice, energy) jobs for K iterations, in threads."""
    def one(job):
        i, e = job
        prm = oracle.AdmParams(mu=MU, rho=RHO, step_rule=oracle.CAUCHY, max_iter=K, tol=0.0)
        f, k, _, _ = oracle.adm_channel(t, BETA[e] * m[i, e].astype(np.float64), prm)
        assert k == K
        return f / BETA[e]
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        return dict(zip(jobs, ex.map(one, jobs)))


def test_paper_size_200_iterations(workload):
    g, plan, t, m = workload
    prm = dect.AdmParams(mu=MU, rho=RHO, beta=BETA, step_rule=dect.CAUCHY, max_iter=200)
    x, reps = dect.adm_tv(plan, torch.tensor(m, device="cuda"), prm)
    x = x.cpu().numpy()
    assert all(r.iters == 200 and not r.converged for r in reps)
    jobs = [(0, 0), (0, 1), (31, 0), (31, 1)]
    want = oracle_channels(t, m, jobs, 200)
    for (i, e), xo in want.items():
        err = rel_l2(x[i, e], xo)
        assert err <= 1e-4, (i, e, err)


def test_benchmark_run_to_the_stop(workload):
    g, plan, t, m = workload
    with open(os.path.join(HERE, "golden", "workload_iterations.json")) as f:
        gold = json.load(f)
    prm = dect.AdmParams(mu=MU, rho=RHO, beta=BETA, step_rule=dect.CAUCHY, max_iter=2000,
                         rel_obj_tol=1e-4, check_every=10)
    x, reps = dect.adm_tv(plan, torch.tensor(m, device="cuda"), prm)
    x = x.cpu().numpy()
    assert all(r.converged and r.rel_change < 1e-4 for r in reps)
    # the carried residual stays on A f - g over the whole run, every channel
    for c, r in enumerate(reps):
        assert r.primal_res > 0 and r.resid_drift <= 1e-4 * r.primal_res, (c, r)
    for ch in gold["channels"]:
        i, e = ch["seed"] - 1000, ch["energy"]
        r = reps[2 * i + e]
        assert abs(r.iters - ch["iterations"]) <= 2, (i, e, r.iters, ch["iterations"])
        k0 = ch["phi_window_first"]
        phi_at_stop = ch["phi_window"][r.iters - k0]
        assert abs(r.objective - phi_at_stop) <= 1e-5 * phi_at_stop, (i, e, r.objective, phi_at_stop)
        # the same objective recomputed by the oracle from the GPU's image
        b = BETA[e]
        phi = oracle.objective(t, b * m[i, e].astype(np.float64), MU, b * x[i, e].astype(np.float64))
        assert abs(r.objective - phi) <= 1e-5 * phi, (i, e, r.objective, phi)
        res = np.linalg.norm(oracle.project(t, b * x[i, e].astype(np.float64)) - b * m[i, e])
        assert abs(r.primal_res - res) <= 1e-5 * res, (i, e, r.primal_res, res)
