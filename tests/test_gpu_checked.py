"""The checked build (libdect_checked.so, index checks of DECT_CHECKED) on
tiny cases (8^2 and 16^2 images): every operator and both solvers run with
no failed check and give the oracle's results, and the self-test shows that
an out-of-range index is caught, reported and not used.  The library is
selected by DECT_CHECKED=1 in a child process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
import oracle, synth
import paper_1607_01650_gb300 as dect
L = dect.load()
assert L.dect_checked_build() == 1
def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))
for n, nv, nb in ((8, 12, 16), (16, 20, 28)):
    g = synth.tiny_geometry(n=n, nv=nv, nb=nb, px=1.0, sod=4.0 * n, sdd=8.0 * n)
    plan = dect.Plan(g)
    t = oracle.table(g)
    rng = np.random.default_rng(n)
    x = rng.random((3, n, n)).astype(np.float32)
    y = rng.random((3, nv, nb)).astype(np.float32)
    xt, yt = torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda")
    for proj, back in ((dect.project, dect.backproject), (dect.project_otf, dect.backproject_otf)):
        p = proj(plan, xt).cpu().numpy()
        b = back(plan, yt).cpu().numpy()
        dect.check_status()
        for k in range(3):
            assert rel(p[k], oracle.project(t, x[k].astype(np.float64))) <= 1e-5
            assert rel(b[k], oracle.backproject(t, y[k].astype(np.float64))) <= 1e-5
    sl = [synth.make_slice(g, seed=s, i0=1e5) for s in (1, 2)]
    m = torch.tensor(np.stack([s.m for s in sl]), dtype=torch.float32, device="cuda")
    prm = dect.AdmParams(mu=16.0, rho=256.0, max_iter=10)
    xa, _ = dect.adm_tv(plan, m, prm)
    [(xb, _)] = dect.adm_tv_batch([(plan, m, None)], prm)
    dect.check_status()
    op = oracle.AdmParams(mu=16.0, rho=256.0, max_iter=10, step_rule=oracle.CAUCHY)
    for i in range(2):
        xo, _ = oracle.adm_dual(t, sl[i].m.astype(np.float32).astype(np.float64), op)
        for e in range(2):
            assert rel(xa[i, e].cpu().numpy(), xo[e]) <= 1e-4
            assert rel(xb[i, e].cpu().numpy(), xo[e]) <= 1e-4
    u, _ = dect.pls_decompose(xa, dect.PlsParams(max_iter=20, tol=0.0))
    fb = dect.fbp(plan, m)
    dect.check_status()
    assert torch.isfinite(u).all() and torch.isfinite(fb).all()
# the checks catch an index outside the array, do not use it, and report it
st = L.dect_selftest_index(8, dect._stream())
assert st == 7, st
assert b"self-test, index 8" in L.dect_last_error()
assert L.dect_selftest_index(3, dect._stream()) == 0
assert float(torch.ones(64, device="cuda").sum()) == 64.0
print("checked ok")
"""


def test_checked_build_tiny_cases():
    env = dict(os.environ, DECT_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
