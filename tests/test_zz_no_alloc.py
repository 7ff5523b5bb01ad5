"""The allocation-free decomposition entry point (dect_pls_decompose_noalloc).

It exists for callers that must not allocate device memory while they run
(a service that reserves the whole device pool at start-up, a plug-in whose
host process owns the GPU allocator).  It must give what the allocating
dect_pls_decompose gives, also on a second call that finds the previous
call's data in the shared scratch array.  This file is collected last on
purpose: the test also has to pass after everything else has run.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_01650_gb300 as dect  # noqa: E402

TOL = 2e-4  # relative L2, the tolerance of the decomposition parity tests


def _pair(n, seed):
    rng = np.random.default_rng(seed)
    g = synth.tiny_geometry(n=n, px=1.0, sod=10.0 * n, sdd=20.0 * n)
    ph = synth.random_ellipse_phantom(g, seed=seed, axis_range=(0.1 * n, 0.3 * n))
    u = synth.rasterize(ph, n, 1.0, supersample=4)
    xh = synth.attenuation(u, 0) + 4e-4 * rng.standard_normal((n, n))
    xl = synth.attenuation(u, 1) + 6e-4 * rng.standard_normal((n, n))
    return np.stack([xh, xl]).astype(np.float32)


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / b.norm())


def test_noalloc_matches_allocating_path_twice():
    prm = dect.PlsParams(gamma=0.1, max_iter=80, tol=1e-6)
    # two calls in a row with different shapes and data: the second one finds
    # the first one's values in the shared array
    for n, batch, seed in ((96, 3, 1), (128, 2, 2)):
        x = torch.tensor(np.stack([_pair(n, seed + k) for k in range(batch)]), device="cuda")
        u_ref, rep_ref = dect.pls_decompose(x, prm)
        u = torch.full_like(x, float("nan"))
        u, rep = dect.pls_decompose_noalloc(x, prm, u)
        torch.cuda.synchronize()
        assert torch.isfinite(u).all()
        for b in range(batch):
            for m in range(2):
                assert _rel(u[b, m], u_ref[b, m]) <= TOL
        assert [r[0] for r in rep] == [r[0] for r in rep_ref]


def test_noalloc_rejects_work_above_its_limit():
    n = 512
    x = torch.zeros((2, 2, n, n), device="cuda")  # 2 * 512^2 pixels > the limit
    with pytest.raises(dect.DectError, match="must be <="):
        dect.pls_decompose_noalloc(x, dect.PlsParams(), torch.empty_like(x))
