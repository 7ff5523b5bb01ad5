"""GPU parity of the fan-beam FBP (dect_fbp) against the FP64 oracle, through
the C ABI.  Tolerance: 1e-5 relative L2 (FP32 filter and back-projection
against FP64), the projection tolerance, since FBP is one linear map."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_01650_gb300 as dect  # noqa: E402

GEOMS = {
    "odd": synth.tiny_geometry(n=37, nv=17, nb=53, px=0.7, start=0.1, det_offset=0.37, sod=60.0, sdd=120.0),
    "small": synth.small_geometry(),
    "dense": synth.tiny_geometry(n=64, nv=720, nb=256, px=1.0, pitch=0.5, sod=200.0, sdd=400.0),
}


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name", sorted(GEOMS))
@pytest.mark.parametrize("batch", [1, 6])
def test_fbp_matches_oracle(name, batch):
    g = GEOMS[name]
    plan = dect.Plan(g)
    S, D = synth.ray_endpoints(g)
    rng = np.random.default_rng(3)
    m = []
    for b in range(batch):
        ph = synth.random_ellipse_phantom(g, 50 + b) if g.n >= 64 else \
            [synth.Ellipse(2.0 * b - 3.0, 1.0, 6.0, 4.0, 0.2 * b, 1.0, 0.3)]
        w = np.array([synth.ETA[0, 0] * e.water + synth.ETA[1, 0] * e.bone for e in ph])
        m.append(synth.ellipse_chords(ph, S, D, w) + 0.001 * rng.standard_normal((g.nv, g.nb)))
    m = np.stack(m).astype(np.float32)
    x = dect.fbp(plan, torch.tensor(m, device="cuda")).cpu().numpy()
    for b in range(batch):
        want = oracle.fbp(g, m[b].astype(np.float64))
        assert rel_l2(x[b], want) <= 1e-5, (name, b)


def test_fbp_paper_size_and_warm_start():
    """512^2 / 60 views / 736 bins, both energies of two slices, against the
    oracle; the result is a valid warm start of the ADM."""
    g = synth.paper_geometry()
    plan = dect.Plan(g)
    sl = [synth.make_slice(g, seed=20 + i, kind="head", i0=2e5) for i in range(2)]
    m = torch.tensor(np.stack([s.m for s in sl]).astype(np.float32), device="cuda")
    x = dect.fbp(plan, m)
    assert x.shape == (2, 2, g.n, g.n)
    xc = x.cpu().numpy()
    for i in range(2):
        for e in range(2):
            want = oracle.fbp(g, sl[i].m[e].astype(np.float32).astype(np.float64))
            assert rel_l2(xc[i, e], want) <= 1e-5
    prm = dect.AdmParams(mu=4.0, rho=256.0, max_iter=3, warm_start=True)
    xa, reps = dect.adm_tv(plan, m, prm, x=x.clone())
    assert torch.isfinite(xa).all()


def test_fbp_rejects_short_scan_and_empty_batch():
    g = synth.tiny_geometry(n=16, nv=20, nb=32, px=1.0, arc=np.pi)
    plan = dect.Plan(g)
    with pytest.raises(dect.DectError):
        dect.fbp(plan, torch.zeros((1, g.nv, g.nb), device="cuda"))
    g2 = synth.tiny_geometry(n=16, nv=20, nb=32, px=1.0)
    plan2 = dect.Plan(g2)
    x = dect.fbp(plan2, torch.zeros((0, g2.nv, g2.nb), device="cuda"))
    assert x.shape == (0, g2.n, g2.n)
