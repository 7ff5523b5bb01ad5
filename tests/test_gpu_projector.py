"""GPU parity of the plan (Siddon table), A x and A^T y against the FP64 oracle.

All calls go through the C ABI (libdect.so via the ctypes binding).
Tolerance for projections: 1e-5 relative L2 (FP32 arithmetic on FP32
lengths against FP64).
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_01650_gb300 as dect  # noqa: E402

GEOMS = {
    "tiny": synth.tiny_geometry(n=8, nv=12, nb=12),
    "odd": synth.tiny_geometry(n=37, nv=17, nb=53, px=0.7, start=0.1, det_offset=0.37),
    "halfarc": synth.tiny_geometry(n=64, nv=30, nb=96, px=0.5, sod=60.0, sdd=130.0, arc=math.pi),
    "small": synth.small_geometry(),
}


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def plans():
    out = {}
    for k, g in GEOMS.items():
        out[k] = (dect.Plan(g), oracle.table(g))
    return out


@pytest.mark.parametrize("name", list(GEOMS))
def test_table_matches_oracle(plans, name):
    plan, t = plans[name]
    rowptr, pix, ln = plan.table()
    assert plan.nnz == t.nnz
    np.testing.assert_array_equal(rowptr, t.rowptr)
    np.testing.assert_array_equal(pix, t.idx)
    # FP64 crossing parameters on both sides, rounded once to FP32
    np.testing.assert_array_equal(ln, t.len.astype(np.float32))
    assert plan.n_grid_aligned == 0


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("batch", [1, 2, 3, 6, 17, 64, 70])
def test_project_parity(plans, name, batch):
    plan, t = plans[name]
    g = GEOMS[name]
    rng = np.random.default_rng(batch)
    x = 0.02 * rng.random((batch, g.n, g.n))
    y = dect.project(plan, torch.tensor(x, dtype=torch.float32, device="cuda"))
    y = y.cpu().numpy()
    for b in range(batch):
        assert rel_l2(y[b], oracle.project(t, x[b])) <= 1e-5


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("batch", [1, 2, 5, 33, 64, 67])
def test_backproject_parity(plans, name, batch):
    plan, t = plans[name]
    g = GEOMS[name]
    rng = np.random.default_rng(10 + batch)
    y = rng.random((batch, g.nv, g.nb))
    x = dect.backproject(plan, torch.tensor(y, dtype=torch.float32, device="cuda")).cpu().numpy()
    for b in range(batch):
        assert rel_l2(x[b], oracle.backproject(t, y[b])) <= 1e-5


def test_adjoint_identity_and_determinism(plans):
    plan, _ = plans["small"]
    g = GEOMS["small"]
    gen = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((2, g.n, g.n), device="cuda", generator=gen)
    y = torch.rand((2, g.nv, g.nb), device="cuda", generator=gen)
    Ax = dect.project(plan, x)
    Aty = dect.backproject(plan, y)
    lhs = (Ax.double() * y.double()).sum().item()
    rhs = (x.double() * Aty.double()).sum().item()
    assert abs(lhs - rhs) / abs(lhs) < 1e-6
    # gather form, fixed order: bitwise reproducible
    assert torch.equal(dect.backproject(plan, y), Aty)
    assert torch.equal(dect.project(plan, x), Ax)


def test_empty_batch_and_bad_args(plans):
    plan, _ = plans["tiny"]
    g = GEOMS["tiny"]
    x = torch.zeros((0, g.n, g.n), device="cuda")
    y = dect.project(plan, x)
    assert y.shape == (0, g.nv, g.nb)
    with pytest.raises(dect.DectError):
        dect.project(plan, torch.zeros((1, g.n, g.n), device="cuda", dtype=torch.float64))
    bad = synth.Geometry(n=8, px=1.0, nv=4, nb=4, pitch=1.0, sod=2.0, sdd=4.0)  # source inside image
    with pytest.raises(dect.DectError):
        dect.Plan(bad)


def test_paper_size_sampled_rays():
    """512^2 / 60 views / 736 bins: sampled rays against the oracle's Siddon walk."""
    g = synth.paper_geometry()
    plan = dect.Plan(g)
    assert 2.5e7 < plan.nnz < 3.3e7
    rowptr, pix, ln = plan.table()
    rng = np.random.default_rng(7)
    x = 0.02 * rng.random((g.n, g.n))
    y = dect.project(plan, torch.tensor(x[None], dtype=torch.float32, device="cuda"))[0].cpu().numpy()
    for r in rng.choice(g.nv * g.nb, 300, replace=False):
        v, b = divmod(int(r), g.nb)
        idx, lens = oracle.siddon_ray(g, v, b)
        s, e = rowptr[r], rowptr[r + 1]
        np.testing.assert_array_equal(pix[s:e], idx)
        np.testing.assert_array_equal(ln[s:e], lens.astype(np.float32))
        want = float(np.dot(lens, x.reshape(-1)[idx]))
        assert abs(y[v, b] - want) <= 1e-5 * max(abs(want), 1e-3)


def test_paper_size_mirror_symmetry():
    """At 512^2 / 60 views / 736 bins, A of the image flipped in y equals A of
    the image with views mirrored ((nv - v) mod nv) and bins reversed: a
    property of the geometry that checks the whole GPU table, not samples.
    No ray of this geometry runs along a grid line (where the midpoint rule
    breaks the symmetry on purpose)."""
    g = synth.paper_geometry()
    plan = dect.Plan(g)
    assert plan.n_grid_aligned == 0
    x = torch.rand((1, g.n, g.n), device="cuda") * 0.02
    y = dect.project(plan, x)[0]
    yf = dect.project(plan, torch.flip(x, dims=[1]).contiguous())[0]
    v = torch.arange(g.nv, device="cuda")
    ym = torch.flip(y[(g.nv - v) % g.nv], dims=[1])
    assert float((yf - ym).norm() / ym.norm()) <= 1e-5


def test_paper_size_64_images():
    """The operators at 512^2 / 60 views / 736 bins on 64 images (one
    interleaved pass over each table): sampled rays of three images against
    the oracle's Siddon walks, and the whole A^T y of those images against the
    oracle's transpose."""
    g = synth.paper_geometry()
    plan = dect.Plan(g)
    rng = np.random.default_rng(11)
    x = (0.02 * rng.random((64, g.n, g.n))).astype(np.float32)
    y = dect.project(plan, torch.tensor(x, device="cuda")).cpu().numpy()
    for b in (0, 31, 63):
        for r in rng.choice(g.nv * g.nb, 60, replace=False):
            v, bn = divmod(int(r), g.nb)
            idx, lens = oracle.siddon_ray(g, v, bn)
            want = float(np.dot(lens, x[b].reshape(-1)[idx].astype(np.float64)))
            assert abs(y[b, v, bn] - want) <= 1e-5 * max(abs(want), 1e-3), (b, v, bn)
    s = rng.random((64, g.nv, g.nb)).astype(np.float32)
    bp = dect.backproject(plan, torch.tensor(s, device="cuda")).cpu().numpy()
    t = oracle.table(g)
    for b in (0, 40, 63):
        assert rel_l2(bp[b], oracle.backproject(t, s[b].astype(np.float64))) <= 1e-5, b
