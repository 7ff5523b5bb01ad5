"""GPU parity of the cone-beam plan (3-D Siddon table, Sec. 2.1 / Fig. 1 with
a flat 2-D detector) and of the 6-neighbour volume decomposition (Eq. (11)-
(15), Eq. (14) in 3-D) against the FP64 oracle, through the C ABI.

Tables: bit-identical to the oracle's (FP64 crossings, one FP32 rounding of
each length).  Projections 1e-5 relative L2; basis maps 2e-4 on inputs whose
edge decision has no voxel within FP32 rounding of tau (tests/edge_band.py).
"""
import dataclasses

import numpy as np
import pytest

import edge_band
import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_01650_gb300 as dect  # noqa: E402

CONES = {
    "small": synth.tiny_cone(n=6, nz=5, nv=7, nr=5, nc=9),
    "offset": synth.tiny_cone(n=9, nz=4, nv=10, nr=6, nc=13, px=0.8, pz=1.3, off_u=0.35, off_v=-0.4),
    "wide": synth.tiny_cone(n=16, nz=7, nv=12, nr=9, nc=24, start=0.4),
}


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def plans():
    return {k: (g, dect.ConePlan(g), oracle.table3(g)) for k, g in CONES.items()}


@pytest.mark.parametrize("name", list(CONES))
def test_cone_table_matches_oracle(plans, name):
    g, plan, t = plans[name]
    rowptr, pix, ln = plan.table()
    np.testing.assert_array_equal(rowptr, t.rowptr)
    np.testing.assert_array_equal(pix, t.idx)
    np.testing.assert_array_equal(ln, t.len.astype(np.float32))
    assert plan.n_pixels == g.n_vox and plan.n_rays == g.n_rays


@pytest.mark.parametrize("name", list(CONES))
@pytest.mark.parametrize("batch", [1, 3])
def test_cone_project_backproject_parity(plans, name, batch):
    g, plan, t = plans[name]
    rng = np.random.default_rng(batch)
    x = rng.random((batch, g.nz, g.n, g.n)).astype(np.float32)
    y = rng.random((batch, g.nv, g.nr, g.nc)).astype(np.float32)
    p = dect.project_cone(plan, torch.tensor(x, device="cuda")).cpu().numpy()
    b = dect.backproject_cone(plan, torch.tensor(y, device="cuda")).cpu().numpy()
    for k in range(batch):
        assert rel_l2(p[k], oracle.project3(t, x[k].astype(np.float64))) <= 1e-5
        assert rel_l2(b[k], oracle.backproject3(t, y[k].astype(np.float64))) <= 1e-5


def test_cone_single_slice_is_the_fan_beam_plan():
    g3 = synth.ConeGeometry(n=24, nz=1, px=1.0, pz=2.0, nv=18, nr=1, nc=40, pu=1.7, pv=1.0, sod=80.0,
                            sdd=160.0, start=0.3, off_u=0.2)
    g2 = synth.tiny_geometry(n=24, nv=18, nb=40, px=1.0, pitch=1.7, sod=80.0, sdd=160.0, start=0.3,
                             det_offset=0.2)
    a, b = dect.ConePlan(g3).table(), dect.Plan(g2).table()
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_cone_sampled_rays_larger_volume():
    """128^2 x 32 voxels, 60 views of 32 x 192 cells: sampled rays against the
    oracle's 3-D Siddon walk, and the z-mirror property on the whole operator."""
    g = synth.ConeGeometry(n=128, nz=33, px=1.0, pz=1.0, nv=60, nr=32, nc=192, pu=1.2, pv=1.2, sod=500.0,
                           sdd=1000.0)
    plan = dect.ConePlan(g)
    assert plan.n_grid_aligned == 0
    rowptr, pix, ln = plan.table()
    rng = np.random.default_rng(9)
    x = (0.02 * rng.random((g.nz, g.n, g.n))).astype(np.float32)
    y = dect.project_cone(plan, torch.tensor(x[None], device="cuda"))[0].cpu().numpy()
    for r in rng.choice(g.n_rays, 200, replace=False):
        v, rem = divmod(int(r), g.nr * g.nc)
        row, c = divmod(rem, g.nc)
        idx, lens = oracle.siddon_ray3(g, v, row, c)
        s, e = rowptr[r], rowptr[r + 1]
        np.testing.assert_array_equal(pix[s:e], idx)
        np.testing.assert_array_equal(ln[s:e], lens.astype(np.float32))
        want = float(np.dot(lens, x.reshape(-1)[idx].astype(np.float64)))
        assert abs(y[v, row, c] - want) <= 1e-5 * max(abs(want), 1e-3)
    yf = dect.project_cone(plan, torch.tensor(x[None, ::-1].copy(), device="cuda"))[0].cpu().numpy()
    assert rel_l2(yf, y[:, ::-1, :]) <= 1e-5


def volumes(n, nz, seed, sig=(4e-4, 6e-4)):
    """Blocky two-material volumes (boxes of water- and bone-like fractions) plus noise."""
    rng = np.random.default_rng(seed)
    u = np.zeros((2, nz, n, n))
    for _ in range(6):
        k0, i0, j0 = rng.integers(0, nz - 1), rng.integers(0, n - 2), rng.integers(0, n - 2)
        k1, i1, j1 = k0 + rng.integers(1, nz - k0 + 1), i0 + rng.integers(2, n - i0 + 1), j0 + rng.integers(2, n - j0 + 1)
        u[rng.integers(0, 2), k0:k1, i0:i1, j0:j1] += rng.uniform(0.3, 1.0)
    xh = synth.attenuation(u, 0) + sig[0] * rng.standard_normal((nz, n, n))
    xl = synth.attenuation(u, 1) + sig[1] * rng.standard_normal((nz, n, n))
    return xh.astype(np.float32), xl.astype(np.float32)


@pytest.mark.parametrize("n,nz,seeds", [(20, 6, (1, 2)), (33, 5, (3,))])
def test_cone_pls_parity_and_mask(n, nz, seeds):
    data = [volumes(n, nz, s) for s in seeds]
    x = torch.tensor(np.stack([np.stack(d) for d in data]), device="cuda")
    mask = dect.pls_edge_mask_cone(x, 0.2).cpu().numpy().astype(bool)
    pp = dect.PlsParams(gamma=0.1, edge_tau=0.2, edge_eps=0.05, max_iter=40, tol=0.0)
    u, reps = dect.pls_decompose_cone(x, pp)
    u = u.cpu().numpy()
    op = oracle.PlsParams(gamma=0.1, tau=0.2, eps=0.05, max_iter=40, tol=0.0)
    for b, (xh, xl) in enumerate(data):
        h, lo = xh.astype(np.float64), xl.astype(np.float64)
        band = edge_band.band3(h, 0.2) | edge_band.band3(lo, 0.2)
        want = oracle.edge_mask3(h, lo, 0.2).astype(bool)
        assert want.any() and not want.all()
        np.testing.assert_array_equal(mask[b][~band], want[~band])
        assert not band.any()
        o1, o2, _, _ = oracle.pls_decompose3(h, lo, op)
        assert rel_l2(u[b, 0], o1) <= 2e-4 and rel_l2(u[b, 1], o2) <= 2e-4
        assert reps[b][0] == (40, 40)
    # gamma = 0: the per-voxel 2x2 solve of Eq. (12), FP64 rounded once
    u0, _ = dect.pls_decompose_cone(x, dataclasses.replace(pp, gamma=0.0, max_iter=5))
    d1, _ = oracle.direct_decompose(synth.ETA, data[0][0].astype(np.float64), data[0][1].astype(np.float64))
    np.testing.assert_array_equal(u0[0, 0].cpu().numpy(), d1.astype(np.float32))


def test_cone_plan_refused_by_fan_beam_solvers(plans):
    g, plan, _ = plans["small"]
    with pytest.raises(dect.DectError):
        dect.load()
        import ctypes as C
        st = dect.load().dect_adm_tv(plan.handle, C.c_void_p(1), C.c_void_p(1), 1,
                                     C.byref(dect.AdmParams()._c()), None, dect._stream())
        dect._check(st, "dect_adm_tv")
    with pytest.raises(dect.DectError):
        import ctypes as C
        dect._check(dect.load().dect_fbp(plan.handle, C.c_void_p(1), C.c_void_p(1), 1, dect._stream()), "dect_fbp")
