"""The on-the-fly projector and the multi-slice ADM (dect_project_otf,
dect_backproject_otf, dect_adm_tv_batch) against the FP64 oracle, through
the C ABI.

The on-the-fly element a_ij is the length of ray i inside pixel j in FP32
(the oracle's Siddon table holds the same lengths in FP64), so projections
match the oracle within 1e-5 relative L2 and reconstructions after a fixed
number of iterations within 1e-4, the tolerances of the table path.  Both
operators evaluate a_ij by one function, so the adjoint identity holds to
the rounding of the sums.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_01650_gb300 as dect  # noqa: E402

MU, RHO = 16.0, 256.0

GEOMS = {
    "small": synth.small_geometry(),
    "odd": synth.tiny_geometry(n=37, nv=23, nb=70, px=0.9, sod=110.0, sdd=230.0, start=0.3),
    "offset": synth.tiny_geometry(n=32, nv=40, nb=64, px=1.0, sod=100.0, sdd=200.0, det_offset=1.7),
    "short_arc": synth.tiny_geometry(n=28, nv=30, nb=50, px=1.0, sod=90.0, sdd=180.0, arc=np.pi * 1.2),
}


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def plans():
    out = {}
    for k, g in GEOMS.items():
        p = dect.Plan(g)
        assert p.n_grid_aligned == 0
        out[k] = (g, p, oracle.table(g))
    return out


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("batch", [1, 2, 3])
def test_otf_project_and_backproject_parity(plans, name, batch):
    g, plan, t = plans[name]
    rng = np.random.default_rng(batch)
    x = (0.02 * rng.random((batch, g.n, g.n))).astype(np.float32)
    y = dect.project_otf(plan, torch.tensor(x, device="cuda")).cpu().numpy()
    s = rng.random((batch, g.nv, g.nb)).astype(np.float32)
    b = dect.backproject_otf(plan, torch.tensor(s, device="cuda")).cpu().numpy()
    for k in range(batch):
        assert rel_l2(y[k], oracle.project(t, x[k].astype(np.float64))) <= 1e-5
        assert rel_l2(b[k], oracle.backproject(t, s[k].astype(np.float64))) <= 1e-5


def test_otf_exact_transpose_and_determinism(plans):
    g, plan, t = plans["odd"]
    rng = np.random.default_rng(5)
    x = torch.tensor(rng.random((2, g.n, g.n)), dtype=torch.float32, device="cuda")
    y = torch.tensor(rng.random((2, g.nv, g.nb)), dtype=torch.float32, device="cuda")
    Ax = dect.project_otf(plan, x)
    Aty = dect.backproject_otf(plan, y)
    lhs = float((Ax.double() * y.double()).sum())
    rhs = float((x.double() * Aty.double()).sum())
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
    assert torch.equal(dect.project_otf(plan, x), Ax)
    assert torch.equal(dect.backproject_otf(plan, y), Aty)
    # and the stored-table operators give the same projections to FP32 rounding
    assert float((dect.project(plan, x) - Ax).norm() / Ax.norm()) <= 1e-5


def test_otf_paper_geometry_sampled():
    """512^2 / 60 views / 736 bins: the on-the-fly projection of a head
    phantom against the stored table on every ray."""
    g = synth.paper_geometry()
    plan = dect.Plan(g)
    x = torch.tensor(synth.make_slice(g, 3, kind="head").truth(supersample=2)[1], dtype=torch.float32,
                     device="cuda")
    a = dect.project_otf(plan, x)
    b = dect.project(plan, x)
    assert float((a - b).norm() / b.norm()) <= 1e-5
    y = torch.rand((2, g.nv, g.nb), device="cuda")
    assert float((dect.backproject_otf(plan, y) - dect.backproject(plan, y)).norm()
                 / dect.backproject(plan, y).norm()) <= 1e-5


UNEVEN = [(40, 30, 60, 2), (56, 180, 90, 1), (32, 47, 48, 3), (48, 96, 72, 1),
          (36, 120, 56, 2), (64, 33, 100, 1), (28, 150, 44, 1), (44, 75, 66, 2)]


def uneven_groups(seed0=600, i0=1e5):
    groups, refs = [], []
    for k, (n, nv, nb, S) in enumerate(UNEVEN):
        g = synth.tiny_geometry(n=n, nv=nv, nb=nb, px=1.0, sod=3.0 * n, sdd=6.0 * n)
        m = np.stack([synth.make_slice(g, seed=seed0 + 10 * k + i, i0=i0).m for i in range(S)]).astype(np.float32)
        plan = dect.Plan(g)
        assert plan.n_grid_aligned == 0
        groups.append((plan, torch.tensor(m, device="cuda"), None))
        refs.append((g, m))
    return groups, refs


@pytest.mark.parametrize("proj", ["otf", "table"])
@pytest.mark.parametrize("opts", [{}, {"joint": True}, {"nonneg": True}, {"xi": 100.0, "step_rule": dect.BB1}])
def test_batch_matches_oracle_fixed_iterations(opts, proj):
    """Eight geometries (28^2 - 64^2, 30 - 180 views), 13 slices in one call,
    the projector on the fly or from the stored tables."""
    groups, refs = uneven_groups()
    K = 15
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=K, **opts)
    res = dect.adm_tv_batch(groups, prm, projector=proj)
    for (x, reps), (g, m) in zip(res, refs):
        t = oracle.table(g)
        x = x.cpu().numpy()
        for i in range(m.shape[0]):
            op = oracle.AdmParams(mu=MU, rho=RHO, max_iter=K, step_rule=opts.get("step_rule", oracle.CAUCHY),
                                  xi=opts.get("xi"), joint=opts.get("joint", False),
                                  nonneg=opts.get("nonneg", False))
            xo, _ = oracle.adm_dual(t, m[i].astype(np.float64), op)
            for e in range(2):
                assert rel_l2(x[i, e], xo[e]) <= 1e-4, (g.n, g.nv, i, e)
            assert all(r.iters == K for r in reps)
            if opts.get("nonneg"):
                assert x.min() >= 0.0


@pytest.mark.parametrize("proj", ["otf", "table"])
def test_batch_stop_and_reports_match_oracle(proj):
    """Run to the 1e-4 relative-objective stop: slices leave the launches as
    they stop; each channel's stop iteration within 2 of the oracle's, its
    image at that count and its reported objective as the oracle's, and the
    carried residual on A f - g."""
    groups, refs = uneven_groups(seed0=700, i0=3e3)
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=3000, rel_obj_tol=1e-4, check_every=10)
    res = dect.adm_tv_batch(groups, prm, projector=proj)
    stops = []
    b = (1.0, 0.6)
    for (x, reps), (g, m) in zip(res, refs):
        t = oracle.table(g)
        x = x.cpu().numpy()
        for i in range(m.shape[0]):
            for e in range(2):
                r = reps[2 * i + e]
                assert r.converged and r.rel_change < 1e-4
                assert r.resid_drift <= 1e-4 * r.primal_res
                op = oracle.AdmParams(mu=MU, rho=RHO, max_iter=3000, tol=1e-4, step_rule=oracle.CAUCHY)
                f, k, phi, _ = oracle.adm_channel(t, b[e] * m[i, e].astype(np.float64), op)
                assert abs(r.iters - k) <= 2, (g.n, g.nv, i, e, r.iters, k)
                op = oracle.AdmParams(mu=MU, rho=RHO, max_iter=r.iters, step_rule=oracle.CAUCHY)
                f, _, _, _ = oracle.adm_channel(t, b[e] * m[i, e].astype(np.float64), op)
                assert rel_l2(x[i, e], f / b[e]) <= 1e-4
                want = oracle.objective(t, b[e] * m[i, e].astype(np.float64), MU, b[e] * x[i, e].astype(np.float64))
                assert abs(r.objective - want) <= 1e-4 * want
                stops.append(r.iters)
    assert max(stops) - min(stops) >= 20  # slices left the launches at different checks


@pytest.mark.parametrize("proj", ["otf", "table"])
def test_batch_equals_single_plan_path(proj):
    """One geometry through dect_adm_tv_batch_ex and through dect_adm_tv
    (stored table): the same iterates to FP32 rounding."""
    g = synth.tiny_geometry(n=48, nv=24, nb=72, px=1.0, sod=120.0, sdd=240.0)
    plan = dect.Plan(g)
    m = torch.tensor(np.stack([synth.make_slice(g, seed=90 + i).m for i in range(3)]), dtype=torch.float32,
                     device="cuda")
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=40)
    xa, _ = dect.adm_tv(plan, m, prm)
    [(xb, _)] = dect.adm_tv_batch([(plan, m, None)], prm, projector=proj)
    assert float((xa - xb).norm() / xa.norm()) <= 1e-5


def test_batch_table_accepts_grid_aligned_rays():
    """Rays along grid lines (the even detector of a centred geometry) are
    refused by the on-the-fly form but run from the stored table, as the
    oracle's Siddon table assigns them."""
    g = synth.tiny_geometry(n=24, nv=12, nb=41, px=1.0, sod=60.0, sdd=120.0)  # odd nb: a ray through the axis
    plan = dect.Plan(g)
    assert plan.n_grid_aligned > 0
    m = np.stack([synth.make_slice(g, seed=40 + i).m for i in range(2)]).astype(np.float32)
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=10)
    with pytest.raises(dect.DectError):
        dect.adm_tv_batch([(plan, torch.tensor(m, device="cuda"), None)], prm, projector="otf")
    [(x, _)] = dect.adm_tv_batch([(plan, torch.tensor(m, device="cuda"), None)], prm, projector="table")
    t = oracle.table(g)
    x = x.cpu().numpy()
    for i in range(2):
        xo, _ = oracle.adm_dual(t, m[i].astype(np.float64),
                                oracle.AdmParams(mu=MU, rho=RHO, max_iter=10, step_rule=oracle.CAUCHY))
        for e in range(2):
            assert rel_l2(x[i, e], xo[e]) <= 1e-4


@pytest.mark.parametrize("proj", ["otf", "table"])
def test_batch_deterministic_and_empty(proj):
    groups, _ = uneven_groups()
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=12)
    a = dect.adm_tv_batch(groups, prm, projector=proj)
    b = dect.adm_tv_batch(groups, prm, projector=proj)
    for (xa, _), (xb, _) in zip(a, b):
        assert torch.equal(xa, xb)
    assert dect.adm_tv_batch([], prm) == []
    g = synth.tiny_geometry(n=16, nv=8, nb=24)
    [(x, reps)] = dect.adm_tv_batch([(dect.Plan(g), torch.zeros((0, 2, 8, 24), device="cuda"), None)], prm)
    assert x.shape == (0, 2, 16, 16)
