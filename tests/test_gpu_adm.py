"""GPU parity of ADM-TV (Eq. (3)-(10)) against the FP64 oracle, through the C ABI.

Tolerance: reconstructions within 1e-4 relative L2 after a fixed number of
iterations (FP32 bulk arithmetic, FP64 norms, against an all-FP64 oracle).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_01650_gb300 as dect  # noqa: E402

MU, RHO = 16.0, 256.0


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def run_both(g, slices, K, rule=dect.CAUCHY, beta=(1.0, 0.6), xi=0.0, tol=0.0, x0=None,
             nonneg=False, joint=False):
    plan = dect.Plan(g)
    t = oracle.table(g)
    m = np.stack([s.m for s in slices])
    prm = dect.AdmParams(mu=MU, rho=RHO, xi=xi, beta=beta, step_rule=rule, max_iter=K,
                         rel_obj_tol=tol, warm_start=x0 is not None, nonneg=nonneg, joint=joint)
    xin = None if x0 is None else torch.tensor(x0, dtype=torch.float32, device="cuda")
    x, reps = dect.adm_tv(plan, torch.tensor(m, dtype=torch.float32, device="cuda"), prm, x=xin)
    x = x.cpu().numpy()
    outs = []
    for i, s in enumerate(slices):
        op = oracle.AdmParams(mu=MU, rho=RHO, xi=(xi if xi > 0 else None), beta=beta,
                              step_rule=rule, max_iter=K, tol=tol, nonneg=nonneg, joint=joint)
        # the oracle reads the same FP32 data the GPU reads
        xo, its = oracle.adm_dual(t, m[i].astype(np.float32).astype(np.float64), op,
                                  x0=None if x0 is None else x0[i].astype(np.float32).astype(np.float64))
        outs.append((xo, its))
    return x, reps, outs, t


def test_small_config_100_iterations():
    g = synth.small_geometry()
    sl = synth.make_slice(g, seed=1, i0=1e5)
    x, reps, outs, t = run_both(g, [sl], 100)
    xo, its = outs[0]
    for e in range(2):
        assert rel_l2(x[0, e], xo[e]) <= 1e-4
        assert reps[e].iters == 100
        phi = oracle.objective(t, 0.0 + (1.0, 0.6)[e] * sl.m[e].astype(np.float32), MU,
                               (1.0, 0.6)[e] * x[0, e].astype(np.float64))
        assert abs(reps[e].objective - phi) <= 1e-4 * phi


@pytest.mark.parametrize("ns", [1, 3, 17, 33])
def test_batched_slices(ns):
    """Batches exercise the 2/8/64-channel interleaved paths and the chunking over 64 channels."""
    g = synth.tiny_geometry(n=48, nv=24, nb=72, px=1.0, sod=120.0, sdd=240.0)
    slices = [synth.make_slice(g, seed=100 + i, i0=1e5) for i in range(ns)]
    x, reps, outs, t = run_both(g, slices, 30)
    for i in range(ns):
        for e in range(2):
            assert rel_l2(x[i, e], outs[i][0][e]) <= 1e-4


def test_chunks_in_flight_equal_chunks_alone():
    """A call of more than 32 slices runs its chunks of 32 two at a time on
    their own streams; each chunk must give, bit for bit, what it gives as a
    call of its own (the same plan, so the same autotuned variants), with the
    relative-objective stop and the narrowing in play."""
    g = synth.tiny_geometry(n=40, nv=20, nb=64, px=1.0, sod=120.0, sdd=240.0)
    doses = [3e2, 1e6, 1e3, 3e5, 1e4]
    ns = 70  # three chunks: 32, 32, 6 slices
    m = np.stack([synth.make_slice(g, seed=900 + i, i0=doses[i % 5]).m for i in range(ns)]).astype(np.float32)
    plan = dect.Plan(g)
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=2000, rel_obj_tol=1e-4, check_every=10)
    md = torch.tensor(m, device="cuda")
    x_all, rep_all = dect.adm_tv(plan, md, prm)
    for c0 in range(0, ns, 32):
        xc, rc = dect.adm_tv(plan, md[c0:c0 + 32].contiguous(), prm)
        assert torch.equal(xc, x_all[c0:c0 + 32])
        for a, b in zip(rc, rep_all[2 * c0: 2 * c0 + 2 * xc.shape[0]]):
            assert (a.iters, a.converged, a.objective, a.rel_change) == (b.iters, b.converged, b.objective,
                                                                         b.rel_change)
    assert len({r.iters for r in rep_all}) > 1  # the stops (and narrowings) differ between channels


def test_bb1_rule_and_xi():
    g = synth.tiny_geometry(n=40, nv=20, nb=64, px=1.0, sod=120.0, sdd=240.0)
    slices = [synth.make_slice(g, seed=7, i0=1e5)]
    x, reps, outs, t = run_both(g, slices, 12, rule=dect.BB1, xi=100.0)
    for e in range(2):
        assert rel_l2(x[0, e], outs[0][0][e]) <= 1e-4


def test_warm_start():
    g = synth.tiny_geometry(n=40, nv=20, nb=64, px=1.0, sod=120.0, sdd=240.0)
    sl = synth.make_slice(g, seed=8, i0=1e5)
    x0 = np.stack([sl.truth()[1]]) * 0.9
    x, reps, outs, t = run_both(g, [sl], 15, x0=x0)
    for e in range(2):
        assert rel_l2(x[0, e], outs[0][0][e]) <= 1e-4


@pytest.mark.parametrize("ns", [1, 5, 20])
def test_nonnegative_projection(ns):
    """f-step projected onto f >= 0 (x in R_+^N, Eq. (1)): parity with the
    oracle's projected iteration, a nonnegative result, and the objective
    reported at it.  Low-dose data makes the unconstrained result negative,
    so the projection is active."""
    g = synth.tiny_geometry(n=48, nv=24, nb=72, px=1.0, sod=120.0, sdd=240.0)
    slices = [synth.make_slice(g, seed=40 + i, i0=2e2) for i in range(ns)]
    x, reps, outs, t = run_both(g, slices, 40, nonneg=True)
    xu, _, _, _ = run_both(g, slices[:1], 40)
    assert xu.min() < 0.0
    assert x.min() >= 0.0
    for i in range(ns):
        for e in range(2):
            xo = outs[i][0][e]
            assert xo.min() >= 0.0
            assert rel_l2(x[i, e], xo) <= 1e-4
    b = (1.0, 0.6)
    for e in range(2):
        phi = oracle.objective(t, b[e] * slices[0].m[e].astype(np.float32), MU,
                               b[e] * x[0, e].astype(np.float64))
        assert abs(reps[e].objective - phi) <= 1e-4 * phi


def test_nonnegative_projection_warm_start_negative():
    """A warm start with negative pixels is used as given by the first step
    (the projection applies to the updated f only), in both implementations."""
    g = synth.tiny_geometry(n=40, nv=20, nb=64, px=1.0, sod=120.0, sdd=240.0)
    sl = synth.make_slice(g, seed=11, i0=1e5)
    rng = np.random.default_rng(3)
    x0 = (np.stack([sl.truth()[1]]) + rng.normal(0.0, 0.02, size=(1, 2, 40, 40))).astype(np.float32)
    assert x0.min() < 0.0
    x, reps, outs, t = run_both(g, [sl], 10, x0=x0, nonneg=True)
    assert x.min() >= 0.0
    for e in range(2):
        assert rel_l2(x[0, e], outs[0][0][e]) <= 1e-4
    # with no iterations the result is the warm start, negative pixels included
    # (up to the FP32 rounding of x -> beta x -> x)
    x1, _, _, _ = run_both(g, [sl], 0, x0=x0, nonneg=True)
    np.testing.assert_allclose(x1, x0, rtol=1e-6, atol=0.0)
    assert x1.min() < 0.0


@pytest.mark.parametrize("ns,rule,xi", [(1, dect.CAUCHY, 0.0), (5, dect.CAUCHY, 0.0), (3, dect.BB1, 100.0), (20, dect.CAUCHY, 0.0)])
def test_joint_tv(ns, rule, xi):
    """TV over both energies of a slice (4-vector shrink, one step per slice):
    parity with the oracle's joint ADM and the slice's joint objective on
    both channels' reports."""
    g = synth.tiny_geometry(n=48, nv=24, nb=72, px=1.0, sod=120.0, sdd=240.0)
    slices = [synth.make_slice(g, seed=60 + i, i0=1e4) for i in range(ns)]
    K = 30
    x, reps, outs, t = run_both(g, slices, K, rule=rule, xi=xi, joint=True)
    for i in range(ns):
        for e in range(2):
            assert rel_l2(x[i, e], outs[i][0][e]) <= 1e-4
        b = np.array([1.0, 0.6]).reshape(2, 1)
        gm = b * slices[i].m.reshape(2, -1).astype(np.float32)
        phi = oracle.objective_joint(t, gm, MU, b.reshape(2, 1, 1) * x[i].astype(np.float64))
        for e in range(2):
            assert reps[2 * i + e].iters == K
            assert abs(reps[2 * i + e].objective - phi) <= 1e-4 * phi
    # the coupling changes the result
    xs, _, _, _ = run_both(g, slices[:1], K)
    assert rel_l2(xs[0], x[0]) > 1e-3


def test_joint_tv_stop_and_projection():
    """Joint TV with the relative-objective stop (one test per slice: both
    channels stop together) and with the projection onto f >= 0."""
    g = synth.tiny_geometry(n=48, nv=24, nb=72, px=1.0, sod=120.0, sdd=240.0)
    sl = [synth.make_slice(g, seed=70 + i, i0=3e2) for i in range(2)]
    x, reps, outs, t = run_both(g, sl, 2000, tol=1e-4, joint=True)
    for i in range(2):
        assert reps[2 * i].iters == reps[2 * i + 1].iters
        assert reps[2 * i].converged and reps[2 * i + 1].converged
        assert abs(reps[2 * i].iters - outs[i][1][0]) <= 2
    x, reps, outs, t = run_both(g, sl, 40, joint=True, nonneg=True)
    assert x.min() >= 0.0
    for i in range(2):
        for e in range(2):
            assert rel_l2(x[i, e], outs[i][0][e]) <= 1e-4


def test_relative_objective_stop():
    g = synth.tiny_geometry(n=48, nv=24, nb=72, px=1.0, sod=120.0, sdd=240.0)
    sl = synth.make_slice(g, seed=9, i0=1e5)
    x, reps, outs, t = run_both(g, [sl], 2000, tol=1e-4)
    xo, its = outs[0]
    for e in range(2):
        assert reps[e].converged
        assert reps[e].rel_change < 1e-4
        # the stopping iteration can move by a step where the test is close to the threshold
        assert abs(reps[e].iters - its[e]) <= 2
    # at the GPU's iteration count the images agree
    x2, _, outs2, _ = run_both(g, [sl], reps[0].iters)
    assert rel_l2(x2[0, 0], outs2[0][0][0]) <= 1e-4


def test_zero_iterations_and_empty():
    g = synth.tiny_geometry(n=16, nv=8, nb=24)
    plan = dect.Plan(g)
    m = torch.zeros((0, 2, g.nv, g.nb), device="cuda")
    x, reps = dect.adm_tv(plan, m, dect.AdmParams(max_iter=5))
    assert x.shape == (0, 2, g.n, g.n)
    m = torch.rand((1, 2, g.nv, g.nb), device="cuda")
    x, reps = dect.adm_tv(plan, m, dect.AdmParams(max_iter=0))
    assert torch.count_nonzero(x) == 0
    with pytest.raises(dect.DectError):
        dect.adm_tv(plan, m, dect.AdmParams(mu=-1.0))


def test_deterministic():
    g = synth.tiny_geometry(n=48, nv=24, nb=72, px=1.0, sod=120.0, sdd=240.0)
    sl = synth.make_slice(g, seed=3)
    plan = dect.Plan(g)
    m = torch.tensor(sl.m[None], dtype=torch.float32, device="cuda")
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=25)
    a, _ = dect.adm_tv(plan, m, prm)
    b, _ = dect.adm_tv(plan, m, prm)
    assert torch.equal(a, b)


def test_paper_size_first_iterations():
    """512^2 / 60 views / 736 bins, two slices as the benchmark runs them: 4 iterations vs the oracle."""
    g = synth.paper_geometry()
    slices = [synth.make_slice(g, seed=20 + i, kind="head", i0=2e5) for i in range(2)]
    x, reps, outs, t = run_both(g, slices, 4)
    for i in range(2):
        for e in range(2):
            assert rel_l2(x[i, e], outs[i][0][e]) <= 1e-4


@pytest.mark.parametrize("ns,joint,tv", [(8, False, None), (6, True, None), (8, False, 1), (6, True, 1)])
def test_narrowing_batch_matches_oracle(ns, joint, tv):
    """Channels whose relative-objective stop comes at different iterations
    (slices of very different dose): once half of a batch has stopped, the
    running channels continue in a batch half as wide.  Every channel ends as
    the oracle does at the channel's own iteration count, with the report of
    that result.  tv = 1: the TMA-staged TV step at every width that has it."""
    g = synth.tiny_geometry(n=48, nv=24, nb=72, px=1.0, sod=120.0, sdd=240.0)
    doses = [3e2, 1e6, 1e3, 3e5, 1e4, 3e3, 1e5, 5e2][:ns]
    slices = [synth.make_slice(g, seed=500 + i, i0=doses[i]) for i in range(ns)]
    plan = dect.Plan(g)
    if tv is not None:
        for w in (4, 8, 16, 32, 64):
            plan.set_tv_tuning(w, tv)
    t = oracle.table(g)
    m = np.stack([s.m for s in slices]).astype(np.float32)
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=3000, rel_obj_tol=1e-4, check_every=10, joint=joint)
    x, reps, prof = dect.adm_tv(plan, torch.tensor(m, device="cuda"), prm, profile=True)
    x = x.cpu().numpy()
    iters = [r.iters for r in reps]
    assert all(r.converged for r in reps)
    assert max(iters) - min(iters) >= 20          # the stops are spread over several checks
    nb = 1 << (2 * ns - 1).bit_length()
    full = 8 * plan.nnz + 8 * (g.nv * g.nb + 1) + 4 * nb * (g.n * g.n + g.nv * g.nb)
    assert prof.table_bytes_fwd < full           # part of the launches ran narrowed
    b = (1.0, 0.6)
    for i in range(ns):
        k = reps[2 * i].iters
        if joint:
            assert reps[2 * i + 1].iters == k
        op = oracle.AdmParams(mu=MU, rho=RHO, max_iter=k, step_rule=oracle.CAUCHY, joint=joint)
        xo, _ = oracle.adm_dual(t, m[i].astype(np.float64), op) if joint else (None, None)
        for e in range(2):
            if not joint:
                op = oracle.AdmParams(mu=MU, rho=RHO, max_iter=reps[2 * i + e].iters, step_rule=oracle.CAUCHY)
                f, _, _, _ = oracle.adm_channel(t, b[e] * m[i, e].astype(np.float64), op)
                xe = f / b[e]
            else:
                xe = xo[e]
            assert rel_l2(x[i, e], xe) <= 1e-4, (i, e)
            if not joint:
                phi = oracle.objective(t, b[e] * m[i, e].astype(np.float64), MU, b[e] * x[i, e].astype(np.float64))
                assert abs(reps[2 * i + e].objective - phi) <= 1e-4 * phi


def test_paper_size_bench_configuration():
    """The benchmark's launch configuration: 32 slices (64 interleaved channels,
    the autotuned 1024-thread table kernels) of the benchmark's inputs at
    512^2 / 60 views / 736 bins with its parameters, 4 iterations; three of
    the slices against the oracle."""
    g = synth.paper_geometry()
    S = 32
    m = np.stack([synth.make_slice(g, seed=1000 + i, kind="head", i0=2e5).m for i in range(S)]).astype(np.float32)
    plan = dect.Plan(g)
    prm = dect.AdmParams(mu=4.0, rho=256.0, beta=(1.0, 0.6), max_iter=4)
    x, reps = dect.adm_tv(plan, torch.tensor(m, device="cuda"), prm)
    x = x.cpu().numpy()
    assert all(r.iters == 4 for r in reps)
    t = oracle.table(g)
    op = oracle.AdmParams(mu=4.0, rho=256.0, beta=(1.0, 0.6), max_iter=4, step_rule=oracle.CAUCHY)
    for i in (0, 17, 31):
        xo, _ = oracle.adm_dual(t, m[i].astype(np.float64), op)
        for e in range(2):
            assert rel_l2(x[i, e], xo[e]) <= 1e-4, (i, e)


def test_zero_data_gives_the_zero_image():
    """m = 0: the minimiser of Eq. (4) is f = 0; no step is taken, nothing
    becomes non-finite, and the stop test fires on the zero objective."""
    g = synth.tiny_geometry(n=24, nv=12, nb=36)
    plan = dect.Plan(g)
    m = torch.zeros((2, 2, g.nv, g.nb), device="cuda")
    x, reps = dect.adm_tv(plan, m, dect.AdmParams(mu=MU, rho=RHO, max_iter=50, rel_obj_tol=1e-4))
    assert torch.count_nonzero(x) == 0
    for r in reps:
        assert r.objective == 0.0 and r.converged
    f, k, phi, _ = oracle.adm_channel(oracle.table(g), np.zeros((g.nv, g.nb)),
                                      oracle.AdmParams(mu=MU, rho=RHO, max_iter=5))
    assert np.count_nonzero(f) == 0 and np.all(phi == 0.0)


@pytest.mark.parametrize("ns", [1, 3, 16, 32])
def test_every_backprojector_variant(ns):
    """Each A^T variant the autotuner can pick gives the oracle's result."""
    g = synth.tiny_geometry(n=52, nv=24, nb=80, px=1.0, sod=130.0, sdd=260.0)
    slices = [synth.make_slice(g, seed=300 + i, i0=1e5) for i in range(ns)]
    plan = dect.Plan(g)
    t = oracle.table(g)
    m = np.stack([s.m for s in slices])
    width = min(64, 1 << (2 * ns - 1).bit_length())
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=12)
    for v in range(dect.BWD_VARIANTS):
        plan.set_tuning(width, v)
        x, _ = dect.adm_tv(plan, torch.tensor(m, dtype=torch.float32, device="cuda"), prm)
        x = x.cpu().numpy()
        for i in range(ns):
            op = oracle.AdmParams(mu=MU, rho=RHO, max_iter=12, step_rule=oracle.CAUCHY)
            xo, _ = oracle.adm_dual(t, m[i].astype(np.float32).astype(np.float64), op)
            for e in range(2):
                assert rel_l2(x[i, e], xo[e]) <= 1e-4, (v, i, e)
    plan.set_tuning(width, -1)
    dect.adm_tv(plan, torch.tensor(m, dtype=torch.float32, device="cuda"), prm)
    choice, us = plan.tuning(width)
    assert 0 <= choice < dect.BWD_VARIANTS and us[choice] > 0


@pytest.mark.parametrize("ns", [1, 3, 32])
@pytest.mark.parametrize("opts", [{}, {"joint": True}, {"nonneg": True}, {"xi": 128.0}, {"rule": dect.BB1}])
def test_every_tv_variant(ns, opts):
    """Each TV-step variant the autotuner can pick gives the oracle's result,
    and both give the same images (the same per-pixel arithmetic; only the
    FP32 partial sums of the norms, hence the reported objective, differ in
    their order).  52 x 52 pixels: two strips of 26 columns at 64 channels,
    more blocks than (strip, row) pairs, so some blocks get no rows."""
    g = synth.tiny_geometry(n=52, nv=24, nb=80, px=1.0, sod=130.0, sdd=260.0)
    slices = [synth.make_slice(g, seed=700 + i, i0=1e5) for i in range(ns)]
    plan = dect.Plan(g)
    t = oracle.table(g)
    m = np.stack([s.m for s in slices])
    width = min(64, 1 << (2 * ns - 1).bit_length())
    K = 12
    rule = opts.get("rule", dect.CAUCHY)
    xi = opts.get("xi", 0.0)
    joint, nonneg = opts.get("joint", False), opts.get("nonneg", False)
    prm = dect.AdmParams(mu=MU, rho=RHO, xi=xi, step_rule=rule, max_iter=K, joint=joint, nonneg=nonneg)
    xs, objs = [], []
    for v in range(dect.TV_VARIANTS):
        plan.set_tv_tuning(width, v)
        x, reps = dect.adm_tv(plan, torch.tensor(m, dtype=torch.float32, device="cuda"), prm)
        xs.append(x.cpu().numpy())
        objs.append([r.objective for r in reps])
        assert all(r.iters == K for r in reps)
    assert np.array_equal(xs[0], xs[1])
    np.testing.assert_allclose(objs[0], objs[1], rtol=1e-6)
    for i in range(ns):
        op = oracle.AdmParams(mu=MU, rho=RHO, xi=(xi if xi > 0 else None), step_rule=rule, max_iter=K,
                              joint=joint, nonneg=nonneg)
        xo, _ = oracle.adm_dual(t, m[i].astype(np.float32).astype(np.float64), op)
        for e in range(2):
            assert rel_l2(xs[1][i, e], xo[e]) <= 1e-4, (i, e)
    plan.set_tv_tuning(width, -1)
    dect.adm_tv(plan, torch.tensor(m, dtype=torch.float32, device="cuda"), prm)
    choice, us = plan.tv_tuning(width)
    assert 0 <= choice < dect.TV_VARIANTS and us[choice] > 0
    if width >= 4:
        assert all(u > 0 for u in us)


def test_uneven_geometry_groups():
    """Slices of different size and view count in one call, each against the oracle."""
    shapes = [(40, 18, 60, 2), (56, 30, 90, 1), (32, 12, 48, 3)]
    groups, refs = [], []
    for k, (n, nv, nb, S) in enumerate(shapes):
        g = synth.tiny_geometry(n=n, nv=nv, nb=nb, px=1.0, sod=3.0 * n, sdd=6.0 * n)
        slices = [synth.make_slice(g, seed=500 + 10 * k + i, i0=1e5) for i in range(S)]
        m = np.stack([s.m for s in slices])
        groups.append((dect.Plan(g), torch.tensor(m, dtype=torch.float32, device="cuda"), None))
        refs.append((g, m))
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=15)
    res = dect.adm_tv_groups(groups, prm, workers=2)
    for (x, reps), (g, m) in zip(res, refs):
        t = oracle.table(g)
        x = x.cpu().numpy()
        for i in range(m.shape[0]):
            op = oracle.AdmParams(mu=MU, rho=RHO, max_iter=15, step_rule=oracle.CAUCHY)
            xo, _ = oracle.adm_dual(t, m[i].astype(np.float32).astype(np.float64), op)
            for e in range(2):
                assert rel_l2(x[i, e], xo[e]) <= 1e-4
        assert all(r.iters == 15 for r in reps)


@pytest.mark.parametrize("ns", [1, 3, 16, 32])
def test_every_projector_variant(ns):
    """Each A variant the autotuner can pick gives the oracle's result, and
    each one's set-up projection r = A f - beta m (checked through a
    one-iteration run from a warm start, whose first step depends on it)."""
    g = synth.tiny_geometry(n=52, nv=24, nb=80, px=1.0, sod=130.0, sdd=260.0)
    slices = [synth.make_slice(g, seed=400 + i, i0=1e5) for i in range(ns)]
    plan = dect.Plan(g)
    t = oracle.table(g)
    m = np.stack([s.m for s in slices])
    width = min(64, 1 << (2 * ns - 1).bit_length())
    prm = dect.AdmParams(mu=MU, rho=RHO, max_iter=12)
    for v in range(dect.FWD_VARIANTS):
        plan.set_fwd_tuning(width, v)
        x, reps = dect.adm_tv(plan, torch.tensor(m, dtype=torch.float32, device="cuda"), prm)
        x = x.cpu().numpy()
        for i in range(ns):
            op = oracle.AdmParams(mu=MU, rho=RHO, max_iter=12, step_rule=oracle.CAUCHY)
            xo, _ = oracle.adm_dual(t, m[i].astype(np.float32).astype(np.float64), op)
            for e in range(2):
                assert rel_l2(x[i, e], xo[e]) <= 1e-4, (v, i, e)
                assert reps[2 * i + e].resid_drift <= 1e-5 * reps[2 * i + e].primal_res, (v, i, e)
    plan.set_fwd_tuning(width, -1)
    dect.adm_tv(plan, torch.tensor(m, dtype=torch.float32, device="cuda"), prm)
    choice, us = plan.fwd_tuning(width)
    assert 0 <= choice < dect.FWD_VARIANTS and us[choice] > 0
