"""Pins of the oracle's joint (channel-coupled) TV ADM.

Reading: the TV of Eq. (4) on the combined image f = (f_h, f_l) is the
per-pixel 2-norm over both channels' gradients, so the z-step of Eq. (8)
shrinks 4-vectors and one step alpha serves the stacked f.  Pinned by the
prox conditions, the gradient of Eq. (6), exact reductions to the
per-channel ADM, and the optimum of an independent primal-dual solver.
"""
import numpy as np

import oracle
import synth

import indep


def test_shrink4_is_prox_of_the_4_norm():
    rng = np.random.default_rng(2)
    t = 0.3
    wh = rng.standard_normal((2, 500)) * 0.3
    wl = rng.standard_normal((2, 500)) * 0.3
    wh[:, :4] = 0.0
    wl[:, :4] = 0.0
    zh, zl = oracle.shrink4(wh, wl, t)
    w = np.concatenate([wh, wl])
    z = np.concatenate([zh, zl])
    nw = np.sqrt((w ** 2).sum(0))
    nz = np.sqrt((z ** 2).sum(0))
    out = nw <= t
    assert np.all(z[:, out] == 0.0)
    act = ~out
    np.testing.assert_allclose((w[:, act] - z[:, act]) / t, z[:, act] / nz[act], rtol=1e-12, atol=1e-12)
    # objective |z| + |z - w|^2 / (2t) is not lowered by random perturbations
    h = lambda zz, ww: np.sqrt((zz ** 2).sum(0)) + ((zz - ww) ** 2).sum(0) / (2 * t)
    base = h(z, w)
    for _ in range(50):
        d = rng.standard_normal(z.shape) * 1e-3
        assert np.all(h(z + d, w) >= base - 1e-15)
    # with a zero second channel it is the 2-vector shrink, bit for bit
    zh2, zl2 = oracle.shrink4(wh, np.zeros_like(wl), t)
    np.testing.assert_array_equal(zh2, oracle.shrink(wh, t))
    assert np.all(zl2 == 0.0)


def test_tv_joint_closed_forms():
    rng = np.random.default_rng(3)
    f = rng.random((9, 9))
    assert oracle.tv_joint(np.stack([f, np.zeros_like(f)])) == oracle.tv(f)
    assert abs(oracle.tv_joint(np.stack([f, f])) - np.sqrt(2.0) * oracle.tv(f)) <= 1e-12 * oracle.tv(f)
    # a ramp along x in one channel and along y in the other: |(0, a, b, 0)| = hypot(a, b)
    n = 6
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a, b = 0.3, 0.4
    f2 = np.stack([a * jj, b * ii]).astype(np.float64)
    # interior pixels (i, j >= 1): 0.5 each; first row: only the x-ramp, first column: only the y-ramp
    expect = (n - 1) ** 2 * 0.5 + (n - 1) * a + (n - 1) * b
    assert abs(oracle.tv_joint(f2) - expect) <= 1e-12
    g = rng.random((2, 9, 9))
    assert abs(oracle.tv_joint(g) - indep.tv_joint_np(g)) <= 1e-12 * indep.tv_joint_np(g)


def _tiny_joint(seed=1, noise=0.002):
    g = synth.tiny_geometry(n=8, nv=12, nb=12)
    t = oracle.table(g)
    A = indep.clip_matrix(g)
    x = np.zeros((2, 8, 8))
    x[0, 2:6, 3:7] = 0.02
    x[0, 1:3, 1:3] = 0.01
    x[1, 2:6, 3:7] = 0.03      # a shared edge and one that only channel 1 has
    x[1, 5:7, 1:3] = 0.015
    rng = np.random.default_rng(seed)
    m = np.stack([A @ x[c].reshape(-1) for c in range(2)]) + noise * rng.standard_normal((2, A.shape[0]))
    return g, t, A, m


def test_joint_G_is_gradient_of_augmented_lagrangian():
    g, t, A, m = _tiny_joint()
    prm = oracle.AdmParams(mu=16.0, rho=8.0, xi=5.0, step_rule=oracle.CAUCHY)
    st = oracle.AdmJointState(np.zeros((2, 8, 8)))
    for _ in range(3):
        oracle.adm_joint_iterate(t, m, prm, st)
    f_k, lam_k = st.f.copy(), st.lam.copy()
    _, G, _ = oracle.adm_joint_iterate(t, m, prm, st)
    z_k1 = st.z.copy()
    h = 1e-6
    fd = np.zeros(128)
    for p in range(128):
        e = np.zeros(128)
        e[p] = h
        e = e.reshape(2, 8, 8)
        fp = indep.aug_lagrangian_joint(A, m, f_k + e, z_k1, lam_k, prm.mu, prm.rho)
        fm = indep.aug_lagrangian_joint(A, m, f_k - e, z_k1, lam_k, prm.mu, prm.rho)
        fd[p] = (fp - fm) / (2 * h)
    np.testing.assert_allclose(G.reshape(-1), fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max())


def test_joint_step_is_exact_and_lagrangian_monotone():
    g, t, A, m = _tiny_joint(seed=2)
    prm = oracle.AdmParams(mu=16.0, rho=16.0, step_rule=oracle.CAUCHY)
    st = oracle.AdmJointState(np.zeros((2, 8, 8)))
    for k in range(30):
        f0, z0, l0 = st.f.copy(), st.z.copy(), st.lam.copy()
        L0 = indep.aug_lagrangian_joint(A, m, f0, z0, l0, prm.mu, prm.rho)
        alpha, G, (gg, aa, dd) = oracle.adm_joint_iterate(t, m, prm, st)
        L1 = indep.aug_lagrangian_joint(A, m, f0, st.z, l0, prm.mu, prm.rho)
        L2 = indep.aug_lagrangian_joint(A, m, st.f, st.z, l0, prm.mu, prm.rho)
        tol = 1e-12 * abs(L0) + 1e-15
        assert L1 <= L0 + tol and L2 <= L1 + tol
        for s in (0.9, 1.1):
            Ls = indep.aug_lagrangian_joint(A, m, f0 - s * alpha * G, st.z, l0, prm.mu, prm.rho)
            assert L2 <= Ls + tol
        # norms over both channels, against the independent operators
        aa_i = sum(float(np.sum((A @ G[c].reshape(-1)) ** 2)) for c in range(2))
        dd_i = sum(float(np.sum(indep.grad_np(G[c]) ** 2)) for c in range(2))
        assert abs(aa - aa_i) <= 1e-12 * aa and abs(dd - dd_i) <= 1e-12 * dd


def test_joint_with_an_empty_channel_is_the_per_channel_adm():
    """With g_l = 0 and f_l = 0 the second channel stays 0, the 4-norm is the
    2-norm of channel h, and the joint iteration is the per-channel one."""
    g, t, A, m = _tiny_joint(seed=3)
    for rule in (oracle.CAUCHY, oracle.BB1):
        prm = oracle.AdmParams(mu=16.0, rho=16.0, xi=9.0, step_rule=rule, max_iter=40)
        mm = np.stack([m[0], np.zeros_like(m[0])])
        fj, kj, phij, aj = oracle.adm_joint(t, mm, prm)
        fs, ks, phis, as_ = oracle.adm_channel(t, m[0], prm)
        assert kj == ks == 40
        np.testing.assert_array_equal(fj[1], 0.0)
        np.testing.assert_array_equal(fj[0], fs)
        np.testing.assert_array_equal(aj, as_)
        np.testing.assert_array_equal(phij, phis)


def test_joint_with_equal_channels_is_a_rescaled_per_channel_problem():
    """g_h = g_l: the joint minimiser has f_h = f_l = f, and sqrt(2) |grad f| +
    mu |A f - g|^2 makes f the per-channel minimiser at mu' = sqrt(2) mu."""
    g, t, A, m = _tiny_joint(seed=4)
    mu = 16.0
    prm = oracle.AdmParams(mu=mu, rho=16.0, step_rule=oracle.CAUCHY, max_iter=20000)
    fj, _, _, _ = oracle.adm_joint(t, np.stack([m[0], m[0]]), prm)
    fs, _, _, _ = oracle.adm_channel(t, m[0], oracle.AdmParams(mu=np.sqrt(2.0) * mu, rho=16.0,
                                                              step_rule=oracle.CAUCHY, max_iter=20000))
    np.testing.assert_array_equal(fj[0], fj[1])
    # Phi_joint(f, f) = sqrt(2) Phi(f; sqrt(2) mu): equal optimal values, close minimisers
    pj = oracle.objective_joint(t, np.stack([m[0], m[0]]), mu, fj)
    ps = oracle.objective(t, m[0], np.sqrt(2.0) * mu, fs)
    assert abs(pj - np.sqrt(2.0) * ps) <= 1e-12 * pj
    assert np.abs(fj[0] - fs).max() <= 1e-10 * np.abs(fs).max()


def _joint_dual_value(A, g, mu, p, n):
    """Fenchel dual of the joint problem for p = [2][2][n][n] with the per-pixel
    4-norm <= 1: D(p) = sum_c min_f <p_c, grad f> + mu/2 |A f - g_c|^2."""
    nrm = np.maximum(1.0, np.sqrt((p ** 2).sum(axis=(0, 1))))
    p = p / nrm
    AtA = A.T @ A
    val = 0.0
    for c in range(2):
        f = np.linalg.solve(AtA, A.T @ g[c] - indep._gradT_np(p[c]).reshape(-1) / mu)
        r = A @ f - g[c]
        val += float((p[c] * indep.grad_np(f.reshape(n, n))).sum()) + 0.5 * mu * float(r @ r)
    return val


def test_joint_adm_reaches_the_minimiser():
    g, t, A, m = _tiny_joint(seed=1)
    mu, rho = 16.0, 16.0
    prm = oracle.AdmParams(mu=mu, rho=rho, step_rule=oracle.CAUCHY)
    st = oracle.AdmJointState(np.zeros((2, 8, 8)))
    for k in range(6000):
        oracle.adm_joint_iterate(t, m, prm, st)
    primal = indep.tv_ls_objective_joint(A, m, st.f, mu)
    assert abs(primal - oracle.objective_joint(t, m, mu, st.f)) <= 1e-12 * primal
    dual = _joint_dual_value(A, m, mu, -st.lam, 8)
    assert dual <= primal + 1e-12
    assert (primal - dual) / primal < 2e-5, (primal, dual)
    fcp = indep.chambolle_pock_joint(A, m, 8, mu, iters=20000)
    pcp = indep.tv_ls_objective_joint(A, m, fcp, mu)
    assert pcp >= dual - 1e-12
    assert abs(pcp - primal) / primal < 5e-3
    # the coupled optimum differs from the per-channel one on this problem
    fs = np.stack([oracle.adm_channel(t, m[c], oracle.AdmParams(mu=mu, rho=rho, max_iter=6000))[0]
                   for c in range(2)])
    assert indep.tv_ls_objective_joint(A, m, fs, mu) > primal * (1 + 1e-4)


def test_adm_dual_joint_uses_beta():
    g, t, A, m = _tiny_joint(seed=5)
    mm = m.reshape(2, 12, 12)
    prm = oracle.AdmParams(mu=16.0, rho=16.0, max_iter=10, beta=(1.0, 0.5), joint=True)
    x, its = oracle.adm_dual(t, mm, prm)
    f, k, _, _ = oracle.adm_joint(t, np.stack([mm[0], 0.5 * mm[1]]), prm)
    assert its == [10, 10]
    np.testing.assert_array_equal(x[0], f[0])
    np.testing.assert_array_equal(x[1], f[1] / 0.5)
