"""Pins of the oracle's TV operators (Eq. (2)), shrinkage (Eq. (8)) and ADM (Eq. (6)-(10)).

References used instead of the oracle itself: numpy restatements of Eq. (2)
and Eq. (6), closed forms, the subgradient optimality conditions of the
z-subproblem, finite differences of the augmented Lagrangian, the exact
power-of-two scaling identity of Eq. (3)-(6), and the Fenchel dual bound of
Eq. (4) (an optimality certificate that no solver produces).
"""
import numpy as np
import pytest

import indep
import oracle
import synth


def test_grad_matches_definition_and_transpose():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((9, 9))
    p = rng.standard_normal((2, 9, 9))
    np.testing.assert_array_equal(oracle.grad(x), indep.grad_np(x))
    np.testing.assert_allclose(oracle.grad_t(p), indep._gradT_np(p), rtol=0, atol=1e-14)
    lhs = float((oracle.grad(x) * p).sum())
    rhs = float((x * oracle.grad_t(p)).sum())
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_tv_closed_forms():
    n = 10
    # vertical step of height h between columns 3 and 4: TV = n h
    x = np.zeros((n, n))
    x[:, 4:] = 0.25
    assert abs(oracle.tv(x) - n * 0.25) < 1e-14
    # plane x_ij = a i + b j: (n-1)^2 sqrt(a^2+b^2) + (n-1)(|a| + |b|)
    a, b = 0.3, -0.7
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = a * i + b * j
    want = (n - 1) ** 2 * np.hypot(a, b) + (n - 1) * (abs(a) + abs(b))
    assert abs(oracle.tv(x) - want) < 1e-12
    d = oracle.grad(x)
    assert np.all(d[0, 1:] == pytest.approx(a)) and np.all(d[0, 0] == 0)
    assert np.all(d[1, :, 1:] == pytest.approx(b)) and np.all(d[1, :, 0] == 0)


def test_shrink_is_prox_of_norm():
    """z = argmin |z| + 1/(2t) |z - w|^2: check the subgradient optimality conditions."""
    rng = np.random.default_rng(1)
    t = 0.3
    w = rng.standard_normal((2, 400)) * 0.5
    w[:, :5] = 0.0
    z = oracle.shrink(w, t)
    nw = np.hypot(w[0], w[1])
    nz = np.hypot(z[0], z[1])
    out = nw <= t
    assert np.all(nz[out] == 0.0)
    # on the active set (w - z)/t must be the unit vector z/|z|
    act = ~out
    g = (w[:, act] - z[:, act]) / t
    np.testing.assert_allclose(g, z[:, act] / nz[act], rtol=1e-12, atol=1e-12)
    # brute force on a grid for a few points
    for k in range(5, 12):
        grid = np.linspace(-2, 2, 801)
        Z0, Z1 = np.meshgrid(grid, grid, indexing="ij")
        h = np.hypot(Z0, Z1) + ((Z0 - w[0, k]) ** 2 + (Z1 - w[1, k]) ** 2) / (2 * t)
        a = np.unravel_index(np.argmin(h), h.shape)
        assert abs(grid[a[0]] - z[0, k]) <= 0.006 and abs(grid[a[1]] - z[1, k]) <= 0.006


def _tiny_problem(seed=1, noise=0.002):
    g = synth.tiny_geometry(n=8, nv=12, nb=12)
    t = oracle.table(g)
    A = indep.clip_matrix(g)
    x = np.zeros((8, 8))
    x[2:6, 3:7] = 0.02
    x[1:3, 1:3] = 0.01
    rng = np.random.default_rng(seed)
    m = A @ x.reshape(-1) + noise * rng.standard_normal(A.shape[0])
    return g, t, A, m


def test_G_is_gradient_of_augmented_lagrangian():
    """G_f of Eq. (9) is d/df of Eq. (6) at (f^k, z^{k+1}, lambda^k)."""
    g, t, A, m = _tiny_problem()
    prm = oracle.AdmParams(mu=16.0, rho=8.0, xi=5.0, step_rule=oracle.CAUCHY)
    st = oracle.AdmState(np.zeros((8, 8)))
    for _ in range(3):
        oracle.adm_iterate(t, m, prm, st)
    f_k = st.f.copy()
    lam_k = st.lam.copy()
    _, G, _ = oracle.adm_iterate(t, m, prm, st)
    z_k1 = st.z.copy()
    h = 1e-6
    fd = np.zeros(64)
    for p in range(64):
        e = np.zeros(64)
        e[p] = h
        fp = indep.aug_lagrangian(A, m, f_k + e.reshape(8, 8), z_k1, lam_k, prm.mu, prm.rho)
        fm = indep.aug_lagrangian(A, m, f_k - e.reshape(8, 8), z_k1, lam_k, prm.mu, prm.rho)
        fd[p] = (fp - fm) / (2 * h)
    np.testing.assert_allclose(G.reshape(-1), fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max())


def test_augmented_lagrangian_monotone_within_iteration():
    """With lambda fixed, the z-step and the exact-step f-step never increase Eq. (6)."""
    g, t, A, m = _tiny_problem(seed=2)
    prm = oracle.AdmParams(mu=16.0, rho=16.0, step_rule=oracle.CAUCHY)
    st = oracle.AdmState(np.zeros((8, 8)))
    for k in range(40):
        f0, z0, l0 = st.f.copy(), st.z.copy(), st.lam.copy()
        L0 = indep.aug_lagrangian(A, m, f0, z0, l0, prm.mu, prm.rho)
        alpha, G, _ = oracle.adm_iterate(t, m, prm, st)
        L1 = indep.aug_lagrangian(A, m, f0, st.z, l0, prm.mu, prm.rho)
        L2 = indep.aug_lagrangian(A, m, st.f, st.z, l0, prm.mu, prm.rho)
        tol = 1e-12 * abs(L0) + 1e-15
        assert L1 <= L0 + tol
        assert L2 <= L1 + tol
        # the step is the exact minimiser along -G
        for s in (0.9, 1.1):
            Ls = indep.aug_lagrangian(A, m, f0 - s * alpha * G, st.z, l0, prm.mu, prm.rho)
            assert L2 <= Ls + tol


def test_bb1_rule_lags_the_exact_step():
    g, t, A, m = _tiny_problem(seed=3)
    prm = oracle.AdmParams(mu=16.0, rho=16.0, step_rule=oracle.BB1)
    st = oracle.AdmState(np.zeros((8, 8)))
    prev = None
    for k in range(6):
        alpha, G, (gg, aa, dd) = oracle.adm_iterate(t, m, prm, st)
        c = gg / (prm.mu * aa + prm.rho * dd)
        # |A G|^2 and |grad G|^2 against the independent operators
        assert abs(aa - float(np.sum((A @ G.reshape(-1)) ** 2))) <= 1e-12 * aa
        assert abs(dd - float(np.sum(indep.grad_np(G) ** 2))) <= 1e-12 * dd
        assert alpha == (c if prev is None else prev)
        prev = c


def test_beta_scaling_identity_is_exact():
    """ADM on (beta m; mu, rho, xi) / beta == ADM on (m; beta mu, beta rho, beta xi), beta = 2^k."""
    g, t, A, m = _tiny_problem(seed=4)
    for beta in (2.0, 0.5):
        a = oracle.AdmParams(mu=16.0, rho=8.0, xi=4.0, step_rule=oracle.CAUCHY, max_iter=25)
        b = oracle.AdmParams(mu=16.0 * beta, rho=8.0 * beta, xi=4.0 * beta,
                             step_rule=oracle.CAUCHY, max_iter=25)
        fa, _, _, _ = oracle.adm_channel(t, beta * m, a)
        fb, _, _, _ = oracle.adm_channel(t, m, b)
        np.testing.assert_allclose(fa / beta, fb, rtol=1e-12, atol=1e-16)


def _dual_value(A, g, mu, p, n):
    """Fenchel dual of Eq. (4): for |p_i| <= 1, D(p) = min_f <p, grad f> + mu/2 |A f - g|^2 <= Phi*."""
    nrm = np.maximum(1.0, np.hypot(p[0], p[1]))
    p = p / nrm
    AtA = A.T @ A
    rhs = A.T @ g - indep._gradT_np(p).reshape(-1) / mu
    f = np.linalg.solve(AtA, rhs)
    r = A @ f - g
    return float((p * indep.grad_np(f.reshape(n, n))).sum()) + 0.5 * mu * float(r @ r)


@pytest.mark.parametrize("rule", [oracle.CAUCHY, oracle.BB1])
def test_adm_reaches_the_minimiser(rule):
    """The ADM limit attains the optimum of Eq. (4): duality gap with p = -lambda -> 0.

    Also checked against an independent primal-dual solver (Chambolle-Pock).
    """
    g, t, A, m = _tiny_problem(seed=1)
    mu, rho = 16.0, 16.0
    prm = oracle.AdmParams(mu=mu, rho=rho, step_rule=rule)
    st = oracle.AdmState(np.zeros((8, 8)))
    for k in range(6000):
        oracle.adm_iterate(t, m, prm, st)
    primal = indep.tv_ls_objective(A, m, st.f, mu)
    dual = _dual_value(A, m, mu, -st.lam, 8)
    assert dual <= primal + 1e-12
    assert (primal - dual) / primal < 2e-5, (primal, dual)
    fcp = indep.chambolle_pock(A, m, 8, mu, iters=20000)
    pcp = indep.tv_ls_objective(A, m, fcp, mu)
    assert pcp >= dual - 1e-12                 # any primal point lies above the dual bound
    assert abs(pcp - primal) / primal < 5e-3   # the primal-dual solver approaches the same value


def test_noiseless_fully_sampled_fit():
    g = synth.tiny_geometry(n=8, nv=40, nb=16)
    t = oracle.table(g)
    A = indep.clip_matrix(g)
    x = np.zeros((8, 8))
    x[2:6, 2:5] = 0.03
    m = A @ x.reshape(-1)
    prm = oracle.AdmParams(mu=1024.0, rho=4.0, step_rule=oracle.CAUCHY, max_iter=400)
    f, k, phi, alpha = oracle.adm_channel(t, m, prm)
    r0 = np.linalg.norm(m)
    r = np.linalg.norm(A @ f.reshape(-1) - m)
    assert r < 2e-2 * r0
    assert phi[-1] < 0.05 * phi[0]
    assert np.abs(f - x).max() < 3e-3


def test_stopping_rule():
    g, t, A, m = _tiny_problem(seed=5)
    prm = oracle.AdmParams(mu=16.0, rho=16.0, step_rule=oracle.CAUCHY, max_iter=5000, tol=1e-4)
    f, k, phi, alpha = oracle.adm_channel(t, m, prm)
    assert k < 5000
    assert abs(phi[k] - phi[k - 1]) / phi[k - 1] < 1e-4
    assert all(abs(phi[i] - phi[i - 1]) / phi[i - 1] >= 1e-4 for i in range(1, k))


def test_dual_energy_wrapper_uses_beta():
    """adm_dual runs each channel on beta_c-scaled data and returns f_c / beta_c."""
    g, t, A, m = _tiny_problem(seed=6)
    mm = np.stack([m.reshape(12, 12), 1.2 * m.reshape(12, 12)])
    prm = oracle.AdmParams(mu=16.0, rho=16.0, step_rule=oracle.CAUCHY, max_iter=10, beta=(1.0, 0.5))
    x, its = oracle.adm_dual(t, mm, prm)
    f1, _, _, _ = oracle.adm_channel(t, 0.5 * mm[1], prm)
    np.testing.assert_array_equal(x[1], f1 / 0.5)


def test_nonnegative_variant():
    """With the projection onto f >= 0 (x in R_+^N, Eq. (1)) every iterate is
    nonnegative, and the limit satisfies the optimality conditions of the
    constrained subproblem: G ~ 0 where f > 0 and G >= 0 where f = 0."""
    g, t, A, m = _tiny_problem(seed=8, noise=0.05)
    prm = oracle.AdmParams(mu=64.0, rho=16.0, step_rule=oracle.CAUCHY, nonneg=True)
    st = oracle.AdmState(np.zeros((8, 8)))
    _, G0, _ = oracle.adm_iterate(t, m, prm, st)
    scale = np.abs(G0).max()
    for k in range(6000):
        _, G, _ = oracle.adm_iterate(t, m, prm, st)
        assert st.f.min() >= 0.0
    free = st.f > 1e-9
    assert np.abs(G[free]).max() < 1e-4 * scale
    assert G[~free].min() > -1e-4 * scale
    assert (~free).sum() > 0   # the constraint is active somewhere
    # the unconstrained run goes negative on this noisy problem
    f_u, _, _, _ = oracle.adm_channel(t, m, oracle.AdmParams(mu=64.0, rho=16.0, max_iter=3000))
    assert f_u.min() < -1e-3
