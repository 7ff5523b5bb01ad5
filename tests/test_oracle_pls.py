"""Pins of the oracle's decomposition (Eq. (11)-(15), Sec. 2.3).

References: exact recovery of noiseless mixtures x = D u, the gamma = 0
special case, a dense Hessian of Eq. (13)-(14) assembled pair by pair from
the definition of R(u), finite differences of Eq. (13), fixed points of the
smoothness term, and a closed-form Prewitt response.
"""
import numpy as np

import indep
import oracle
import synth

ETA = synth.ETA


def _mix(u1, u2):
    xh = ETA[0, 0] * u1 + ETA[1, 0] * u2
    xl = ETA[0, 1] * u1 + ETA[1, 1] * u2
    return xh, xl


def test_direct_decomposition_recovers_noiseless_mixtures():
    rng = np.random.default_rng(0)
    u1, u2 = rng.random((2, 32, 32))
    xh, xl = _mix(u1, u2)
    d1, d2 = oracle.direct_decompose(ETA, xh, xl)
    np.testing.assert_allclose(d1, u1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(d2, u2, rtol=0, atol=1e-12)
    # and against a general 2x2 solve
    D = np.array([[ETA[0, 0], ETA[1, 0]], [ETA[0, 1], ETA[1, 1]]])
    sol = np.linalg.solve(D, np.stack([xh.reshape(-1), xl.reshape(-1)]))
    np.testing.assert_allclose(d1.reshape(-1), sol[0], atol=1e-12)


def test_gamma_zero_is_direct_decomposition():
    rng = np.random.default_rng(1)
    xh, xl = 0.02 * rng.random((2, 24, 24))
    prm = oracle.PlsParams(gamma=0.0)
    u1, u2, mask, its = oracle.pls_decompose(xh, xl, prm)
    d1, d2 = oracle.direct_decompose(ETA, xh, xl)
    np.testing.assert_array_equal(u1, d1)
    np.testing.assert_array_equal(u2, d2)


def test_pls_operator_equals_hessian_of_objective():
    """(I + gamma L_e) equals half the Hessian of Eq. (13) with R of Eq. (14)."""
    rng = np.random.default_rng(2)
    n = 9
    mask = (rng.random((n, n)) < 0.25).astype(np.uint8)
    gamma, eps = 0.7, 0.05
    H = indep.pls_matrix(mask, gamma, eps)
    U = rng.standard_normal((n, n))
    np.testing.assert_allclose(oracle.pls_apply(mask, gamma, eps, U).reshape(-1),
                               H @ U.reshape(-1), rtol=1e-13, atol=1e-13)


def test_pcg_matches_dense_solve_and_optimality():
    rng = np.random.default_rng(3)
    n = 16
    mask = (rng.random((n, n)) < 0.2).astype(np.uint8)
    gamma, eps = 0.8, 0.05
    d = rng.standard_normal((n, n))
    u, it, rr = oracle.pls_pcg(mask, gamma, eps, d, 500, 1e-14)
    H = indep.pls_matrix(mask, gamma, eps)
    want = np.linalg.solve(H, d.reshape(-1))
    np.testing.assert_allclose(u.reshape(-1), want, rtol=1e-10, atol=1e-10)
    # first-order optimality of Eq. (13): finite-difference gradient vanishes
    h = 1e-5
    for p in rng.choice(n * n, 12, replace=False):
        e = np.zeros(n * n)
        e[p] = h
        e = e.reshape(n, n)
        gp = (indep.pls_objective(u + e, d, mask, gamma, eps)
              - indep.pls_objective(u - e, d, mask, gamma, eps)) / (2 * h)
        assert abs(gp) < 1e-7


def test_constant_and_piecewise_constant_fixed_points():
    n = 12
    mask = np.zeros((n, n), np.uint8)
    d = np.full((n, n), 0.4)
    u, it, rr = oracle.pls_pcg(mask, 0.5, 0.05, d, 50, 1e-14)
    np.testing.assert_allclose(u, d, atol=1e-14)
    # two pieces separated by an edge band with eps = 0 stay unsmoothed
    d = np.zeros((n, n))
    d[:, 6:] = 1.0
    mask[:, 5:7] = 1
    u, it, rr = oracle.pls_pcg(mask, 0.5, 0.0, d, 50, 1e-14)
    np.testing.assert_allclose(u, d, atol=1e-13)


def test_prewitt_closed_form_and_mask():
    n = 10
    h = 0.3
    x = np.zeros((n, n))
    x[:, 5:] = h
    mag = oracle.prewitt(x)
    want = np.zeros((n, n))
    want[:, 4:6] = 3 * h
    np.testing.assert_allclose(mag, want, atol=1e-14)
    # horizontal step: same response on rows
    np.testing.assert_allclose(oracle.prewitt(x.T), want.T, atol=1e-14)
    # mask: either image above tau (after normalising by its own maximum)
    y = np.zeros((n, n))
    y[3:, :] = 0.01
    m = oracle.edge_mask(x, y, 0.5)
    want_m = (want > 0) | (oracle.prewitt(y) / oracle.prewitt(y).max() > 0.5)
    np.testing.assert_array_equal(m.astype(bool), want_m)


def test_prewitt_of_a_plane_and_mask_threshold():
    """A plane x = a i + b j has Prewitt components 6b (along j) and 6a (along i)
    inside the image and half of that on a replicated border; the mask keeps
    exactly the pixels whose magnitude over the maximum exceeds tau."""
    n, a, b = 9, 0.013, -0.004
    i, j = np.mgrid[0:n, 0:n].astype(np.float64)
    mag = oracle.prewitt(a * i + b * j)
    fi = np.where((i == 0) | (i == n - 1), 3.0, 6.0)
    fj = np.where((j == 0) | (j == n - 1), 3.0, 6.0)
    want = np.hypot(fi * a, fj * b)
    np.testing.assert_allclose(mag, want, rtol=1e-13, atol=1e-15)
    # the magnitudes take 4 distinct values: tau between them selects whole classes
    levels = np.unique(np.round(want / want.max(), 12))
    for lo, hi in zip(levels[:-1], levels[1:]):
        tau = 0.5 * (lo + hi)
        m = oracle.edge_mask(a * i + b * j, np.zeros((n, n)), tau)
        np.testing.assert_array_equal(m.astype(bool), want / want.max() > tau)
    # an empty image has no edges
    assert not oracle.edge_mask(np.zeros((n, n)), np.zeros((n, n)), 0.2).any()


def test_jacobi_diagonal_is_hessian_diagonal():
    """The PCG preconditioner is the diagonal of (I + gamma L_e) assembled pair
    by pair from Eq. (14); closed forms: 1 + gamma * (number of in-image
    neighbours) without edges, 1 + gamma * eps * (that number) when every
    pixel is an edge."""
    rng = np.random.default_rng(7)
    for n, frac in ((7, 0.3), (12, 0.1), (5, 1.0)):
        mask = (rng.random((n, n)) < frac).astype(np.uint8)
        gamma, eps = 0.37, 0.05
        want = np.diag(indep.pls_matrix(mask, gamma, eps)).reshape(n, n)
        np.testing.assert_allclose(oracle.pls_diag(mask, gamma, eps), want, rtol=1e-15, atol=1e-15)
    n, gamma, eps = 6, 0.5, 0.05
    deg = np.full((n, n), 4.0)
    deg[0, :] -= 1
    deg[-1, :] -= 1
    deg[:, 0] -= 1
    deg[:, -1] -= 1
    np.testing.assert_array_equal(oracle.pls_diag(np.zeros((n, n), np.uint8), gamma, eps), 1 + gamma * deg)
    np.testing.assert_allclose(oracle.pls_diag(np.ones((n, n), np.uint8), gamma, eps),
                               1 + gamma * eps * deg, rtol=1e-15)
    # one edge pixel lowers the weight of its own four links and of each neighbour's link to it
    mask = np.zeros((n, n), np.uint8)
    mask[2, 3] = 1
    d = oracle.pls_diag(mask, gamma, eps)
    assert d[2, 3] == 1 + gamma * 4 * eps
    for (ii, jj) in ((1, 3), (3, 3), (2, 2), (2, 4)):
        assert abs(d[ii, jj] - (1 + gamma * (3 + eps))) < 1e-15


def test_pls_reduces_noise_on_mixture():
    """On a noisy piecewise-constant mixture PLS is closer to u than D^{-1} x (Sec. 2.3)."""
    g = synth.small_geometry()
    ph = synth.random_ellipse_phantom(g, seed=4)
    u = synth.rasterize(ph, 64, 2.0, supersample=4)
    xh, xl = _mix(u[0], u[1])
    rng = np.random.default_rng(5)
    xh_n = xh + 4e-4 * rng.standard_normal(xh.shape)
    xl_n = xl + 6e-4 * rng.standard_normal(xl.shape)
    prm = oracle.PlsParams(gamma=0.5, tau=0.2, eps=0.05)
    u1, u2, mask, its = oracle.pls_decompose(xh_n, xl_n, prm)
    d1, d2 = oracle.direct_decompose(ETA, xh_n, xl_n)
    assert np.linalg.norm(u1 - u[0]) < 0.7 * np.linalg.norm(d1 - u[0])
    assert np.linalg.norm(u2 - u[1]) < 0.7 * np.linalg.norm(d2 - u[1])
