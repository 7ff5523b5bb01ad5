"""GPU parity of the PLS decomposition (Eq. (11)-(15)) against the FP64 oracle, through the C ABI.

Tolerance for basis maps: 2e-4 relative L2.

The edge map of Eq. (14) is an integer decided by floating point: the GPU
decides in FP32, the oracle in FP64.  The GPU map must equal the oracle's at
every pixel outside the rounding band of tests/edge_band.py, and that band
must be nearly empty; the basis maps are compared on inputs whose band the
test first shows to be empty, so both sides solve the same system.
"""
import numpy as np
import pytest

import edge_band
import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1607_01650_gb300 as dect  # noqa: E402


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def noisy_mixture(n, px, seed, sig=(4e-4, 6e-4)):
    g = synth.tiny_geometry(n=n, px=px, sod=10 * n * px, sdd=20 * n * px)
    ph = synth.random_ellipse_phantom(g, seed=seed, axis_range=(0.1 * n * px, 0.3 * n * px))
    u = synth.rasterize(ph, n, px, supersample=4)
    rng = np.random.default_rng(seed)
    xh = synth.attenuation(u, 0) + sig[0] * rng.standard_normal((n, n))
    xl = synth.attenuation(u, 1) + sig[1] * rng.standard_normal((n, n))
    return xh.astype(np.float32), xl.astype(np.float32), u


def no_band(xh, xl, tau=0.2):
    """The inputs leave no pixel within rounding of the edge threshold."""
    return not edge_band.mask_band(xh.astype(np.float64), xl.astype(np.float64), tau).any()


def run(xh, xl, gamma=0.1, K=60, tol=0.0, tau=0.2, eps=0.05):
    pp = dect.PlsParams(gamma=gamma, edge_tau=tau, edge_eps=eps, max_iter=K, tol=tol)
    x = torch.tensor(np.stack([xh, xl], axis=1), device="cuda")
    u, reps = dect.pls_decompose(x, pp)
    u = u.cpu().numpy()
    return u[:, 0], u[:, 1], reps


@pytest.mark.parametrize("n,batch", [(128, 1), (37, 3), (64, 2)])
def test_pls_fixed_iterations(n, batch):
    data = [noisy_mixture(n, 1.0, 30 + b) for b in range(batch)]
    xh = np.stack([d[0] for d in data])
    xl = np.stack([d[1] for d in data])
    u1, u2, reps = run(xh, xl)
    for b in range(batch):
        assert no_band(xh[b], xl[b])
        op = oracle.PlsParams(gamma=0.1, tau=0.2, eps=0.05, max_iter=60, tol=0.0)
        o1, o2, mask, its = oracle.pls_decompose(xh[b].astype(np.float64), xl[b].astype(np.float64), op)
        assert rel_l2(u1[b], o1) <= 2e-4
        assert rel_l2(u2[b], o2) <= 2e-4
        assert reps[b][0] == (60, 60)


def test_gamma_zero_is_direct_decomposition():
    xh, xl, _ = noisy_mixture(50, 1.0, 5)
    u1, u2, reps = run(xh[None], xl[None], gamma=0.0, K=10)
    d1, d2 = oracle.direct_decompose(synth.ETA, xh.astype(np.float64), xl.astype(np.float64))
    # FP64 2x2 solve rounded once to FP32 on both sides
    np.testing.assert_array_equal(u1[0], d1.astype(np.float32))
    np.testing.assert_array_equal(u2[0], d2.astype(np.float32))


def test_noiseless_mixture_is_recovered():
    n = 64
    rng = np.random.default_rng(2)
    U = rng.random((2, n, n))
    xh = (synth.ETA[0, 0] * U[0] + synth.ETA[1, 0] * U[1]).astype(np.float32)
    xl = (synth.ETA[0, 1] * U[0] + synth.ETA[1, 1] * U[1]).astype(np.float32)
    u1, u2, _ = run(xh[None], xl[None], gamma=0.0, K=0)
    # FP32 inputs: the error is the 2x2 condition number times FP32 rounding
    assert np.abs(u1[0] - U[0]).max() < 1e-4 and np.abs(u2[0] - U[1]).max() < 1e-4


def test_tolerance_stop():
    xh, xl, _ = noisy_mixture(96, 1.0, 6)
    u1, u2, reps = run(xh[None], xl[None], K=500, tol=1e-6)
    its, rr = reps[0]
    assert max(its) < 500 and max(rr) < 1e-6
    assert no_band(xh, xl)
    op = oracle.PlsParams(gamma=0.1, tau=0.2, eps=0.05, max_iter=500, tol=1e-10)
    o1, o2, _, _ = oracle.pls_decompose(xh.astype(np.float64), xl.astype(np.float64), op)
    assert rel_l2(u1[0], o1) <= 2e-4 and rel_l2(u2[0], o2) <= 2e-4


def test_paper_size_sampled():
    """512^2 slice, gamma 0.1, full PCG: compare with the oracle on the whole map."""
    xh, xl, _ = noisy_mixture(512, 0.5, 9)
    assert no_band(xh, xl)
    u1, u2, reps = run(xh[None], xl[None], K=500, tol=1e-6)
    op = oracle.PlsParams(gamma=0.1, tau=0.2, eps=0.05, max_iter=500, tol=1e-10)
    o1, o2, _, _ = oracle.pls_decompose(xh.astype(np.float64), xl.astype(np.float64), op)
    assert rel_l2(u1[0], o1) <= 2e-4 and rel_l2(u2[0], o2) <= 2e-4


def test_paper_size_bench_batch():
    """The benchmark's launch configuration: 32 slices of 512^2 in one call
    (PCG to 1e-6, as the benchmark runs it); the first and last slices against
    the oracle."""
    maps = [noisy_mixture(512, 0.5, 40 + s) for s in range(32)]
    xh = np.stack([m[0] for m in maps])
    xl = np.stack([m[1] for m in maps])
    u1, u2, reps = run(xh, xl, K=500, tol=1e-6)
    op = oracle.PlsParams(gamma=0.1, tau=0.2, eps=0.05, max_iter=500, tol=1e-10)
    for s in (0, 31):
        assert no_band(xh[s], xl[s]), s
        o1, o2, _, _ = oracle.pls_decompose(xh[s].astype(np.float64), xl[s].astype(np.float64), op)
        assert rel_l2(u1[s], o1) <= 2e-4 and rel_l2(u2[s], o2) <= 2e-4, s


@pytest.mark.parametrize("n,px,seeds,tau", [(128, 1.0, (30,), 0.2), (37, 1.0, (30, 31, 32), 0.2),
                                            (512, 0.5, tuple(range(40, 72)), 0.2),
                                            (96, 1.0, (6, 7), 0.05), (64, 1.0, (8,), 0.6)])
def test_edge_mask_equals_fp64_decision_outside_rounding_band(n, px, seeds, tau):
    """Eq. (14): the GPU's FP32 edge map against the oracle's FP64 map."""
    maps = [noisy_mixture(n, px, s) for s in seeds]
    xh = np.stack([m[0] for m in maps])
    xl = np.stack([m[1] for m in maps])
    x = torch.tensor(np.stack([xh, xl], axis=1), device="cuda")
    got = dect.pls_edge_mask(x, tau).cpu().numpy().astype(bool)
    in_band = 0
    for b in range(len(seeds)):
        h, lo = xh[b].astype(np.float64), xl[b].astype(np.float64)
        want = oracle.edge_mask(h, lo, tau).astype(bool)
        band = edge_band.mask_band(h, lo, tau)
        assert want.any() and not want.all()
        np.testing.assert_array_equal(got[b][~band], want[~band])
        in_band += int(band.sum())
    assert in_band <= max(4, 1e-4 * len(seeds) * n * n)


def test_edge_mask_special_cases():
    """An empty image has no edges; a single step edge is found in both images alone."""
    n = 40
    z = np.zeros((n, n), np.float32)
    step = z.copy()
    step[:, n // 2:] = 0.02
    x = torch.tensor(np.stack([np.stack([z, z]), np.stack([step, z]), np.stack([z, step])]), device="cuda")
    got = dect.pls_edge_mask(x, 0.2).cpu().numpy()
    assert not got[0].any()
    want = oracle.edge_mask(step.astype(np.float64), z.astype(np.float64), 0.2)
    np.testing.assert_array_equal(got[1], want)
    np.testing.assert_array_equal(got[2], want)
    assert got[1][:, n // 2 - 1: n // 2 + 1].all() and got[1].sum() == 2 * n
