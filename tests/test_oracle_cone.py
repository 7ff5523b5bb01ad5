"""Pins of the oracle's cone-beam Siddon table and 3-D decomposition (Sec. 2.1,
Fig. 1 with a flat 2-D detector; Sec. 2.3, Eq. (13)-(15) with the 6 neighbours
of a voxel; Sec. 3).

References: an independent slab-clipping of every ray against every voxel
box, the ray's chord through the volume box, the exact reduction to the
fan-beam table when the volume is one slice and the detector one central
row, the mirror symmetry in z, the dense Hessian of Eq. (13)-(14) assembled
pair by pair, closed-form 3-D Prewitt responses, and the reduction of the
3-D decomposition to the 2-D one for a single slice.
"""
import dataclasses

import numpy as np
import pytest

import indep
import oracle
import synth

CONES = {
    "small": synth.tiny_cone(n=6, nz=4, nv=7, nr=5, nc=9),
    "offset": synth.tiny_cone(n=5, nz=3, nv=5, nr=4, nc=7, px=0.8, pz=1.3, off_u=0.35, off_v=-0.4),
    "flat_slab": synth.tiny_cone(n=6, nz=2, nv=6, nr=3, nc=8, pz=0.5, start=0.71),
}


def dense(t):
    A = np.zeros((t.m, t.npix))
    for r in range(t.m):
        s, e = t.rowptr[r], t.rowptr[r + 1]
        np.add.at(A[r], t.idx[s:e], t.len[s:e])
    return A


@pytest.mark.parametrize("name", list(CONES))
def test_siddon3_equals_voxel_clipping(name):
    g = CONES[name]
    t = oracle.table3(g)
    A = dense(t)
    B = indep.clip_matrix3(g)
    assert t.nnz > 0.5 * g.n_rays
    np.testing.assert_allclose(A, B, rtol=0, atol=1e-12 * max(1.0, B.max()))
    np.testing.assert_allclose(A.sum(1), indep.box_chord3(g), rtol=0, atol=1e-11)
    # one element per (ray, voxel)
    for r in range(t.m):
        s, e = t.rowptr[r], t.rowptr[r + 1]
        assert len(np.unique(t.idx[s:e])) == e - s


def test_project3_backproject3_use_the_table():
    g = CONES["small"]
    t = oracle.table3(g)
    A = indep.clip_matrix3(g)
    rng = np.random.default_rng(1)
    x = rng.random((g.nz, g.n, g.n))
    y = rng.random((g.nv, g.nr, g.nc))
    np.testing.assert_allclose(oracle.project3(t, x).reshape(-1), A @ x.reshape(-1), atol=1e-11)
    np.testing.assert_allclose(oracle.backproject3(t, y).reshape(-1), A.T @ y.reshape(-1), atol=1e-11)


def test_single_slice_central_row_is_the_fan_beam_table():
    """nz = 1 and one detector row at z = 0: every ray runs in the plane z = 0
    inside the slab, and the cone table equals the fan-beam table of the same
    in-plane geometry."""
    g3 = synth.ConeGeometry(n=9, nz=1, px=1.0, pz=2.0, nv=11, nr=1, nc=17, pu=1.9, pv=1.0, sod=40.0,
                            sdd=80.0, start=0.3, off_u=0.2)
    g2 = synth.tiny_geometry(n=9, nv=11, nb=17, px=1.0, pitch=1.9, sod=40.0, sdd=80.0, start=0.3,
                             det_offset=0.2)
    t3, t2 = oracle.table3(g3), oracle.table(g2)
    np.testing.assert_array_equal(t3.rowptr, t2.rowptr)
    np.testing.assert_array_equal(t3.idx, t2.idx)
    np.testing.assert_allclose(t3.len, t2.len, rtol=1e-15, atol=0)


def test_mirror_symmetry_in_z():
    """Flipping the volume in z mirrors the projections across the detector's
    centre row (rows reversed) when the detector is not offset in z.  The
    volume has an odd number of slices, so that the centre row's rays (in the
    plane z = 0) do not run along a slice boundary, where the midpoint rule
    gives them to the +z side on purpose."""
    g = synth.tiny_cone(n=6, nz=5, nv=7, nr=5, nc=9)
    t = oracle.table3(g)
    x = np.random.default_rng(3).random((g.nz, g.n, g.n))
    y = oracle.project3(t, x)
    yf = oracle.project3(t, x[::-1].copy())
    np.testing.assert_allclose(yf, y[:, ::-1, :], rtol=1e-12, atol=1e-12)


def test_pls3_operator_diagonal_and_solve():
    rng = np.random.default_rng(4)
    nz, n = 3, 4
    mask = (rng.random((nz, n, n)) < 0.25).astype(np.uint8)
    gamma, eps = 0.6, 0.05
    H = indep.pls_matrix3(mask, gamma, eps)
    U = rng.standard_normal((nz, n, n))
    np.testing.assert_allclose(oracle.pls_apply3(mask, gamma, eps, U).reshape(-1), H @ U.reshape(-1),
                               rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.pls_diag3(mask, gamma, eps).reshape(-1), np.diag(H), rtol=1e-15, atol=1e-15)
    d = rng.standard_normal((nz, n, n))
    u, it, rr = oracle.pls_pcg3(mask, gamma, eps, d, 500, 1e-14)
    np.testing.assert_allclose(u.reshape(-1), np.linalg.solve(H, d.reshape(-1)), rtol=1e-10, atol=1e-10)
    # no edges: 1 + gamma * (number of in-volume neighbours), 3 at a corner .. 6 inside
    deg = np.full((nz, n, n), 6.0)
    for ax, m in ((0, nz), (1, n), (2, n)):
        sl = [slice(None)] * 3
        sl[ax] = 0
        deg[tuple(sl)] -= 1
        sl[ax] = m - 1
        deg[tuple(sl)] -= 1
    np.testing.assert_array_equal(oracle.pls_diag3(np.zeros((nz, n, n), np.uint8), gamma, eps), 1 + gamma * deg)


def test_prewitt3_closed_forms():
    """A linear volume a j + b i + c k: each component is 18 times the slope
    inside and 9 times on a replicated border; a step along z responds in the
    two slices next to it only."""
    nz, n = 5, 6
    k, i, j = np.mgrid[0:nz, 0:n, 0:n].astype(np.float64)
    a, b, c = 0.01, -0.02, 0.005
    mag = oracle.prewitt3(a * j + b * i + c * k)
    f = lambda idx, m: np.where((idx == 0) | (idx == m - 1), 9.0, 18.0)  # noqa: E731
    want = np.sqrt((f(j, n) * a) ** 2 + (f(i, n) * b) ** 2 + (f(k, nz) * c) ** 2)
    np.testing.assert_allclose(mag, want, rtol=1e-13, atol=1e-15)
    step = np.zeros((nz, n, n))
    step[3:] = 0.3
    m = oracle.prewitt3(step)
    want = np.zeros((nz, n, n))
    want[2:4] = 9 * 0.3
    np.testing.assert_allclose(m, want, atol=1e-14)


def test_single_slice_decomposition_is_the_2d_one():
    """nz = 1: the 6-neighbour stencil loses its z links and the 3-D Prewitt
    magnitude is three times the 2-D one, so the edge map, the operator and
    the decomposition are the 2-D ones."""
    rng = np.random.default_rng(6)
    n = 12
    xh = 0.02 * rng.random((n, n))
    xl = 0.03 * rng.random((n, n))
    np.testing.assert_allclose(oracle.prewitt3(xh[None])[0], 3 * oracle.prewitt(xh), rtol=1e-14, atol=1e-16)
    prm = oracle.PlsParams(gamma=0.3, tau=0.2, eps=0.05, max_iter=40, tol=0.0)
    u1, u2, mask, _ = oracle.pls_decompose(xh, xl, prm)
    v1, v2, mask3, _ = oracle.pls_decompose3(xh[None], xl[None], prm)
    np.testing.assert_array_equal(mask3[0], mask)
    np.testing.assert_allclose(v1[0], u1, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(v2[0], u2, rtol=1e-13, atol=1e-15)
    # gamma = 0: the per-voxel 2x2 solve of Eq. (12)
    v1, v2, _, _ = oracle.pls_decompose3(xh[None], xl[None], dataclasses.replace(prm, gamma=0.0))
    d1, d2 = oracle.direct_decompose(synth.ETA, xh, xl)
    np.testing.assert_array_equal(v1[0], d1)
