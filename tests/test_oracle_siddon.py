"""Pins of the oracle's Siddon system matrix A (Eq. (1), Siddon's method [42]).

Each test compares the oracle against something other than itself: a
pixel-driven clip of every ray against every pixel square, closed-form box
chords, the exact 90-degree rotation symmetry of the fan-beam geometry,
and analytic ellipse line integrals.
"""
import math

import numpy as np
import pytest

import indep
import oracle
import synth


GEOMS = [
    synth.tiny_geometry(n=8, nv=12, nb=12),
    synth.tiny_geometry(n=7, nv=9, nb=16, px=0.7, start=0.1, det_offset=0.37),
    synth.tiny_geometry(n=16, nv=20, nb=24, px=0.5, sod=30.0, sdd=70.0, arc=math.pi),
    synth.tiny_geometry(n=1, nv=8, nb=5, px=2.0, sod=10.0, sdd=20.0, pitch=0.9),
]


@pytest.mark.parametrize("geom", GEOMS)
def test_siddon_equals_pixel_clip(geom):
    """Every entry of A equals the chord of the ray through that pixel square."""
    A = oracle.table(geom).dense()
    B = indep.clip_matrix(geom)
    assert A.shape == B.shape
    assert np.abs(A - B).max() <= 1e-12 * max(1.0, geom.sdd)


@pytest.mark.parametrize("geom", GEOMS)
def test_row_sums_are_box_chords(geom):
    """A applied to a constant image c gives c times the chord through the image box."""
    t = oracle.table(geom)
    c = 0.37
    y = oracle.project(t, np.full((geom.n, geom.n), c)).reshape(-1)
    want = c * indep.box_chord(geom)
    np.testing.assert_allclose(y, want, rtol=1e-12, atol=1e-12)


def test_single_pixel_closed_form():
    """n = 1: each entry is the segment length of the ray inside one square."""
    g = GEOMS[3]
    t = oracle.table(g)
    S, D = indep.rays_np(g)
    half = 0.5 * g.px
    for r in range(g.nv * g.nb):
        s, d = S[r], D[r] - S[r]
        # closed form: slab intersection of the infinite line with the square
        with np.errstate(divide="ignore"):
            tx = sorted(((-half - s[0]) / d[0], (half - s[0]) / d[0]))
            ty = sorted(((-half - s[1]) / d[1], (half - s[1]) / d[1]))
        lo, hi = max(tx[0], ty[0]), min(tx[1], ty[1])
        want = max(hi - lo, 0.0) * math.hypot(d[0], d[1])
        got = t.len[t.rowptr[r]:t.rowptr[r + 1]].sum()
        assert abs(got - want) <= 1e-12


def test_rotation_by_quarter_turn_shifts_views():
    """Rotating the image by 90 degrees rotates the sinogram by nv/4 views."""
    g = synth.tiny_geometry(n=12, nv=16, nb=20, px=1.0)
    t = oracle.table(g)
    x = synth.random_image(g.n, 5)
    n = g.n
    xr = np.empty_like(x)
    for i in range(n):
        for j in range(n):
            xr[j, n - 1 - i] = x[i, j]     # point (x, y) -> (-y, x)
    y = oracle.project(t, x)
    yr = oracle.project(t, xr)
    np.testing.assert_allclose(np.roll(yr, -g.nv // 4, axis=0), y, rtol=1e-12, atol=1e-14)


def test_mirror_flip_reverses_views_and_bins():
    """Mirroring the image in y (row i -> n - 1 - i) mirrors the source orbit
    (view angle t -> -t) and the detector axis (u -> -u): ray (v, b) of the
    flipped image is ray ((nv - v) mod nv, nb - 1 - b) of the original.  The
    image side is odd so that no ray runs along a grid line (there the
    midpoint rule gives the +side pixel, which mirroring does not keep)."""
    g = synth.tiny_geometry(n=11, nv=18, nb=21, px=1.0)
    t = oracle.table(g)
    x = synth.random_image(g.n, 6)
    y = oracle.project(t, x)
    yf = oracle.project(t, x[::-1, :].copy())
    v = np.arange(g.nv)
    np.testing.assert_allclose(yf, y[(g.nv - v) % g.nv][:, ::-1], rtol=1e-12, atol=1e-14)


def test_adjoint_identity():
    """<A x, y> = <x, A^T y> to 1e-12, and A^T equals the pixel-clip transpose."""
    g = GEOMS[1]
    t = oracle.table(g)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((g.n, g.n))
    y = rng.standard_normal((g.nv, g.nb))
    lhs = float((oracle.project(t, x) * y).sum())
    rhs = float((x * oracle.backproject(t, y)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    B = indep.clip_matrix(g)
    np.testing.assert_allclose(oracle.backproject(t, y).reshape(-1), B.T @ y.reshape(-1),
                               rtol=1e-11, atol=1e-12)


def test_ellipse_line_integrals():
    """A of a finely rasterised ellipse phantom matches analytic line integrals to O(px)."""
    g = synth.small_geometry()
    t = oracle.table(g)
    ph = synth.random_ellipse_phantom(g, seed=11)
    u = synth.rasterize(ph, g.n, g.px, supersample=16)
    for e in (synth.HIGH, synth.LOW):
        y = oracle.project(t, synth.attenuation(u, e))
        ref = synth.analytic_sinogram(ph, g, e)
        rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert rel < 2e-2, rel
        # a coarser rasterisation is further from the continuous integrals
    uc = synth.rasterize(ph, g.n // 2, 2 * g.px, supersample=16)
    gc = synth.Geometry(n=g.n // 2, px=2 * g.px, nv=g.nv, nb=g.nb, pitch=g.pitch, sod=g.sod, sdd=g.sdd)
    yc = oracle.project(oracle.table(gc), synth.attenuation(uc, 0))
    ref = synth.analytic_sinogram(ph, g, 0)
    y = oracle.project(t, synth.attenuation(u, 0))
    assert np.linalg.norm(yc - ref) > np.linalg.norm(y - ref)


def test_small_geometry_has_no_grid_aligned_rays():
    """The small workload's rays never run along a pixel grid line."""
    g = synth.small_geometry()
    S, D = indep.rays_np(g)
    d = D - S
    assert np.all(np.abs(d[:, 0]) > 1e-9) and np.all(np.abs(d[:, 1]) > 1e-9)


def test_nnz_estimate_small():
    t = oracle.table(synth.small_geometry())
    assert 1.7e6 < t.nnz < 2.1e6
    assert t.idx.min() >= 0 and t.idx.max() < 128 * 128
    assert np.all(t.len > 0)


def test_one_element_per_ray_and_pixel():
    """Rays through grid corners (rational slopes) still give one element a_ij per pixel."""
    g = synth.tiny_geometry(n=64, nv=30, nb=96, px=0.5, sod=60.0, sdd=130.0, arc=math.pi)
    t = oracle.table(g)
    for r in range(g.nv * g.nb):
        idx = t.idx[t.rowptr[r]:t.rowptr[r + 1]]
        assert len(np.unique(idx)) == len(idx)
    sub = synth.tiny_geometry(n=16, nv=6, nb=24, px=0.5, sod=60.0, sdd=130.0, arc=math.pi)
    np.testing.assert_allclose(oracle.table(sub).dense(), indep.clip_matrix(sub), rtol=0, atol=1e-11)
