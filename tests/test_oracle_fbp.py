"""Pins of the oracle's fan-beam FBP (the analytic reconstruction the paper
uses in Sec. 2.4 and Sec. 3; textbook algorithm for an equally spaced flat
detector over 360 degrees) against exact line integrals of ellipses."""
import numpy as np

import oracle
import synth

MU = 0.02


def _geom():
    # 720 views, bins of 0.25 mm at the isocentre: sampling fine enough that
    # the discretisation error of the ramp filter stays well below 1 %
    return synth.tiny_geometry(n=64, nv=720, nb=256, px=1.0, pitch=0.5, sod=200.0, sdd=400.0)


def _grid(n):
    c = (np.arange(n) + 0.5) - n / 2
    return np.meshgrid(c, c)  # X (column), Y (row)


def _sino(g, phantom, w=MU):
    S, D = synth.ray_endpoints(g)
    return synth.ellipse_chords(phantom, S, D, np.full(len(phantom), w))


def test_uniform_disk_value():
    """A disk of attenuation mu is reconstructed as mu inside and 0 outside."""
    g = _geom()
    f = oracle.fbp(g, _sino(g, [synth.Ellipse(0.0, 0.0, 20.0, 20.0, 0.0, 1.0, 0.0)]))
    X, Y = _grid(g.n)
    r = np.hypot(X, Y)
    inside = f[r < 16]
    assert abs(inside.mean() - MU) < 1e-3 * MU
    assert np.abs(inside - MU).max() < 5e-3 * MU
    assert np.abs(f[(r > 24) & (r < 30)]).max() < 2e-2 * MU


def test_wide_fan_disk_value():
    """A wide fan (half-angle ~20 degrees at the FOV edge) needs the cosine
    pre-weight and the (SOD / L)^2 back-projection weight to get mu."""
    g = synth.tiny_geometry(n=64, nv=720, nb=256, px=1.0, pitch=0.5, sod=80.0, sdd=160.0)
    f = oracle.fbp(g, _sino(g, [synth.Ellipse(0.0, 0.0, 26.0, 26.0, 0.0, 1.0, 0.0)]))
    X, Y = _grid(g.n)
    r = np.hypot(X, Y)
    assert np.abs(f[r < 22] - MU).max() < 5e-3 * MU


def test_small_object_with_detector_offset():
    """A 2 mm disk stays sharp with the detector shifted by 4 mm: the offset
    enters the bin positions with the right sign."""
    g = synth.tiny_geometry(n=64, nv=720, nb=288, px=1.0, pitch=0.5, sod=200.0, sdd=400.0,
                            det_offset=4.0)
    f = oracle.fbp(g, _sino(g, [synth.Ellipse(10.5, 4.5, 2.0, 2.0, 0.0, 1.0, 0.0)]))
    assert abs(f[int(4.5 + 32), int(10.5 + 32)] - MU) < 0.05 * MU


def test_off_centre_ellipse_position_and_orientation():
    """An ellipse away from the centre lands where it is (row = y, column = x):
    a flipped or rotated back-projection moves its centroid."""
    g = _geom()
    e = [synth.Ellipse(15.0, -8.0, 5.0, 3.0, 0.3, 1.0, 0.0)]
    f = oracle.fbp(g, _sino(g, e))
    X, Y = _grid(g.n)
    u = synth.rasterize(e, g.n, g.px, 8)[0] * MU
    cx, cy = (f * X).sum() / f.sum(), (f * Y).sum() / f.sum()
    assert abs(cx - 15.0) < 0.2 and abs(cy + 8.0) < 0.2
    # the pixel at the ellipse centre is mu; its mirror images are empty
    at = lambda x, y: f[int(y + g.n / 2), int(x + g.n / 2)]
    assert abs(at(15.0, -8.0) - MU) < 0.05 * MU
    for x, y in ((-15.0, -8.0), (15.0, 8.0), (-8.0, 15.0)):
        assert abs(at(x, y)) < 0.05 * MU
    roi = np.hypot(X - 15.0, Y + 8.0) < 10
    assert abs(f[roi].sum() - u.sum()) < 1e-2 * u.sum()   # edges blur, the mass agrees


def test_detector_offset_and_start_angle():
    """A shifted detector and a rotated start angle reconstruct the same object
    in the same place (a sign error in either moves or rotates it)."""
    g2 = synth.tiny_geometry(n=64, nv=720, nb=264, px=1.0, pitch=0.5, sod=200.0, sdd=400.0,
                             start=0.7, det_offset=1.5)
    e = [synth.Ellipse(-6.0, 9.0, 7.0, 4.0, -0.5, 1.0, 0.0)]
    X, Y = _grid(g2.n)
    f = oracle.fbp(g2, _sino(g2, e))
    core = synth.rasterize([synth.Ellipse(-6.0, 9.0, 5.0, 2.5, -0.5, 1.0, 0.0)], g2.n, g2.px, 4)[0] > 0.999
    assert np.abs(f[core] - MU).max() < 5e-3 * MU
    roi = np.hypot(X + 6.0, Y - 9.0) < 12
    w = f * roi
    assert abs((w * X).sum() / w.sum() + 6.0) < 0.1 and abs((w * Y).sum() / w.sum() - 9.0) < 0.1


def test_ramp_filter_kernel():
    """The filter of one bin impulse is ds * h: h(0) = 1/(4 ds^2), zero at even
    offsets, -1/(pi^2 k^2 ds^2) at odd ones (times the cosine weight)."""
    g = synth.tiny_geometry(n=8, nv=1, nb=41, px=1.0, pitch=0.5, sod=1e7, sdd=2e7)
    p = np.zeros((1, 41))
    p[0, 20] = 1.0
    qf = oracle.fbp_filter(g, p)[0]
    ds = 0.25
    k = np.arange(41) - 20
    want = np.where(k == 0, 1 / (4 * ds * ds), np.where(k % 2 == 0, 0.0, -1 / (np.pi ** 2 * k ** 2 * ds * ds))) * ds
    np.testing.assert_allclose(qf, want, rtol=1e-9, atol=1e-12)


def test_linear_in_the_data():
    g = _geom()
    rng = np.random.default_rng(0)
    p = rng.random((g.nv, g.nb))
    np.testing.assert_array_equal(oracle.fbp(g, 2.0 * p), 2.0 * oracle.fbp(g, p))
