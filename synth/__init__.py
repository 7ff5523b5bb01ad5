"""Seeded synthetic inputs for the dual-energy CT hot path.

This module only *describes* workloads and draws random numbers; it holds
none of the reconstruction method's arithmetic (no Siddon walk, no ADM, no
PLS).  Both the FP64 oracle and the CUDA library read what it produces.

What it makes
-------------
* ``Geometry``: the fan-beam slice geometry (Sec. 2.1, Fig. 1 of the paper:
  source on a circle of radius SOD, flat 1-D detector at SDD).
* Phantoms: sums of ellipses, each carrying an additive amount of two basis
  materials (water-like, bone-like), i.e. the material maps ``u`` of Eq. (11).
  Sums (not clipped overlays) keep every line integral analytic.
* ``analytic_sinogram``: exact line integrals of the continuous ellipse
  phantom along each source-to-bin ray, per energy, with the attenuation
  ``mu_E = eta_1E * u_1 + eta_2E * u_2`` of Eq. (11)-(12).  This is the
  physics of the measurement, not the discrete model ``A`` of Eq. (1): the
  reconstruction therefore sees the usual continuous-to-discrete mismatch,
  as with real data.
* ``poisson_log``: Poisson counts at ``I0`` photons/bin and the log
  transform back to line integrals (the paper uses measured data; this is
  the stand-in).
* ``rasterize``: supersampled area-fraction images of a phantom (for
  ground-truth images in tests).

Rays
----
The generator states the ray geometry for its own use: view ``v`` has angle
``theta_v = start + v * (arc / nv)``, the source sits at
``SOD * (cos theta, sin theta)``, the detector centre at
``(SOD - SDD) * (cos theta, sin theta)``, the detector axis is
``(-sin theta, cos theta)`` and bin ``b`` is centred at
``u_b = (b - (nb - 1) / 2) * pitch + det_offset``.  The image is ``n x n``
pixels of side ``px`` centred on the isocentre; row index = y, column = x.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

# Basis-material attenuation (1/mm) at (high, low) energy.  Material 1 is
# water-like, material 2 bone-like.  eta[m][e]: m = material, e = 0 high, 1 low.
ETA = np.array([[0.0184, 0.0227],
                [0.0342, 0.0573]], dtype=np.float64)

HIGH, LOW = 0, 1


@dataclasses.dataclass(frozen=True)
class Geometry:
    n: int                 # image is n x n pixels
    px: float              # pixel side, mm
    nv: int                # number of views
    nb: int                # detector bins
    pitch: float           # bin pitch, mm
    sod: float             # source to isocentre, mm
    sdd: float             # source to detector, mm
    start: float = 0.0     # angle of view 0, rad
    arc: float = 2.0 * math.pi
    det_offset: float = 0.0

    @property
    def n_pix(self) -> int:
        return self.n * self.n

    @property
    def n_rays(self) -> int:
        return self.nv * self.nb

    def fov_radius(self) -> float:
        """Radius of the disk seen by every view (mm)."""
        half = 0.5 * self.nb * self.pitch
        return half * self.sod / math.hypot(self.sdd, half)


def small_geometry() -> Geometry:
    """128^2 at 1 mm, 60 views over 360 deg, 192 bins x 1.2 mm, SOD 500, SDD 1000."""
    return Geometry(n=128, px=1.0, nv=60, nb=192, pitch=1.2, sod=500.0, sdd=1000.0)


def paper_geometry() -> Geometry:
    """512^2 at 0.5 mm, sparse 60 views over 360 deg, 736 bins (pitch 0.6 mm)."""
    return Geometry(n=512, px=0.5, nv=60, nb=736, pitch=0.6, sod=500.0, sdd=1000.0)


def stress_geometry() -> Geometry:
    """1024^2 at 0.25 mm, 360 views, 1472 bins x 0.3 mm."""
    return Geometry(n=1024, px=0.25, nv=360, nb=1472, pitch=0.3, sod=500.0, sdd=1000.0)


def batched_geometry(n: int, nv: int) -> Geometry:
    """Uneven-slice workload: n in {256..512} at 0.5 mm, nv views, bins scaled with n."""
    nb = 368 + int(round((n - 256) / 256.0 * 368))
    return Geometry(n=n, px=0.5, nv=nv, nb=nb, pitch=0.6, sod=500.0, sdd=1000.0)


def tiny_geometry(n: int = 8, nv: int = 12, nb: int = 12, px: float = 1.0,
                  pitch: float = None, sod: float = 40.0, sdd: float = 80.0,
                  start: float = 0.0, arc: float = 2.0 * math.pi,
                  det_offset: float = 0.0) -> Geometry:
    """Small geometry for oracle pins and quick parity cases."""
    if pitch is None:
        # cover the image diagonal on the detector with some margin
        pitch = 1.6 * n * px * (sdd / sod) / nb
    return Geometry(n=n, px=px, nv=nv, nb=nb, pitch=pitch, sod=sod, sdd=sdd,
                    start=start, arc=arc, det_offset=det_offset)


@dataclasses.dataclass(frozen=True)
class ConeGeometry:
    """Circular cone-beam geometry with a flat 2-D detector (Sec. 2.1, Fig. 1;
    Sec. 3): source orbit in the plane z = 0; detector cell (row r, column c)
    at u_c = (c - (nc - 1) / 2) pu + off_u, z_r = (r - (nr - 1) / 2) pv + off_v;
    an n x n x nz volume of px x px x pz voxels centred on the origin."""
    n: int
    nz: int
    px: float
    pz: float
    nv: int
    nr: int
    nc: int
    pu: float
    pv: float
    sod: float
    sdd: float
    start: float = 0.0
    arc: float = 2.0 * math.pi
    off_u: float = 0.0
    off_v: float = 0.0

    @property
    def n_vox(self) -> int:
        return self.n * self.n * self.nz

    @property
    def n_rays(self) -> int:
        return self.nv * self.nr * self.nc


def tiny_cone(n: int = 4, nz: int = 3, nv: int = 6, nr: int = 3, nc: int = 5, px: float = 1.0,
              pz: float = 1.0, sod: float = 20.0, sdd: float = 40.0, start: float = 0.2,
              off_u: float = 0.0, off_v: float = 0.0) -> ConeGeometry:
    """Small cone geometry for oracle pins and quick parity cases: the
    detector covers the volume's footprint with some margin."""
    mag = sdd / (sod - 0.75 * n * px)
    pu = 1.6 * n * px * mag / nc
    pv = 1.4 * nz * pz * mag / nr
    return ConeGeometry(n=n, nz=nz, px=px, pz=pz, nv=nv, nr=nr, nc=nc, pu=pu, pv=pv, sod=sod, sdd=sdd,
                        start=start, off_u=off_u, off_v=off_v)


def cone_geometry() -> ConeGeometry:
    """A cone-beam stand-in for the paper's scan (Sec. 3) at the benchmark's
    scale: 256^2 x 64 voxels of 0.5 mm, 60 views over 360 deg, 64 rows x 368
    columns of 0.6 mm at SOD 500 / SDD 1000."""
    return ConeGeometry(n=256, nz=64, px=0.5, pz=0.5, nv=60, nr=64, nc=368, pu=0.6, pv=0.6,
                        sod=500.0, sdd=1000.0)


# --------------------------------------------------------------------------
# Phantoms
# --------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Ellipse:
    cx: float
    cy: float
    a: float               # semi-axis along the rotated x axis, mm
    b: float               # semi-axis along the rotated y axis, mm
    phi: float             # rotation, rad
    water: float           # additive water-like fraction
    bone: float            # additive bone-like fraction


def random_ellipse_phantom(geom: Geometry, seed: int, k_range=(4, 10),
                           axis_range=(5.0, 40.0)) -> List[Ellipse]:
    """K random ellipses inside 0.95 x the FOV disk and the image box.

    Each ellipse adds a water or bone fraction in (0.2, 0.6]; the sums stay
    well inside [0, 2].
    """
    rng = np.random.default_rng(seed)
    lim = 0.95 * min(geom.fov_radius(), 0.5 * geom.n * geom.px)
    k = int(rng.integers(k_range[0], k_range[1] + 1))
    out = []
    amin, amax = axis_range
    amax = min(amax, 0.45 * lim)
    amin = min(amin, 0.5 * amax)
    for _ in range(k):
        a = float(rng.uniform(amin, amax))
        b = float(rng.uniform(amin, amax))
        r_max = lim - max(a, b)
        rr = float(rng.uniform(0.0, max(r_max, 0.0)))
        ang = float(rng.uniform(0.0, 2.0 * math.pi))
        phi = float(rng.uniform(0.0, math.pi))
        frac = float(rng.uniform(0.2, 0.6))
        if rng.random() < 0.6:
            out.append(Ellipse(rr * math.cos(ang), rr * math.sin(ang), a, b, phi, frac, 0.0))
        else:
            out.append(Ellipse(rr * math.cos(ang), rr * math.sin(ang), a, b, phi, 0.0, frac))
    return out


def head_phantom(geom: Geometry, seed: int) -> List[Ellipse]:
    """Head-like phantom: soft tissue, a 4-7 mm bone shell and 6-12 small inserts.

    Built additively so that all line integrals stay analytic:
    outer tissue ellipse (water 1); skull ellipse (bone +1, water -1);
    brain ellipse inside it (bone -1, water +1); inserts of 2-6 mm diameter
    inside the brain that swap some water for bone or add water.
    """
    rng = np.random.default_rng(seed)
    lim = 0.95 * min(geom.fov_radius(), 0.5 * geom.n * geom.px)
    scale = min(1.0, lim / 108.0)
    A, B = 90.0 * scale, 105.0 * scale
    tilt = float(rng.uniform(-0.1, 0.1))
    skull = float(rng.uniform(4.0, 7.0)) * scale
    scalp = 3.0 * scale
    out = [Ellipse(0.0, 0.0, A, B, tilt, 1.0, 0.0),
           Ellipse(0.0, 0.0, A - scalp, B - scalp, tilt, -1.0, 1.0),
           Ellipse(0.0, 0.0, A - scalp - skull, B - scalp - skull, tilt, 1.0, -1.0)]
    ai, bi = A - scalp - skull, B - scalp - skull
    n_ins = int(rng.integers(6, 13))
    for _ in range(n_ins):
        d = float(rng.uniform(2.0, 6.0)) * max(scale, 0.25)
        # a point well inside the brain ellipse
        rr = math.sqrt(float(rng.uniform(0.0, 1.0))) * 0.75
        ang = float(rng.uniform(0.0, 2.0 * math.pi))
        cx, cy = rr * ai * math.cos(ang), rr * bi * math.sin(ang)
        c, s = math.cos(tilt), math.sin(tilt)
        cx, cy = c * cx - s * cy, s * cx + c * cy
        kind = rng.integers(0, 3)
        if kind == 0:          # bone-like insert
            dw, db = -0.5, 0.5
        elif kind == 1:        # dense bone
            dw, db = -1.0, 1.0
        else:                  # denser soft tissue
            dw, db = 0.3, 0.0
        e = float(rng.uniform(0.6, 1.0))
        out.append(Ellipse(cx, cy, 0.5 * d, 0.5 * d * e, float(rng.uniform(0, math.pi)), dw, db))
    return out


def rasterize(phantom: Sequence[Ellipse], n: int, px: float, supersample: int = 8) -> np.ndarray:
    """Area-fraction material maps u[2][n][n] (float64), row = y, col = x."""
    s = supersample
    x0 = -0.5 * n * px
    sub = (np.arange(n * s) + 0.5) * (px / s) + x0
    X, Y = np.meshgrid(sub, sub)          # Y varies along rows
    u = np.zeros((2, n * s, n * s))
    for e in phantom:
        c, sn = math.cos(e.phi), math.sin(e.phi)
        xr = c * (X - e.cx) + sn * (Y - e.cy)
        yr = -sn * (X - e.cx) + c * (Y - e.cy)
        inside = (xr / e.a) ** 2 + (yr / e.b) ** 2 <= 1.0
        u[0][inside] += e.water
        u[1][inside] += e.bone
    return u.reshape(2, n, s, n, s).mean(axis=(2, 4))


def attenuation(u: np.ndarray, energy: int) -> np.ndarray:
    """mu_E = eta_1E u_1 + eta_2E u_2 (1/mm), Eq. (11)-(12)."""
    return ETA[0, energy] * u[0] + ETA[1, energy] * u[1]


# --------------------------------------------------------------------------
# Measurements
# --------------------------------------------------------------------------

def ray_endpoints(geom: Geometry) -> Tuple[np.ndarray, np.ndarray]:
    """Source and bin-centre points, arrays [nv, nb, 2] (float64)."""
    v = np.arange(geom.nv, dtype=np.float64)
    th = geom.start + v * (geom.arc / geom.nv)
    c, s = np.cos(th), np.sin(th)
    S = np.stack([geom.sod * c, geom.sod * s], axis=-1)[:, None, :]
    C = np.stack([(geom.sod - geom.sdd) * c, (geom.sod - geom.sdd) * s], axis=-1)
    u = (np.arange(geom.nb, dtype=np.float64) - 0.5 * (geom.nb - 1)) * geom.pitch + geom.det_offset
    ax = np.stack([-s, c], axis=-1)
    D = C[:, None, :] + u[None, :, None] * ax[:, None, :]
    S = np.broadcast_to(S, D.shape).copy()
    return S, D


def ellipse_chords(phantom: Sequence[Ellipse], S: np.ndarray, D: np.ndarray,
                   weights: np.ndarray) -> np.ndarray:
    """Sum over ellipses of weight * chord length of the line S->D (mm)."""
    d = D - S
    L = np.linalg.norm(d, axis=-1)
    dn = d / L[..., None]
    out = np.zeros(S.shape[:-1])
    for e, w in zip(phantom, weights):
        if w == 0.0:
            continue
        c, sn = math.cos(e.phi), math.sin(e.phi)
        px_ = S[..., 0] - e.cx
        py_ = S[..., 1] - e.cy
        ox = c * px_ + sn * py_
        oy = -sn * px_ + c * py_
        dx = c * dn[..., 0] + sn * dn[..., 1]
        dy = -sn * dn[..., 0] + c * dn[..., 1]
        qa = (dx / e.a) ** 2 + (dy / e.b) ** 2
        qb = 2.0 * (ox * dx / e.a ** 2 + oy * dy / e.b ** 2)
        qc = (ox / e.a) ** 2 + (oy / e.b) ** 2 - 1.0
        disc = qb * qb - 4.0 * qa * qc
        chord = np.where(disc > 0.0, np.sqrt(np.maximum(disc, 0.0)) / qa, 0.0)
        out += w * chord
    return out


def analytic_sinogram(phantom: Sequence[Ellipse], geom: Geometry, energy: int) -> np.ndarray:
    """Exact line integrals of mu_E along every ray, [nv][nb] float64."""
    S, D = ray_endpoints(geom)
    w = np.array([ETA[0, energy] * e.water + ETA[1, energy] * e.bone for e in phantom])
    return ellipse_chords(phantom, S, D, w)


def poisson_log(p: np.ndarray, i0: float, seed: int) -> np.ndarray:
    """Noisy line integrals -ln(max(N, 1) / I0), N ~ Poisson(I0 exp(-p))."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(i0 * np.exp(-p))
    return -np.log(np.maximum(counts, 1) / i0)


@dataclasses.dataclass
class Slice:
    """One dual-energy slice: geometry, phantom and measured data m_E."""
    geom: Geometry
    phantom: List[Ellipse]
    m: np.ndarray          # [2][nv][nb] float64, index 0 = high, 1 = low energy

    def truth(self, supersample: int = 8) -> Tuple[np.ndarray, np.ndarray]:
        u = rasterize(self.phantom, self.geom.n, self.geom.px, supersample)
        x = np.stack([attenuation(u, HIGH), attenuation(u, LOW)])
        return u, x


def make_slice(geom: Geometry, seed: int, kind: str = "ellipses", i0: float = 1e5,
               noise: bool = True) -> Slice:
    """Seeded dual-energy slice.  kind: 'ellipses' (random) or 'head'."""
    ph = head_phantom(geom, seed) if kind == "head" else random_ellipse_phantom(geom, seed)
    m = np.stack([analytic_sinogram(ph, geom, HIGH), analytic_sinogram(ph, geom, LOW)])
    if noise:
        m = np.stack([poisson_log(m[e], i0, seed * 7919 + 17 + e) for e in range(2)])
    return Slice(geom, ph, m)


def random_image(n: int, seed: int, scale: float = 0.02) -> np.ndarray:
    """Plain random test image (float64), for operator-level tests."""
    return scale * np.random.default_rng(seed).random((n, n))


def random_batched_shapes(count: int, seed: int) -> List[Tuple[int, int]]:
    """(n, nv) pairs of the uneven-slice workload: n in {256,...,512}, nv in [30, 180]."""
    rng = np.random.default_rng(seed)
    ns = [256, 320, 384, 448, 512]
    return [(int(ns[rng.integers(0, 5)]), int(rng.integers(30, 181))) for _ in range(count)]


# ---------------------------------------------------------------------------
# Initial weights of the warm-start network (the learned part of the
# workload; not in the paper).  Random numbers only: the network itself is
# defined by the CUDA library and by the oracle, each in its own code.
# ---------------------------------------------------------------------------

# (input, output) channels of the ten 3x3 convolutions, in parameter order;
# the 1x1 head (32 weights + 1 bias) follows them.
CNN_LAYERS = [(1, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (192, 64), (64, 64),
              (96, 32), (32, 32)]


def cnn_num_params() -> int:
    return sum(co * ci * 9 + co for ci, co in CNN_LAYERS) + 33


def cnn_init(seed: int) -> np.ndarray:
    """He-normal 3x3 weights (std sqrt(2 / (9 Cin))), zero biases and a zero
    head, so that the untrained network x + s * net(x / s) is the identity.
    Flat float64 vector in the layout of dect_cnn_set_params."""
    rng = np.random.default_rng(seed)
    parts = []
    for cin, cout in CNN_LAYERS:
        parts.append(rng.standard_normal(cout * cin * 9) * np.sqrt(2.0 / (cin * 9)))
        parts.append(np.zeros(cout))
    parts.append(np.zeros(33))
    return np.concatenate(parts)
