"""Independent numpy restatements used to pin the oracle.

Nothing here calls the oracle or the CUDA library.  Each routine computes a
quantity from its definition by a different route than the oracle does:

* ``clip_matrix``: the system matrix of Eq. (1) by clipping every ray
  against every pixel square (a pixel-driven Liang-Barsky clip, half-open
  squares), instead of Siddon's merged crossing list.
* ``box_chord``: length of a ray inside the whole image box.
* ``grad_np`` / ``tv_np``: Eq. (2) with numpy slicing.
* ``aug_lagrangian``: Eq. (6) for one channel.
* ``pls_matrix``: the Hessian of the PLS objective Eq. (13)-(14), assembled
  pair by pair from the definition of R(u).
* ``chambolle_pock``: an independent primal-dual solver of Eq. (4).
* ``tv_joint_np`` / ``aug_lagrangian_joint`` / ``chambolle_pock_joint``: the
  same for the channel-coupled TV (the norm taken over both channels'
  gradients at every pixel).
"""
from __future__ import annotations

import math

import numpy as np


def rays_np(geom):
    """Source and bin points [M, 2] (same geometry statement as the paper's Fig. 1)."""
    v = np.arange(geom.nv, dtype=np.float64)
    th = geom.start + v * (geom.arc / geom.nv)
    c, s = np.cos(th), np.sin(th)
    u = (np.arange(geom.nb) - 0.5 * (geom.nb - 1)) * geom.pitch + geom.det_offset
    S = np.stack([geom.sod * c, geom.sod * s], -1)
    Cd = np.stack([(geom.sod - geom.sdd) * c, (geom.sod - geom.sdd) * s], -1)
    D = Cd[:, None, :] + u[None, :, None] * np.stack([-s, c], -1)[:, None, :]
    S = np.broadcast_to(S[:, None, :], D.shape)
    return S.reshape(-1, 2), D.reshape(-1, 2)


def _clip_interval(s0, d0, lo, hi):
    """Parameter interval of s0 + a d0 inside [lo, hi) (arrays broadcast)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (lo - s0) / d0
        t1 = (hi - s0) / d0
    a_lo = np.where(d0 != 0, np.minimum(t0, t1), np.where((s0 >= lo) & (s0 < hi), -np.inf, np.inf))
    a_hi = np.where(d0 != 0, np.maximum(t0, t1), np.where((s0 >= lo) & (s0 < hi), np.inf, -np.inf))
    return a_lo, a_hi


def clip_matrix(geom) -> np.ndarray:
    """Dense A[M, N]: length of each ray inside each pixel square (mm)."""
    S, D = rays_np(geom)
    d = D - S
    L = np.hypot(d[:, 0], d[:, 1])
    n, px = geom.n, geom.px
    lo = -0.5 * n * px
    edges = lo + np.arange(n) * px
    ax_lo, ax_hi = _clip_interval(S[:, 0:1], d[:, 0:1], edges[None, :], edges[None, :] + px)  # [M, n] cols
    ay_lo, ay_hi = _clip_interval(S[:, 1:2], d[:, 1:2], edges[None, :], edges[None, :] + px)  # [M, n] rows
    a_lo = np.maximum(np.maximum(ay_lo[:, :, None], ax_lo[:, None, :]), 0.0)
    a_hi = np.minimum(np.minimum(ay_hi[:, :, None], ax_hi[:, None, :]), 1.0)
    A = np.clip(a_hi - a_lo, 0.0, None) * L[:, None, None]
    return A.reshape(S.shape[0], n * n)


def box_chord(geom) -> np.ndarray:
    """Length of each ray inside the image box [M]."""
    S, D = rays_np(geom)
    d = D - S
    L = np.hypot(d[:, 0], d[:, 1])
    lo = -0.5 * geom.n * geom.px
    hi = lo + geom.n * geom.px
    ax_lo, ax_hi = _clip_interval(S[:, 0], d[:, 0], lo, hi)
    ay_lo, ay_hi = _clip_interval(S[:, 1], d[:, 1], lo, hi)
    a_lo = np.maximum(np.maximum(ax_lo, ay_lo), 0.0)
    a_hi = np.minimum(np.minimum(ax_hi, ay_hi), 1.0)
    return np.clip(a_hi - a_lo, 0.0, None) * L


def grad_np(x: np.ndarray) -> np.ndarray:
    """Eq. (2) backward differences, zero on the first row / column."""
    d = np.zeros((2,) + x.shape)
    d[0, 1:, :] = x[1:, :] - x[:-1, :]
    d[1, :, 1:] = x[:, 1:] - x[:, :-1]
    return d


def tv_np(x: np.ndarray) -> float:
    d = grad_np(x)
    return float(np.sqrt(d[0] ** 2 + d[1] ** 2).sum())


def aug_lagrangian(A, g, f, z, lam, mu, rho) -> float:
    """Eq. (6) for one channel: |z| - <lam, grad f - z> + rho/2 |grad f - z|^2 + mu/2 |A f - g|^2."""
    df = grad_np(f)
    zn = float(np.sqrt(z[0] ** 2 + z[1] ** 2).sum())
    e = df - z
    r = A @ f.reshape(-1) - g.reshape(-1)
    return zn - float((lam * e).sum()) + 0.5 * rho * float((e * e).sum()) + 0.5 * mu * float(r @ r)


def tv_ls_objective(A, g, f, mu) -> float:
    """Eq. (4) for one channel."""
    r = A @ f.reshape(-1) - g.reshape(-1)
    return tv_np(f) + 0.5 * mu * float(r @ r)


def chambolle_pock(A, g, n, mu, iters=200000, f0=None):
    """Primal-dual (Chambolle-Pock 2011) solver of min |grad f|_TV + mu/2 |A f - g|^2.

    K = [grad; A] with dual variables p (TV, projected on the unit disk per
    pixel) and q (data term, prox of the conjugate of mu/2|. - g|^2).
    """
    N = n * n
    # operator norm estimate by power iteration
    v = np.random.default_rng(0).random(N)
    for _ in range(200):
        w = grad_np(v.reshape(n, n))
        u = A @ v
        v = _gradT_np(w) .reshape(-1) + A.T @ u
        v /= np.linalg.norm(v)
    Lk = math.sqrt(np.linalg.norm(_gradT_np(grad_np(v.reshape(n, n))).reshape(-1) + A.T @ (A @ v)))
    tau = sigma = 0.99 / Lk
    f = np.zeros(N) if f0 is None else f0.reshape(-1).copy()
    fb = f.copy()
    p = np.zeros((2, n, n))
    q = np.zeros(A.shape[0])
    gg = g.reshape(-1)
    for _ in range(iters):
        p = p + sigma * grad_np(fb.reshape(n, n))
        nrm = np.maximum(1.0, np.sqrt(p[0] ** 2 + p[1] ** 2))
        p = p / nrm
        q = (q + sigma * (A @ fb - gg)) / (1.0 + sigma / mu)
        f_new = f - tau * (_gradT_np(p).reshape(-1) + A.T @ q)
        fb = 2.0 * f_new - f
        f = f_new
    return f.reshape(n, n)


def _gradT_np(d: np.ndarray) -> np.ndarray:
    out = np.zeros(d.shape[1:])
    out[1:, :] += d[0, 1:, :]
    out[:-1, :] -= d[0, 1:, :]
    out[:, 1:] += d[1, :, 1:]
    out[:, :-1] -= d[1, :, 1:]
    return out


def pls_matrix(mask: np.ndarray, gamma: float, eps: float) -> np.ndarray:
    """Half the Hessian of |u - d|^2 + gamma R(u), R of Eq. (14), one material.

    R(u) = 1/2 sum_i sum_{k in N_i} e_ik (u_i - u_k)^2 is assembled from its
    definition: every ordered (i, k) pair adds e_ik (u_i - u_k)^2 / 2, whose
    Hessian puts +e_ik at (i,i), (k,k) and -e_ik at (i,k), (k,i).
    """
    n = mask.shape[0]
    N = n * n
    H = 2.0 * np.eye(N)        # Hessian of |u - d|^2
    for i in range(n):
        for j in range(n):
            p = i * n + j
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n:
                    k = ii * n + jj
                    e = eps if (mask[i, j] or mask[ii, jj]) else 1.0
                    w = gamma * 0.5 * e * 2.0      # gamma * (1/2) * Hessian of e (u_i-u_k)^2
                    H[p, p] += w
                    H[k, k] += w
                    H[p, k] -= w
                    H[k, p] -= w
    return 0.5 * H


def pls_objective(u: np.ndarray, d: np.ndarray, mask: np.ndarray, gamma: float, eps: float) -> float:
    """Eq. (13) for one material with R of Eq. (14)."""
    n = u.shape[0]
    r = 0.0
    for i in range(n):
        for j in range(n):
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n:
                    e = eps if (mask[i, j] or mask[ii, jj]) else 1.0
                    r += 0.5 * e * (u[i, j] - u[ii, jj]) ** 2
    return float(((u - d) ** 2).sum() + gamma * r)


def tv_joint_np(f: np.ndarray) -> float:
    """sum_p |(grad f_0, grad f_1)_p|_2 for f = [2][n][n]."""
    d0, d1 = grad_np(f[0]), grad_np(f[1])
    return float(np.sqrt(d0[0] ** 2 + d0[1] ** 2 + d1[0] ** 2 + d1[1] ** 2).sum())


def tv_ls_objective_joint(A, g, f, mu) -> float:
    """Joint form of Eq. (4): tv_joint + mu/2 sum_c |A f_c - g_c|^2, g = [2][M]."""
    s = 0.0
    for c in range(2):
        r = A @ f[c].reshape(-1) - g[c].reshape(-1)
        s += float(r @ r)
    return tv_joint_np(f) + 0.5 * mu * s


def aug_lagrangian_joint(A, g, f, z, lam, mu, rho) -> float:
    """Eq. (6) for the stacked f = [2][n][n]; z, lam = [2][2][n][n]; the
    z-norm is the per-pixel 4-norm."""
    zn = float(np.sqrt((z ** 2).sum(axis=(0, 1))).sum())
    val = zn
    for c in range(2):
        e = grad_np(f[c]) - z[c]
        r = A @ f[c].reshape(-1) - g[c].reshape(-1)
        val += -float((lam[c] * e).sum()) + 0.5 * rho * float((e * e).sum()) + 0.5 * mu * float(r @ r)
    return val


def chambolle_pock_joint(A, g, n, mu, iters=20000):
    """Chambolle-Pock for the joint problem: the dual variable of the TV term
    is projected per pixel onto the unit ball of R^4 (both channels)."""
    N = n * n
    v = np.random.default_rng(0).random(N)
    for _ in range(200):
        v = _gradT_np(grad_np(v.reshape(n, n))).reshape(-1) + A.T @ (A @ v)
        v /= np.linalg.norm(v)
    Lk = math.sqrt(np.linalg.norm(_gradT_np(grad_np(v.reshape(n, n))).reshape(-1) + A.T @ (A @ v)))
    tau = sigma = 0.99 / Lk
    f = np.zeros((2, N))
    fb = f.copy()
    p = np.zeros((2, 2, n, n))
    q = np.zeros((2, A.shape[0]))
    gg = g.reshape(2, -1)
    for _ in range(iters):
        for c in range(2):
            p[c] = p[c] + sigma * grad_np(fb[c].reshape(n, n))
        nrm = np.maximum(1.0, np.sqrt((p ** 2).sum(axis=(0, 1))))
        p = p / nrm
        f_new = np.empty_like(f)
        for c in range(2):
            q[c] = (q[c] + sigma * (A @ fb[c] - gg[c])) / (1.0 + sigma / mu)
            f_new[c] = f[c] - tau * (_gradT_np(p[c]).reshape(-1) + A.T @ q[c])
        fb = 2.0 * f_new - f
        f = f_new
    return f.reshape(2, n, n)


# ---------------------------------------------------------------------------
# Cone-beam (3-D) counterparts
# ---------------------------------------------------------------------------

def rays3_np(geom):
    """Source and detector-cell points [M, 3], ray order (v, r, c) (Fig. 1 with a 2-D detector)."""
    v = np.arange(geom.nv, dtype=np.float64)
    th = geom.start + v * (geom.arc / geom.nv)
    c, s = np.cos(th), np.sin(th)
    u = (np.arange(geom.nc) - 0.5 * (geom.nc - 1)) * geom.pu + geom.off_u
    z = (np.arange(geom.nr) - 0.5 * (geom.nr - 1)) * geom.pv + geom.off_v
    S = np.stack([geom.sod * c, geom.sod * s, np.zeros_like(c)], -1)                  # [nv, 3]
    Cd = np.stack([(geom.sod - geom.sdd) * c, (geom.sod - geom.sdd) * s, np.zeros_like(c)], -1)
    eu = np.stack([-s, c, np.zeros_like(c)], -1)
    D = (Cd[:, None, None, :] + u[None, None, :, None] * eu[:, None, None, :]
         + z[None, :, None, None] * np.array([0.0, 0.0, 1.0])[None, None, None, :])    # [nv, nr, nc, 3]
    S = np.broadcast_to(S[:, None, None, :], D.shape)
    return S.reshape(-1, 3), D.reshape(-1, 3)


def clip_matrix3(geom) -> np.ndarray:
    """Dense A[M, N]: length of each ray inside each voxel box (mm), by slab clipping."""
    S, D = rays3_np(geom)
    d = D - S
    L = np.sqrt((d * d).sum(-1))
    n, nz = geom.n, geom.nz
    ex = -0.5 * n * geom.px + np.arange(n) * geom.px
    ez = -0.5 * nz * geom.pz + np.arange(nz) * geom.pz
    ax_lo, ax_hi = _clip_interval(S[:, 0:1], d[:, 0:1], ex[None, :], ex[None, :] + geom.px)   # [M, n] cols
    ay_lo, ay_hi = _clip_interval(S[:, 1:2], d[:, 1:2], ex[None, :], ex[None, :] + geom.px)   # [M, n] rows
    az_lo, az_hi = _clip_interval(S[:, 2:3], d[:, 2:3], ez[None, :], ez[None, :] + geom.pz)   # [M, nz]
    a_lo = np.maximum(np.maximum(np.maximum(az_lo[:, :, None, None], ay_lo[:, None, :, None]),
                                 ax_lo[:, None, None, :]), 0.0)
    a_hi = np.minimum(np.minimum(np.minimum(az_hi[:, :, None, None], ay_hi[:, None, :, None]),
                                 ax_hi[:, None, None, :]), 1.0)
    A = np.clip(a_hi - a_lo, 0.0, None) * L[:, None, None, None]
    return A.reshape(S.shape[0], nz * n * n)


def box_chord3(geom) -> np.ndarray:
    """Length of each ray inside the volume box [M]."""
    S, D = rays3_np(geom)
    d = D - S
    L = np.sqrt((d * d).sum(-1))
    lo = np.array([-0.5 * geom.n * geom.px] * 2 + [-0.5 * geom.nz * geom.pz])
    hi = -lo
    a_lo, a_hi = np.zeros(len(S)), np.ones(len(S))
    for a in range(3):
        l, h = _clip_interval(S[:, a], d[:, a], lo[a], hi[a])
        a_lo = np.maximum(a_lo, l)
        a_hi = np.minimum(a_hi, h)
    return np.clip(a_hi - a_lo, 0.0, None) * L


def pls_matrix3(mask: np.ndarray, gamma: float, eps: float) -> np.ndarray:
    """Half the Hessian of |u - d|^2 + gamma R(u) with R of Eq. (14) over the 6
    neighbours of each voxel, assembled pair by pair (as pls_matrix)."""
    nz, n, _ = mask.shape
    N = nz * n * n
    H = 2.0 * np.eye(N)
    for k in range(nz):
        for i in range(n):
            for j in range(n):
                p = (k * n + i) * n + j
                for dk, di, dj in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
                    kk, ii, jj = k + dk, i + di, j + dj
                    if 0 <= kk < nz and 0 <= ii < n and 0 <= jj < n:
                        q = (kk * n + ii) * n + jj
                        e = eps if (mask[k, i, j] or mask[kk, ii, jj]) else 1.0
                        w = gamma * e
                        H[p, p] += w
                        H[q, q] += w
                        H[p, q] -= w
                        H[q, p] -= w
    return 0.5 * H
