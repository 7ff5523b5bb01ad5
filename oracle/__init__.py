"""FP64 CPU oracle for the dual-energy CT hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (``paper_1607_01650_gb300``)
never does, and this package never imports the product: the two share no
code.  The arithmetic lives in ``dect_oracle.c`` (plain C, FP64, compiled
with ``-ffp-contract=off``); this module only marshals numpy arrays.

Every function cites the passage of the paper it restates; the readings
R1-R16 used where the paper is silent or garbled are listed in the C file's
header.  Parity status: every function here is pinned by a ``-m "not gpu"``
test against closed forms, brute force or an independent solver, except the
choice of parameter values (mu, rho, xi, beta, tau, eps, gamma), which the
paper does not fix.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dect_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (seconds).  Returns the library path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Geom(C.Structure):
    _fields_ = [("n", C.c_int), ("px", C.c_double), ("nv", C.c_int), ("nb", C.c_int),
                ("pitch", C.c_double), ("sod", C.c_double), ("sdd", C.c_double),
                ("start", C.c_double), ("arc", C.c_double), ("det_offset", C.c_double)]


class _Geom3(C.Structure):
    _fields_ = [("n", C.c_int), ("nz", C.c_int), ("px", C.c_double), ("pz", C.c_double),
                ("nv", C.c_int), ("nr", C.c_int), ("nc", C.c_int), ("pu", C.c_double), ("pv", C.c_double),
                ("sod", C.c_double), ("sdd", C.c_double), ("start", C.c_double), ("arc", C.c_double),
                ("off_u", C.c_double), ("off_v", C.c_double)]


class _AdmParams(C.Structure):
    _fields_ = [("mu", C.c_double), ("rho", C.c_double), ("xi", C.c_double),
                ("step_rule", C.c_int), ("max_iter", C.c_int), ("tol", C.c_double),
                ("nonneg", C.c_int)]


class _AdmState(C.Structure):
    _fields_ = [("f", C.POINTER(C.c_double)), ("z", C.POINTER(C.c_double)),
                ("lam", C.POINTER(C.c_double)), ("alpha_prev", C.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        i32 = C.POINTER(C.c_int32)
        i64 = C.POINTER(C.c_int64)
        u8 = C.POINTER(C.c_uint8)
        G = C.POINTER(_Geom)
        sig = {
            "orc_ray": (None, [G, C.c_int, C.c_int, d, d]),
            "orc_siddon_ray": (C.c_int, [G, C.c_int, C.c_int, i32, d, C.c_int]),
            "orc_table_nnz": (C.c_int64, [G]),
            "orc_table_build": (None, [G, i64, i32, d]),
            "orc_project": (None, [C.c_int64, i64, i32, d, d, d]),
            "orc_backproject": (None, [C.c_int64, C.c_int64, i64, i32, d, d, d]),
            "orc_grad": (None, [C.c_int, d, d]),
            "orc_grad_t": (None, [C.c_int, d, d]),
            "orc_tv": (C.c_double, [C.c_int, d]),
            "orc_shrink": (None, [C.c_int64, d, C.c_double, d]),
            "orc_adm_iterate": (C.c_double, [C.c_int, C.c_int64, i64, i32, d, d,
                                             C.POINTER(_AdmParams), C.POINTER(_AdmState), d, d]),
            "orc_objective": (C.c_double, [C.c_int, C.c_int64, i64, i32, d, d, C.c_double, d]),
            "orc_adm_run": (C.c_int, [C.c_int, C.c_int64, i64, i32, d, d,
                                      C.POINTER(_AdmParams), d, d, d]),
            "orc_shrink4": (None, [C.c_int64, d, d, C.c_double, d, d]),
            "orc_fbp_filter": (None, [G, d, d]),
            "orc_fbp": (None, [G, d, d]),
            "orc_tv_joint": (C.c_double, [C.c_int, d]),
            "orc_objective_joint": (C.c_double, [C.c_int, C.c_int64, i64, i32, d, d, C.c_double, d]),
            "orc_adm_joint_iterate": (C.c_double, [C.c_int, C.c_int64, i64, i32, d, d,
                                                   C.POINTER(_AdmParams), C.POINTER(_AdmState), d, d]),
            "orc_adm_joint_run": (C.c_int, [C.c_int, C.c_int64, i64, i32, d, d,
                                            C.POINTER(_AdmParams), d, d, d]),
            "orc_direct_decompose": (None, [C.c_int64, d, d, d, d, d]),
            "orc_prewitt": (None, [C.c_int, d, d]),
            "orc_edge_mask": (None, [C.c_int, d, d, C.c_double, u8]),
            "orc_pls_apply": (None, [C.c_int, u8, C.c_double, C.c_double, d, d]),
            "orc_pls_diag": (None, [C.c_int, u8, C.c_double, C.c_double, d]),
            "orc_pls_pcg": (C.c_int, [C.c_int, u8, C.c_double, C.c_double, d, d,
                                      C.c_int, C.c_double, d]),
            "orc3_ray": (None, [C.POINTER(_Geom3), C.c_int, C.c_int, C.c_int, d, d]),
            "orc3_siddon_ray": (C.c_int, [C.POINTER(_Geom3), C.c_int, C.c_int, C.c_int, i32, d, C.c_int]),
            "orc3_table_nnz": (C.c_int64, [C.POINTER(_Geom3)]),
            "orc3_table_build": (None, [C.POINTER(_Geom3), i64, i32, d]),
            "orc3_prewitt": (None, [C.c_int, C.c_int, d, d]),
            "orc3_edge_mask": (None, [C.c_int, C.c_int, d, d, C.c_double, u8]),
            "orc3_pls_apply": (None, [C.c_int, C.c_int, u8, C.c_double, C.c_double, d, d]),
            "orc3_pls_diag": (None, [C.c_int, C.c_int, u8, C.c_double, C.c_double, d]),
            "orc3_pls_pcg": (C.c_int, [C.c_int, C.c_int, u8, C.c_double, C.c_double, d, d,
                                       C.c_int, C.c_double, d]),
            "orc_cnn_num_params": (C.c_int64, []),
            "orc_cnn_run": (None, [d, C.c_double, d, C.c_int, C.c_int, d, d, d, d]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _geom(g) -> _Geom:
    return _Geom(g.n, g.px, g.nv, g.nb, g.pitch, g.sod, g.sdd, g.start, g.arc, g.det_offset)


# ---------------------------------------------------------------------------
# Sec. 2.1: geometry and the Siddon system matrix A of Eq. (1)
# ---------------------------------------------------------------------------

def ray(geom, v: int, b: int) -> Tuple[np.ndarray, np.ndarray]:
    """Source point and bin-centre point of ray (v, b)."""
    S = np.zeros(2)
    D = np.zeros(2)
    _load().orc_ray(C.byref(_geom(geom)), v, b, _d(S), _d(D))
    return S, D


def siddon_ray(geom, v: int, b: int) -> Tuple[np.ndarray, np.ndarray]:
    """(pixel indices, lengths in mm) of ray (v, b), Siddon's method (ref. [42])."""
    cap = 4 * geom.n + 8
    idx = np.zeros(cap, np.int32)
    ln = np.zeros(cap)
    c = _load().orc_siddon_ray(C.byref(_geom(geom)), v, b,
                               idx.ctypes.data_as(C.POINTER(C.c_int32)), _d(ln), cap)
    return idx[:c].copy(), ln[:c].copy()


@dataclasses.dataclass
class Table:
    """Ray-major table of A: row r = v * nb + b."""
    geom: object
    rowptr: np.ndarray   # int64 [M + 1]
    idx: np.ndarray      # int32 [nnz]
    len: np.ndarray      # float64 [nnz]

    @property
    def m(self) -> int:
        return self.geom.nv * self.geom.nb

    @property
    def npix(self) -> int:
        return self.geom.n * self.geom.n

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def _args(self):
        return (C.c_int64(self.m), self.rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                self.idx.ctypes.data_as(C.POINTER(C.c_int32)), _d(self.len))

    def dense(self) -> np.ndarray:
        A = np.zeros((self.m, self.npix))
        for r in range(self.m):
            s, e = self.rowptr[r], self.rowptr[r + 1]
            np.add.at(A[r], self.idx[s:e], self.len[s:e])
        return A


def table(geom) -> Table:
    """Build the Siddon table of the whole geometry."""
    lib = _load()
    g = _geom(geom)
    nnz = lib.orc_table_nnz(C.byref(g))
    M = geom.nv * geom.nb
    rowptr = np.zeros(M + 1, np.int64)
    idx = np.zeros(max(nnz, 1), np.int32)
    ln = np.zeros(max(nnz, 1))
    lib.orc_table_build(C.byref(g), rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                        idx.ctypes.data_as(C.POINTER(C.c_int32)), _d(ln))
    return Table(geom, rowptr, idx[:nnz], ln[:nnz])


def project(t: Table, x) -> np.ndarray:
    """y = A x, Eq. (1).  x: [n][n] -> y: [nv][nb]."""
    x = _f64(x).reshape(-1)
    y = np.zeros(t.m)
    _load().orc_project(*t._args(), _d(x), _d(y))
    return y.reshape(t.geom.nv, t.geom.nb)


def backproject(t: Table, y) -> np.ndarray:
    """x = A^T y (the transpose used by G_f of Eq. (9)).  y: [nv][nb] -> [n][n]."""
    y = _f64(y).reshape(-1)
    x = np.zeros(t.npix)
    m, rp, ix, ln = t._args()
    _load().orc_backproject(m, C.c_int64(t.npix), rp, ix, ln, _d(y), _d(x))
    return x.reshape(t.geom.n, t.geom.n)


# ---------------------------------------------------------------------------
# Sec. 2.2: TV, shrinkage, ADM
# ---------------------------------------------------------------------------

def grad(x) -> np.ndarray:
    """Backward differences of Eq. (2): [n][n] -> [2][n][n]."""
    x = _f64(x)
    n = x.shape[-1]
    d = np.zeros((2, n, n))
    _load().orc_grad(n, _d(x), _d(d))
    return d


def grad_t(d) -> np.ndarray:
    """Transpose of grad: [2][n][n] -> [n][n]."""
    d = _f64(d)
    n = d.shape[-1]
    out = np.zeros((n, n))
    _load().orc_grad_t(n, _d(d), _d(out))
    return out


def tv(x) -> float:
    """Isotropic TV norm, Eq. (2)."""
    x = _f64(x)
    return float(_load().orc_tv(x.shape[-1], _d(x)))


def shrink(w, t: float) -> np.ndarray:
    """Isotropic shrinkage of Eq. (8) (reading R1) on [2][...] vectors."""
    w = _f64(w)
    npix = w[0].size
    z = np.zeros_like(w)
    _load().orc_shrink(C.c_int64(npix), _d(w), t, _d(z))
    return z


BB1, CAUCHY = 0, 1


@dataclasses.dataclass
class AdmParams:
    """Eq. (6)-(10) parameters (values are readings; the paper gives ranges only)."""
    mu: float = 4.0
    rho: float = 256.0
    xi: Optional[float] = None     # None -> xi = rho
    step_rule: int = CAUCHY
    max_iter: int = 100
    tol: float = 0.0
    beta: Tuple[float, float] = (1.0, 0.6)   # (beta_1 for x_h, beta_2 for x_l), Eq. (3)
    nonneg: bool = False                     # project f onto f >= 0 after each f-step
    joint: bool = False                      # adm_dual: TV coupled over both channels

    def c(self) -> _AdmParams:
        xi = self.rho if self.xi is None else self.xi
        return _AdmParams(self.mu, self.rho, xi, self.step_rule, self.max_iter, self.tol,
                          1 if self.nonneg else 0)


class AdmState:
    """State (f, z, lambda, previous step) of one channel's ADM."""

    def __init__(self, f0):
        f0 = _f64(f0)
        n = f0.shape[-1]
        self.f = f0.copy()
        self.z = np.zeros((2, n, n))
        self.lam = np.zeros((2, n, n))
        self.alpha_prev = -1.0


def adm_iterate(t: Table, g, prm: AdmParams, st: AdmState):
    """One iteration of Eq. (10).  Returns (alpha, G, (|G|^2, |AG|^2, |grad G|^2))."""
    g = _f64(g).reshape(-1)
    n = t.geom.n
    cst = _AdmState(_d(st.f), _d(st.z), _d(st.lam), st.alpha_prev)
    G = np.zeros((n, n))
    norms = np.zeros(3)
    cp = prm.c()
    m, rp, ix, ln = t._args()
    a = _load().orc_adm_iterate(n, m, rp, ix, ln, _d(g), C.byref(cp), C.byref(cst), _d(G), _d(norms))
    st.alpha_prev = cst.alpha_prev
    return float(a), G, tuple(norms)


def objective(t: Table, g, mu: float, f) -> float:
    """Phi(f) = ||grad f||_TV + mu/2 ||A f - g||^2, Eq. (4) for one channel."""
    g = _f64(g).reshape(-1)
    f = _f64(f)
    m, rp, ix, ln = t._args()
    return float(_load().orc_objective(t.geom.n, m, rp, ix, ln, _d(g), mu, _d(f)))


def adm_channel(t: Table, g, prm: AdmParams, f0=None):
    """ADM of Eq. (10) for one channel from f0 (default 0).

    Returns (f, iterations, phi[0..iters], alpha[0..iters-1]).
    """
    n = t.geom.n
    g = _f64(g).reshape(-1)
    f = np.zeros((n, n)) if f0 is None else _f64(f0).copy()
    phi = np.zeros(prm.max_iter + 1)
    alpha = np.zeros(max(prm.max_iter, 1))
    cp = prm.c()
    m, rp, ix, ln = t._args()
    k = _load().orc_adm_run(n, m, rp, ix, ln, _d(g), C.byref(cp), _d(f), _d(phi), _d(alpha))
    return f, int(k), phi[:k + 1].copy(), alpha[:k].copy()


def adm_dual(t: Table, m_he, prm: AdmParams, x0=None):
    """Dual-energy reconstruction, Eq. (3)-(10) under reading R3.

    m_he: [2][nv][nb] (high, low).  Each channel runs on f_c = beta_c x_c
    against g_c = beta_c m_c; returns x[2][n][n] = f_c / beta_c and the
    per-channel iteration counts.
    """
    if prm.joint:
        b = np.array(prm.beta, np.float64).reshape(2, 1, 1)
        f0 = None if x0 is None else b * _f64(x0)
        g = b * _f64(m_he).reshape(2, t.geom.nv, t.geom.nb)
        f, k, _, _ = adm_joint(t, g, prm, f0)
        return f / b, [k, k]
    xs, its = [], []
    for c in range(2):
        b = prm.beta[c]
        f0 = None if x0 is None else b * _f64(x0[c])
        f, k, _, _ = adm_channel(t, b * _f64(m_he[c]), prm, f0)
        xs.append(f / b)
        its.append(k)
    return np.stack(xs), its


# ---------------------------------------------------------------------------
# Fan-beam FBP (the analytic reconstruction of Sec. 2.4 and Sec. 3; textbook
# algorithm for an equally spaced flat detector over 360 degrees)
# ---------------------------------------------------------------------------

def fbp_filter(geom, p) -> np.ndarray:
    """Cosine-weighted, ramp-filtered projections [nv][nb] (see dect_oracle.c)."""
    p = _f64(p).reshape(geom.nv, geom.nb)
    qf = np.zeros_like(p)
    _load().orc_fbp_filter(C.byref(_geom(geom)), _d(p), _d(qf))
    return qf


def fbp(geom, p) -> np.ndarray:
    """FBP image [n][n] from projections [nv][nb]."""
    p = _f64(p).reshape(geom.nv, geom.nb)
    f = np.zeros((geom.n, geom.n))
    _load().orc_fbp(C.byref(_geom(geom)), _d(p), _d(f))
    return f


# ---------------------------------------------------------------------------
# Joint TV: Eq. (4) with the TV norm taken over both channels per pixel
# ---------------------------------------------------------------------------

def shrink4(wh, wl, t: float):
    """Prox of the per-pixel 4-norm: z = max(|w| - t, 0) w / |w| on
    w = (wh[0], wh[1], wl[0], wl[1]).  Returns (zh, zl), each [2][...]."""
    wh, wl = _f64(wh), _f64(wl)
    zh, zl = np.zeros_like(wh), np.zeros_like(wl)
    _load().orc_shrink4(wh[0].size, _d(wh), _d(wl), t, _d(zh), _d(zl))
    return zh, zl


def tv_joint(f) -> float:
    """sum_p |(grad f_h, grad f_l)_p|_2 for f = [2][n][n]."""
    f = _f64(f)
    return float(_load().orc_tv_joint(f.shape[-1], _d(f)))


def objective_joint(t: Table, g, mu: float, f) -> float:
    """Joint objective: tv_joint(f) + mu/2 sum_c |A f_c - g_c|^2; g = [2][M]."""
    g = _f64(g).reshape(-1)
    f = _f64(f)
    m, rp, ix, ln = t._args()
    return float(_load().orc_objective_joint(t.geom.n, m, rp, ix, ln, _d(g), mu, _d(f)))


class AdmJointState:
    """State of the joint ADM: f [2][n][n], z and lambda [2][2][n][n]."""

    def __init__(self, f0):
        f0 = _f64(f0)
        n = f0.shape[-1]
        self.f = f0.copy()
        self.z = np.zeros((2, 2, n, n))
        self.lam = np.zeros((2, 2, n, n))
        self.alpha_prev = -1.0


def adm_joint_iterate(t: Table, g, prm: AdmParams, st: AdmJointState):
    """One joint iteration of Eq. (10).  g = [2][M].
    Returns (alpha, G [2][n][n], (|G|^2, |AG|^2, |grad G|^2) over both channels)."""
    g = _f64(g).reshape(-1)
    n = t.geom.n
    cst = _AdmState(_d(st.f), _d(st.z), _d(st.lam), st.alpha_prev)
    G = np.zeros((2, n, n))
    norms = np.zeros(3)
    cp = prm.c()
    m, rp, ix, ln = t._args()
    a = _load().orc_adm_joint_iterate(n, m, rp, ix, ln, _d(g), C.byref(cp), C.byref(cst), _d(G),
                                      _d(norms))
    st.alpha_prev = cst.alpha_prev
    return float(a), G, tuple(norms)


def adm_joint(t: Table, g, prm: AdmParams, f0=None):
    """Joint ADM from f0 ([2][n][n], default 0) against g = [2][M].
    Returns (f, iterations, phi[0..iters], alpha[0..iters-1])."""
    n = t.geom.n
    g = _f64(g).reshape(-1)
    f = np.zeros((2, n, n)) if f0 is None else _f64(f0).copy()
    phi = np.zeros(prm.max_iter + 1)
    alpha = np.zeros(max(prm.max_iter, 1))
    cp = prm.c()
    m, rp, ix, ln = t._args()
    k = _load().orc_adm_joint_run(n, m, rp, ix, ln, _d(g), C.byref(cp), _d(f), _d(phi), _d(alpha))
    return f, int(k), phi[:k + 1].copy(), alpha[:k].copy()


# ---------------------------------------------------------------------------
# Sec. 2.3: decomposition
# ---------------------------------------------------------------------------

def eta_array(eta) -> np.ndarray:
    """eta[material][energy] as a flat float64 [4] (m * 2 + e)."""
    e = _f64(eta).reshape(2, 2)
    return e.reshape(-1).copy()


def direct_decompose(eta, xh, xl) -> Tuple[np.ndarray, np.ndarray]:
    """D^{-1} x per pixel, Eq. (11)-(12)."""
    xh, xl = _f64(xh), _f64(xl)
    e = eta_array(eta)
    d1 = np.zeros_like(xh)
    d2 = np.zeros_like(xh)
    _load().orc_direct_decompose(C.c_int64(xh.size), _d(e), _d(xh), _d(xl), _d(d1), _d(d2))
    return d1, d2


def prewitt(x) -> np.ndarray:
    """3x3 Prewitt gradient magnitude, replicate padding (reading R14)."""
    x = _f64(x)
    out = np.zeros_like(x)
    _load().orc_prewitt(x.shape[-1], _d(x), _d(out))
    return out


def edge_mask(xh, xl, tau: float) -> np.ndarray:
    """Edge pixels (uint8) from both energy images (reading R14)."""
    xh, xl = _f64(xh), _f64(xl)
    mask = np.zeros(xh.shape, np.uint8)
    _load().orc_edge_mask(xh.shape[-1], _d(xh), _d(xl), tau,
                          mask.ctypes.data_as(C.POINTER(C.c_uint8)))
    return mask


def pls_diag(mask, gamma: float, eps: float) -> np.ndarray:
    """Jacobi diagonal 1 + gamma sum_k e_ik of (I + gamma L_e) (readings R13, R16)."""
    mask = np.ascontiguousarray(mask, np.uint8)
    out = np.zeros(mask.shape, np.float64)
    _load().orc_pls_diag(mask.shape[-1], mask.ctypes.data_as(C.POINTER(C.c_uint8)), gamma, eps, _d(out))
    return out


def pls_apply(mask, gamma: float, eps: float, u) -> np.ndarray:
    """(I + gamma L_e) u, Eq. (14)-(15) under reading R13."""
    u = _f64(u)
    mask = np.ascontiguousarray(mask, np.uint8)
    out = np.zeros_like(u)
    _load().orc_pls_apply(u.shape[-1], mask.ctypes.data_as(C.POINTER(C.c_uint8)),
                          gamma, eps, _d(u), _d(out))
    return out


def pls_pcg(mask, gamma: float, eps: float, d, max_iter: int, tol: float):
    """Jacobi PCG for (I + gamma L_e) u = d from u = d.  Returns (u, iters, relres)."""
    d = _f64(d)
    mask = np.ascontiguousarray(mask, np.uint8)
    u = np.zeros_like(d)
    rr = C.c_double(0.0)
    it = _load().orc_pls_pcg(d.shape[-1], mask.ctypes.data_as(C.POINTER(C.c_uint8)),
                             gamma, eps, _d(d), _d(u), max_iter, tol, C.byref(rr))
    return u, int(it), float(rr.value)


@dataclasses.dataclass
class PlsParams:
    eta: np.ndarray = dataclasses.field(default_factory=lambda: np.array([[0.0184, 0.0227],
                                                                         [0.0342, 0.0573]]))
    gamma: float = 0.1
    tau: float = 0.2
    eps: float = 0.05
    max_iter: int = 500
    tol: float = 1e-10


def pls_decompose(xh, xl, prm: PlsParams):
    """PLS decomposition, Eq. (13)-(15): returns (u1, u2, mask, iters)."""
    d1, d2 = direct_decompose(prm.eta, xh, xl)
    mask = edge_mask(xh, xl, prm.tau)
    u1, i1, _ = pls_pcg(mask, prm.gamma, prm.eps, d1, prm.max_iter, prm.tol)
    u2, i2, _ = pls_pcg(mask, prm.gamma, prm.eps, d2, prm.max_iter, prm.tol)
    return u1, u2, mask, (i1, i2)


# ---------------------------------------------------------------------------
# CNN warm start (not in the paper; the learned part of the workload)
# ---------------------------------------------------------------------------

def cnn_num_params() -> int:
    return int(_load().orc_cnn_num_params())


def cnn_forward(params, x, scale: float) -> np.ndarray:
    """Encoder-decoder output x + s * net(x / s) for one image x [H][W] (H, W multiples of 4)."""
    params = _f64(params)
    x = _f64(x)
    out = np.zeros_like(x)
    _load().orc_cnn_run(_d(params), scale, _d(x), x.shape[0], x.shape[1], _d(out), None, None, None)
    return out


def cnn_loss_grad(params, x, target, scale: float):
    """(loss, dloss/dparams) for L = mean (out - target)^2 on one image."""
    params = _f64(params)
    x = _f64(x)
    target = _f64(target)
    grad = np.zeros_like(params)
    loss = C.c_double(0.0)
    _load().orc_cnn_run(_d(params), scale, _d(x), x.shape[0], x.shape[1], None, _d(target), _d(grad),
                        C.byref(loss))
    return float(loss.value), grad



# ---------------------------------------------------------------------------
# Cone-beam geometry and 3-D decomposition (Sec. 2.1, Fig. 1; Sec. 2.3,
# Eq. (14) with 6 neighbours; Sec. 3)
# ---------------------------------------------------------------------------

def _geom3(g) -> _Geom3:
    return _Geom3(g.n, g.nz, g.px, g.pz, g.nv, g.nr, g.nc, g.pu, g.pv, g.sod, g.sdd, g.start, g.arc,
                  g.off_u, g.off_v)


def ray3(geom, v: int, r: int, c: int):
    """(S, D): source and detector-cell centre of ray (v, r, c), mm."""
    S = np.zeros(3)
    D = np.zeros(3)
    _load().orc3_ray(C.byref(_geom3(geom)), v, r, c, _d(S), _d(D))
    return S, D


def siddon_ray3(geom, v: int, r: int, c: int):
    """(voxel indices, lengths in mm) of ray (v, r, c), in walk order."""
    cap = 2 * geom.n + geom.nz + 8
    idx = np.zeros(cap, np.int32)
    ln = np.zeros(cap)
    k = _load().orc3_siddon_ray(C.byref(_geom3(geom)), v, r, c, idx.ctypes.data_as(C.POINTER(C.c_int32)),
                                _d(ln), cap)
    return idx[:k].copy(), ln[:k].copy()


@dataclasses.dataclass
class Table3:
    """Ray-major table of the cone-beam A: row (v nr + r) nc + c."""
    geom: object
    rowptr: np.ndarray
    idx: np.ndarray
    len: np.ndarray

    @property
    def m(self) -> int:
        return self.geom.nv * self.geom.nr * self.geom.nc

    @property
    def npix(self) -> int:
        return self.geom.n * self.geom.n * self.geom.nz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def _args(self):
        return (C.c_int64(self.m), self.rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                self.idx.ctypes.data_as(C.POINTER(C.c_int32)), _d(self.len))


def table3(geom) -> Table3:
    lib = _load()
    g = _geom3(geom)
    nnz = lib.orc3_table_nnz(C.byref(g))
    M = geom.nv * geom.nr * geom.nc
    rowptr = np.zeros(M + 1, np.int64)
    idx = np.zeros(max(nnz, 1), np.int32)
    ln = np.zeros(max(nnz, 1))
    lib.orc3_table_build(C.byref(g), rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                         idx.ctypes.data_as(C.POINTER(C.c_int32)), _d(ln))
    return Table3(geom, rowptr, idx[:nnz], ln[:nnz])


def project3(t: Table3, x) -> np.ndarray:
    """y = A x: volume [nz][n][n] -> projections [nv][nr][nc]."""
    x = _f64(x).reshape(-1)
    y = np.zeros(t.m)
    _load().orc_project(*t._args(), _d(x), _d(y))
    return y.reshape(t.geom.nv, t.geom.nr, t.geom.nc)


def backproject3(t: Table3, y) -> np.ndarray:
    """x = A^T y: [nv][nr][nc] -> [nz][n][n]."""
    y = _f64(y).reshape(-1)
    x = np.zeros(t.npix)
    m, rp, ix, ln = t._args()
    _load().orc_backproject(m, C.c_int64(t.npix), rp, ix, ln, _d(y), _d(x))
    return x.reshape(t.geom.nz, t.geom.n, t.geom.n)


def prewitt3(x) -> np.ndarray:
    """3-D Prewitt magnitude, replicate padding: x [nz][n][n]."""
    x = _f64(x)
    out = np.zeros_like(x)
    _load().orc3_prewitt(x.shape[-1], x.shape[0], _d(x), _d(out))
    return out


def edge_mask3(xh, xl, tau: float) -> np.ndarray:
    xh, xl = _f64(xh), _f64(xl)
    mask = np.zeros(xh.shape, np.uint8)
    _load().orc3_edge_mask(xh.shape[-1], xh.shape[0], _d(xh), _d(xl), tau,
                           mask.ctypes.data_as(C.POINTER(C.c_uint8)))
    return mask


def pls_apply3(mask, gamma: float, eps: float, u) -> np.ndarray:
    u = _f64(u)
    mask = np.ascontiguousarray(mask, np.uint8)
    out = np.zeros_like(u)
    _load().orc3_pls_apply(u.shape[-1], u.shape[0], mask.ctypes.data_as(C.POINTER(C.c_uint8)), gamma, eps,
                           _d(u), _d(out))
    return out


def pls_diag3(mask, gamma: float, eps: float) -> np.ndarray:
    mask = np.ascontiguousarray(mask, np.uint8)
    out = np.zeros(mask.shape, np.float64)
    _load().orc3_pls_diag(mask.shape[-1], mask.shape[0], mask.ctypes.data_as(C.POINTER(C.c_uint8)), gamma, eps,
                          _d(out))
    return out


def pls_pcg3(mask, gamma: float, eps: float, d, max_iter: int, tol: float):
    d = _f64(d)
    mask = np.ascontiguousarray(mask, np.uint8)
    u = np.zeros_like(d)
    rr = C.c_double(0.0)
    it = _load().orc3_pls_pcg(d.shape[-1], d.shape[0], mask.ctypes.data_as(C.POINTER(C.c_uint8)), gamma, eps,
                              _d(d), _d(u), max_iter, tol, C.byref(rr))
    return u, int(it), float(rr.value)


def pls_decompose3(xh, xl, prm: PlsParams):
    """3-D PLS decomposition (Eq. (13)-(15), 6 neighbours): volumes [nz][n][n]."""
    d1, d2 = direct_decompose(prm.eta, xh, xl)
    mask = edge_mask3(xh, xl, prm.tau)
    u1, i1, _ = pls_pcg3(mask, prm.gamma, prm.eps, d1, prm.max_iter, prm.tol)
    u2, i2, _ = pls_pcg3(mask, prm.gamma, prm.eps, d2, prm.max_iter, prm.tol)
    return u1, u2, mask, (i1, i2)
