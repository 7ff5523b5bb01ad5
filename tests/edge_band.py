"""Where an FP32 edge decision may differ from the FP64 one (Eq. (14), reading R14).

The GPU takes the edge decision of Eq. (14) in FP32; the oracle takes it in
FP64.  Both start from the same FP32 image values.  This helper bounds, per
pixel, how far the FP32 normalised Prewitt magnitude |g| / max|g| can lie
from the FP64 one, from standard floating-point error analysis with unit
roundoff u = 2^-24:

  - each Prewitt component is a sum of three rounded differences, summed in
    order: |error| <= 3u * S (S = the sum of the absolute differences, plus
    second-order terms), so the vector error is <= 3u * hypot(S_x, S_y);
  - squaring, adding and the square root add a relative error <= 3u of |g|;
  - the maximum of the magnitudes moves by at most the largest of the
    per-pixel errors; the division adds a relative u.

The band is twice that bound.  Pixels outside it must get the same decision
on both sides; pixels inside it may legitimately differ.
"""
import numpy as np

import oracle

U32 = 2.0 ** -24


def _abs_terms(x: np.ndarray) -> np.ndarray:
    """hypot of the sums of absolute differences of the two Prewitt components."""
    n = x.shape[0]
    idx = np.arange(n)
    cl = lambda a: np.clip(a, 0, n - 1)  # noqa: E731 (replicate padding)
    sx = np.zeros_like(x)
    sy = np.zeros_like(x)
    for t in (-1, 0, 1):
        sx += np.abs(x[cl(idx + t)][:, cl(idx + 1)] - x[cl(idx + t)][:, cl(idx - 1)])
        sy += np.abs(x[cl(idx + 1)][:, cl(idx + t)] - x[cl(idx - 1)][:, cl(idx + t)])
    return np.hypot(sx, sy)


def band(x: np.ndarray, tau: float) -> np.ndarray:
    """Boolean map of the pixels of image x (FP32 values) whose FP32 decision
    against tau may differ from the FP64 one."""
    x = np.asarray(x, np.float64)
    m = oracle.prewitt(x)
    big = m.max()
    if big == 0.0:
        return np.zeros(x.shape, bool)
    err = 4 * U32 * _abs_terms(x) + 3 * U32 * m
    r = m / big
    width = 2 * ((err + r * err.max()) / big + 2 * U32 * r)
    return np.abs(r - tau) <= width


def mask_band(xh: np.ndarray, xl: np.ndarray, tau: float) -> np.ndarray:
    """Pixels whose edge/non-edge decision from either image is within rounding of tau."""
    return band(xh, tau) | band(xl, tau)


def _abs_terms3(x: np.ndarray) -> np.ndarray:
    """3-D counterpart of _abs_terms: x [nz][n][n], nine differences per component."""
    nz, n = x.shape[0], x.shape[1]
    ci = lambda a: np.clip(a, 0, n - 1)  # noqa: E731
    ck = lambda a: np.clip(a, 0, nz - 1)  # noqa: E731
    ii, kk = np.arange(n), np.arange(nz)
    sx = np.zeros_like(x)
    sy = np.zeros_like(x)
    sz = np.zeros_like(x)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            sx += np.abs(x[ck(kk + a)][:, ci(ii + b)][:, :, ci(ii + 1)] - x[ck(kk + a)][:, ci(ii + b)][:, :, ci(ii - 1)])
            sy += np.abs(x[ck(kk + a)][:, ci(ii + 1)][:, :, ci(ii + b)] - x[ck(kk + a)][:, ci(ii - 1)][:, :, ci(ii + b)])
            sz += np.abs(x[ck(kk + 1)][:, ci(ii + a)][:, :, ci(ii + b)] - x[ck(kk - 1)][:, ci(ii + a)][:, :, ci(ii + b)])
    return np.sqrt(sx * sx + sy * sy + sz * sz)


def band3(x: np.ndarray, tau: float) -> np.ndarray:
    """band() for volumes [nz][n][n] and the 3-D Prewitt of nine terms per component."""
    x = np.asarray(x, np.float64)
    m = oracle.prewitt3(x)
    big = m.max()
    if big == 0.0:
        return np.zeros(x.shape, bool)
    err = 10 * U32 * _abs_terms3(x) + 4 * U32 * m
    r = m / big
    width = 2 * ((err + r * err.max()) / big + 2 * U32 * r)
    return np.abs(r - tau) <= width
