"""Oracle discrete Fourier transforms (test infrastructure, FP64).

Only tests, the smoke check and the CPU-baseline leg of the benchmark may use
this package; the product path never imports it.

* ``dft_dense``: the DFT written out as a matrix product,
  ``X[k] = sum_n x[n] exp(sign * 2 pi i n k / N)``, O(N^2) per axis.
* ``fft``: a plain recursive decimation-in-time FFT (radix 2 and radix 3,
  dense DFT for any other odd length), vectorised over the other axes.

Both are unnormalised; ``inverse=True`` uses ``sign = +1`` and divides by
``N``.  The recursive transform is checked against the dense one and against
closed forms in the ``-m "not gpu"`` tests.  Sec. 3.3 of the paper fixes 3D
Fourier transforms for all spatial derivatives; these are those transforms.
"""

from __future__ import annotations

import numpy as np


def _dense_axis0(x, sign):
    n = x.shape[0]
    j = np.arange(n)
    w = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
    return np.tensordot(w, x, axes=([1], [0]))


def _fft_axis0(x, sign):
    n = x.shape[0]
    if n == 1:
        return x.copy()
    bshape = (-1,) + (1,) * (x.ndim - 1)
    if n % 2 == 0:
        e = _fft_axis0(x[0::2], sign)
        o = _fft_axis0(x[1::2], sign)
        k = np.arange(n // 2)
        t = np.exp(sign * 2j * np.pi * k / n).reshape(bshape) * o
        return np.concatenate([e + t, e - t], axis=0)
    if n % 3 == 0:
        m = n // 3
        k = np.arange(n)
        out = np.zeros(x.shape, dtype=np.complex128)
        for r in range(3):
            y = _fft_axis0(x[r::3], sign)
            out += np.exp(sign * 2j * np.pi * r * k / n).reshape(bshape) * y[k % m]
        return out
    return _dense_axis0(x, sign)


def _along(fn, x, axis, inverse):
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, 0)
    y = fn(x, +1.0 if inverse else -1.0)
    if inverse:
        y = y / x.shape[0]
    return np.moveaxis(y, 0, axis)


def fft(x, axis, inverse=False):
    """Recursive FFT along ``axis``."""
    return _along(_fft_axis0, x, axis, inverse)


def dft_dense(x, axis, inverse=False):
    """Dense-matrix DFT along ``axis``."""
    return _along(_dense_axis0, x, axis, inverse)


# threads of the ``"scipy"`` kind (the library transform split over cores,
# for long oracle runs on large grids)
SCIPY_WORKERS = 1


def fftn(x, inverse=False, kind="recursive"):
    """3D transform: one 1D transform per axis (``kind``: ``"recursive"``,
    ``"dense"``, ``"numpy"`` for the library routine, or ``"scipy"`` for the
    library routine on ``SCIPY_WORKERS`` threads)."""
    if kind == "numpy":
        return np.fft.ifftn(x) if inverse else np.fft.fftn(x)
    if kind == "scipy":
        import scipy.fft as sf
        return sf.ifftn(x, workers=SCIPY_WORKERS) if inverse else sf.fftn(x, workers=SCIPY_WORKERS)
    f = fft if kind == "recursive" else dft_dense
    y = np.asarray(x, dtype=np.complex128)
    for a in range(y.ndim):
        y = f(y, a, inverse)
    return y
