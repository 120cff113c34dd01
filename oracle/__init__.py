"""Oracle for the permutation-avoiding FFT convolution — TEST INFRASTRUCTURE.

Plain, slow, obviously correct FP64 CPU implementations of what the CUDA
path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's
CPU-baseline / reference legs may import this package; the library under
``paper_2506_12718_gb300`` never does, and this package imports nothing from
it.  The two share no code; only the seeded input generators
(``pac_inputs``) serve both.

Routes (all FP64, interleaved complex, row-major with the last index fastest):

* ``conv_direct``         O1: y[k] = sum_j h[j] x[(k-j) mod n] (the convolution of
                          Section 2 / Section 4 written out), O(N^2)
* ``conv_direct_points``  O1 at chosen output indices
* ``conv_separable``      O2: separable filter, one 1-D definition per axis
* ``dft`` / ``idft``      O3: naive per-axis DFT (Section 2, w_n = exp(-2 pi i/n))
* ``unordered_forward``   A^T x = P^T F x per axis, with P from the paper's
                          definition (``paper_forms.pos_to_freq``)
* ``paper_forms``         the paper's matrix forms for tiny n (Eq. 25, Eq. 35, Eq. 80),
                          the mixed-radix A_rho, P_rho (Section 7.1) and the prime factor
                          maps and convolution (Section 7.2)

Parity: every route is pinned by ``tests/test_oracle_pins.py`` (brute force,
library routines, closed forms and invariants); none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

from . import paper_forms  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc (-O2, OpenMP, IEEE arithmetic) into liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_conv_direct.argtypes = [ctypes.c_int, i64p, p, p, p]
        lib.oracle_conv_direct_points.argtypes = [ctypes.c_int, i64p, p, p, ctypes.c_int64, i64p, p]
        lib.oracle_conv_separable.argtypes = [ctypes.c_int, i64p, ctypes.POINTER(ctypes.c_void_p), p, p, p]
        lib.oracle_dft.argtypes = [ctypes.c_int, i64p, p, p, ctypes.c_int, p]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.complex128)


def _dims(shape):
    d = np.ascontiguousarray(np.asarray(shape, dtype=np.int64))
    return d, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def num_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def conv_direct(h, x) -> np.ndarray:
    """O1: circular convolution of x with h from its definition (FP64)."""
    h, x = _c128(h), _c128(x)
    assert h.shape == x.shape
    y = np.empty_like(x)
    d, dp = _dims(x.shape)
    rc = _load().oracle_conv_direct(len(x.shape), dp, h.ctypes.data, x.ctypes.data, y.ctypes.data)
    assert rc == 0
    return y


def conv_direct_points(h, x, idx) -> np.ndarray:
    """O1 at linear output indices ``idx`` (row-major)."""
    h, x = _c128(h), _c128(x)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.empty(idx.shape[0], np.complex128)
    d, dp = _dims(x.shape)
    rc = _load().oracle_conv_direct_points(len(x.shape), dp, h.ctypes.data, x.ctypes.data,
                                           idx.shape[0], idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           out.ctypes.data)
    assert rc == 0
    return out


def conv_separable(factors, x) -> np.ndarray:
    """O2: convolution with h = outer(factors) as one 1-D definition per axis (FP64)."""
    x = _c128(x)
    fs = [_c128(f) for f in factors]
    assert len(fs) == x.ndim and all(f.shape == (n,) for f, n in zip(fs, x.shape))
    ptrs = (ctypes.c_void_p * len(fs))(*[f.ctypes.data for f in fs])
    y = np.empty_like(x)
    work = np.empty_like(x)
    d, dp = _dims(x.shape)
    rc = _load().oracle_conv_separable(x.ndim, dp, ptrs, x.ctypes.data, y.ctypes.data, work.ctypes.data)
    assert rc == 0
    return y


def dft(x, sign: int = -1) -> np.ndarray:
    """O3: naive d-D DFT, w_n = exp(sign 2 pi i / n) per axis, unnormalised."""
    x = _c128(x)
    out = np.empty_like(x)
    work = np.empty_like(x)
    d, dp = _dims(x.shape)
    rc = _load().oracle_dft(x.ndim, dp, x.ctypes.data, out.ctypes.data, int(sign), work.ctypes.data)
    assert rc == 0
    return out


def idft(X) -> np.ndarray:
    """Inverse of ``dft``: conjugate-sign naive DFT divided by N."""
    return dft(X, +1) / np.prod(np.asarray(X).shape)


def conv_via_dft(h, x) -> np.ndarray:
    """F_h(x) = DFT^-1(DFT(h) o DFT(x)) through the naive DFT (a second route to O1)."""
    return idft(dft(h) * dft(x))


def unordered_forward(x, stages_per_axis) -> np.ndarray:
    """A^T x per axis (DIF output): DFT then the paper's index-reversal order.

    Along each axis position p holds frequency pos_to_freq(stages)[p]
    (F = P A^T, Section 2.1; F = P_rho A_rho^T, Section 7.1).
    """
    X = dft(x)
    for a, st in enumerate(stages_per_axis):
        X = np.take(X, paper_forms.pos_to_freq(st), axis=a)
    return np.ascontiguousarray(X)


def rel_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2 accumulated in FP64."""
    a = np.asarray(a, dtype=np.complex128).reshape(-1)
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
