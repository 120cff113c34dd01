"""Seeded synthetic inputs for the permutation-avoiding FFT convolution.

This module is shared by the tests, the bench and the oracle's callers.  It
holds input construction only (random signals, filters, workload mixes) and
none of the convolution arithmetic: no DFT, no butterfly, no index reversal.

Workloads follow the shapes the paper benchmarks (1-D, 2-D and 3-D arrays
whose axes are powers of the radix, Section 6) with the distributions stated
for this build's five workloads:

* ``c1``: 1-D n=2^10, radix 2, complex FP64, x and h with re/im ~ U[-1,1].
* ``c2``: 3-D 128^3, radix 2/4/8, complex FP32 and FP64; x ~ N(0,1) re/im;
  h a periodised isotropic Gaussian (sigma = 4 cells), normalised to sum 1.
* ``c3``: 2-D 2187^2 (radix 3) and 3125^2 (radix 5); x ~ U[-1,1];
  h a periodised separable exponential exp(-|i|/20 - |j|/20).
* ``c4``: 4096 independent FP32 convolutions, sizes drawn from 20 classes.
* ``c5``: Poisson request stream of mixed shapes/radices/precisions.

The paper itself prints no input distributions; the choices above, the
minimum-image periodisation and the size-sampling rules are this build's
readings and are listed in the design notes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------- signals


def complex_uniform(shape, seed: int) -> np.ndarray:
    """Complex128 array with real and imaginary parts i.i.d. U[-1, 1]."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-1.0, 1.0, size=shape)
    im = rng.uniform(-1.0, 1.0, size=shape)
    return (re + 1j * im).astype(np.complex128)


def complex_normal(shape, seed: int) -> np.ndarray:
    """Complex128 array with real and imaginary parts i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(size=shape)
    im = rng.standard_normal(size=shape)
    return (re + 1j * im).astype(np.complex128)


def as_dtype(a: np.ndarray, dtype: str) -> np.ndarray:
    """Round a complex128 array once to the working precision.

    ``dtype`` is "c64" (complex FP32), or "c128" / "c128df" (complex FP64
    arrays, computed in FP64 or in double-float arithmetic).  The oracle is
    then run on the rounded values promoted back to FP64, so an error measure
    reflects the algorithm only, not the input rounding.
    """
    if dtype == "c64":
        return a.astype(np.complex64)
    if dtype in ("c128", "c128df"):
        return a.astype(np.complex128)
    raise ValueError(f"unknown dtype {dtype!r}")


# ---------------------------------------------------------------- filters


def _min_image(n: int) -> np.ndarray:
    """Periodic distance of each index to 0 on a ring of n cells."""
    i = np.arange(n)
    return np.minimum(i, n - i).astype(np.float64)


def gaussian_factors(dims, sigma: float) -> list[np.ndarray]:
    """Per-axis factors of a periodised isotropic Gaussian, each summing to 1.

    The full filter is their outer product: h[i] = prod_a g_a(i_a) with
    g_a(d) = exp(-d^2 / (2 sigma^2)) at the minimum-image distance d, so h is
    real, even and sums to 1.
    """
    out = []
    for n in dims:
        d = _min_image(int(n))
        g = np.exp(-(d * d) / (2.0 * sigma * sigma))
        out.append((g / g.sum()).astype(np.complex128))
    return out


def exponential_factors(dims, length: float) -> list[np.ndarray]:
    """Per-axis factors exp(-d/length) at the minimum-image distance (unnormalised)."""
    return [np.exp(-_min_image(int(n)) / length).astype(np.complex128) for n in dims]


def outer(factors: list[np.ndarray]) -> np.ndarray:
    """Dense separable filter from its per-axis factors (row-major, last axis fastest)."""
    h = factors[0]
    for f in factors[1:]:
        h = np.multiply.outer(h, f)
    return np.ascontiguousarray(h)


# ---------------------------------------------------------------- workloads


@dataclass(frozen=True)
class Conv:
    """One convolution problem: shape, radix, precision and its inputs' recipe."""

    dims: tuple
    radix: int
    dtype: str  # "c64" | "c128"
    x_kind: str  # "uniform" | "normal"
    h_kind: str  # "uniform" | "gauss" | "exp"
    seed: int
    h_param: float = 0.0  # sigma (gauss) or length (exp); unused for "uniform"
    h_seed: int = 0

    @property
    def n_total(self) -> int:
        return int(np.prod(self.dims))

    @property
    def elem_bytes(self) -> int:
        return 8 if self.dtype == "c64" else 16


def make_x(c: Conv) -> np.ndarray:
    """Input signal of problem ``c`` rounded to its precision."""
    gen = complex_uniform if c.x_kind == "uniform" else complex_normal
    return as_dtype(gen(c.dims, c.seed), c.dtype)


def make_h(c: Conv):
    """Filter of problem ``c`` rounded to its precision, plus its FP64 factors.

    Returns ``(h, factors)``; ``factors`` is None for non-separable filters.
    The factors are the exact FP64 factors; for FP32 the dense filter is the
    rounded outer product, which the oracle uses promoted to FP64.
    """
    if c.h_kind == "uniform":
        return as_dtype(complex_uniform(c.dims, c.h_seed), c.dtype), None
    if c.h_kind == "gauss":
        f = gaussian_factors(c.dims, c.h_param)
    elif c.h_kind == "exp":
        f = exponential_factors(c.dims, c.h_param)
    elif c.h_kind == "delta":
        f = []
        for n in c.dims:
            e = np.zeros(n, np.complex128)
            e[0] = 1.0
            f.append(e)
    else:
        raise ValueError(c.h_kind)
    return as_dtype(outer(f), c.dtype), f


def c1() -> Conv:
    """1-D circular convolution, n = 2^10, radix 2, complex FP64, seed 1."""
    return Conv((1024,), 2, "c128", "uniform", "uniform", seed=1, h_seed=101)


def c2(radix: int = 8, dtype: str = "c64", n: int = 128) -> Conv:
    """3-D periodic convolution n^3 with a sigma=4 periodised Gaussian, seed 2."""
    return Conv((n, n, n), radix, dtype, "normal", "gauss", seed=2, h_param=4.0)


def c3(radix: int = 3, dtype: str = "c64") -> Conv:
    """2-D 2187^2 (radix 3) or 3125^2 (radix 5) with a separable exponential, seed 3."""
    n = {3: 2187, 5: 3125}[radix]
    return Conv((n, n), radix, dtype, "uniform", "exp", seed=3, h_param=20.0)


def mixed(dims=(1000, 1000), dtype: str = "c64") -> Conv:
    """Mixed-radix shapes, every dim 2^a 3^b 5^c (radix 0), with c3's recipe
    (x ~ U[-1,1], separable exponential of length 20), seed 6."""
    return Conv(tuple(int(d) for d in dims), 0, dtype, "uniform", "exp", seed=6, h_param=20.0)


def aniso(dims=(2 ** 24, 2), dtype: str = "c64") -> Conv:
    """The paper's anisotropic shapes, n x 2 and n x 2 x 2 (radix 2), with c3's
    recipe (x ~ U[-1,1], separable exponential of length 20), seed 8."""
    return Conv(tuple(int(d) for d in dims), 2, dtype, "uniform", "exp", seed=8, h_param=20.0)


# Size classes of the batched workload: 1-D {2^8..2^16} (9 classes),
# 1-D {3^5..3^10} (6 classes) and 2-D {2^6..2^10}^2 (5 classes).
C4_CLASSES = ([((2 ** e,), 2) for e in range(8, 17)]
              + [((3 ** e,), 3) for e in range(5, 11)]
              + [((2 ** e, 2 ** e), 2) for e in range(6, 11)])


def c4_instances(count: int = 4096, seed: int = 4, n_filters: int = 64):
    """Batched workload: ``count`` FP32 problems, classes drawn uniformly.

    Each instance uses filter id f in [0, n_filters); a filter id seeds an
    i.i.d. U[-1,1] filter generated at that instance's shape, so instances of
    the same (f, shape) share one filter spectrum.
    """
    rng = np.random.default_rng(seed)
    cls = rng.integers(0, len(C4_CLASSES), size=count)
    fid = rng.integers(0, n_filters, size=count)
    out = []
    for i in range(count):
        dims, radix = C4_CLASSES[int(cls[i])]
        out.append(Conv(dims, radix, "c64", "normal", "uniform",
                        seed=10_000 + i, h_seed=20_000 + int(fid[i])))
    return out


@dataclass
class Request:
    """One serving request: arrival time (s) and its problem."""

    t_arrive: float
    conv: Conv
    filter_id: int


def c5_filter_pool(seed: int = 5, n: int = 32):
    """32 filters: 16 Gaussians with sigma ~ U[1,8], 16 exponentials with length ~ U[5,40]."""
    rng = np.random.default_rng(seed + 1000)
    pool = []
    for i in range(n):
        if i < n // 2:
            pool.append(("gauss", float(rng.uniform(1.0, 8.0))))
        else:
            pool.append(("exp", float(rng.uniform(5.0, 40.0))))
    return pool


def c5_shape(rng) -> tuple:
    """Draw (dims, radix) for a serving request.

    Dimension uniform over {1,2,3}; radix 2 or 3 with probability 1/2 each;
    the size uniform over the powers of that radix inside the stated ranges
    (radix 2: 1-D 2^12..2^20, 2-D 256..2048 per axis, 3-D 32..256 per axis;
    radix 3: 1-D 3^8..3^12, 2-D 3^5..3^7, 3-D 3^4..3^5).
    """
    d = int(rng.integers(1, 4))
    r = 2 if rng.random() < 0.5 else 3
    ranges = {(1, 2): (12, 20), (2, 2): (8, 11), (3, 2): (5, 8),
              (1, 3): (8, 12), (2, 3): (5, 7), (3, 3): (4, 5)}
    lo, hi = ranges[(d, r)]
    e = int(rng.integers(lo, hi + 1))
    return tuple([r ** e] * d), r


def c5_requests(duration_s: float, rate: float = 2000.0, seed: int = 5,
                max_elems: int | None = None):
    """Poisson arrivals at ``rate`` req/s for ``duration_s`` seconds.

    70 % FP32 / 30 % FP64; x ~ N(0,1); filters from the 32-entry pool.
    ``max_elems`` (optional) redraws shapes above that element count, so a
    short test can keep the mix small.
    """
    rng = np.random.default_rng(seed)
    pool = c5_filter_pool(seed)
    t = 0.0
    out = []
    i = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration_s:
            break
        while True:
            dims, r = c5_shape(rng)
            if max_elems is None or math.prod(dims) <= max_elems:
                break
        dtype = "c64" if rng.random() < 0.7 else "c128"
        fid = int(rng.integers(0, len(pool)))
        kind, param = pool[fid]
        out.append(Request(t, Conv(dims, r, dtype, "normal", kind, seed=50_000 + i,
                                   h_param=param), fid))
        i += 1
    return out


def sample_points(n_total: int, count: int, seed: int) -> np.ndarray:
    """Seeded distinct linear output indices for point-sampled checks (sorted)."""
    rng = np.random.default_rng(seed)
    count = min(count, n_total)
    return np.sort(rng.choice(n_total, size=count, replace=False)).astype(np.int64)
