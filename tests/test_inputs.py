"""The seeded input recipes (pac_inputs) match the workloads' stated recipes.

These run on the CPU and pin what the tests and the bench feed both sides:
seeds determine every array, the distributions and filter normalisations are
the stated ones, and the batched / served mixes have the stated proportions.
"""
import math

import numpy as np
import pytest

import pac_inputs as pin


def test_seeds_determine_arrays():
    a, b = pin.complex_uniform((64, 3), 7), pin.complex_uniform((64, 3), 7)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, pin.complex_uniform((64, 3), 8))
    assert np.array_equal(pin.complex_normal((50,), 3), pin.complex_normal((50,), 3))


def test_signal_distributions():
    u = pin.complex_uniform((200_000,), 1)
    assert u.dtype == np.complex128
    assert np.all(np.abs(u.real) <= 1) and np.all(np.abs(u.imag) <= 1)
    assert abs(u.real.mean()) < 0.01 and abs(u.real.var() - 1 / 3) < 0.01
    g = pin.complex_normal((200_000,), 2)
    assert abs(g.real.mean()) < 0.01 and abs(g.imag.std() - 1) < 0.01


def test_rounding_to_working_precision():
    x = pin.complex_uniform((16,), 4)
    assert pin.as_dtype(x, "c64").dtype == np.complex64
    assert pin.as_dtype(x, "c128").dtype == np.complex128
    assert np.max(np.abs(pin.as_dtype(x, "c64") - x)) < 1e-7
    with pytest.raises(ValueError):
        pin.as_dtype(x, "c32")


@pytest.mark.parametrize("n,sigma", [(128, 4.0), (81, 2.5), (25, 1.0), (2, 4.0)])
def test_gaussian_factor_is_periodised_even_and_normalised(n, sigma):
    (g,) = pin.gaussian_factors((n,), sigma)
    assert abs(g.sum() - 1) < 1e-14
    assert np.all(g.imag == 0) and np.all(g.real > 0)
    assert np.allclose(g[1:], g[1:][::-1], rtol=0, atol=1e-17)  # g[i] = g[n - i]
    assert g[0].real == g.real.max()


def test_exponential_factor_at_minimum_image_distance():
    (e,) = pin.exponential_factors((10,), 20.0)
    d = np.array([0, 1, 2, 3, 4, 5, 4, 3, 2, 1])
    assert np.allclose(e, np.exp(-d / 20.0), rtol=0, atol=1e-16)


def test_outer_is_row_major_separable():
    f = [np.arange(1, 4, dtype=np.complex128), np.arange(1, 6, dtype=np.complex128)]
    h = pin.outer(f)
    assert h.shape == (3, 5) and h.flags.c_contiguous
    assert h[2, 4] == 3 * 5


def test_workload_shapes():
    assert pin.c1().dims == (1024,) and pin.c1().dtype == "c128" and pin.c1().radix == 2
    for r in (2, 4, 8):
        assert pin.c2(r).dims == (128, 128, 128)
    assert pin.c3(3).dims == (2187, 2187) and pin.c3(5).dims == (3125, 3125)
    assert pin.mixed((1000, 1000)).radix == 0
    assert pin.aniso((2 ** 22, 2, 2)).n_total == 2 ** 24
    h, fs = pin.make_h(pin.c2(4))
    assert fs is not None and h.shape == (128, 128, 128) and abs(h.sum() - 1) < 1e-5
    h1, f1 = pin.make_h(pin.c1())
    assert f1 is None and h1.shape == (1024,)


def test_batched_mix_is_uniform_over_classes():
    insts = pin.c4_instances(4096)
    assert len(insts) == 4096 and len(pin.C4_CLASSES) == 20
    counts = {}
    for c in insts:
        counts[(c.dims, c.radix)] = counts.get((c.dims, c.radix), 0) + 1
        assert c.dtype == "c64" and 20_000 <= c.h_seed < 20_064
    assert set(counts) == set(pin.C4_CLASSES)
    expect = 4096 / 20
    assert all(abs(v - expect) < 5 * math.sqrt(expect) for v in counts.values())


def test_served_mix_rate_precision_and_shapes():
    reqs = pin.c5_requests(2.0)
    n = len(reqs)
    assert abs(n - 4000) < 5 * math.sqrt(4000)
    assert all(a.t_arrive < b.t_arrive for a, b in zip(reqs, reqs[1:]))
    frac32 = sum(r.conv.dtype == "c64" for r in reqs) / n
    assert abs(frac32 - 0.7) < 0.03
    for r in reqs:
        d, radix = r.conv.dims, r.conv.radix
        assert len(d) in (1, 2, 3) and radix in (2, 3) and len(set(d)) == 1
        e = round(math.log(d[0], radix))
        assert radix ** e == d[0]
        lo, hi = {(1, 2): (12, 20), (2, 2): (8, 11), (3, 2): (5, 8),
                  (1, 3): (8, 12), (2, 3): (5, 7), (3, 3): (4, 5)}[(len(d), radix)]
        assert lo <= e <= hi
        assert 0 <= r.filter_id < 32
    small = pin.c5_requests(0.05, max_elems=1 << 16)
    assert all(r.conv.n_total <= 1 << 16 for r in small)


def test_sample_points_are_distinct_sorted_and_in_range():
    p = pin.sample_points(1000, 64, seed=3)
    assert len(p) == 64 and np.all(np.diff(p) > 0) and p[0] >= 0 and p[-1] < 1000
    assert np.array_equal(p, pin.sample_points(1000, 64, seed=3))
    assert len(pin.sample_points(10, 64, seed=1)) == 10
