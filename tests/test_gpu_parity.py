"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Tolerances (relative L2 over the whole output, accumulated in FP64):
  complex FP64: <= 1e-12;  complex FP32: <= 1e-5 * log2(N).
FP32 inputs are generated in FP64 and rounded once; the oracle runs on the
rounded values promoted to FP64.  For separable filters the oracle's
per-axis route (O2) uses the FP64 factors while the GPU gets the rounded
dense filter; the difference (<= 6e-8 relative for FP32, ~1e-16 for FP64) is
far below the tolerances.
"""
import math
import os
import time

import numpy as np
import pytest

import oracle
import pac_inputs as pin
from oracle import paper_forms as pf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_12718_gb300 import _build
    _build.build()
    import paper_2506_12718_gb300 as pac
    pac.load()
    return pac


def pac_mod():
    import paper_2506_12718_gb300 as pac
    return pac


def tol(dtype, n):
    # complex FP64 arrays, computed in FP64 ("c128") or double-float arithmetic ("c128df"): the FP64 bound
    return 1e-12 if dtype in ("c128", "c128df") else 1e-5 * max(1.0, math.log2(n))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_conv(dims, radix, dtype, h, x, permuted=False):
    pac = pac_mod()
    plan = pac.Plan(dims, radix, dtype)
    try:
        plan.filter_spectrum(dev(h))
        xd = dev(x)
        y = plan.convolve_permuted(xd) if permuted else plan.convolve(xd)
        torch.cuda.synchronize()
        return y.cpu().numpy()
    finally:
        plan.close()


def separable_case(dims, dtype, seed):
    fs = [pin.complex_uniform((n,), seed + 100 + a) for a, n in enumerate(dims)]
    h = pin.as_dtype(pin.outer(fs), dtype)
    x = pin.as_dtype(pin.complex_uniform(dims, seed), dtype)
    return fs, h, x


def check(y, ref, dtype, n, what=""):
    err = oracle.rel_l2(y, ref)
    assert err <= tol(dtype, n), f"{what} rel_l2={err:.3e} tol={tol(dtype, n):.1e}"
    return err


# ------------------------------------------------------------------ configs


def test_c1_full_definition():
    """1-D n = 2^10, radix 2, complex FP64 against the direct definition (O1)."""
    c = pin.c1()
    x, (h, _) = pin.make_x(c), pin.make_h(c)
    y = gpu_conv(c.dims, c.radix, c.dtype, h, x)
    check(y, oracle.conv_direct(h, x), c.dtype, c.n_total, "c1")


@pytest.mark.parametrize("dtype", ["c64", "c128", "c128df"])
@pytest.mark.parametrize("radix", [2, 4, 8])
def test_c2_128_cubed_gaussian(radix, dtype):
    """3-D 128^3 periodic convolution with the sigma=4 Gaussian, full array (O2)."""
    c = pin.c2(radix, dtype)
    x, (h, fs) = pin.make_x(c), pin.make_h(c)
    y = gpu_conv(c.dims, c.radix, c.dtype, h, x)
    ref = _c2_ref(dtype)
    check(y, ref, dtype, c.n_total, f"c2 r{radix} {dtype}")


_C2_CACHE = {}


def _c2_ref(dtype):
    if dtype not in _C2_CACHE:
        c = pin.c2(2, dtype)
        x, (_, fs) = pin.make_x(c), pin.make_h(c)
        _C2_CACHE[dtype] = oracle.conv_separable(fs, x)
    return _C2_CACHE[dtype]


@pytest.mark.parametrize("dtype", ["c64", "c128", "c128df"])
@pytest.mark.parametrize("radix", [3, 5])
def test_c3_large_2d_exponential(radix, dtype):
    """2-D 2187^2 (radix 3) and 3125^2 (radix 5) with the separable exponential (O2)."""
    c = pin.c3(radix, dtype)
    x, (h, fs) = pin.make_x(c), pin.make_h(c)
    y = gpu_conv(c.dims, c.radix, c.dtype, h, x)
    check(y, oracle.conv_separable(fs, x), dtype, c.n_total, f"c3 r{radix} {dtype}")


# --------------------------------------------------------- shapes and radices

SHAPES = [
    ((2,), 2), ((8,), 2), ((64,), 4), ((128,), 8), ((256,), 2), ((1024,), 4), ((4096,), 2),
    ((8192,), 2), ((16384,), 4), ((32768,), 8), ((3,), 3), ((27,), 3), ((243,), 3), ((2187,), 3),
    ((6561,), 3), ((5,), 5), ((125,), 5), ((3125,), 5), ((15625,), 5),
    ((8, 8), 2), ((64, 32), 4), ((27, 81), 3), ((25, 125), 5), ((2, 1024), 2), ((1024, 2), 8),
    ((1, 64), 2), ((64, 1), 4), ((243, 9), 3), ((4, 4, 4), 4), ((8, 16, 32), 8), ((27, 9, 3), 3),
    ((2, 2, 2), 2), ((32, 32, 32), 2), ((5, 25, 5), 5), ((16, 1, 8), 2),
    # anisotropic shapes of the paper's experiments: n x 2 and n x 2 x 2
    ((16384, 2), 2), ((65536, 2), 4), ((4096, 2, 2), 2), ((16384, 2, 2), 8), ((6561, 3), 3),
]


@pytest.mark.parametrize("dtype", ["c64", "c128", "c128df"])
@pytest.mark.parametrize("dims,radix", SHAPES, ids=[f"{'x'.join(map(str, d))}-r{r}" for d, r in SHAPES])
def test_shapes_separable(dims, radix, dtype):
    fs, h, x = separable_case(dims, dtype, seed=hash((dims, radix)) % 1000)
    y = gpu_conv(dims, radix, dtype, h, x)
    check(y, oracle.conv_separable(fs, x), dtype, int(np.prod(dims)), f"{dims} r{radix}")


PLANE_SHAPES = [((128, 128), 4, "c64"), ((64, 64), 2, "c64"), ((2, 32, 32), 8, "c64"), ((16, 16), 2, "c64"),
                ((4, 64, 128), 2, "c64"), ((2, 128, 64), 4, "c64"), ((81, 81), 3, "c64"), ((27, 27), 3, "c64"),
                ((25, 25), 5, "c64"), ((125, 125), 5, "c64"), ((9, 9), 3, "c64"), ((64, 64), 4, "c128"),
                ((4, 32, 32), 2, "c128"), ((81, 81), 3, "c128"), ((25, 25), 5, "c128"), ((16, 16), 8, "c128"),
                ((3, 27, 27), 3, "c128")]


@pytest.mark.parametrize("dims,radix,dtype", PLANE_SHAPES,
                         ids=[f"{'x'.join(map(str, d))}-r{r}-{t}" for d, r, t in PLANE_SHAPES])
def test_plane_pass_shapes(dims, radix, dtype, monkeypatch):
    """Shapes whose last two axes run as one plane pass (whole planes in one
    CTA): against the oracle, and equal to the per-axis passes (PAC_PLANE=0)."""
    pac = pac_mod()
    fs, h, x = separable_case(dims, dtype, seed=len(dims) * 100 + dims[-1])
    ref = oracle.conv_separable(fs, x)
    y = gpu_conv(dims, radix, dtype, h, x)
    check(y, ref, dtype, int(np.prod(dims)), f"plane {dims}")
    plan = pac.Plan(dims, radix, dtype)
    try:
        assert plan.query(pac.Q_LAUNCHES_CONVOLVE) == 2 * (len(dims) - 2) + 1
    finally:
        plan.close()
    monkeypatch.setenv("PAC_PLANE", "0")
    y2 = gpu_conv(dims, radix, dtype, h, x)
    check(y2, ref, dtype, int(np.prod(dims)), f"per-axis {dims}")


@pytest.mark.parametrize("dims,radix", [((16,), 2), ((9, 27), 3), ((8, 4, 16), 4), ((25, 5), 5), ((64, 64), 8)])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_nonseparable_direct(dims, radix, dtype):
    h = pin.as_dtype(pin.complex_uniform(dims, 5), dtype)
    x = pin.as_dtype(pin.complex_normal(dims, 6), dtype)
    y = gpu_conv(dims, radix, dtype, h, x)
    check(y, oracle.conv_direct(h, x), dtype, int(np.prod(dims)))


MAX_SHAPES = [((1 << 28,), 4, "c64"), ((16384, 16384), 2, "c64"), ((512, 512, 512), 8, "c64"),
              ((1 << 27,), 2, "c128"), ((59049, 2187), 3, "c64")]


@pytest.mark.parametrize("dims,radix,dtype", MAX_SHAPES,
                         ids=[f"{'x'.join(map(str, d))}-r{r}-{t}" for d, r, t in MAX_SHAPES])
def test_maximum_sizes_sampled(dims, radix, dtype):
    """The largest arrays a plan takes (N up to 2^28, offsets near the 32-bit
    limit of the kernels), checked at 6 seeded output points against the
    direct definition (O1); inputs generated on the device from a seed."""
    pac = pac_mod()
    n = int(np.prod(dims))
    real = torch.float32 if dtype == "c64" else torch.float64
    g = torch.Generator(device="cuda")
    g.manual_seed(n % 1000003)
    x = torch.view_as_complex(torch.rand(*dims, 2, generator=g, device="cuda", dtype=real) * 2 - 1)
    h = torch.view_as_complex(torch.rand(*dims, 2, generator=g, device="cuda", dtype=real) * 2 - 1)
    plan = pac.Plan(dims, radix, dtype)
    try:
        plan.filter_spectrum(h)
        y = plan.convolve(x)
        torch.cuda.synchronize()
        idx = pin.sample_points(n, 6, seed=n % 7919)
        ref = oracle.conv_direct_points(h.cpu().numpy(), x.cpu().numpy(), idx)
        got = y.reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
        err = oracle.rel_l2(got, ref)
        assert err <= tol(dtype, n), f"{dims}: rel_l2 {err:.3e}"
    finally:
        plan.close()
        del x, h
        torch.cuda.empty_cache()


def test_empty_batch_and_n1_in_batch():
    pac = pac_mod()
    pac.pac_convolve_many([], [], [])  # nothing to do
    p1 = pac.Plan((1,), 2, "c128")
    p2 = pac.Plan((64,), 4, "c128")
    try:
        h1 = torch.tensor([2.0 - 1.0j], dtype=torch.complex128, device="cuda")
        x1 = torch.tensor([0.5 + 3.0j], dtype=torch.complex128, device="cuda")
        p1.filter_spectrum(h1)
        fs, h2, x2 = separable_case((64,), "c128", 3)
        p2.filter_spectrum(dev(h2))
        x2d = dev(x2)
        y1, y2 = torch.empty_like(x1), torch.empty_like(x2d)
        pac.pac_convolve_many([p1.handle, p2.handle], [x1, x2d], [y1, y2])
        torch.cuda.synchronize()
        assert abs(y1.item() - (2.0 - 1.0j) * (0.5 + 3.0j)) < 1e-15
        check(y2.cpu().numpy(), oracle.conv_separable(fs, x2), "c128", 64, "batch with N = 1")
    finally:
        p1.close()
        p2.close()


def test_shared_tables_outlive_another_plan():
    """Plans of one problem share their device tables (reference counted):
    destroying one leaves the others' tables in place."""
    pac = pac_mod()
    dims, radix, dtype = (64, 64), 4, "c64"
    fs, h, x = separable_case(dims, dtype, seed=71)
    ref = oracle.conv_separable(fs, x)
    plans = [pac.Plan(dims, radix, dtype) for _ in range(3)]
    try:
        for p in plans:
            p.filter_spectrum(dev(h))
        plans[0].close()
        plans[1].close()
        y = plans[2].convolve(dev(x))
        torch.cuda.synchronize()
        check(y.cpu().numpy(), ref, dtype, x.size, "after two plans of the same problem were destroyed")
        again = pac.Plan(dims, radix, dtype)  # takes the surviving copy
        try:
            again.filter_spectrum(dev(h))
            check(again.convolve(dev(x)).cpu().numpy(), ref, dtype, x.size, "a new plan of the same problem")
        finally:
            again.close()
    finally:
        for p in plans:
            p.close()


def test_single_element():
    h = np.array([2.0 - 1.0j], np.complex128)
    x = np.array([0.5 + 3.0j], np.complex128)
    y = gpu_conv((1,), 2, "c128", h, x)
    assert abs(y[0] - h[0] * x[0]) < 1e-15


def test_delta_filter_is_identity_fp64():
    dims = (64, 32, 16)
    h = np.zeros(dims, np.complex128)
    h[0, 0, 0] = 1.0
    x = pin.complex_normal(dims, 9)
    y = gpu_conv(dims, 4, "c128", h, x)
    assert oracle.rel_l2(y, x) < 1e-14


def test_shifted_delta_is_roll():
    dims = (81, 27)
    h = np.zeros(dims, np.complex128)
    h[5, 20] = 1.0
    x = pin.complex_normal(dims, 10)
    y = gpu_conv(dims, 3, "c128", h, x)
    assert oracle.rel_l2(y, np.roll(x, (5, 20), axis=(0, 1))) < 1e-13


LARGE_GROUP_SHAPES = [((2187, 2187), 3, "c64"), ((3125, 3125), 5, "c64"), ((729, 81), 3, "c64"), ((625, 25), 5, "c64"),
                ((2187, 9), 3, "c128"), ((3125, 5), 5, "c128"), ((27, 729), 3, "c64"), ((3, 2187), 3, "c128"),
                ((25, 625), 5, "c128")]


@pytest.mark.parametrize("dims,radix,dtype", LARGE_GROUP_SHAPES,
                         ids=[f"{'x'.join(map(str, d))}-r{r}-{t}" for d, r, t in LARGE_GROUP_SHAPES])
def test_large_groups_match_oracle(dims, radix, dtype):
    """Large groups (729, 2187, 625, 3125 rows or lines; forward, fused and
    inverse passes): the convolution against the oracle and the forward
    transform against the DFT in index-reversed order."""
    fs, h, x = separable_case(dims, dtype, seed=dims[0] + dims[-1])
    ref = oracle.conv_separable(fs, x)
    y = gpu_conv(dims, radix, dtype, h, x)
    check(y, ref, dtype, int(np.prod(dims)), f"large group {dims}")
    pac = pac_mod()
    xu = pin.as_dtype(pin.complex_uniform(dims, 5), dtype)
    plan = pac.Plan(dims, radix, dtype)
    try:
        stages = [plan.stages(a) for a in range(len(dims))]
        xh = plan.forward_unordered(dev(xu))
        torch.cuda.synchronize()
        check(xh.cpu().numpy(), oracle.unordered_forward(xu, stages), dtype, xu.size, "large group A^T x")
    finally:
        plan.close()


# ------------------------------------------------------- unordered transform


@pytest.mark.parametrize("dims,radix,dtype", [
    ((128,), 2, "c128"), ((128,), 4, "c128"), ((128,), 8, "c128"), ((81,), 3, "c128"), ((125,), 5, "c128"),
    ((16, 8), 4, "c128"), ((4, 8, 16), 8, "c128"), ((8192,), 2, "c128"), ((8192,), 4, "c64"),
    ((6561,), 3, "c128"), ((32, 64), 8, "c64"), ((2187,), 3, "c64"),
])
def test_forward_is_dft_in_index_reversed_order(dims, radix, dtype):
    """The fixed fact of the method: A^T x = P^T F x, per axis (Sections 2.1, 7.1)."""
    pac = pac_mod()
    x = pin.as_dtype(pin.complex_uniform(dims, 11), dtype)
    plan = pac.Plan(dims, radix, dtype)
    try:
        stages = [plan.stages(a) for a in range(len(dims))]
        for a in range(len(dims)):
            assert plan.stages(a) == pac.pac_stage_list(dims[a], radix)
            assert np.array_equal(np.array(plan.reverse_table(a)), pf.pos_to_freq(stages[a]))
        xh = plan.forward_unordered(dev(x))
        torch.cuda.synchronize()
        got = xh.cpu().numpy()
    finally:
        plan.close()
    ref = oracle.unordered_forward(x, stages)
    check(got, ref, dtype, int(np.prod(dims)), "A^T x")


# -------------------------------------------------------- ordered transforms


@pytest.mark.parametrize("dims,radix,dtype", [((128,), 4, "c128"), ((81,), 3, "c128"), ((16, 32), 8, "c128"),
                                             ((8, 4, 16), 2, "c64"), ((125, 25), 5, "c64"), ((4096,), 2, "c64")])
def test_ordered_fft_is_the_dft(dims, radix, dtype):
    """pac_fft: forward = the naive DFT (O3) in natural order; inverse(forward(x)) = x; inverse = O3's inverse."""
    pac = pac_mod()
    x = pin.as_dtype(pin.complex_uniform(dims, 15), dtype)
    plan = pac.Plan(dims, radix, dtype)
    try:
        xd = dev(x)
        X = torch.empty_like(xd)
        pac.pac_fft(plan.handle, xd, X)
        back = torch.empty_like(xd)
        pac.pac_fft(plan.handle, X, back, inverse=True)
        torch.cuda.synchronize()
        Xn = X.cpu().numpy()
        check(Xn, oracle.dft(x), dtype, x.size, "F x")
        check(back.cpu().numpy(), x, dtype, x.size, "F^-1 F x")
        y = torch.empty_like(xd)
        pac.pac_fft(plan.handle, dev(Xn), y, inverse=True)
        torch.cuda.synchronize()
        check(y.cpu().numpy(), oracle.idft(Xn), dtype, x.size, "F^-1 X")
    finally:
        plan.close()


# ------------------------------------------------------------- mixed radix

MIXED_SHAPES = [((30,), "c128"), ((360,), "c64"), ((1000,), "c128"), ((2700,), "c64"), ((6000,), "c64"),
                ((12, 20), "c128"), ((60, 90), "c64"), ((100, 120), "c128"), ((250, 48), "c64"), ((1, 45), "c64"),
                ((6, 10, 15), "c128"), ((12, 20, 30), "c64"), ((40, 36, 50), "c64"), ((96, 2, 2), "c128"),
                ((1000, 1000), "c64"), ((48, 1000), "c128"), ((120, 120, 120), "c64")]


@pytest.mark.parametrize("dims,dtype", MIXED_SHAPES, ids=[f"{'x'.join(map(str, d))}-{t}" for d, t in MIXED_SHAPES])
def test_mixed_radix_plans(dims, dtype):
    """radix 0, n = 2^a 3^b 5^c per axis (Section 7.1): one pass per run of one
    prime base, external twiddles of non-prime-power lengths; the
    convolution against the oracle."""
    fs, h, x = separable_case(dims, dtype, seed=sum(dims))
    y = gpu_conv(dims, 0, dtype, h, x)
    check(y, oracle.conv_separable(fs, x), dtype, int(np.prod(dims)), f"mixed {dims}")


@pytest.mark.parametrize("dims,dtype,mixed_launches,onebase_launches",
                         [((1000, 1000), "c64", 3, 7), ((120, 120, 120), "c64", 5, 17), ((60, 90), "c128", 3, 11),
                          ((6000,), "c64", (1, 3), 5), ((6000, 6), "c128", (3, 5), 9), ((30,), "c128", 1, 5),
                          ((72, 75), "c64", 3, 7)])
def test_mixed_groups_against_one_base_groups(dims, dtype, mixed_launches, onebase_launches, monkeypatch):
    """Groups spanning prime bases (compiled kernels where they exist,
    PAC_MIXED=1, a 6000-point axis as one compiled group; the runtime-radix
    kernel for all of them, PAC_MIXED=rt, which stops at 2048 points) against
    one-base groups (PAC_MIXED=0): fewer launches, the same convolution."""
    pac = pac_mod()
    fs, h, x = separable_case(dims, dtype, seed=3 * sum(dims))
    ref = oracle.conv_separable(fs, x)
    n = int(np.prod(dims))
    for k, mode in enumerate(("1", "rt")):
        monkeypatch.setenv("PAC_MIXED", mode)
        plan = pac.Plan(dims, 0, dtype)
        want = mixed_launches[k] if isinstance(mixed_launches, tuple) else mixed_launches
        try:
            assert plan.query(pac.Q_LAUNCHES_CONVOLVE) == want
        finally:
            plan.close()
        check(gpu_conv(dims, 0, dtype, h, x), ref, dtype, n, f"mixed groups {dims} ({mode})")
    monkeypatch.setenv("PAC_MIXED", "0")
    plan = pac.Plan(dims, 0, dtype)
    try:
        assert plan.query(pac.Q_LAUNCHES_CONVOLVE) == onebase_launches
    finally:
        plan.close()
    check(gpu_conv(dims, 0, dtype, h, x), ref, dtype, n, f"one-base groups {dims}")


STAGE_ORDERS = [((60,), [[3, 4, 5]], "c128"), ((60,), [[5, 3, 2, 2]], "c128"), ((1000,), [[5, 2, 5, 4, 5]], "c64"),
                ((120, 90), [[2, 3, 4, 5], [3, 5, 2, 3]], "c64"), ((18, 20, 24), [[3, 2, 3], [5, 4], [4, 3, 2]], "c128"),
                ((1024,), [[2] * 10], "c64"), ((72, 1), [[2, 3, 4, 3], []], "c128"), ((25, 27), [[5, 5], [3, 9]], "c64"),
                ((64, 48), [[16, 4], [16, 3]], "c64")]


@pytest.mark.parametrize("mixed", ["0", "1", "rt"])
@pytest.mark.parametrize("dims,stages,dtype", STAGE_ORDERS,
                         ids=[f"{'x'.join(map(str, d))}-{'_'.join('.'.join(map(str, s)) for s in st)}-{t}"
                              for d, st, t in STAGE_ORDERS])
def test_explicit_stage_lists(dims, stages, dtype, mixed, monkeypatch):
    """Any stage order (Section 7.1, A_rho with rho = the DIF list reversed):
    the unordered transform is the DFT in that list's digit-reversed order
    (the oracle's P_rho), and the convolution does not depend on the order;
    with one-base groups and with groups spanning bases."""
    monkeypatch.setenv("PAC_MIXED", mixed)
    pac = pac_mod()
    fs, h, x = separable_case(dims, dtype, seed=7 * len(dims))
    plan = pac.Plan(dims, 0, dtype, stages=stages)
    try:
        for a in range(len(dims)):
            assert plan.stages(a) == list(stages[a])
            assert np.array_equal(np.array(plan.reverse_table(a)), pf.pos_to_freq(stages[a]))
        plan.filter_spectrum(dev(h))
        y = plan.convolve(dev(x))
        xh = plan.forward_unordered(dev(x))
        torch.cuda.synchronize()
        n = int(np.prod(dims))
        check(y.cpu().numpy(), oracle.conv_separable(fs, x), dtype, n, f"stages {stages}")
        check(xh.cpu().numpy(), oracle.unordered_forward(x, stages), dtype, n, f"A^T x, stages {stages}")
    finally:
        plan.close()


@pytest.mark.parametrize("dims,dtype", [((60, 90), "c128"), ((1000,), "c64"), ((12, 20, 30), "c64")])
def test_mixed_radix_comparator_and_ordered_fft(dims, dtype):
    """The permuted form (explicit index reversals) and the ordered transform
    on mixed-radix plans."""
    pac = pac_mod()
    fs, h, x = separable_case(dims, dtype, seed=21)
    ref = oracle.conv_separable(fs, x)
    check(gpu_conv(dims, 0, dtype, h, x, permuted=True), ref, dtype, int(np.prod(dims)), "mixed permuted")
    plan = pac.Plan(dims, 0, dtype)
    try:
        xd = dev(x)
        X = torch.empty_like(xd)
        pac.pac_fft(plan.handle, xd, X)
        torch.cuda.synchronize()
        check(X.cpu().numpy(), oracle.dft(x), dtype, x.size, "mixed F x")
    finally:
        plan.close()


@pytest.mark.parametrize("mixed", ["0", "1", "rt"])
def test_mixed_radix_in_a_batch(mixed, monkeypatch):
    """Mixed-radix plans merged with uniform-radix ones in one pac_convolve_many
    call (with groups spanning bases: the batched compiled mixed kernels, or
    the batched runtime-radix kernel with PAC_MIXED=rt)."""
    monkeypatch.setenv("PAC_MIXED", mixed)
    pac = pac_mod()
    cases = [((60, 90), 0), ((1000,), 0), ((64, 64), 4), ((360,), 0), ((1000,), 0)]
    plans, xs, ys, refs = [], [], [], []
    try:
        for i, (dims, radix) in enumerate(cases):
            fs, h, x = separable_case(dims, "c64", seed=40 + i)
            p = pac.Plan(dims, radix, "c64")
            plans.append(p)
            p.filter_spectrum(dev(h))
            xs.append(dev(x))
            ys.append(torch.empty_like(xs[-1]))
            refs.append(oracle.conv_separable(fs, x))
        pac.pac_convolve_many([p.handle for p in plans], xs, ys)
        torch.cuda.synchronize()
        for (dims, _), y, ref in zip(cases, ys, refs):
            check(y.cpu().numpy(), ref, "c64", int(np.prod(dims)), f"batched mixed {dims}")
    finally:
        for p in plans:
            p.close()


@pytest.mark.parametrize("dims,dtype", [((6000, 6000), "c64"), ((1024 * 243 * 125,), "c64"), ((360, 360, 360), "c64"),
                                        ((2 ** 10 * 3 ** 4 * 5 ** 3,), "c128")])
def test_mixed_radix_large_sampled(dims, dtype):
    """Large mixed-radix arrays at 6 seeded output points against the direct definition."""
    pac = pac_mod()
    n = int(np.prod(dims))
    real = torch.float32 if dtype == "c64" else torch.float64
    g = torch.Generator(device="cuda")
    g.manual_seed(n % 1000003)
    x = torch.view_as_complex(torch.rand(*dims, 2, generator=g, device="cuda", dtype=real) * 2 - 1)
    h = torch.view_as_complex(torch.rand(*dims, 2, generator=g, device="cuda", dtype=real) * 2 - 1)
    plan = pac.Plan(dims, 0, dtype)
    try:
        plan.filter_spectrum(h)
        y = plan.convolve(x)
        torch.cuda.synchronize()
        idx = pin.sample_points(n, 6, seed=n % 7919)
        ref = oracle.conv_direct_points(h.cpu().numpy(), x.cpu().numpy(), idx)
        got = y.reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
        assert oracle.rel_l2(got, ref) <= tol(dtype, n)
    finally:
        plan.close()
        del x, h
        torch.cuda.empty_cache()


# ------------------------------------------------ prime factor form (Section 7.2)

PFA_CASES = [(6, "c128"), (10, "c64"), (12, "c128"), (60, "c128"), (360, "c64"), (1000, "c128"), (6000, "c64"),
             (81, "c64"), (1, "c128"), (2 ** 6 * 3 ** 3 * 5 ** 2, "c64"), (2 ** 5 * 125, "c128")]


@pytest.mark.parametrize("n,dtype", PFA_CASES, ids=[f"{n}-{t}" for n, t in PFA_CASES])
def test_prime_factor_convolution(n, dtype):
    """Three permutations around a t-D convolution of shape (n_t, ..., n_1)
    (Section 7.2): against the definition, in place, and equal to the
    permutation-free mixed-radix 1-D plan."""
    pac = pac_mod()
    h = pin.as_dtype(pin.complex_uniform((n,), 50 + n % 97), dtype)
    x = pin.as_dtype(pin.complex_normal((n,), 51 + n % 89), dtype)
    ref = oracle.conv_direct(h, x)
    p = pac.Pfa(n, dtype)
    try:
        assert p.shape == tuple(reversed(pf.coprime_factors(n))) or (n == 1 and p.shape == (1,))
        p.filter_spectrum(dev(h))
        y = p.convolve(dev(x))
        xd = dev(x)
        p.convolve(xd, xd)  # in place
        torch.cuda.synchronize()
        check(y.cpu().numpy(), ref, dtype, n, f"pfa {n}")
        check(xd.cpu().numpy(), ref, dtype, n, f"pfa {n} in place")
        assert p.query(pac.Q_LAUNCHES_CONVOLVE) >= 3
    finally:
        p.close()
    check(gpu_conv((n,), 0, dtype, h, x), ref, dtype, n, f"mixed radix 1-D {n}")


def test_prime_factor_convolution_large_sampled():
    """n = 2^10 3^5 5^3 (31.1 M points, FP32): 6 seeded outputs against the definition."""
    pac = pac_mod()
    n = 2 ** 10 * 3 ** 5 * 5 ** 3
    g = torch.Generator(device="cuda")
    g.manual_seed(17)
    x = torch.view_as_complex(torch.rand(n, 2, generator=g, device="cuda") * 2 - 1)
    h = torch.view_as_complex(torch.rand(n, 2, generator=g, device="cuda") * 2 - 1)
    p = pac.Pfa(n, "c64")
    try:
        assert p.shape == (1024, 243, 125)
        p.filter_spectrum(h)
        y = p.convolve(x)
        torch.cuda.synchronize()
        idx = pin.sample_points(n, 6, seed=23)
        ref = oracle.conv_direct_points(h.cpu().numpy(), x.cpu().numpy(), idx)
        got = y[torch.from_numpy(idx).cuda()].cpu().numpy()
        assert oracle.rel_l2(got, ref) <= tol("c64", n)
    finally:
        p.close()
        del x, h
        torch.cuda.empty_cache()


def test_prime_factor_without_spectrum_fails():
    pac = pac_mod()
    p = pac.Pfa(60, "c64")
    try:
        x = torch.zeros(60, dtype=torch.complex64, device="cuda")
        with pytest.raises(pac.PacError) as ei:
            p.convolve(x)
        assert ei.value.status == pac.Status.ERR_NO_SPECTRUM
    finally:
        p.close()


# -------------------------------------------------------------- comparator


@pytest.mark.parametrize("dims,radix,dtype", [((128, 128, 128), 4, "c64"), ((243, 81), 3, "c128"),
                                             ((8192,), 2, "c64"), ((32, 16), 8, "c128")])
def test_permuted_form_matches(dims, radix, dtype):
    fs, h, x = separable_case(dims, dtype, seed=12)
    ref = oracle.conv_separable(fs, x)
    yp = gpu_conv(dims, radix, dtype, h, x, permuted=True)
    check(yp, ref, dtype, int(np.prod(dims)), "permuted")


# ------------------------------------------------------------ API behaviour


def test_in_place_and_host_buffers():
    pac = pac_mod()
    dims, radix, dtype = (64, 128), 4, "c64"
    fs, h, x = separable_case(dims, dtype, seed=13)
    ref = oracle.conv_separable(fs, x)
    plan = pac.Plan(dims, radix, dtype)
    try:
        plan.filter_spectrum(dev(h))
        xd = dev(x)
        plan.convolve(xd, xd)  # y == x
        torch.cuda.synchronize()
        check(xd.cpu().numpy(), ref, dtype, x.size, "in place")
        xh = torch.from_numpy(x.copy()).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        s = torch.cuda.Stream()
        pac.pac_convolve_host(plan.handle, xh, yh, s)
        check(yh.numpy(), ref, dtype, x.size, "host buffers")
    finally:
        plan.close()


@pytest.mark.parametrize("dims,radix,dtype", [((4096, 2048), 2, "c64"), ((243, 243, 243), 3, "c64"),
                                             ((2187, 2187), 3, "c128"), ((3125, 1500), 0, "c128"),
                                             ((81, 110592), 0, "c64"), ((512, 512), 2, "c64")])
def test_host_buffers_in_column_blocks(dims, radix, dtype):
    """pac_convolve_host on arrays of 64 MiB and more copies the array in
    column blocks of the first pass (one strided copy each, on its own
    stream) while that pass runs on the blocks already in, and copies the
    result out block by block behind the last pass; smaller arrays (the last
    case) take one copy each way.  Twice in a row, the result is bit for bit
    the device-buffer convolution's (the same kernels on the same tiles) and
    matches the direct definition (O1) at 64 seeded points (ragged last tile
    and last block included)."""
    pac = pac_mod()
    n = int(np.prod(dims))
    x = pin.as_dtype(pin.complex_uniform(dims, 70 + len(dims)), dtype)
    h = pin.as_dtype(pin.complex_uniform(dims, 80 + len(dims)), dtype)
    plan = pac.Plan(dims, radix, dtype)
    try:
        plan.filter_spectrum(dev(h))
        yd = plan.convolve(dev(x)).cpu().numpy()
        idx = pin.sample_points(n, 64, seed=n % 7919)
        ref = oracle.conv_direct_points(h, x, idx)
        err = oracle.rel_l2(yd.reshape(-1)[idx], ref)
        assert err <= tol(dtype, n), f"{dims}: rel_l2 {err:.3e}"
        xh = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        s = torch.cuda.Stream()
        for rep in range(2):
            yh = torch.full_like(xh, float("nan")).pin_memory()
            pac.pac_convolve_host(plan.handle, xh, yh, s)
            assert np.array_equal(yh.numpy(), yd), f"{dims}: host-buffer result #{rep} differs"
    finally:
        plan.close()


def test_errors():
    pac = pac_mod()
    plan = pac.Plan((64,), 2, "c64")
    try:
        x = torch.zeros(64, dtype=torch.complex64, device="cuda")
        with pytest.raises(pac.PacError) as ei:
            plan.convolve(x)
        assert ei.value.status == pac.Status.ERR_NO_SPECTRUM
        plan.filter_spectrum(x)
        buf = torch.zeros(80, dtype=torch.complex64, device="cuda")
        with pytest.raises(pac.PacError) as ei:
            pac.pac_convolve(plan.handle, buf.data_ptr() + 8, buf.data_ptr() + 16)
        assert ei.value.status == pac.Status.ERR_ARG
        assert plan.query(pac.Q_HAS_SPECTRUM) == 1
        assert plan.query(pac.Q_N_TOTAL) == 64
    finally:
        plan.close()
    with pytest.raises(pac.PacError) as ei:
        pac.Plan((96,), 2, "c64")
    assert ei.value.status == pac.Status.ERR_SIZE


def test_convolve_many_matches_single():
    pac = pac_mod()
    cases = [((4096,), 2, 1), ((27, 81), 3, 2), ((64, 64), 8, 3), ((3125,), 5, 4), ((4096,), 2, 5)]
    plans, xs, ys, refs = [], [], [], []
    try:
        for dims, radix, seed in cases:
            fs, h, x = separable_case(dims, "c64", seed)
            p = pac.Plan(dims, radix, "c64")
            p.filter_spectrum(dev(h))
            plans.append(p)
            xs.append(dev(x))
            ys.append(torch.empty_like(xs[-1]))
            refs.append(oracle.conv_separable(fs, x))
        pac.pac_convolve_many([p.handle for p in plans], xs, ys)
        torch.cuda.synchronize()
        for y, ref, (dims, _, _) in zip(ys, refs, cases):
            check(y.cpu().numpy(), ref, "c64", int(np.prod(dims)), f"many {dims}")
    finally:
        for p in plans:
            p.close()


def test_convolve_many_graph_replay_and_plan_reuse():
    """A batch replays its captured graph on the second call (same result),
    a changed batch (new y pointers) is captured anew, and destroying a plan
    drops the cached batches that used it."""
    pac = pac_mod()
    cases = [((256,), 2, 7), ((81, 27), 3, 8), ((32, 32, 32), 4, 9), ((16384,), 8, 10), ((125,), 5, 11)]
    plans, xs, refs = [], [], []
    try:
        for dims, radix, seed in cases:
            fs, h, x = separable_case(dims, "c64", seed)
            p = pac.Plan(dims, radix, "c64")
            p.filter_spectrum(dev(h))
            plans.append(p)
            xs.append(dev(x))
            refs.append(oracle.conv_separable(fs, x))
        handles = [p.handle for p in plans] * 3  # plans repeat across instances
        xs3 = xs * 3
        for attempt in range(2):
            ys = [torch.full_like(x, float("nan")) for x in xs3]
            for _ in range(2):
                pac.pac_convolve_many(handles, xs3, ys)
            torch.cuda.synchronize()
            for k, y in enumerate(ys):
                dims = cases[k % len(cases)][0]
                check(y.cpu().numpy(), refs[k % len(cases)], "c64", int(np.prod(dims)), f"many[{k}] {dims}")
        plans[1].close()
        rest = [p.handle for i, p in enumerate(plans) if i != 1]
        xr = [x for i, x in enumerate(xs) if i != 1]
        yr = [torch.empty_like(x) for x in xr]
        pac.pac_convolve_many(rest, xr, yr)
        torch.cuda.synchronize()
        for y, ref, (dims, _, _) in zip(yr, [r for i, r in enumerate(refs) if i != 1],
                                        [c for i, c in enumerate(cases) if i != 1]):
            check(y.cpu().numpy(), ref, "c64", int(np.prod(dims)), f"after destroy {dims}")
    finally:
        for p in plans:
            p.close()


def test_convolve_many_batched_workload_sample():
    """96 instances drawn from the batched workload's 20 size classes (FP32,
    64 filter ids), checked at 48 seeded output points each against the
    direct definition (O1)."""
    pac = pac_mod()
    insts = pin.c4_instances(96)
    plans, xs, ys, hs = {}, [], [], []
    try:
        handles = []
        for c in insts:
            key = (c.dims, c.radix, c.h_seed)
            h, _ = pin.make_h(c)
            if key not in plans:
                p = pac.Plan(c.dims, c.radix, c.dtype)
                p.filter_spectrum(dev(h))
                plans[key] = p
            handles.append(plans[key].handle)
            x = pin.make_x(c)
            xs.append(x)
            hs.append(h)
        xd = [dev(x) for x in xs]
        yd = [torch.empty_like(x) for x in xd]
        pac.pac_convolve_many(handles, xd, yd)
        torch.cuda.synchronize()
        for i, (c, h, x, y) in enumerate(zip(insts, hs, xs, yd)):
            idx = pin.sample_points(c.n_total, 48, seed=500 + i)
            ref = oracle.conv_direct_points(h, x, idx)
            got = y.cpu().numpy().reshape(-1)[idx]
            err = oracle.rel_l2(got, ref)
            assert err <= tol("c64", c.n_total), f"instance {i} {c.dims}: rel_l2 {err:.3e}"
    finally:
        for p in plans.values():
            p.close()


@pytest.mark.parametrize("dims,radix,dtype", [((4096,), 2, "c64"), ((243, 243), 3, "c64"), ((32, 64, 64), 4, "c128"),
                                             ((65536,), 4, "c64"), ((1000, 1000), 0, "c64"), ((60, 90, 30), 0, "c128")])
def test_autotuned_schedule_matches_oracle(dims, radix, dtype):
    """pac_tune times the candidate pass schedules and keeps the fastest; a
    plan created afterwards uses it and still matches the oracle."""
    pac = pac_mod()
    us = pac.pac_tune(dims, radix, dtype, reps=3)
    assert us > 0
    fs, h, x = separable_case(dims, dtype, seed=77)
    plan = pac.Plan(dims, radix, dtype)
    try:
        cap = plan.query(pac.Q_GROUP_CAP)
        assert cap >= 1  # a tuned schedule always carries its cap
        assert plan.query(pac.Q_GROUPS) >= len(dims)
    finally:
        plan.close()
    y = gpu_conv(dims, radix, dtype, h, x)
    check(y, oracle.conv_separable(fs, x), dtype, int(np.prod(dims)), f"tuned {dims}")


def test_tune_file_round_trip(tmp_path):
    """With PAC_TUNE_FILE set, a schedule tuned in one process is used by
    plans of a later process."""
    import subprocess
    import sys
    path = tmp_path / "tune.txt"
    env = dict(os.environ, PAC_TUNE_FILE=str(path))
    code1 = ("import paper_2506_12718_gb300 as pac; pac.load(); import torch; torch.cuda.init(); "
             "print(pac.pac_tune((2187, 2187), 3, 'c64', 2))")
    subprocess.run([sys.executable, "-c", code1], env=env, check=True, cwd=os.path.dirname(os.path.dirname(__file__)))
    line = path.read_text().split()
    assert len(line) == 9 and line[0] == "2" and line[1] == "2187"
    code2 = ("import paper_2506_12718_gb300 as pac; pac.load(); import torch; torch.cuda.init(); "
             "p = pac.Plan((2187, 2187), 3, 'c64'); print(p.query(pac.Q_GROUP_CAP)); p.close()")
    out = subprocess.run([sys.executable, "-c", code2], env=env, check=True, capture_output=True, text=True,
                         cwd=os.path.dirname(os.path.dirname(__file__)))
    assert int(out.stdout.strip().splitlines()[-1]) == int(line[6])


def test_tuner_chooses_the_plane_tile(tmp_path):
    """The tuner's candidates include the plane pass' tile: a whole 81 x 81
    plane per CTA or the plane split over a 3-CTA cluster.  The tune file
    records the winner (flags bit 0 the plane pass, bits 4-7 its split, 0 =
    the default rule), a later plan uses it, and both tiles' convolutions
    match the oracle."""
    import subprocess
    import sys
    path = tmp_path / "tune.txt"
    env = dict(os.environ, PAC_TUNE_FILE=str(path))
    root = os.path.dirname(os.path.dirname(__file__))
    code1 = ("import paper_2506_12718_gb300 as pac; pac.load(); import torch; torch.cuda.init(); "
             "print(pac.pac_tune((81, 81), 3, 'c64', 3))")
    subprocess.run([sys.executable, "-c", code1], env=env, check=True, cwd=root)
    line = path.read_text().split()
    assert len(line) == 9 and line[1] == "81"
    k = (int(line[7]) >> 4) & 15
    code2 = ("import paper_2506_12718_gb300 as pac; pac.load(); import torch; torch.cuda.init(); "
             "p = pac.Plan((81, 81), 3, 'c64'); print(p.query(pac.Q_PLANE)); p.close()")
    out = subprocess.run([sys.executable, "-c", code2], env=env, check=True, capture_output=True, text=True, cwd=root)
    plane = int(out.stdout.strip().splitlines()[-1])
    if int(line[7]) & 1:  # the winner has the plane pass: the tile it recorded
        assert plane in (1, 3) and (k == 0 or plane == k)
    else:  # per-axis passes won (e.g. with narrow tiles)
        assert plane == 0
    fs, h, x = separable_case((81, 81), "c64", seed=181)
    ref = oracle.conv_separable(fs, x)
    pac = pac_mod()
    for forced in (1, 3):  # both tiles give the convolution
        os.environ["PAC_PLANE_K"] = str(forced)
        try:
            plan = pac.Plan((81, 81), 3, "c64")
            try:
                assert plan.query(pac.Q_PLANE) == forced
            finally:
                plan.close()
            check(gpu_conv((81, 81), 3, "c64", h, x), ref, "c64", 81 * 81, f"plane tile {forced}")
        finally:
            del os.environ["PAC_PLANE_K"]


NARROW_SHAPES = [((128, 128, 128), 4, "c64", "1"), ((128, 128, 128), 4, "c64", "0"), ((64, 64), 2, "c128", "0"),
                 ((16, 4096), 2, "c64", "0"), ((25, 25, 25), 5, "c128", "0"), ((27, 81), 3, "c64", "0"),
                 ((8, 32, 32), 8, "c64", "0")]


@pytest.mark.parametrize("dims,radix,dtype,plane", NARROW_SHAPES,
                         ids=[f"{'x'.join(map(str, d))}-r{r}-{t}-plane{p}" for d, r, t, p in NARROW_SHAPES])
def test_narrow_tile_matches_oracle(dims, radix, dtype, plane, monkeypatch):
    """The narrow tile of the group passes (half the columns, PAC_NARROW=1),
    rows and lines layouts, with and without the plane pass: the plan takes
    it for at least one group and the convolution matches the oracle and
    the default tile."""
    pac = pac_mod()
    fs, h, x = separable_case(dims, dtype, seed=7 + dims[-1])
    ref = oracle.conv_separable(fs, x)
    monkeypatch.setenv("PAC_PLANE", plane)
    monkeypatch.setenv("PAC_NARROW", "1")
    plan = pac.Plan(dims, radix, dtype)
    try:
        assert plan.query(pac.Q_NARROW) >= 1
    finally:
        plan.close()
    y = gpu_conv(dims, radix, dtype, h, x)
    check(y, ref, dtype, int(np.prod(dims)), f"narrow {dims}")
    monkeypatch.setenv("PAC_NARROW", "0")
    y0 = gpu_conv(dims, radix, dtype, h, x)
    check(y0, ref, dtype, int(np.prod(dims)), f"default tile {dims}")
    assert oracle.rel_l2(y, y0) <= tol(dtype, int(np.prod(dims)))


def test_narrow_tile_in_a_batch(monkeypatch):
    """Plans with narrow tiles in pac_convolve_many: merged per-level launches
    of the narrow kernels (PAC_BATCH=graph), and the persistent kernel, which
    runs the same passes in its own default tiles."""
    pac = pac_mod()
    monkeypatch.setenv("PAC_NARROW", "1")
    monkeypatch.setenv("PAC_PLANE", "0")
    cases = [((128, 128), 2, 11), ((64, 64), 8, 12), ((4096,), 2, 13), ((27, 81), 3, 14)]
    plans, xs, ys, refs = [], [], [], []
    try:
        for dims, radix, seed in cases:
            fs, h, x = separable_case(dims, "c64", seed)
            p = pac.Plan(dims, radix, "c64")
            p.filter_spectrum(dev(h))
            plans.append(p)
            xs.append(dev(x))
            ys.append(torch.empty_like(xs[-1]))
            refs.append(oracle.conv_separable(fs, x))
        assert sum(p.query(pac.Q_NARROW) for p in plans) >= 1
        for batch in ("graph", "persistent"):
            monkeypatch.setenv("PAC_BATCH", batch)
            for rep in range(2):
                for y in ys:
                    y.fill_(float("nan"))
                pac.pac_convolve_many([p.handle for p in plans], xs, ys)
                torch.cuda.synchronize()
                for y, ref, (dims, _, _) in zip(ys, refs, cases):
                    check(y.cpu().numpy(), ref, "c64", int(np.prod(dims)), f"many narrow {batch} {dims} rep {rep}")
        # a narrow forward / inverse pass (axis 0) with a default-tile fused pass: the persistent
        # kernel takes the batch (one launch) in its own tiles
        dims = (128, 512)
        fs, h, x = separable_case(dims, "c64", 15)
        p = pac.Plan(dims, 2, "c64")
        plans.append(p)
        p.filter_spectrum(dev(h))
        assert p.query(pac.Q_NARROW) == 1
        assert pac.pac_convolve_many_launches([p.handle, p.handle]) == 1
        xd = dev(x)
        yd = [torch.full_like(xd, float("nan")) for _ in range(2)]
        pac.pac_convolve_many([p.handle, p.handle], [xd, xd], yd)
        torch.cuda.synchronize()
        ref = oracle.conv_separable(fs, x)
        for y in yd:
            check(y.cpu().numpy(), ref, "c64", int(np.prod(dims)), "persistent, narrow axis-0 passes")
    finally:
        for p in plans:
            p.close()


def test_tune_file_narrow_flag(tmp_path):
    """A tune-file line with flags bit 2 set makes later plans of that problem
    take the narrow tile; the tuner's own run on the same problem records a
    valid line, and its schedule matches the oracle."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(__file__))
    path = tmp_path / "tune.txt"
    # ndim n0 n1 n2 radix dtype cap flags us: 128^3 radix 4 c64, cap 0 (none), plane on, narrow
    path.write_text("3 128 128 128 4 0 0 5 1.0\n")
    env = dict(os.environ, PAC_TUNE_FILE=str(path))
    code = ("import paper_2506_12718_gb300 as pac; pac.load(); import torch; torch.cuda.init(); "
            "p = pac.Plan((128, 128, 128), 4, 'c64'); print(p.query(pac.Q_NARROW), p.query(pac.Q_PLANE)); p.close()")
    out = subprocess.run([sys.executable, "-c", code], env=env, check=True, capture_output=True, text=True, cwd=root)
    nv, plane = map(int, out.stdout.strip().splitlines()[-1].split())
    assert nv >= 1 and plane >= 1
    path2 = tmp_path / "tune2.txt"
    env2 = dict(os.environ, PAC_TUNE_FILE=str(path2))
    code1 = ("import paper_2506_12718_gb300 as pac; pac.load(); import torch; torch.cuda.init(); "
             "print(pac.pac_tune((64, 64, 64), 4, 'c64', 3))")
    subprocess.run([sys.executable, "-c", code1], env=env2, check=True, cwd=root)
    line = path2.read_text().split()
    assert len(line) == 9 and line[1] == "64" and int(line[7]) & ~0xF7 == 0


DF_SHAPES = [((4096,), 2), ((3125,), 5), ((2187,), 3), ((25, 125), 5), ((81, 81), 3), ((64, 64, 64), 4),
             ((2, 1024), 2), ((27, 9, 3), 3), ((16384, 2), 2)]


@pytest.mark.parametrize("dims,radix", DF_SHAPES, ids=[f"{'x'.join(map(str, d))}-r{r}" for d, r in DF_SHAPES])
def test_double_float_plans_match_the_oracle_and_fp64(dims, radix):
    """PAC_C128_DF: complex FP64 arrays in and out, double-float arithmetic
    inside; against the oracle within the FP64 bound, and against the plain
    FP64 plan on the same inputs; the device and host-buffer calls agree."""
    pac = pac_mod()
    fs, h, x = separable_case(dims, "c128", seed=31 + dims[0])
    ref = oracle.conv_separable(fs, x)
    n = int(np.prod(dims))
    y = gpu_conv(dims, radix, "c128df", h, x)
    check(y, ref, "c128df", n, f"df {dims}")
    y64 = gpu_conv(dims, radix, "c128", h, x)
    assert oracle.rel_l2(y, y64) <= tol("c128df", n)
    plan = pac.Plan(dims, radix, "c128df")
    try:
        assert plan.query(pac.Q_PLANE) == 0
        plan.filter_spectrum(dev(h))
        xh = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        pac.pac_convolve_host(plan.handle, xh, yh)
        assert np.array_equal(yh.numpy(), y)
    finally:
        plan.close()


def test_double_float_large_host_buffers_in_column_blocks():
    """3125^2 in double-float, device call and the host-buffer call (column
    blocks: the first pass reads complex FP64 blocks in place, the last writes
    them): both against the oracle, equal bit for bit."""
    pac = pac_mod()
    dims = (3125, 3125)
    fs, h, x = separable_case(dims, "c128", seed=5)
    ref = oracle.conv_separable(fs, x)
    y = gpu_conv(dims, 5, "c128df", h, x)
    check(y, ref, "c128df", 3125 * 3125, "df 3125^2")
    plan = pac.Plan(dims, 5, "c128df")
    try:
        plan.filter_spectrum(dev(h))
        xh = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        pac.pac_convolve_host(plan.handle, xh, yh)
        assert np.array_equal(yh.numpy(), y)
    finally:
        plan.close()


def test_double_float_entry_points_and_queue():
    """Entry points that do not take double-float plans say so (PAC_ERR_ARG);
    the request queue runs them (same result as pac_convolve)."""
    pac = pac_mod()
    dims = (243, 27)
    fs, h, x = separable_case(dims, "c128", seed=9)
    plan = pac.Plan(dims, 3, "c128df")
    try:
        plan.filter_spectrum(dev(h))
        xd = dev(x)
        y = plan.convolve(xd)
        torch.cuda.synchronize()
        check(y.cpu().numpy(), oracle.conv_separable(fs, x), "c128df", 243 * 27, "df queue case")
        yp = torch.empty_like(xd)
        for call in (lambda: plan.convolve_permuted(xd),
                     lambda: pac.pac_convolve_many([plan.handle], [xd], [yp]),
                     lambda: pac.pac_forward_unordered(plan.handle, xd, yp)):
            with pytest.raises(pac.PacError) as ei:
                call()
            assert ei.value.status == pac.Status.ERR_ARG
        q = pac.pac_queue_create(1 << 30, 2)
        try:
            yq = torch.empty_like(xd)
            t = pac.pac_submit(q, plan.handle, xd, yq)
            pac.pac_queue_drain(q)
            assert pac.pac_poll(q, t)[0] == pac.Status.OK
            assert torch.equal(yq, y)
        finally:
            pac.pac_queue_destroy(q)
    finally:
        plan.close()


def test_tune_search_at_plan_creation_and_plan_log():
    """PAC_TUNE=search tunes a problem when its first plan is made; PAC_LOG=1
    prints the plan's pass schedule."""
    import subprocess
    import sys
    env = dict(os.environ, PAC_TUNE="search", PAC_LOG="1")
    env.pop("PAC_TUNE_FILE", None)
    code = ("import paper_2506_12718_gb300 as pac; pac.load(); import torch; torch.cuda.init(); "
            "p = pac.Plan((64, 64, 64), 2, 'c64'); print('cap', p.query(pac.Q_GROUP_CAP)); p.close()")
    out = subprocess.run([sys.executable, "-c", code], env=env, check=True, capture_output=True, text=True,
                         cwd=os.path.dirname(os.path.dirname(__file__)))
    cap = int(out.stdout.strip().splitlines()[-1].split()[1])
    assert cap >= 1  # a tuned schedule (an untuned plan reports 0)
    assert "pac: plan dims 64 64 64 radix 2 c64" in out.stderr


def _queue_setup(n_req=24):
    pac = pac_mod()
    shapes = [((4096,), 2), ((81, 81), 3), ((32, 32, 32), 2), ((125, 25), 5), ((1024,), 4)]
    plans = {}
    reqs = []
    for i in range(n_req):
        dims, radix = shapes[i % len(shapes)]
        dtype = "c64" if i % 3 else "c128"
        key = (dims, radix, dtype)
        if key not in plans:
            _, h, _ = separable_case(dims, dtype, 40 + len(plans))
            p = pac.Plan(dims, radix, dtype)
            p.filter_spectrum(dev(h))
            plans[key] = p
        x = pin.as_dtype(pin.complex_normal(dims, 1000 + i), dtype)
        reqs.append((plans[key], dev(x)))
    return plans, reqs


def test_queue_alone_and_in_the_mix_agree():
    """Continuous batching: each result is the same alone and in the mix."""
    pac = pac_mod()
    plans, reqs = _queue_setup()
    try:
        alone = []
        for p, x in reqs:
            y = p.convolve(x)
            torch.cuda.synchronize()
            alone.append(y.cpu().numpy())
        q = pac.pac_queue_create(1 << 30, 6)
        ys = [torch.empty_like(x) for _, x in reqs]
        tickets = [pac.pac_submit(q, p.handle, x, y) for (p, x), y in zip(reqs, ys)]
        pac.pac_queue_drain(q, 60000)
        lats = []
        for t in tickets:
            st, lat = pac.pac_poll(q, t)
            assert st == pac.Status.OK
            lats.append(lat)
        with pytest.raises(pac.PacError) as ei:
            pac.pac_poll(q, tickets[0])
        assert ei.value.status == pac.Status.ERR_NOT_FOUND
        pac.pac_queue_destroy(q)
        for a, y, (p, _) in zip(alone, ys, reqs):
            got = y.cpu().numpy()
            dtype = p.dtype
            assert oracle.rel_l2(got, a) <= tol(dtype, got.size)
        assert all(lat > 0 for lat in lats)
    finally:
        for p in plans.values():
            p.close()


def test_mixed_radix_host_buffers_and_queue():
    """Mixed-radix plans through the host-buffer call and the request queue."""
    pac = pac_mod()
    cases = [((60, 90), "c64"), ((1000,), "c128"), ((12, 20, 30), "c64")]
    plans, xs, refs = [], [], []
    try:
        for i, (dims, dtype) in enumerate(cases):
            fs, h, x = separable_case(dims, dtype, seed=60 + i)
            p = pac.Plan(dims, 0, dtype)
            p.filter_spectrum(dev(h))
            plans.append(p)
            xs.append(x)
            refs.append(oracle.conv_separable(fs, x))
        for p, x, ref, (dims, dtype) in zip(plans, xs, refs, cases):
            xh = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
            yh = torch.empty_like(xh).pin_memory()
            pac.pac_convolve_host(p.handle, xh, yh)
            torch.cuda.synchronize()
            check(yh.numpy(), ref, dtype, x.size, f"host {dims}")
        q = pac.pac_queue_create(1 << 30, 4)
        xd = [dev(x) for x in xs]
        ys = [torch.empty_like(x) for x in xd]
        tickets = [pac.pac_submit(q, p.handle, x, y) for p, x, y in zip(plans, xd, ys)]
        pac.pac_queue_drain(q, 60000)
        for t in tickets:
            assert pac.pac_poll(q, t)[0] == pac.Status.OK
        pac.pac_queue_destroy(q)
        for y, ref, (dims, dtype) in zip(ys, refs, cases):
            check(y.cpu().numpy(), ref, dtype, ref.size, f"queue {dims}")
    finally:
        for p in plans:
            p.close()


def test_served_workload_sample_matches_oracle():
    """Requests drawn from the serving workload's recipe (1-D/2-D/3-D, radix 2
    or 3, FP32 and FP64, Gaussian / exponential filters from the pool), kept
    to at most 2^16 elements, pushed through the queue together; each result
    is checked against the direct definition (O1) at 32 seeded points."""
    pac = pac_mod()
    reqs = pin.c5_requests(0.02, max_elems=1 << 16)[:32]
    assert len(reqs) >= 16
    pool = pin.c5_filter_pool()
    plans, items = {}, []
    try:
        for i, r in enumerate(reqs):
            c = r.conv
            kind, param = pool[r.filter_id]
            fs = pin.gaussian_factors(c.dims, param) if kind == "gauss" else pin.exponential_factors(c.dims, param)
            h = pin.as_dtype(pin.outer(fs), c.dtype)
            key = (c.dims, c.radix, c.dtype, r.filter_id)
            if key not in plans:
                p = pac.Plan(c.dims, c.radix, c.dtype)
                p.filter_spectrum(dev(h))
                plans[key] = p
            x = pin.make_x(c)
            xd = dev(x)
            items.append((plans[key], c, h, x, xd, torch.empty_like(xd)))
        q = pac.pac_queue_create(1 << 30, 8)
        tickets = [pac.pac_submit(q, p.handle, xd, yd) for p, _, _, _, xd, yd in items]
        pac.pac_queue_drain(q, 60000)
        for t in tickets:
            assert pac.pac_poll(q, t)[0] == pac.Status.OK
        pac.pac_queue_destroy(q)
        for i, (_, c, h, x, _, yd) in enumerate(items):
            idx = pin.sample_points(c.n_total, 32, seed=900 + i)
            ref = oracle.conv_direct_points(h, x, idx)
            got = yd.cpu().numpy().reshape(-1)[idx]
            assert oracle.rel_l2(got, ref) <= tol(c.dtype, c.n_total), f"request {i} {c.dims} {c.dtype}"
    finally:
        for p in plans.values():
            p.close()


def test_queue_injected_launch_failure_isolated(monkeypatch):
    pac = pac_mod()
    plans, reqs = _queue_setup(8)
    monkeypatch.setenv("PAC_FAULT", "launch:3")
    try:
        q = pac.pac_queue_create(1 << 30, 2)
        monkeypatch.delenv("PAC_FAULT")
        ys = [torch.empty_like(x) for _, x in reqs]
        tickets = [pac.pac_submit(q, p.handle, x, y) for (p, x), y in zip(reqs, ys)]
        pac.pac_queue_drain(q, 60000)
        failed = 0
        for i, t in enumerate(tickets):
            try:
                st, _ = pac.pac_poll(q, t)
                assert st == pac.Status.OK
            except pac.PacError as e:
                assert e.status == pac.Status.ERR_CUDA and i == 2
                failed += 1
        assert failed == 1
        pac.pac_queue_destroy(q)
    finally:
        for p in plans.values():
            p.close()


def test_queue_tiny_budget_serialises_but_completes():
    pac = pac_mod()
    plans, reqs = _queue_setup(6)
    try:
        q = pac.pac_queue_create(1024, 4)  # smaller than any request: one at a time
        ys = [torch.empty_like(x) for _, x in reqs]
        tickets = [pac.pac_submit(q, p.handle, x, y) for (p, x), y in zip(reqs, ys)]
        pac.pac_queue_drain(q, 60000)
        for t in tickets:
            assert pac.pac_poll(q, t)[0] == pac.Status.OK
        pac.pac_queue_destroy(q)
    finally:
        for p in plans.values():
            p.close()


@pytest.mark.parametrize("dims,radix,dtype", [((128, 128, 128), 4, "c64"), ((243, 243), 3, "c64"),
                                             ((64, 64, 64), 2, "c128"), ((1024, 1024), 8, "c64")])
def test_single_launch_repeatable_and_barrier_clean(dims, radix, dtype, monkeypatch):
    """The whole convolution as one cooperative launch (opt-in per plan): 30
    back-to-back runs are bit-identical (deterministic kernels, no stale data
    across the phases), match the oracle, and no bounded barrier wait gave up."""
    pac = pac_mod()
    fs, h, x = separable_case(dims, dtype, seed=21)
    monkeypatch.setenv("PAC_SINGLE_LAUNCH", "1")
    monkeypatch.setenv("PAC_PLANE", "0")  # the single launch runs the per-axis pass sequence
    plan = pac.Plan(dims, radix, dtype)
    monkeypatch.delenv("PAC_SINGLE_LAUNCH")
    monkeypatch.delenv("PAC_PLANE")
    try:
        plan.filter_spectrum(dev(h))
        xd = dev(x)
        ys = [torch.empty_like(xd) for _ in range(30)]
        for y in ys:
            plan.convolve(xd, y)
        torch.cuda.synchronize()
        first = ys[0].cpu().numpy()
        for y in ys[1:]:
            assert np.array_equal(y.cpu().numpy(), first)
        assert plan.query(pac.Q_DEVICE_ERROR) == 0
        assert plan.query(pac.Q_LAUNCHES_CONVOLVE) == 1
    finally:
        plan.close()
    check(first, oracle.conv_separable(fs, x), dtype, int(np.prod(dims)), "single launch")


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_bounded_barrier_wait_runs_out_and_reports(dtype):
    """The grid barrier of the single-launch kernel waits with a bound: with a
    target no launch reaches (one arrival more than the grid makes) and a
    limit of 64 polls, every wait runs out.  The kernel still ends promptly,
    the device error word reads 1 (and 0 once read), and the next ordinary
    convolution on the same context matches the oracle."""
    pac = pac_mod()
    dims = (1 << 16,)
    h = pin.as_dtype(pin.complex_uniform(dims, 31), dtype)
    x = pin.as_dtype(pin.complex_uniform(dims, 32), dtype)
    plan = pac.Plan(dims, 2, dtype)
    try:
        plan.filter_spectrum(dev(h))
        xd = dev(x)
        y = torch.empty_like(xd)
        assert plan.query(pac.Q_DEVICE_ERROR) == 0
        t0 = time.perf_counter()
        pac.pac_test_barrier_timeout(plan.handle, xd, y, 64)
        torch.cuda.synchronize()
        assert time.perf_counter() - t0 < 10.0
        assert plan.query(pac.Q_DEVICE_ERROR) == 1
        assert plan.query(pac.Q_DEVICE_ERROR) == 0
        with pytest.raises(pac.PacError) as ei:
            pac.pac_test_barrier_timeout(plan.handle, xd, y, 0)
        assert ei.value.status == pac.Status.ERR_ARG
        plan.convolve(xd, y)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert plan.query(pac.Q_DEVICE_ERROR) == 0
    finally:
        plan.close()
    pts = pin.sample_points(int(np.prod(dims)), 1024, 33)
    err = oracle.rel_l2(got.reshape(-1)[pts], oracle.conv_direct_points(h, x, pts))
    tol = 1e-12 if dtype == "c128" else 1e-5 * math.log2(np.prod(dims))
    assert err <= tol, f"after a timed-out launch: rel_l2 {err:.3e} > {tol:.1e}"



PERSIST_CASES = [((4096,), 2, 1), ((27, 81), 3, 2), ((64, 64), 8, 3), ((3125,), 5, 4), ((32, 32, 32), 4, 5),
                 ((128, 128), 2, 6), ((1 << 16,), 2, 7), ((2187,), 3, 8), ((1024, 1024), 2, 9), ((729, 9), 3, 10)]


def test_persistent_batch_is_one_launch_and_matches_the_merged_form(monkeypatch):
    """A batch whose passes all have shapes the persistent kernel carries runs
    as one launch (replayed from a graph): every instance matches the oracle,
    the same batch in the merged-launch form (PAC_BATCH=graph) to rounding,
    and a second call (the replay, counters reset by the kernel) gives the
    same result bit for bit.  (The default tiles: a schedule tuned earlier in
    the process may otherwise give a fused pass the narrow tile, which the
    persistent kernel does not carry.)"""
    pac = pac_mod()
    monkeypatch.setenv("PAC_NARROW", "0")
    plans, xs, refs = [], [], []
    try:
        for dims, radix, seed in PERSIST_CASES:
            fs, h, x = separable_case(dims, "c64", seed)
            p = pac.Plan(dims, radix, "c64")
            p.filter_spectrum(dev(h))
            plans.append(p)
            xs.append(dev(x))
            refs.append(oracle.conv_separable(fs, x))
        handles = [p.handle for p in plans] * 2
        xs2 = xs * 2
        assert pac.pac_convolve_many_launches(handles) == 1
        ys = [torch.full_like(x, float("nan")) for x in xs2]
        pac.pac_convolve_many(handles, xs2, ys)
        torch.cuda.synchronize()
        first = [y.cpu().numpy() for y in ys]
        pac.pac_convolve_many(handles, xs2, ys)  # replay
        torch.cuda.synchronize()
        for k, y in enumerate(ys):
            assert np.array_equal(y.cpu().numpy(), first[k])
        monkeypatch.setenv("PAC_BATCH", "graph")
        assert pac.pac_convolve_many_launches(handles) > 1
        yg = [torch.empty_like(x) for x in xs2]
        pac.pac_convolve_many(handles, xs2, yg)
        torch.cuda.synchronize()
        monkeypatch.delenv("PAC_BATCH")
        for k in range(len(handles)):
            dims = PERSIST_CASES[k % len(PERSIST_CASES)][0]
            n = int(np.prod(dims))
            check(first[k], refs[k % len(PERSIST_CASES)], "c64", n, f"persistent {dims}")
            assert oracle.rel_l2(first[k], yg[k].cpu().numpy()) <= tol("c64", n)
        assert plans[0].query(pac.Q_DEVICE_ERROR) == 0
    finally:
        for p in plans:
            p.close()


def test_persistent_batch_bounded_wait_runs_out_and_reports():
    """The persistent kernel's dependency waits are bounded: with every
    target one tile beyond what the pass before has and a limit of about
    200 us, each dependent wait runs out; the launch ends, the device error
    word reads 1 (then 0), and the next ordinary batch matches the oracle."""
    pac = pac_mod()
    cases = [((1 << 16,), 2, 21), ((32, 32, 32), 4, 22), ((27, 81), 3, 23)]
    plans, xs, refs = [], [], []
    try:
        for dims, radix, seed in cases:
            fs, h, x = separable_case(dims, "c64", seed)
            p = pac.Plan(dims, radix, "c64")
            p.filter_spectrum(dev(h))
            plans.append(p)
            xs.append(dev(x))
            refs.append(oracle.conv_separable(fs, x))
        handles = [p.handle for p in plans]
        ys = [torch.empty_like(x) for x in xs]
        assert plans[0].query(pac.Q_DEVICE_ERROR) == 0
        t0 = time.perf_counter()
        pac.pac_test_batch_timeout(handles, xs, ys, 200)
        assert time.perf_counter() - t0 < 30.0
        assert plans[0].query(pac.Q_DEVICE_ERROR) == 1
        assert plans[0].query(pac.Q_DEVICE_ERROR) == 0
        pac.pac_convolve_many(handles, xs, ys)
        torch.cuda.synchronize()
        for y, ref, (dims, _, _) in zip(ys, refs, cases):
            check(y.cpu().numpy(), ref, "c64", int(np.prod(dims)), f"after timeouts {dims}")
        assert plans[0].query(pac.Q_DEVICE_ERROR) == 0
    finally:
        for p in plans:
            p.close()
