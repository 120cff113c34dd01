"""The allocation-free permuted convolution against the ordinary permuted one.

pac_convolve_permuted_noalloc serves callers that cannot allocate device
memory (their GPU memory is owned by another allocator, or capped by a quota,
or their path cannot tolerate cudaMalloc's synchronisation): its scratch is a
fixed 8 MiB static buffer inside the library.  This file is collected last
(tests/test_zz_*) so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import math
import os

import numpy as np
import pytest

import pac_inputs as pin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pac():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_12718_gb300 import _build
    _build.build()
    import paper_2506_12718_gb300 as pac
    pac.load()
    return pac


def rel_l2(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims,radix,dtype", [((64, 64, 64), 4, "c64"), ((243, 81), 3, "c128"),
                                             ((1024, 1024), 8, "c64"), ((3125,), 5, "c128"),
                                             ((60, 90), 0, "c128"), ((1000,), 0, "c64"), ((360,), -1, "c64")])
def test_noalloc_matches_permuted_twice(pac, dims, radix, dtype):
    tol = 1e-12 if dtype == "c128" else 1e-5 * math.log2(int(np.prod(dims)))
    h = pin.as_dtype(pin.complex_uniform(dims, 31), dtype)
    x = pin.as_dtype(pin.complex_normal(dims, 32), dtype)
    if radix == -1:  # a mixed group (runtime-radix kernel)
        os.environ["PAC_MIXED"] = "1"
        try:
            plan = pac.Plan(dims, 0, dtype)
        finally:
            del os.environ["PAC_MIXED"]
    else:
        plan = pac.Plan(dims, radix, dtype)
    try:
        plan.filter_spectrum(torch.from_numpy(h).cuda())
        xd = torch.from_numpy(x).cuda()
        ref = plan.convolve_permuted(xd)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
        for _ in range(2):  # two calls in a row share the static scratch
            y = torch.full_like(xd, float("nan"))
            pac.pac_convolve_permuted_noalloc(plan.handle, xd, y)
            torch.cuda.synchronize()
            assert rel_l2(y.cpu().numpy(), ref) <= tol
        yi = xd.clone()  # in place
        pac.pac_convolve_permuted_noalloc(plan.handle, yi, yi)
        torch.cuda.synchronize()
        assert rel_l2(yi.cpu().numpy(), ref) <= tol
    finally:
        plan.close()


@pytest.mark.parametrize("dims,radix,dtype", [((27, 81), 3, "c128"), ((32, 16, 8), 2, "c64")])
def test_noalloc_matches_the_oracle(pac, dims, radix, dtype):
    """The allocation-free form against the FP64 oracle directly (the
    definition of the convolution, route O1), on two calls in a row."""
    import oracle
    tol = 1e-12 if dtype == "c128" else 1e-5 * math.log2(int(np.prod(dims)))
    h = pin.as_dtype(pin.complex_uniform(dims, 41), dtype)
    x = pin.as_dtype(pin.complex_normal(dims, 42), dtype)
    ref = oracle.conv_direct(h, x)
    plan = pac.Plan(dims, radix, dtype)
    try:
        plan.filter_spectrum(torch.from_numpy(h).cuda())
        xd = torch.from_numpy(x).cuda()
        for _ in range(2):
            y = torch.full_like(xd, float("nan"))
            pac.pac_convolve_permuted_noalloc(plan.handle, xd, y)
            torch.cuda.synchronize()
            assert oracle.rel_l2(y.cpu().numpy(), ref) <= tol
    finally:
        plan.close()


def test_noalloc_rejects_plans_above_the_static_buffer(pac):
    plan = pac.Plan((128, 128, 128), 2, "c64")  # 16 MiB > 8 MiB
    try:
        x = torch.zeros(128, 128, 128, dtype=torch.complex64, device="cuda")
        plan.filter_spectrum(x)
        with pytest.raises(pac.PacError) as ei:
            pac.pac_convolve_permuted_noalloc(plan.handle, x, x)
        assert ei.value.status == pac.Status.ERR_SIZE
        assert "static buffer" in str(ei.value)
    finally:
        plan.close()
