"""CPU emulation of the pass kernels against the FP64 oracle (no GPU).

tests/c/emulate.cpp builds the kernels' own device code (csrc/fft_device.cuh:
run_phase, the rounds, the placement tables' use, the spectrum order and the
double-float loads and stores) for the host and runs each pass as one CTA of
NT host threads (__syncthreads a barrier of those threads, the exchange
buffer in host memory), driven by the library's step records
(pac_test_host_steps: the plan builder's groups, tables and pass arguments).
So the whole convolution path, apart from the launch and the hardware, is
checked on the CPU: complex FP32, FP64 and double-float, 1-D to 3-D, rows
and lines passes, fused single-group plans, external twiddles (a group cap
that splits an axis), the plane pass with one CTA per plane (complex FP32
and FP64), the compiled groups spanning prime bases (48, 120, 1000) and the
runtime-radix kernel of the other groups spanning bases.  Results against the oracle (O2, separable
filters) within the GPU tests' tolerances.

PAC_EMULATE_SANITIZE=1 in the environment builds the emulator with
AddressSanitizer and UndefinedBehaviorSanitizer (about ten minutes of
compilation): every access of the kernels' code to the arrays, tables and
exchange buffer is then checked on the CPU.
"""
import glob
import hashlib
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import pac_inputs as pin

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
PKG = os.path.join(ROOT, "paper_2506_12718_gb300")
CODES = {"c64": 0, "c128": 1, "c128df": 2}

CASES = [((25, 125), 5, 0), ((64, 32), 4, 0), ((27, 81), 3, 0), ((2048,), 2, 0), ((3, 9, 27), 3, 0),
         ((3125,), 5, 2), ((4096,), 4, 3), ((5, 25, 5), 5, 0), ((2, 8, 16), 2, 0)]
# plane passes (one CTA per plane): 3-D with the two innermost axes as planes, and an n x 2 shape
PLANE_CASES = [((4, 64, 64), 4, "c64"), ((2, 128, 128), 2, "c64"), ((3, 27, 27), 3, "c64"), ((5, 25, 25), 5, "c64"),
               ((128, 2), 2, "c64"), ((4, 64, 64), 2, "c128"), ((3, 27, 27), 3, "c128"), ((25, 25), 5, "c128"),
               ((128, 2), 2, "c128")]


@pytest.fixture(scope="module")
def emulate():
    if not shutil.which("g++") or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    from paper_2506_12718_gb300 import _build
    _build.build()
    sanitize = os.environ.get("PAC_EMULATE_SANITIZE") == "1"
    san = ["-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined"] if sanitize else []
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0") if sanitize else None
    # the emulator is rebuilt only when its sources change (it links libpac.so at run time)
    h = hashlib.sha256(" ".join(san).encode())
    srcs = [os.path.join(ROOT, "tests", "c", "emulate.cpp"), os.path.join(ROOT, "include", "pac.h")]
    srcs += sorted(glob.glob(os.path.join(PKG, "csrc", "*.cuh")) + glob.glob(os.path.join(PKG, "csrc", "*.h")))
    for f in srcs:
        h.update(open(f, "rb").read())
    cache = os.path.join(PKG, "_build")
    os.makedirs(cache, exist_ok=True)
    exe = os.path.join(cache, "emulate_" + h.hexdigest()[:16])
    if not os.path.exists(exe):
        tmp = exe + ".tmp%d" % os.getpid()
        r = subprocess.run(["g++", "-O1"] + san + ["-std=c++20", "-ffp-contract=off", "-pthread", "-I", CUDA_INC, "-I",
                            os.path.join(ROOT, "include"), "-I", os.path.join(PKG, "csrc"), srcs[0], "-L", PKG,
                            "-lpac", "-Wl,-rpath," + PKG, "-o", tmp], capture_output=True, text=True)
        if r.returncode:
            pytest.fail("emulator build failed:\n" + r.stderr[-2000:])
        os.replace(tmp, exe)

    def run(dims, radix, dtype, cap, h, x, flags=0):
        d = tempfile.mkdtemp()
        hf, xf, yf = (os.path.join(d, n) for n in ("h", "x", "y"))
        h.tofile(hf)
        x.tofile(xf)
        args = ([exe, str(CODES[dtype]), str(radix), str(cap), str(flags), str(len(dims))] + [str(v) for v in dims] +
                [hf, xf, yf])
        r = subprocess.run(args, capture_output=True, text=True, timeout=600, env=env)
        assert r.returncode == 0, r.stderr
        return np.fromfile(yf, dtype=x.dtype).reshape(dims)
    return run


def tol(dtype, n):
    return 1e-12 if dtype in ("c128", "c128df") else 1e-5 * max(1.0, math.log2(n))


@pytest.mark.parametrize("dtype", list(CODES))
@pytest.mark.parametrize("dims,radix,cap", CASES, ids=[f"{'x'.join(map(str, d))}-r{r}-cap{c}" for d, r, c in CASES])
def test_emulated_kernels_match_the_oracle(emulate, dims, radix, cap, dtype):
    seed = 17 + dims[0]
    fs = [pin.complex_uniform((n,), seed + 100 + a) for a, n in enumerate(dims)]
    store = "c64" if dtype == "c64" else "c128"
    h = pin.as_dtype(pin.outer(fs), store)
    x = pin.as_dtype(pin.complex_uniform(dims, seed), store)
    y = emulate(dims, radix, dtype, cap, h, x)
    ref = oracle.conv_separable(fs, x)
    n = int(np.prod(dims))
    err = oracle.rel_l2(y, ref)
    assert err <= tol(dtype, n), f"{dims} r{radix} cap {cap} {dtype}: rel_l2 {err:.3e}"
    if dtype == "c128df":  # a different arithmetic from FP64, within the same bound
        assert err > 0


MIXED_CASES = [((120, 120), "c64"), ((1000,), "c128"), ((48, 125), "c64"), ((120, 8), "c128"), ((1000, 3), "c64")]


@pytest.mark.parametrize("dims,dtype", MIXED_CASES, ids=[f"{'x'.join(map(str, d))}-{t}" for d, t in MIXED_CASES])
def test_emulated_compiled_mixed_groups_match_the_oracle(emulate, dims, dtype):
    """Groups spanning prime bases with compiled kernels (48, 120, 1000 points;
    mixed radix, radix 0), against the oracle."""
    seed = 41 + dims[0]
    fs = [pin.complex_uniform((n,), seed + 100 + a) for a, n in enumerate(dims)]
    h = pin.as_dtype(pin.outer(fs), dtype)
    x = pin.as_dtype(pin.complex_uniform(dims, seed), dtype)
    y = emulate(dims, 0, dtype, 0, h, x, flags=2)
    err = oracle.rel_l2(y, oracle.conv_separable(fs, x))
    assert err <= tol(dtype, int(np.prod(dims))), f"mixed {dims} {dtype}: rel_l2 {err:.3e}"


RUNTIME_CASES = [((60, 90), "c64"), ((360,), "c128"), ((12, 20, 30), "c64"), ((2000,), "c64"), ((240, 6), "c128")]


@pytest.mark.parametrize("dims,dtype", RUNTIME_CASES, ids=[f"{'x'.join(map(str, d))}-{t}" for d, t in RUNTIME_CASES])
def test_emulated_runtime_radix_kernel_matches_the_oracle(emulate, dims, dtype):
    """Every group spanning prime bases in the runtime-radix kernel (as
    PAC_MIXED=rt), against the oracle."""
    seed = 53 + dims[0]
    fs = [pin.complex_uniform((n,), seed + 100 + a) for a, n in enumerate(dims)]
    h = pin.as_dtype(pin.outer(fs), dtype)
    x = pin.as_dtype(pin.complex_uniform(dims, seed), dtype)
    y = emulate(dims, 0, dtype, 0, h, x, flags=4)
    err = oracle.rel_l2(y, oracle.conv_separable(fs, x))
    assert err <= tol(dtype, int(np.prod(dims))), f"runtime radix {dims} {dtype}: rel_l2 {err:.3e}"


@pytest.mark.parametrize("dims,radix,dtype", PLANE_CASES, ids=[f"{'x'.join(map(str, d))}-r{r}-{t}" for d, r, t in PLANE_CASES])
def test_emulated_plane_pass_matches_the_oracle(emulate, dims, radix, dtype):
    seed = 29 + dims[-1]
    fs = [pin.complex_uniform((n,), seed + 100 + a) for a, n in enumerate(dims)]
    h = pin.as_dtype(pin.outer(fs), dtype)
    x = pin.as_dtype(pin.complex_uniform(dims, seed), dtype)
    y = emulate(dims, radix, dtype, 0, h, x, flags=1)
    ref = oracle.conv_separable(fs, x)
    n = int(np.prod(dims))
    err = oracle.rel_l2(y, ref)
    assert err <= tol(dtype, n), f"plane {dims} r{radix} {dtype}: rel_l2 {err:.3e}"
