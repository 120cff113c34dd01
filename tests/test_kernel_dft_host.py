"""CPU tests of the kernels' own in-register DFT code (no GPU).

csrc/fft_device.cuh's dft<R, INV, V> templates (the factored twiddles, the
stage-2 butterflies with the twiddles' real factors folded into their
constants, the FP32 plain-twiddle splits, and every radix the pass kernels
use: 2, 3, 4, 5, 8, 9, 16, 25, 27, 32) are compiled for the host
(tests/c/dft_host.cpp gives the device intrinsics host definitions with the
same IEEE rounding) for complex FP32, complex FP64 and double-float
elements, and compared with numpy's FFT on random vectors and on every
basis vector (a wrong constant or a wrong output slot anywhere shows):
FP32 within 2.5e-6 log2 R, FP64 within 4e-15 log2 R, double-float within
2e-14 (its inputs carry the 48-bit split of the FP64 values).
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
RADICES = [2, 3, 4, 5, 8, 9, 16, 25, 27, 32]
TYPES = {"c64": (0, 2.5e-6), "c128": (1, 4e-15), "c128df": (2, 2e-14)}


@pytest.fixture(scope="module")
def dft_host():
    if not shutil.which("g++") or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = os.path.join(tempfile.mkdtemp(), "dft_host")
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-I", CUDA_INC, "-I",
                    os.path.join(ROOT, "paper_2506_12718_gb300", "csrc"), os.path.join(ROOT, "tests", "c", "dft_host.cpp"),
                    "-o", exe], check=True, capture_output=True)

    def run(code, R, inv, vectors):
        lines = [f"{code} {R} {inv} " + " ".join(float(v).hex() for c in x for v in (c.real, c.imag)) for x in vectors]
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
        res = []
        for ln in out.strip().splitlines():
            t = [float.fromhex(s) for s in ln.split()]
            res.append(np.array(t[0::2]) + 1j * np.array(t[1::2]))
        return res
    return run


@pytest.mark.parametrize("dtype", list(TYPES))
@pytest.mark.parametrize("R", RADICES)
@pytest.mark.parametrize("inv", [0, 1])
def test_kernel_dft_is_the_dft(dft_host, dtype, R, inv):
    code, tol = TYPES[dtype]
    rng = np.random.default_rng(1000 * R + 10 * inv + code)
    rand = [rng.standard_normal(R) + 1j * rng.standard_normal(R) for _ in range(4)]
    basis = [np.eye(R)[k].astype(complex) for k in range(R)]
    got = dft_host(code, R, inv, rand + basis)
    F = np.exp((2j if inv else -2j) * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
    bound = tol * max(1.0, np.log2(R)) if dtype != "c128df" else tol
    for x, y in zip(rand + basis, got):
        want = F @ x
        assert np.linalg.norm(y - want) <= bound * np.linalg.norm(want), (dtype, R, inv)
