"""CPU tests of the C-ABI library: it loads, exports every declared symbol, and
its host-only rules (stage lists, index-reversal tables) match the oracle's
reading of the paper bit for bit.  No compute call needs a GPU here."""
import os
import re
import time

import numpy as np
import pytest

import paper_2506_12718_gb300 as pac
from oracle import paper_forms as pf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_12718_gb300 import _build
    _build.build()
    pac.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pac_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 20
    lib = pac.load()
    for n in names:
        assert hasattr(lib, n), n
    # and the binding mirrors each name
    for n in names:
        assert callable(getattr(pac, n)), n


def test_version():
    assert "sm_103a" in pac.pac_version()


@pytest.mark.parametrize("n,radix,want", [
    (128, 2, [2] * 7), (128, 4, [4, 4, 4, 2]), (128, 8, [8, 8, 2]), (1024, 4, [4] * 5),
    (2187, 3, [3] * 7), (3125, 5, [5] * 5), (64, 8, [8, 8]), (2, 8, [2]), (1, 2, []), (32, 4, [4, 4, 2]),
    # radix 0: mixed radix (Section 7.1), 2^a as radix-4 stages (a leftover 2 last), then 3s, then 5s
    (1000, 0, [4, 2, 5, 5, 5]), (360, 0, [4, 2, 3, 3, 5]), (128, 0, [4, 4, 4, 2]), (81, 0, [3] * 4),
    (30, 0, [2, 3, 5]), (1, 0, []), (5, 0, [5]), (6000, 0, [4, 4, 3, 5, 5, 5]),
])
def test_stage_list(n, radix, want):
    assert pac.pac_stage_list(n, radix) == want


@pytest.mark.parametrize("n,radix,status", [
    (100, 2, pac.Status.ERR_SIZE), (96, 4, pac.Status.ERR_SIZE), (243, 2, pac.Status.ERR_SIZE),
    (64, 6, pac.Status.ERR_ARG), (64, 7, pac.Status.ERR_ARG), (0, 2, pac.Status.ERR_SIZE),
    (7, 0, pac.Status.ERR_SIZE), (14, 0, pac.Status.ERR_SIZE), (0, 0, pac.Status.ERR_SIZE),
])
def test_stage_list_errors(n, radix, status):
    with pytest.raises(pac.PacError) as ei:
        pac.pac_stage_list(n, radix)
    assert ei.value.status == status
    assert pac.pac_last_error()


STAGE_LISTS = [[2] * 7, [4, 4, 4, 2], [8, 8, 2], [3] * 7, [5] * 5, [2, 4, 4, 4], [2, 8, 8], [2, 3, 4],
               [4] * 5, [8] * 4, [3, 3], [16, 4], [2], [4, 2, 5, 5, 5], [4, 2, 3, 3, 5], [5, 2, 5, 4, 5],
               [3, 5, 2, 3], [5, 3, 4]]


@pytest.mark.parametrize("stages", STAGE_LISTS)
def test_reverse_table_matches_paper_permutation(stages):
    """Bit-exact: the library's position->frequency table equals P^T idx from the
    paper's modulo-r sorts (uniform radix) or perfect shuffles (mixed radix)."""
    got = np.array(pac.pac_reverse_table(stages))
    assert np.array_equal(got, pf.pos_to_freq(stages))


@pytest.mark.parametrize("r,t", [(2, 10), (4, 5), (8, 4), (3, 7), (5, 5)])
def test_reverse_table_is_involution_for_uniform_radix(r, t):
    p = np.array(pac.pac_reverse_table([r] * t))
    assert np.array_equal(p[p], np.arange(r ** t))


def test_plan_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pac.PacError) as ei:
        pac.pac_plan_create(1, [64], 2, pac.C64)
    assert ei.value.status in (pac.Status.ERR_CUDA, pac.Status.ERR_NOMEM)


@pytest.mark.parametrize("dims,stages,status", [
    ([12], [[2, 3]], pac.Status.ERR_SIZE),          # product 6, not 12
    ([14], [[2, 7]], pac.Status.ERR_SIZE),          # 7 is no stage
    ([12], [[6, 2]], pac.Status.ERR_SIZE),          # 6 is not a prime power
    ([64], [[64]], pac.Status.ERR_SIZE),            # a stage above 32
    ([4, 6], [[4], []], pac.Status.ERR_SIZE),       # an empty list for a dim > 1
    ([2, 2, 2, 2], [[2]] * 4, pac.Status.ERR_ARG),  # ndim 4
    ([0], [[]], pac.Status.ERR_SIZE),
])
def test_plan_create_stages_rejects_bad_lists_before_touching_the_device(dims, stages, status):
    with pytest.raises(pac.PacError) as ei:
        pac.pac_plan_create_stages(dims, stages, pac.C64)
    assert ei.value.status == status


def test_plan_create_rejects_arrays_of_2_31_elements_or_more():
    with pytest.raises(pac.PacError) as ei:
        pac.pac_plan_create(3, [2048, 2048, 512], 2, pac.C64)
    assert ei.value.status == pac.Status.ERR_SIZE
    assert "2147483648" in str(ei.value)


@pytest.mark.parametrize("dims,text", [([1 << 30, 1 << 30, 16], "18446744073709551616"),
                                       ([1 << 30, 1 << 30, 2], "2305843009213693952"),
                                       ([1 << 30, 4, 1], "4294967296")])
def test_plan_create_rejects_products_that_overflow_64_bits(dims, text):
    # each dim is in range, but the product of three of them exceeds 2^63: the
    # check must come before the multiply, not after a wrapped product
    t0 = time.perf_counter()
    with pytest.raises(pac.PacError) as ei:
        pac.pac_plan_create(3, dims, 2, pac.C64)
    assert ei.value.status == pac.Status.ERR_SIZE
    assert text in str(ei.value)
    assert time.perf_counter() - t0 < 5.0


def test_plan_create_stages_wants_one_list_per_axis():
    with pytest.raises(ValueError):
        pac.pac_plan_create_stages([4, 6], [[4]], pac.C64)


def test_plan_create_rejects_bad_arguments_before_touching_the_device():
    with pytest.raises(pac.PacError) as ei:
        pac.pac_plan_create(1, [100], 2, pac.C64)
    assert ei.value.status == pac.Status.ERR_SIZE
    with pytest.raises(pac.PacError) as ei:
        pac.pac_plan_create(4, [2, 2, 2, 2], 2, pac.C64)
    assert ei.value.status == pac.Status.ERR_ARG
    with pytest.raises(pac.PacError) as ei:
        pac.pac_plan_create(1, [64], 7, pac.C64)
    assert ei.value.status == pac.Status.ERR_ARG


@pytest.mark.parametrize("n,status", [(7, pac.Status.ERR_SIZE), (0, pac.Status.ERR_SIZE), (1 << 31, pac.Status.ERR_SIZE),
                                      (2 * 7 * 5, pac.Status.ERR_SIZE)])
def test_prime_factor_object_rejects_bad_lengths_before_touching_the_device(n, status):
    with pytest.raises(pac.PacError) as ei:
        pac.pac_pfa_create(n, pac.C64)
    assert ei.value.status == status
    with pytest.raises(pac.PacError) as ei:
        pac.pac_pfa_create(60, 7)
    assert ei.value.status == pac.Status.ERR_ARG


# ---------------------------------------------------------- pass schedule (host only)

@pytest.mark.parametrize("dims,radix,dtype,mixed,cap,want", [
    ((128, 128, 128), 4, 0, False, 0, [(0, 128, [16, 8]), (1, 128, [16, 8]), (2, 128, [16, 8])]),
    ((3125, 3125), 5, 0, False, 0, [(0, 3125, [25, 25, 5]), (1, 3125, [25, 25, 5])]),
    ((2187,), 3, 0, False, 0, [(0, 2187, [27, 9, 9])]),
    ((2187,), 3, 1, False, 0, [(0, 2187, [9, 9, 9, 3])]),             # FP64 rounds of base 3 stop at 9
    ((1 << 20,), 4, 0, False, 0, [(0, 1024, [16, 8, 8]), (0, 1024, [16, 8, 8])]),
    ((1 << 20,), 4, 0, False, 9, [(0, 64, [8, 8]), (0, 64, [8, 8]), (0, 256, [16, 16])]),  # a schedule's cap
    ((4096,), 2, 1, False, 0, [(0, 64, [8, 8]), (0, 64, [8, 8])]),     # FP64 groups stop at 2048
    ((1000,), 0, 0, False, 0, [(0, 8, [8]), (0, 125, [25, 5])]),       # one-base groups (PAC_MIXED=0)
    ((1000,), 0, 0, True, 0, [(0, 1000, [25, 8, 5])]),                 # one group spanning bases
    ((6000,), 0, 0, False, 0, [(0, 16, [16]), (0, 3, [3]), (0, 125, [25, 5])]),
    ((6000,), 0, 0, True, 0, [(0, 6000, [25, 16, 5, 3])]),             # the whole axis: a compiled group
    ((2 ** 10 * 3 ** 5 * 5 ** 3,), 0, 0, True, 0,                       # spanning bases would not be fewer
     [(0, 1024, [16, 8, 8]), (0, 243, [27, 9]), (0, 125, [25, 5])]),
    # the default rule: groups spanning bases where each has a compiled kernel (48, 120, 1000 points)
    ((1000,), 0, 0, None, 0, [(0, 1000, [25, 8, 5])]),
    ((1000,), 0, 1, None, 0, [(0, 1000, [25, 8, 5])]),
    ((6000,), 0, 0, None, 0, [(0, 6000, [25, 16, 5, 3])]),
    ((6000,), 0, 0, True, 9, [(0, 48, [16, 3]), (0, 125, [25, 5])]),  # a cap: groups of at most 2048
    ((120, 120), 0, 0, None, 0, [(0, 120, [8, 5, 3]), (1, 120, [8, 5, 3])]),
    ((360,), 0, 0, None, 0, [(0, 8, [8]), (0, 9, [9]), (0, 5, [5])]),   # 360 has no compiled kernel
    ((360,), 0, 0, True, 0, [(0, 360, [9, 8, 5])]),
])
def test_plan_groups(dims, radix, dtype, mixed, cap, want):
    """The pass schedule rules, pinned on the host: one-base runs split evenly
    under the CTA's group limit (or a cap), groups spanning bases only when
    fewer, and each group's in-CTA round radices."""
    assert pac.pac_plan_groups(dims, radix, dtype, mixed, cap) == want


@pytest.mark.parametrize("dims", [(30,), (360, 360), (12, 20, 30), (6000, 6000), (2 ** 7 * 3 ** 4 * 5 ** 2,), (64, 81, 25),
                                  (2, 3, 5), (1, 1000), (4 * 27 * 125,), (3 ** 7 * 2,)])
@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("mixed", [False, True, None])
def test_plan_groups_invariants(dims, dtype, mixed):
    """Any 2^a 3^b 5^c shape: per axis the group sizes multiply to the dim,
    each group's rounds multiply to its size and are radices the kernels have,
    one-base groups stay within the CTA limit, groups spanning bases within 2048,
    and allowing groups spanning bases never adds groups."""
    groups = pac.pac_plan_groups(dims, 0, dtype, mixed)
    for a, n in enumerate(dims):
        sizes = [m for ax, m, _ in groups if ax == a]
        assert int(np.prod(sizes)) == n
    limits = {2: 4096 if dtype == 0 else 2048, 3: 2187, 5: 3125}
    for _, m, rounds in groups:
        assert int(np.prod(rounds)) == m
        assert set(rounds) <= {2, 3, 4, 5, 8, 9, 16, 25, 27}
        bases = {p for p in (2, 3, 5) if m % p == 0}
        if len(bases) == 1:
            assert m <= limits[bases.pop()]
        else:
            assert mixed is not False and (m <= 2048 or m == 6000)  # 6000: a compiled whole axis
            if mixed is None:  # the default rule forms only groups with compiled kernels
                assert m in (48, 120, 1000, 6000)
    assert len(groups) <= len(pac.pac_plan_groups(dims, 0, dtype, False))


@pytest.mark.parametrize("dims,radix", [((3125, 3125), 5), ((2187, 2187), 3), ((128, 128, 128), 2), ((4096, 4096), 4),
                                        ((1 << 20,), 4), ((1000, 1000), 0), ((60, 90, 30), 0), ((6000,), 0)])
def test_double_float_plan_groups(dims, radix):
    """Double-float plans (PAC_C128_DF) get the FP64 plans' one-base groups
    (the same sizes, axes and order; groups spanning bases are never formed,
    whatever the flags) and their own rounds: at most 4 points for base 2,
    3 for base 3, 5 for base 5, larger rounds first, multiplying to the group."""
    df = pac.pac_plan_groups(dims, radix, pac.C128_DF, None)
    assert [(a, m) for a, m, _ in df] == [(a, m) for a, m, _ in pac.pac_plan_groups(dims, radix, pac.C128, False)]
    assert df == pac.pac_plan_groups(dims, radix, pac.C128_DF, True)
    for _, m, rounds in df:
        base = 2 if m % 2 == 0 else (3 if m % 3 == 0 else 5)
        assert int(np.prod(rounds)) == m
        assert all(r <= {2: 4, 3: 3, 5: 5}[base] and r % base == 0 for r in rounds)
        assert rounds == sorted(rounds, reverse=True)
    if dims == (3125, 3125):
        assert df == [(0, 3125, [5] * 5), (1, 3125, [5] * 5)]


def test_plan_groups_rejects_bad_problems():
    for dims, radix, status in [((7,), 0, pac.Status.ERR_SIZE), ((100,), 2, pac.Status.ERR_SIZE),
                                ((64,), 6, pac.Status.ERR_ARG), ((2, 2, 2, 2), 2, pac.Status.ERR_ARG)]:
        with pytest.raises(pac.PacError) as ei:
            pac.pac_plan_groups(dims, radix)
        assert ei.value.status == status


def test_header_is_c_and_the_library_links_from_c():
    """include/pac.h compiles as C99 with warnings as errors, a C program links
    libpac.so and calls the host-only entry points (no GPU)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lib_dir = os.path.dirname(pac.LIB_PATH)
    exe = os.path.join(lib_dir, "_build", "abi_host")  # beside the library's other build products
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_host.c"), "-L", lib_dir, "-lpac", f"-Wl,-rpath,{lib_dir}",
                    "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.splitlines()
    assert out[0] == "stages 4 2 5 5 5"
    assert out[1] == "reverse " + " ".join(str(v) for v in pf.pos_to_freq([4, 4, 2])[[0, 1, 31]])
    assert out[2] == "groups 1 6000"  # the whole 6000-point axis as one compiled group
    assert out[3] == f"error {int(pac.Status.ERR_SIZE)} message"
    assert out[4].startswith("version ") and "sm_103a" in out[4]
