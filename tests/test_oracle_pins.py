"""Pins for the oracle: each route checked against something other than itself.

Sources of truth used here: values the paper prints (the F_2/F_4/F_8 matrices
of Appendix A, the modulo-r sort of eq. (r-ary-sorting)), hand-worked small
convolutions, a library FFT (numpy's pocketfft), closed forms (delta, shifted
delta, constant filter, Parseval) and the paper's identities F = P A^T,
F^-1 = conj(A) P / n and Eq. (35)/(80), which tie the matrix forms of
``oracle.paper_forms`` to the definition-based routes of ``oracle``.

The mutation tests at the end plant plausible mistakes in oracle functions
(on the CPU, via monkeypatch) and check that a pin catches each one.
"""
import os

import numpy as np
import pytest

import oracle
import pac_inputs as pin
from oracle import paper_forms as pf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RADIX_LISTS = [[2] * 4, [4, 4], [8, 8], [3, 3, 3], [5, 5], [2] * 6, [3] * 4,
               [4, 4, 4, 2], [2, 4, 4, 4], [8, 8, 2], [2, 8, 8], [2, 3, 4], [4, 2, 2],
               # mixed prime bases in any order (Section 7.1): 2^a 3^b 5^c
               [2, 3, 5], [5, 3, 2, 2], [3, 5, 2, 3], [4, 2, 5, 5], [5, 2, 5, 4]]


def rand_c(shape, seed):
    return pin.complex_uniform(shape, seed)


# ------------------------------------------------------------------ golden


def _sym(s):
    a = (1 - 1j) / np.sqrt(2)
    b = -(1 + 1j) / np.sqrt(2)
    table = {"1": 1, "-1": -1, "i": 1j, "-i": -1j, "a": a, "-a": -a, "b": b, "-b": -b}
    return table[s]


def load_fourier_golden():
    mats, cur, name = {}, [], None
    for line in open(os.path.join(GOLDEN, "fourier_matrices.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("F"):
            if name:
                mats[name] = np.array(cur)
            name, cur = int(line[1:]), []
        else:
            cur.append([_sym(t) for t in line.split()])
    mats[name] = np.array(cur)
    return mats


def test_fourier_matches_paper_matrices():
    for n, m in load_fourier_golden().items():
        assert m.shape == (n, n)
        np.testing.assert_allclose(pf.fourier(n), m, atol=1e-15)


def test_oracle_dft_matches_paper_matrices():
    # the naive DFT applied to unit vectors gives the columns of F_n
    for n, m in load_fourier_golden().items():
        got = np.stack([oracle.dft(np.eye(n)[k]) for k in range(n)], axis=1)
        np.testing.assert_allclose(got, m, atol=1e-15)


def load_reversal_golden():
    out = []
    for line in open(os.path.join(GOLDEN, "index_reversal.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, vals = line.split(":")
        kind, r, n = head.split()
        out.append((kind, int(r.split("=")[1]), int(n.split("=")[1]), [int(v) for v in vals.split()]))
    return out


def test_index_reversal_golden():
    for kind, r, n, perm in load_reversal_golden():
        got = pf.mod_sort(r, n) if kind == "mod_sort" else pf.index_reversal(r, n)
        assert list(got) == perm, (kind, r, n)


def load_conv_golden():
    out = []
    for line in open(os.path.join(GOLDEN, "conv_small.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        shape, h, x, y = [t.strip() for t in line.split("|")]
        shape = tuple(int(s) for s in shape.split("x"))
        conv = lambda s: np.array([complex(eval(t)) for t in s.split()]).reshape(shape)  # noqa: E731
        out.append((shape, conv(h), conv(x), conv(y)))
    return out


@pytest.mark.parametrize("route", ["direct", "via_dft", "points"])
def test_conv_hand_worked(route):
    for shape, h, x, y in load_conv_golden():
        if route == "direct":
            got = oracle.conv_direct(h, x)
        elif route == "via_dft":
            got = oracle.conv_via_dft(h, x)
        else:
            got = oracle.conv_direct_points(h, x, np.arange(h.size)).reshape(shape)
        np.testing.assert_allclose(got, y, atol=1e-14)


# --------------------------------------------------------- library routines


@pytest.mark.parametrize("shape", [(12,), (27,), (6, 10), (4, 6, 5), (8, 8, 8)])
def test_dft_matches_numpy_fft(shape):
    x = rand_c(shape, 7)
    np.testing.assert_allclose(oracle.dft(x), np.fft.fftn(x), atol=1e-12 * np.sqrt(x.size))
    np.testing.assert_allclose(oracle.idft(oracle.dft(x)), x, atol=1e-13)


@pytest.mark.parametrize("shape", [(16,), (9,), (25,), (8, 4), (3, 9), (4, 4, 4), (3, 5, 2)])
def test_conv_direct_matches_fft_convolution(shape):
    h, x = rand_c(shape, 1), rand_c(shape, 2)
    ref = np.fft.ifftn(np.fft.fftn(h) * np.fft.fftn(x))
    got = oracle.conv_direct(h, x)
    assert oracle.rel_l2(got, ref) < 1e-14
    assert oracle.rel_l2(oracle.conv_via_dft(h, x), ref) < 1e-13


# ------------------------------------------------------------ closed forms


@pytest.mark.parametrize("shape", [(32,), (8, 6), (4, 3, 5)])
def test_delta_filter_returns_input(shape):
    x = rand_c(shape, 3)
    h = np.zeros(shape, complex)
    h[(0,) * len(shape)] = 1.0
    np.testing.assert_allclose(oracle.conv_direct(h, x), x, atol=1e-15)


@pytest.mark.parametrize("shape,shift", [((32,), (5,)), ((8, 6), (3, 4)), ((4, 3, 5), (1, 2, 4))])
def test_shifted_delta_is_exact_roll(shape, shift):
    x = rand_c(shape, 4)
    h = np.zeros(shape, complex)
    h[shift] = 1.0
    got = oracle.conv_direct(h, x)
    assert np.array_equal(got, np.roll(x, shift, axis=tuple(range(len(shape)))))


@pytest.mark.parametrize("shape", [(16,), (6, 4), (3, 3, 3)])
def test_constant_filter_gives_total_sum(shape):
    x = rand_c(shape, 5)
    got = oracle.conv_direct(np.ones(shape, complex), x)
    np.testing.assert_allclose(got, np.full(shape, x.sum()), atol=1e-13)


@pytest.mark.parametrize("shape", [(20,), (5, 7), (3, 4, 2)])
def test_commutative_and_linear(shape):
    h, x, z = rand_c(shape, 6), rand_c(shape, 7), rand_c(shape, 8)
    np.testing.assert_allclose(oracle.conv_direct(h, x), oracle.conv_direct(x, h), atol=1e-14)
    a, b = 0.3 - 1.2j, -2.0 + 0.5j
    lhs = oracle.conv_direct(h, a * x + b * z)
    rhs = a * oracle.conv_direct(h, x) + b * oracle.conv_direct(h, z)
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


@pytest.mark.parametrize("shape", [(16,), (8, 6), (4, 6, 5), (9, 25)])
def test_separable_matches_direct(shape):
    # distinct factors per axis catch a transposed axis or a swapped factor
    fs = [rand_c((n,), 30 + a) for a, n in enumerate(shape)]
    x = rand_c(shape, 9)
    ref = oracle.conv_direct(pin.outer(fs), x)
    assert oracle.rel_l2(oracle.conv_separable(fs, x), ref) < 1e-14


def test_points_match_full():
    shape = (6, 5, 4)
    h, x = rand_c(shape, 10), rand_c(shape, 11)
    full = oracle.conv_direct(h, x).reshape(-1)
    idx = pin.sample_points(full.size, 37, seed=3)
    np.testing.assert_array_equal(oracle.conv_direct_points(h, x, idx), full[idx])


def test_compensated_sum_accuracy():
    # y[0] = h0 x0 + h1 x[-1] + h2 x[-2] = 1e16 + 1 - 1e16 = 1 exactly; a plain
    # left-to-right FP64 sum returns 0 (1e16 + 1 rounds to 1e16)
    n = 64
    x = np.zeros(n, complex)
    x[0] = x[n - 1] = x[n - 2] = 1.0
    h = np.zeros(n, complex)
    h[0], h[1], h[2] = 1e16, 1.0, -1e16
    assert (1e16 + 1.0) - 1e16 == 0.0
    y = oracle.conv_direct(h, x)
    assert y[0] == 1.0


# ------------------------------------------------------ the paper's identities


@pytest.mark.parametrize("r,n", [(2, 8), (2, 64), (3, 27), (4, 64), (5, 25), (8, 64), (3, 81)])
def test_index_reversal_symmetric_involution(r, n):
    p = pf.index_reversal(r, n)
    assert np.array_equal(pf.compose(p, p), np.arange(n))  # P P = I (Section 2.1)
    m = pf.perm_matrix(p)
    assert np.array_equal(m, m.T)  # P = P^T


@pytest.mark.parametrize("r,n", [(2, 16), (3, 27), (4, 64), (5, 25), (8, 64)])
def test_fourier_factorisation_uniform(r, n):
    a = pf.a_uniform(r, n)
    p = pf.perm_matrix(pf.index_reversal(r, n))
    f = pf.fourier(n)
    np.testing.assert_allclose(a @ p, f, atol=1e-12)  # F = A P
    np.testing.assert_allclose(p @ a.T, f, atol=1e-12)  # F = P A^T
    np.testing.assert_allclose(np.conj(a) @ p / n, np.linalg.inv(f), atol=1e-12)  # F^-1


@pytest.mark.parametrize("stages", RADIX_LISTS)
def test_dif_output_is_dft_in_reversed_order(stages):
    """The fixed fact: A^T x equals DFT(x) in index-reversed order (F = P A^T)."""
    n = int(np.prod(stages))
    x = rand_c((n,), 12)
    lhs = pf.a_transpose(stages) @ x
    rhs = oracle.dft(x)[pf.pos_to_freq(stages)]
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
    np.testing.assert_allclose(oracle.unordered_forward(x, [stages]), lhs, atol=1e-12)


@pytest.mark.parametrize("stages", RADIX_LISTS)
def test_pos_to_freq_digit_formula(stages):
    """Mixed-radix position: k = k1 + s1 k2 + s1 s2 k3 ... lands at sum_i k_i prod_{j>i} s_j."""
    n = int(np.prod(stages))
    want = np.empty(n, np.int64)
    for k in range(n):
        rem, pos = k, 0
        for i, s in enumerate(stages):
            pos += (rem % s) * int(np.prod(stages[i + 1:]))
            rem //= s
        want[pos] = k
    assert np.array_equal(pf.pos_to_freq(stages), want)


@pytest.mark.parametrize("stages", RADIX_LISTS)
def test_eq35_equals_definition(stages):
    n = int(np.prod(stages))
    h, x = rand_c((n,), 13), rand_c((n,), 14)
    assert oracle.rel_l2(pf.conv_eq35(h, x, stages), oracle.conv_direct(h, x)) < 1e-13


@pytest.mark.parametrize("stage_lists", [([2, 2, 2], [4, 2]), ([3, 3], [3, 3, 3]), ([5], [5, 5]),
                                         ([2, 2], [2, 2], [2, 2]), ([4], [2, 2], [8]), ([2, 3], [5, 2]),
                                         ([3, 2], [2], [5])])
def test_eq80_equals_definition(stage_lists):
    shape = tuple(int(np.prod(s)) for s in stage_lists)
    h, x = rand_c(shape, 15), rand_c(shape, 16)
    assert oracle.rel_l2(pf.conv_eq80(h, x, stage_lists), oracle.conv_direct(h, x)) < 1e-13


def test_wrong_plan_pairing_is_wrong():
    """Forward in radix-2 order with an inverse in radix-4 order does not convolve."""
    n = 64
    h, x = rand_c((n,), 17), rand_c((n,), 18)
    a2t = pf.a_transpose([2] * 6)
    a4t = pf.a_transpose([4] * 3)
    mixed = np.conj(a4t.T) @ ((a2t @ h) * (a2t @ x)) / n
    assert oracle.rel_l2(mixed, oracle.conv_direct(h, x)) > 0.1


@pytest.mark.parametrize("stages", [[2] * 7, [4, 4, 4, 2], [8, 8, 2], [3] * 5, [5] * 3])
def test_parseval_on_unordered_output(stages):
    n = int(np.prod(stages))
    x = rand_c((n,), 19)
    xh = oracle.unordered_forward(x, [stages])
    np.testing.assert_allclose(np.vdot(xh, xh).real, n * np.vdot(x, x).real, rtol=1e-13)


@pytest.mark.parametrize("dims,sigma", [((128,), 4.0), ((32, 24, 16), 1.5)])
def test_gaussian_spectrum_real_nonnegative(dims, sigma):
    # exact periodisation needs the ring much wider than sigma (images below 1e-15)
    h = pin.outer(pin.gaussian_factors(dims, sigma))
    H = oracle.dft(h)
    assert np.abs(H.imag).max() < 1e-15
    assert H.real.min() > -1e-15
    assert abs(H.real.reshape(-1)[0] - 1.0) < 1e-14  # normalised to sum 1


# ------------------------------------------------------------- mutation tests


def test_mutation_wrong_dft_sign_caught(monkeypatch):
    real = oracle.dft
    monkeypatch.setattr(oracle, "dft", lambda x, sign=-1: real(x, -sign))
    x = rand_c((16,), 20)
    assert not np.allclose(oracle.dft(x), np.fft.fft(x), atol=1e-10)


def test_mutation_wrong_mod_sort_caught(monkeypatch):
    # a plausible off-by-one reading of eq. (r-ary-sorting): sort by p div r
    monkeypatch.setattr(pf, "mod_sort", lambda r, n: (np.arange(n) % r) * (n // r) + np.arange(n) // r)
    golden = [g for g in load_reversal_golden() if g[0] == "reversal" and g[1] == 2 and g[2] == 16][0]
    assert list(pf.index_reversal(2, 16)) != golden[3]


def test_mutation_butterfly_missing_twiddle_caught(monkeypatch):
    # drop the Omega diagonal of Eq. (25): A^T x no longer matches the reordered DFT
    monkeypatch.setattr(pf, "butterfly", lambda r, k: np.kron(pf.fourier(r), np.eye(k // r)))
    x = rand_c((16,), 21)
    lhs = pf.a_transpose([2] * 4) @ x
    assert not np.allclose(lhs, oracle.dft(x)[pf.pos_to_freq([2] * 4)], atol=1e-6)


def test_mutation_transposed_stage_list_caught():
    # using rho in place of the DIF stage list (forgetting the reversal) breaks mixed radix
    stages = [4, 4, 2]
    x = rand_c((32,), 22)
    wrong = pf.inverse_perm(pf.p_mixed(stages))
    assert not np.allclose(pf.a_transpose(stages) @ x, oracle.dft(x)[wrong], atol=1e-6)


# ----------------------------------------------- prime factor framework (Section 7.2)


@pytest.mark.parametrize("n,want", [(6, [2, 3]), (10, [2, 5]), (60, [3, 4, 5]), (1000, [8, 125]), (81, [81]),
                                    (1, []), (2 ** 10 * 3 ** 5 * 5 ** 3, [125, 243, 1024])])
def test_coprime_factors(n, want):
    assert pf.coprime_factors(n) == want


@pytest.mark.parametrize("n", [6, 10, 12, 15, 30, 60, 90])
def test_prime_factor_fourier_factorisation(n):
    """Section 7.2: F_n = Gamma (F_{n_t} (x) ... (x) F_{n_1}) Upsilon^T with Gamma the
    Chinese-remainder output map and Upsilon the Ruritanian input map; both are
    permutations.  Where the two maps differ (n / n_q != 1 mod n_q for some q;
    for n = 30 they coincide), Gamma on both sides does not factor F_n."""
    f = pf.coprime_factors(n)
    g, u = pf.crt_gamma(f), pf.ruritanian_upsilon(f)
    assert sorted(g) == list(range(n)) and sorted(u) == list(range(n))
    lhs = pf.perm_matrix(g) @ pf.kron_fourier(f) @ pf.perm_matrix(u).T
    np.testing.assert_allclose(lhs, pf.fourier(n), atol=1e-12)
    if not np.array_equal(g, u):
        wrong = pf.perm_matrix(g) @ pf.kron_fourier(f) @ pf.perm_matrix(g).T
        assert not np.allclose(wrong, pf.fourier(n), atol=1e-6)


@pytest.mark.parametrize("n", [6, 10, 12, 15, 30, 60, 90, 120])
def test_prime_factor_convolution_equals_definition(n):
    """Section 7.2's convolution with three permutations equals the definition (O1)."""
    h, x = rand_c((n,), 30 + n), rand_c((n,), 31 + n)
    assert oracle.rel_l2(pf.conv_pfa(h, x, pf.coprime_factors(n)), oracle.conv_direct(h, x)) < 1e-13


def test_gamma_is_additive():
    """Gamma^T takes a cyclic shift by s to the tensor shift by (s mod n_q) per axis,
    which is why a cyclic convolution of length n becomes a d-D cyclic one."""
    f = [4, 3, 5]
    n = 60
    gt = pf.inverse_perm(pf.crt_gamma(f))
    x = rand_c((n,), 32)
    s = 7
    lhs = np.roll(x, s)[gt].reshape(5, 3, 4)
    rhs = np.roll(x[gt].reshape(5, 3, 4), (s % 5, s % 3, s % 4), axis=(0, 1, 2))
    np.testing.assert_allclose(lhs, rhs, atol=0)


def test_mutation_pfa_with_ruritanian_gather_caught():
    # gathering with Upsilon^T but scattering with Gamma mixes two maps: wrong result
    n = 60
    f = pf.coprime_factors(n)
    h, x = rand_c((n,), 33), rand_c((n,), 34)
    g, u = pf.crt_gamma(f), pf.ruritanian_upsilon(f)
    ut = pf.inverse_perm(u)
    shape = tuple(reversed(f))
    y = pf.conv_eq80(h[ut].reshape(shape), x[ut].reshape(shape), [[m] for m in shape]).reshape(-1)[g]
    assert oracle.rel_l2(y, oracle.conv_direct(h, x)) > 0.1
