"""Oracle, part 2: the paper's matrix forms, written out literally (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Dense matrices, so
only for small n (a few hundred at most).  Each function follows the paper's
definitions in its notation; nothing is blocked, fused or reordered.

* ``fourier(n)``                F_n with (F_n)_{jk} = w_n^{jk}, w_n = exp(-2 pi i/n)   (Section 2)
* ``mod_sort(r, n)``            R_{r,n}: the modulo-r sort of eq. (r-ary-sorting)     (Section 2.1)
* ``index_reversal(r, n)``      P_{r,n} = R_{r,t,n} ... R_{r,1,n}                      (Section 2.1)
* ``butterfly(r, k)``           B_{r,k} = (F_r (x) I_{k/r}) diag(I, W, ..., W^{r-1})    (Eq. 25)
* ``a_uniform(r, n)``           A_{r,n} = B_{r,t,n} ... B_{r,1,n}                      (Section 2.1)
* ``a_mixed(rho)``, ``p_mixed(rho)``  A_rho and P_rho of the mixed-radix framework   (Section 7.1)
* ``conv_eq35(h, x, ...)``      conj(A)((A^T h) o (A^T x)) / n                          (Eq. 35)
* ``conv_eq80(H, X, ...)``      the 2-D / d-D Kronecker form                           (Eq. 80, Sections 3.1 and 4.1)
* ``coprime_factors(n)``, ``crt_gamma``, ``ruritanian_upsilon``, ``conv_pfa``
                                the prime factor framework: F_n = Gamma (F_{n_t} (x) ... (x) F_{n_1}) Upsilon^T
                                and the convolution with three permutations               (Section 7.2)

Index conventions are zero-based.  A permutation matrix is returned as an
index array ``perm`` with (P v)[p] = v[perm[p]].
"""
from __future__ import annotations

import numpy as np


def omega(n: int) -> complex:
    """w_n = exp(-2 pi i / n) (Section 2)."""
    return np.exp(-2j * np.pi / n)


def fourier(n: int) -> np.ndarray:
    """Dense Fourier matrix F_n, (F_n)_{jk} = w_n^{jk}, exponent reduced mod n."""
    j = np.arange(n)
    e = np.outer(j, j) % n
    return np.exp(-2j * np.pi * e / n)


def perm_matrix(perm) -> np.ndarray:
    """Dense matrix of the permutation index array ``perm``: (P v)[p] = v[perm[p]]."""
    n = len(perm)
    m = np.zeros((n, n))
    m[np.arange(n), np.asarray(perm)] = 1.0
    return m


def compose(p_outer, p_inner):
    """Index array of the product P_outer P_inner (P_inner applied first)."""
    p_outer = np.asarray(p_outer)
    p_inner = np.asarray(p_inner)
    # (P_o P_i v)[p] = (P_i v)[p_o[p]] = v[p_i[p_o[p]]]
    return p_inner[p_outer]


def kron_identity_perm(blocks: int, perm) -> np.ndarray:
    """I_blocks (x) P as an index array."""
    perm = np.asarray(perm)
    m = len(perm)
    return (np.arange(blocks)[:, None] * m + perm[None, :]).reshape(-1)


def mod_sort(r: int, n: int) -> np.ndarray:
    """R_{r,n} of eq. (r-ary-sorting): group entries by residue mod r.

    R_{r,n} x = [x_0, x_r, x_2r, ..., x_1, x_{r+1}, ..., x_{r-1}, x_{2r-1}, ...]
    (zero-based), i.e. position p holds x[(p mod (n/r)) * r + p div (n/r)].
    """
    assert n % r == 0
    m = n // r
    p = np.arange(n)
    return (p % m) * r + p // m


def perfect_shuffle(r: int, n: int) -> np.ndarray:
    """Pi_{r,n}: the inverse of the modulo-r sort (Section 7.1)."""
    s = mod_sort(r, n)
    inv = np.empty_like(s)
    inv[s] = np.arange(n)
    return inv


def index_reversal(r: int, n: int) -> np.ndarray:
    """P_{r,n} = R_{r,t,n} R_{r,t-1,n} ... R_{r,1,n} with R_{r,q,n} = I_{r^{q-1}} (x) R_{r,n/r^{q-1}}."""
    t = int(round(np.log(n) / np.log(r)))
    assert r ** t == n
    perm = np.arange(n)  # identity
    for q in range(1, t + 1):  # R_{r,1,n} is applied first
        rq = kron_identity_perm(r ** (q - 1), mod_sort(r, n // r ** (q - 1)))
        perm = compose(rq, perm)
    return perm


def big_omega(r: int, m: int) -> np.ndarray:
    """Omega_{r,m} = diag(1, w_{rm}, w_{rm}^2, ..., w_{rm}^{m-1}) as a vector."""
    j = np.arange(m)
    return np.exp(-2j * np.pi * j / (r * m))


def butterfly(r: int, k: int) -> np.ndarray:
    """B_{r,k} = (F_r (x) I_{k/r}) diag(I_{k/r}, W, W^2, ..., W^{r-1}), W = Omega_{r,k/r} (Eq. 25)."""
    m = k // r
    w = big_omega(r, m)
    d = np.concatenate([w ** p for p in range(r)])
    return np.kron(fourier(r), np.eye(m)) @ np.diag(d)


def a_uniform(r: int, n: int) -> np.ndarray:
    """A_{r,n} = B_{r,t,n} ... B_{r,1,n}, B_{r,q,n} = I_{n/r^q} (x) B_{r,r^q}."""
    t = int(round(np.log(n) / np.log(r)))
    assert r ** t == n
    a = np.eye(n, dtype=complex)
    for q in range(1, t + 1):
        bq = np.kron(np.eye(n // r ** q), butterfly(r, r ** q))
        a = bq @ a
    return a


def a_mixed(rho) -> np.ndarray:
    """A_rho = B_{r_t,n} (I (x) B_{r_{t-1}, r_1..r_{t-1}}) ... (I_{n/r_1} (x) B_{r_1,r_1}) (Section 7.1)."""
    n = int(np.prod(rho))
    a = np.eye(n, dtype=complex)
    k = 1
    for r in rho:  # r_1 acts first, on blocks of size r_1
        k *= r
        a = np.kron(np.eye(n // k), butterfly(r, k)) @ a
    return a


def p_mixed(rho) -> np.ndarray:
    """P_rho = Pi_{r_t,n} (I (x) Pi_{r_{t-1}, r_1..r_{t-1}}) ... (I_{n/r_1} (x) Pi_{r_1,r_1}) (Section 7.1)."""
    n = int(np.prod(rho))
    perm = np.arange(n)
    k = 1
    for r in rho:
        k *= r
        perm = compose(kron_identity_perm(n // k, perfect_shuffle(r, k)), perm)
    return perm


def inverse_perm(perm) -> np.ndarray:
    perm = np.asarray(perm)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    return inv


def rho_of_dif_stages(stages) -> list:
    """The paper's rho = [r_1..r_t] for a DIF stage list (s_1 acts first on the full length).

    A_rho^T applies B_{r_t,n}^T first, so s_1 = r_t, ..., s_T = r_1.
    """
    return list(reversed(list(stages)))


def pos_to_freq(stages) -> np.ndarray:
    """Frequency held at each position of the DIF (A^T) output for a stage list.

    From F = P A^T with P symmetric (uniform radix, Section 2.1) or
    F = P_rho A_rho^T (Section 7.1): A^T x = P^T F x, so position p holds
    frequency (P^T idx)[p].
    """
    stages = list(stages)
    n = int(np.prod(stages))
    if len(set(stages)) == 1:
        perm = index_reversal(stages[0], n)  # symmetric: P^T = P
        return perm
    return inverse_perm(p_mixed(rho_of_dif_stages(stages)))


def a_transpose(stages) -> np.ndarray:
    """A^T for a DIF stage list (uniform or mixed radix)."""
    stages = list(stages)
    n = int(np.prod(stages))
    if len(set(stages)) == 1:
        return a_uniform(stages[0], n).T
    return a_mixed(rho_of_dif_stages(stages)).T


def conv_eq35(h: np.ndarray, x: np.ndarray, stages) -> np.ndarray:
    """Permutation-avoiding 1-D convolution, Eq. (35): conj(A)((A^T h) o (A^T x)) / n."""
    at = a_transpose(stages)
    n = at.shape[0]
    return np.conj(at.T) @ ((at @ h) * (at @ x)) / n


def conv_eq80(h: np.ndarray, x: np.ndarray, stages_per_axis) -> np.ndarray:
    """d-D permutation-avoiding convolution (Eq. 80 of Section 3.1 and its d-D form, Section 4.1), Kronecker form.

    vec(F_H(X)) = (conj A_1 (x) ... (x) conj A_d)[((A_1^T (x)..) vec H) o ((A_1^T (x)..) vec X)] / N
    with row-major vec (last index fastest).
    """
    ats = [a_transpose(s) for s in stages_per_axis]
    kt = ats[0]
    for a in ats[1:]:
        kt = np.kron(kt, a)
    n = kt.shape[0]
    hv = h.reshape(-1)
    xv = x.reshape(-1)
    y = np.conj(kt.T) @ ((kt @ hv) * (kt @ xv)) / n
    return y.reshape(x.shape)


# ------------------------------------------------- prime factor framework (Section 7.2)


def coprime_factors(n: int) -> list:
    """n = 2^a 3^b 5^c as its pairwise coprime prime powers [n_1, ..., n_t], ascending
    (the factors of Section 7.2; [] for n = 1)."""
    out = []
    for p in (2, 3, 5):
        q = 1
        while n % p == 0:
            n //= p
            q *= p
        if q > 1:
            out.append(q)
    if n != 1:
        raise ValueError("n is not of the form 2^a 3^b 5^c")
    return sorted(out)


def _tensor_index(idx, factors) -> int:
    """Row-major position of (i_t, ..., i_1) in the tensor of shape (n_t, ..., n_1),
    idx[q] = i_{q+1}: the ordering of F_{n_t} (x) ... (x) F_{n_1}."""
    pos = 0
    for q in reversed(range(len(factors))):
        pos = pos * factors[q] + idx[q]
    return pos


def crt_gamma(factors) -> np.ndarray:
    """Gamma of Section 7.2 as an index array, (Gamma v)[k] = v[gamma[k]]: output k of
    the length-n transform is tensor entry (k mod n_t, ..., k mod n_1) (Chinese remainders)."""
    n = int(np.prod(factors)) if len(factors) else 1
    return np.array([_tensor_index([k % m for m in factors], factors) for k in range(n)], dtype=np.int64)


def ruritanian_upsilon(factors) -> np.ndarray:
    """Upsilon of Section 7.2 as an index array, (Upsilon v)[i] = v[upsilon[i]]: input
    i = sum_q (n / n_q) i_q mod n is tensor entry (i_t, ..., i_1), i.e.
    i_q = i (n / n_q)^{-1} mod n_q."""
    n = int(np.prod(factors)) if len(factors) else 1
    inv = [pow((n // m) % m, -1, m) if m > 1 else 0 for m in factors]
    return np.array([_tensor_index([(i * inv[q]) % m for q, m in enumerate(factors)], factors)
                     for i in range(n)], dtype=np.int64)


def kron_fourier(factors) -> np.ndarray:
    """F_{n_t} (x) ... (x) F_{n_1} (dense)."""
    k = np.eye(1, dtype=complex)
    for m in reversed(list(factors)):
        k = np.kron(k, fourier(m))
    return k


def conv_pfa(h: np.ndarray, x: np.ndarray, factors) -> np.ndarray:
    """Prime factor convolution of Section 7.2 for a 1-D length n = n_1 ... n_t:
    Gamma (conj A_{n_t} (x) ... (x) conj A_{n_1}) [((A^T ...) Gamma^T h) o ((A^T ...) Gamma^T x)] / n,
    the three permutations being Gamma^T h, Gamma^T x and Gamma.  Each A_{n_q} is
    the uniform-radix A of its prime (Section 2.1); the bracket is the d-D form of
    Eq. (80) on the tensor of shape (n_t, ..., n_1)."""
    g = crt_gamma(factors)
    gt = inverse_perm(g)  # (Gamma^T v)[j] = v[gt[j]]
    shape = tuple(reversed(list(factors)))
    stages = []
    for m in shape:
        p = next(q for q in (2, 3, 5) if m % q == 0)
        stages.append([p] * int(round(np.log(m) / np.log(p))))
    hh = np.asarray(h, dtype=complex)[gt].reshape(shape)
    xx = np.asarray(x, dtype=complex)[gt].reshape(shape)
    y = conv_eq80(hh, xx, stages).reshape(-1)
    return y[g]
