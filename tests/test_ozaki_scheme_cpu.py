"""The arithmetic of the Ozaki scheme used by ACSE_OZAKI (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms
59, 2012), emulated exactly with Python integers and fractions on the CPU: the claims the GPU kernels
rest on, checked without the kernels.

* A row scaled by 2^-e (|a| 2^-e < 1/2) and rounded to the fixed point X = round(a 2^(6S-e)) splits
  into S balanced base-64 digits in [-32, 32] (exact in bf16) that give back X exactly.
* A digit matrix product summed over K stays below K 2^10 in magnitude, so g products with
  g K 2^10 < 2^24 add exactly in FP32; the worst case (every digit 32, one sign) reaches the bound.
* Keeping the levels s + t <= S + 1 leaves an error of order 2^(-6S) of the row and column scales
  times K, falling by about 2^6 per added slice.

The O(r^6) GEMMs use the modular form of the scheme (K. Ozaki, Y. Uchino, T. Imamura, Ozaki Scheme II,
2025); its claims are checked the same way:
* The moduli are pairwise coprime.  A residue taken as v - round(v / p) p with the float reciprocal of p
  (no correction step) is congruent to v and at most 64 in magnitude for |v| < 2^23 (65 for |v| <= 2^24),
  exact in bf16; a K chunk of 64 * 64 products of such residues stays within 2^24 (exact FP32
  accumulation), 65 blocks would not.
* The number T of moduli chosen for S slices covers 4 K 2^(2 min(6S, 53)) for the longest contraction.
* The reconstruction (s = sum_t w_t P / p_t in FP32 sums of base-2^11 limbs for one chunk, base-2^10
  for two, each an integer below 2^22; q = round(s / P) estimated in FP32 from those sums; x = s - q P)
  returns every x with |x| <= P / 4, for every T.
* The whole product (integer rows, residues, chunked exact sums, reconstruction) equals the exact
  product of the integer rows, and its error against the real product falls by about 2^6 a slice.
The CUDA path (paper_2604_02550_gb300/csrc/gemm_oz.cu) is checked against the oracle on the GPU in
tests/test_gpu_ozaki.py.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest


def fixed_point(a, S, e):
    """round(a 2^(6S - e)) for a float a (exact, ties away from zero as in the kernel)."""
    x = Fraction(float(a)) * Fraction(2) ** (6 * S - e)
    sgn = -1 if x < 0 else 1
    q = abs(x)
    n = int(q)
    if q - n >= Fraction(1, 2):
        n += 1
    return sgn * n


def digits(X, S):
    """Balanced base-64 digits, most significant first."""
    out = []
    for t in range(S):
        if t < S - 1:
            d = ((X + 32) & 63) - 32
            X = (X - d) >> 6
        else:
            d = X
        out.append(d)
    return out[::-1]


def row_exponent(row):
    m = max(abs(float(x)) for x in row)
    return 0 if m == 0 else int(np.frexp(m)[1]) + 1     # m < 2^(frexp exponent) => e = that + 1


def slices(Mat, S):
    """Digit matrices D_s (s = 1..S) and row exponents of a float matrix."""
    R, K = Mat.shape
    e = [row_exponent(Mat[i]) for i in range(R)]
    D = np.zeros((S, R, K), dtype=np.int64)
    for i in range(R):
        for k in range(K):
            X = fixed_point(Mat[i, k], S, e[i])
            assert abs(X) < 2 ** (6 * S - 1)
            D[:, i, k] = digits(X, S)
    return D, e


@pytest.mark.parametrize("S", [4, 6, 8])
def test_digits_exact_and_bounded(S):
    rng = np.random.default_rng(S)
    row = rng.standard_normal(64) * 10.0 ** rng.integers(-6, 6, 64)
    e = row_exponent(row)
    assert max(abs(row)) * 2.0 ** -e < 0.5
    for a in row:
        X = fixed_point(a, S, e)
        d = digits(X, S)
        assert all(-32 <= v <= 32 for v in d)
        assert sum(v * 64 ** (S - 1 - i) for i, v in enumerate(d)) == X
        # the fixed point is within half a unit of the scaled value
        assert abs(Fraction(float(a)) * Fraction(2) ** (6 * S - e) - X) <= Fraction(1, 2)


@pytest.mark.parametrize("K", [1128, 2304, 4608])
def test_group_bound_exact_in_fp32(K):
    g = ((1 << 24) - 1) // (K << 10)
    assert g >= 1
    worst = g * K * 32 * 32            # every digit 32, one sign
    assert worst < 2 ** 24             # exact in FP32: every partial sum is an integer below 2^24
    assert (g + 1) * K * 1024 >= 2 ** 24   # g is the largest such count
    # the same products as FP32 sums really are exact at the bound (sequential FP32 accumulation)
    acc = np.float32(0)
    for _ in range(g * K):
        acc = np.float32(acc + np.float32(1024))
    assert int(acc) == g * K * 1024


def ozaki_product(A, B, S):
    """C = A B^T from the levels s + t <= S + 1 of the digit products, summed exactly."""
    DA, ea = slices(A, S)
    DB, eb = slices(B, S)
    M, N = A.shape[0], B.shape[0]
    C = [[Fraction(0)] * N for _ in range(M)]
    for s in range(1, S + 1):
        for t in range(1, S + 2 - s):
            P = DA[s - 1] @ DB[t - 1].T                      # exact integer matrix
            w = Fraction(2) ** (-6 * (s + t))
            for i in range(M):
                for j in range(N):
                    C[i][j] += int(P[i, j]) * w
    return [[float(C[i][j] * Fraction(2) ** (ea[i] + eb[j])) for j in range(N)] for i in range(M)], ea, eb


def test_truncation_error_falls_with_slices():
    rng = np.random.default_rng(3)
    K = 40
    A = rng.standard_normal((3, K)) * np.exp(rng.standard_normal((3, K)))
    B = rng.standard_normal((4, K)) * np.exp(rng.standard_normal((4, K)))
    exact = [[sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[i], B[j])) for j in range(4)]
             for i in range(3)]
    errs = {}
    for S in (3, 4, 5, 6, 8):
        C, ea, eb = ozaki_product(A, B, S)
        # error relative to the scales 2^(ea + eb) K of the bound
        errs[S] = max(abs(Fraction(C[i][j]) - exact[i][j]) / (Fraction(2) ** (ea[i] + eb[j]) * K)
                      for i in range(3) for j in range(4))
        assert errs[S] <= Fraction(2) ** (-6 * S + 3), S
    for S in (3, 4, 5):
        assert errs[S + 1] < errs[S] / 8
    # with 8 slices the error is of the order of FP64 FMA rounding: below 2^-44 max|a| max|b| K
    C, _, _ = ozaki_product(A, B, 8)
    for i in range(3):
        for j in range(4):
            scale = np.abs(A[i]).max() * np.abs(B[j]).max() * K
            assert abs(C[i][j] - float(exact[i][j])) <= 2.0 ** -44 * scale


# ------------------------------------------------------------------ the modular form (Ozaki scheme II)
MODULI = [127, 125, 123, 121, 119, 113, 109, 107, 103, 101, 97, 89, 83, 79, 73, 71, 67, 61, 59]
LIMBS = {1: (11, 12), 2: (10, 14)}   # limbs of the reconstruction by K chunks: (bits, count)


def moduli_count(S, Kmax):
    """Least T whose product covers 4 Kmax 2^(2 bits), bits = min(6S, 53) (all 19 at most)."""
    bits = min(6 * S, 53)
    P, T = 1, 0
    while T < len(MODULI) and P < (Kmax << (2 * bits + 2)):
        P *= MODULI[T]
        T += 1
    return T, P, bits


def crt_constants(T):
    P = math.prod(MODULI[:T])
    Q = [P // p for p in MODULI[:T]]
    y = [pow(Q[t] % MODULI[t], -1, MODULI[t]) for t in range(T)]
    return P, Q, y


def balanced(v, p):
    r = v % p
    return r - p if r > (p - 1) // 2 else r


def limbs(v, nch):
    lb, nl = LIMBS[nch]
    return [(v >> (lb * l)) & ((1 << lb) - 1) for l in range(nl)]


def limb_sums(ws, Q, nch):
    """FP32 limb sums of s = sum_t w_t Q_t: every partial sum is an integer below 2^22 (exact)."""
    f = np.float32
    acc = [f(0)] * LIMBS[nch][1]
    for w, q in zip(ws, Q):
        for l, ql in enumerate(limbs(q, nch)):
            acc[l] = f(acc[l] + f(w) * f(ql))
            assert abs(float(acc[l])) < 2 ** 22
    return acc


def reconstruct(acc, P, nch):
    """x from the limb sums: q from an FP32 estimate of s / P summed from the limb sums as they are,
    then exact integer steps."""
    f = np.float32
    lb = LIMBS[nch][0]
    sf = f(0)
    for l in range(len(acc)):
        sf = f(sf + acc[l] * f(2.0 ** (lb * l - 120)))
    q = int(np.rint(sf * f(2.0 ** 120 / float(P))))
    return sum(int(a) * (1 << (lb * l)) for l, a in enumerate(acc)) - q * P


def test_moduli_coprime_and_residues_exact_in_bf16():
    torch = pytest.importorskip("torch")
    for i in range(len(MODULI)):
        assert all(math.gcd(MODULI[i], MODULI[j]) == 1 for j in range(i))
    r = torch.arange(-64, 65, dtype=torch.float32)
    assert torch.equal(r.to(torch.bfloat16).to(torch.float32), r)
    # one chunk: 64 blocks of 64 products of magnitude <= 64^2 stay within 2^24 (every integer up to 2^24
    # is a float), 65 blocks do not
    assert 64 * 64 * 64 * 64 == 2 ** 24 < 65 * 64 * 64 * 64
    assert float(np.float32(2 ** 24)) == 2 ** 24 and float(np.float32(2 ** 24 + 1)) != 2 ** 24 + 1


@pytest.mark.parametrize("p", MODULI)
def test_rounded_residue_bounds(p):
    """r = v - q p with q = round-half-even(v * fl(1/p)) (the fused multiply-add with 1.5 * 2^23), exactly
    evaluated: r = v mod p, |r| <= 64 for |v| < 2^23, |r| <= 65 for |v| <= 2^24."""
    pinv = np.float32(1.0) / np.float32(p)
    m, ex = np.frexp(np.float64(pinv))
    mant = int(m * 2 ** 24)                     # pinv = mant 2^(ex - 24) exactly
    sh = 24 - int(ex)
    rng = np.random.default_rng(p)
    for lim in (2 ** 23 - 1, 2 ** 24):
        v = np.concatenate([rng.integers(-lim, lim + 1, 400000), np.arange(-3000, 3000),
                            np.array([lim, -lim, lim - 1, -lim + 1])]).astype(np.int64)
        # half-integer quotients and their neighbours: v = p n + (p - 1) / 2 + {0, 1}
        n = rng.integers(-lim // p, lim // p, 20000)
        v = np.concatenate([v, p * n + (p - 1) // 2, p * n + (p + 1) // 2])
        v = v[np.abs(v) <= lim]
        prod = v * mant                         # exact: below 2^48
        q = prod >> sh                          # floor, then round half to even
        rem = prod - (q << sh)
        half = 1 << (sh - 1)
        q = q + ((rem > half) | ((rem == half) & (q & 1 == 1)))
        r = v - q * p
        assert np.all((v - r) % p == 0)
        assert np.abs(r).max() <= (64 if lim < 2 ** 23 else 65)


@pytest.mark.parametrize("S", [4, 5, 6, 7, 8, 9, 10])
def test_moduli_count_covers_the_products(S):
    for Kmax in (9, 162, 1152, 4608, 8192):
        T, P, bits = moduli_count(S, Kmax)
        assert 4 * Kmax * 2 ** (2 * bits) <= P
        assert T == 1 or 4 * Kmax * 2 ** (2 * bits) > P // MODULI[T - 1]   # least such T
    assert moduli_count(8, 4608)[0] == 17 and moduli_count(6, 4608)[0] == 13


@pytest.mark.parametrize("T", list(range(1, 20)))
def test_reconstruction_exact_within_quarter_P(T):
    """Every |x| <= P / 4, from residues split over 1..2 chunks (unreduced sums of residues up to 65 in
    magnitude), comes back exactly from FP32 limb sums: the FP32 quotient estimate never misses by a whole
    P, small P included."""
    P, Q, y = crt_constants(T)
    rnd = random.Random(T)
    xs = [0, 1, -1, P // 4, -(P // 4), P // 4 - 1] + [rnd.randint(-(P // 4), P // 4) for _ in range(300)]
    for x in xs:
        nch = rnd.randint(1, 2)
        wt = []
        for t, p in enumerate(MODULI[:T]):
            ws = [rnd.randint(-65, 65) for _ in range(nch - 1)]
            last = balanced(x * y[t] - sum(ws), p)
            ws.append(last + p if last < 0 and rnd.random() < 0.3 and last + p <= 65 else last)
            wt.append(sum(ws))
        assert reconstruct(limb_sums(wt, Q, nch), P, nch) == x


def modular_product(A, B, S, Kmax=None):
    """The modular scheme end to end on exact integers: integer rows, residues (B times y_t), chunked
    residue products (each chunk below 2^24), balanced chunk residues, limb sums, reconstruction."""
    K = A.shape[1]
    T, P, bits = moduli_count(S, Kmax or K)
    P, Q, y = crt_constants(T)
    b = bits
    while b > 0 and (K << (2 * b + 2)) > P:
        b -= 1
    nb = b + 1
    ea = [row_exponent(r) for r in A]
    eb = [row_exponent(r) for r in B]
    XA = [[fixed_point(a, 0, ea[i] - nb) for a in A[i]] for i in range(A.shape[0])]
    XB = [[fixed_point(v, 0, eb[j] - nb) for v in B[j]] for j in range(B.shape[0])]
    kb = (K + 63) // 64
    nch = (kb + 63) // 64
    cb = (kb + nch - 1) // nch
    C = np.zeros((A.shape[0], B.shape[0]))
    for i in range(A.shape[0]):
        for j in range(B.shape[0]):
            wt = []
            for t, p in enumerate(MODULI[:T]):
                ra = [balanced(x, p) for x in XA[i]]
                rb = [balanced(x * y[t], p) for x in XB[j]]
                w = 0
                for c in range(nch):
                    part = sum(ra[k] * rb[k] for k in range(c * cb * 64, min(K, (c + 1) * cb * 64)))
                    assert abs(part) <= 2 ** 24
                    w += balanced(part, p)
                wt.append(w)
            x = reconstruct(limb_sums(wt, Q, nch), P, nch)
            assert x == sum(a * v for a, v in zip(XA[i], XB[j]))
            C[i, j] = float(Fraction(x) * Fraction(2) ** (ea[i] + eb[j] - 2 * nb))
    return C


def test_modular_product_error_falls_with_slices():
    rng = np.random.default_rng(11)
    K = 162
    A = rng.standard_normal((2, K)) * np.exp(rng.standard_normal((2, K)))
    B = rng.standard_normal((2, K)) * np.exp(rng.standard_normal((2, K)))
    exact = [[sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[i], B[j])) for j in range(2)]
             for i in range(2)]
    errs = {}
    for S in (4, 5, 6, 8):
        C = modular_product(A, B, S)
        errs[S] = max(abs(Fraction(C[i][j]) - exact[i][j]) / (Fraction(2) ** (row_exponent(A[i]) + row_exponent(B[j])) * K)
                      for i in range(2) for j in range(2))
        assert errs[S] <= Fraction(2) ** (-6 * S), S
    for S in (4, 5):
        assert errs[S + 1] < errs[S] / 8
    C = modular_product(A, B, 8)
    for i in range(2):
        for j in range(2):
            scale = np.abs(A[i]).max() * np.abs(B[j]).max() * K
            assert abs(C[i][j] - float(exact[i][j])) <= 2.0 ** -46 * scale


def test_modular_product_two_chunks():
    """K above 64 * 64 runs as two exactly accumulated chunks per modulus."""
    rng = np.random.default_rng(12)
    K = 4300
    A = rng.standard_normal((1, K))
    B = rng.standard_normal((1, K))
    C = modular_product(A, B, 8, Kmax=8192)
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[0], B[0]))
    assert abs(C[0][0] - float(exact)) <= 2.0 ** -46 * np.abs(A).max() * np.abs(B).max() * K
