"""The arithmetic of the Ozaki scheme used by ACSE_OZAKI (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms
59, 2012), emulated exactly with Python integers and fractions on the CPU: the claims the GPU kernels
rest on, checked without the kernels.

* A row scaled by 2^-e (|a| 2^-e < 1/2) and rounded to the fixed point X = round(a 2^(6S-e)) splits
  into S balanced base-64 digits in [-32, 32] (exact in bf16) that give back X exactly.
* A digit matrix product summed over K stays below K 2^10 in magnitude, so g products with
  g K 2^10 < 2^24 add exactly in FP32; the worst case (every digit 32, one sign) reaches the bound.
* Keeping the levels s + t <= S + 1 leaves an error of order 2^(-6S) of the row and column scales
  times K, falling by about 2^6 per added slice.
The CUDA path (paper_2604_02550_gb300/csrc/gemm_oz.cu) is checked against the oracle on the GPU in
tests/test_gpu_ozaki.py.
"""
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
