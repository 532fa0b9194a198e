"""The host side of the modular Ozaki GEMM (`acse_ozaki_plan_info`, no device access) against the rules
the CPU pins of tests/test_ozaki_scheme_cpu.py check: the moduli (pairwise coprime, largest first), the
least moduli count T whose product covers 4 Kmax 2^(2 min(6S, 53)), the bits kept for a GEMM of
contraction length k (the largest b <= min(6S, 53) with 4 k 2^(2b) <= P) and its K chunks of at most
64 * 64 elements."""
import math

import pytest

from tests.test_ozaki_scheme_cpu import MODULI, moduli_count


@pytest.fixture(scope="module")
def lib():
    from paper_2604_02550_gb300 import _lib
    import os
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _lib


def _bits(S, kmax, k):
    T, P, bits = moduli_count(S, kmax)
    b = bits
    while b > 0 and (k << (2 * b + 2)) > P:
        b -= 1
    return T, b


@pytest.mark.parametrize("S", [4, 5, 6, 7, 8, 9, 10])
def test_plan_matches_the_rules(lib, S):
    for kmax in (1, 9, 162, 1152, 2304, 4608, 8192):
        for k in sorted({1, min(36, kmax), (kmax + 1) // 2, kmax}):
            got = lib.acse_ozaki_plan_info(S, kmax, k)
            T, b = _bits(S, kmax, k)
            assert got["moduli_count"] == T
            assert got["moduli"] == MODULI[:T]
            assert got["bits"] == b
            assert got["chunks"] == -(-((k + 63) // 64) // 64)
            # the product of the moduli covers every integer product of the plan
            assert 4 * k * 2 ** (2 * got["bits"]) <= math.prod(got["moduli"])


def test_plan_at_the_benchmark_sizes(lib):
    """r = 48: Kmax = 2 r^2 = 4608; 17 moduli and 48 bits at S = 8 (13 moduli, 36 bits at S = 6), one
    chunk for K = r^2, two for K = 2 r^2."""
    p = lib.acse_ozaki_plan_info(8, 4608, 2304)
    assert (p["moduli_count"], p["bits"], p["chunks"]) == (17, 48, 1)
    assert lib.acse_ozaki_plan_info(8, 4608, 4608)["chunks"] == 2
    p = lib.acse_ozaki_plan_info(6, 4608, 1128)
    assert (p["moduli_count"], p["bits"], p["chunks"]) == (13, 36, 1)
    assert lib.acse_ozaki_plan_info(10, 8192, 8192)["bits"] == 53


@pytest.mark.parametrize("args", [(3, 100, 10), (11, 100, 10), (8, 0, 1), (8, 8193, 10), (8, 100, 0),
                                  (8, 100, 101)])
def test_plan_rejects_arguments_out_of_range(lib, args):
    with pytest.raises(lib.AcseError):
        lib.acse_ozaki_plan_info(*args)
