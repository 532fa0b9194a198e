"""CPU check of the same-spin pair packing that the split-precision path's GEMMs rely on.

In the alpha-alpha and beta-beta sectors the rows (ij), the columns (kp) and the contraction index
pair (rs) of X = [M; D] W^T are antisymmetric pairs.  The tensor-core path therefore multiplies
matrices over the pairs a < b only (P = r(r-1)/2 rows and columns, row-major numbering pk(a, b)) with
alpha = 2 for the halved (rs) sum, and recovers every element by antisymmetry:
    X[(i,j)][(k,p)] = s_ij s_kp Xp[pk(i,j)][pk(k,p)],  s_ab = +1 (a < b), -1 (a > b), 0 (a = b).
The Q partial trace Q[k][i] = sum_p X[(i,p)][(k,p)] is read from the packed output the same way.
These identities are checked here in numpy against the unpacked contraction on random antisymmetric
tensors; nothing of the library is used.
"""
import numpy as np
import pytest


def pk(r, a, b):
    """Row-major number of the pair a < b among the r(r-1)/2 pairs."""
    return a * r - a * (a + 1) // 2 + (b - a - 1)


def antisym_pairs(rng, r):
    """A random tensor T[i,j,k,l] antisymmetric in (i, j) and in (k, l)."""
    t = rng.standard_normal((r, r, r, r))
    t = t - t.transpose(1, 0, 2, 3)
    return t - t.transpose(0, 1, 3, 2)


def packed(t, r):
    P = r * (r - 1) // 2
    out = np.zeros((P, P))
    for i in range(r):
        for j in range(i + 1, r):
            for k in range(r):
                for l in range(k + 1, r):
                    out[pk(r, i, j), pk(r, k, l)] = t[i, j, k, l]
    return out


def sign(a, b):
    return 0.0 if a == b else (1.0 if a < b else -1.0)


@pytest.mark.parametrize("r", [2, 3, 5, 8])
def test_pair_numbering_is_a_bijection(r):
    P = r * (r - 1) // 2
    seen = sorted(pk(r, a, b) for a in range(r) for b in range(a + 1, r))
    assert seen == list(range(P))


@pytest.mark.parametrize("r", [2, 3, 4, 7])
def test_packed_gemm_with_alpha_two_reproduces_every_element(r):
    rng = np.random.default_rng(100 + r)
    M = antisym_pairs(rng, r)
    W = antisym_pairs(rng, r)
    # X^{ij}_{kp} = sum_{rs} M^{ij}_{rs} W^{kp}_{rs}, every (r, s) order
    X = np.einsum("ijrs,kprs->ijkp", M, W)
    Xp = 2.0 * packed(M, r) @ packed(W, r).T
    for i in range(r):
        for j in range(r):
            for k in range(r):
                for p in range(r):
                    s = sign(i, j) * sign(k, p)
                    want = X[i, j, k, p]
                    got = 0.0 if s == 0.0 else s * Xp[pk(r, min(i, j), max(i, j)), pk(r, min(k, p), max(k, p))]
                    assert got == pytest.approx(want, abs=1e-12 * max(1.0, np.abs(X).max()))


@pytest.mark.parametrize("r", [3, 6])
def test_partial_trace_from_packed_output(r):
    rng = np.random.default_rng(200 + r)
    M = antisym_pairs(rng, r)
    W = antisym_pairs(rng, r)
    X = np.einsum("ijrs,kprs->ijkp", M, W)
    Q_full = np.einsum("ipkp->ki", X)
    Xp = 2.0 * packed(M, r) @ packed(W, r).T
    Q_packed = np.zeros((r, r))
    for k in range(r):
        for i in range(r):
            acc = 0.0
            for p in range(r):
                if i == p or k == p:
                    continue
                v = Xp[pk(r, min(i, p), max(i, p)), pk(r, min(k, p), max(k, p))]
                acc += v if (i < p) == (k < p) else -v
            Q_packed[k, i] = acc
    np.testing.assert_allclose(Q_packed, Q_full, rtol=0, atol=1e-12 * max(1.0, np.abs(Q_full).max()))
