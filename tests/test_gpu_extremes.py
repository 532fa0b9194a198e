"""The size limits of every precision: the smallest problem (r = 2, one alpha and one beta electron:
one same-spin pair, P = 1), r above the limit (rejected), and the largest supported r = 64
(128 spin orbitals: 2r^2 = 8192 contraction rows, the 2 x 64^2 K of the particle-hole GEMM, every
tile ragged against the 128 x 256 GEMM tile), checked against the oracle on sampled entries.
"""
import numpy as np
import pytest

import acse_inputs as I
from oracle import acse_oracle as O
from tests.gpu_helpers import maxrel, oracle_residual_blocks, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# split precisions: about five times the largest error measured on a GB300 at r = 2 (1.2e-5, 3.4e-7, 7.1e-4)
TOL = {"fp64": 1e-12, "ozaki": 1e-12, "bf16x3": 6e-5, "tf32x3": 2e-6, "tf32": 3.5e-3}


@pytest.fixture(scope="module")
def acse():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import api
    return api


@pytest.mark.parametrize("prec,singlet", [("fp64", False), ("ozaki", False), ("bf16x3", False), ("tf32x3", False),
                                          ("tf32", False), ("bf16x3", True)])
def test_smallest_problem(acse, prec, singlet):
    h, V = I.make_integrals(2, 4)
    Daa, Dab, Dbb = I.random_pair_tensor_blocks(2, 5, hermitian=1, scale=0.2)
    if singlet:
        s = 0.5 * (Daa + Dbb)
        Daa, Dab, Dbb = s, 0.5 * (Dab + Dab.transpose(1, 0, 3, 2)), s.copy()
    p = I.Problem("r2", 2, 1, 1, h, V, Daa, Dab, Dbb)
    Db = (p.Daa, p.Dab, p.Dbb)
    ctx = acse.ACSE(2, 1, 1, p.h, p.V, prec, singlet=singlet)
    A, n2 = ctx.residual(ctx.to_blocks(Db))
    want, n2w = oracle_residual_blocks(p, Db)
    err = maxrel(to_np(A), want)
    print(f"r=2 {prec} singlet={singlet}: max rel err {err:.3e}")
    assert err < TOL[prec]
    assert float(n2) == pytest.approx(n2w, rel=max(1e-12, 4 * TOL[prec]))
    D = ctx.to_blocks(Db)
    E, _, _ = ctx.step(D, 1e-3)
    assert np.isfinite(float(E))
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "ozaki", "bf16x3", "tf32x3", "tf32"])
def test_above_the_limit_is_rejected(acse, prec):
    from paper_2604_02550_gb300 import _lib
    h = np.zeros((65, 65))
    V = np.zeros((2, 2, 2, 2))     # never read: the shape check comes first
    with pytest.raises(_lib.AcseError) as ei:
        _lib.acse_create(65, 4, 4, h, V, prec)
    assert ei.value.status == -2


R = 64


@pytest.fixture(scope="module")
def largest():
    """A random pair-Hermitian 2-RDM at r = 64 and the oracle's values of 12 sampled entries
    (the six-term equation with each 3-RDM element formed on the fly)."""
    h, V = I.make_integrals(R, 91)
    D = I.random_pair_tensor_blocks(R, 92, hermitian=1, scale=0.02)
    p = I.Problem("pair64", R, 12, 12, h, V, *D)
    rng = np.random.default_rng(93)
    ent = []
    for blk, sector in enumerate(("aa", "ab", "bb")):
        for _ in range(4):
            while True:
                i, j, k, l = (int(x) for x in rng.integers(0, R, 4))
                if sector == "ab" or (i != j and k != l):
                    break
            off = {"aa": (0, 0, 0, 0), "ab": (0, R, 0, R), "bb": (R, R, R, R)}[sector]
            ent.append((tuple(x + o for x, o in zip((i, j, k, l), off)), blk, (i, j, k, l)))
    want = O.residual_entries(p.h, p.V, p.N, p.Daa, p.Dab, p.Dbb, [so for so, _, _ in ent])
    return p, ent, want


@pytest.mark.parametrize("prec", ["bf16x3", "ozaki", "fp64"])
def test_largest_problem_sampled_entries(acse, largest, prec):
    p, ent, want = largest
    ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec)
    A, n2 = ctx.residual(ctx.to_blocks((p.Daa, p.Dab, p.Dbb)))
    Ab = to_np(A)
    got = np.array([Ab[blk][idx] for _, blk, idx in ent])
    scale = np.abs(want).max()
    err = np.abs(got - want).max() / scale
    print(f"r=64 {prec}: sampled max |A| {scale:.3e}, max rel err {err:.3e}")
    assert scale > 0
    assert err < {"fp64": 1e-11, "ozaki": 1e-11, "bf16x3": 5e-4}[prec]
    # the norm is the spin-orbital Frobenius norm of the returned blocks
    assert float(n2) == pytest.approx(np.sum(Ab[0] ** 2) + np.sum(Ab[2] ** 2) + 4 * np.sum(Ab[1] ** 2), rel=1e-12)
    ctx.close()
