"""NY reconstruction (opts.recon = ACSE_RECON_NY) on the GPU vs the FP64 oracle with sigma given.

The oracle's NY path is pinned in test_oracle_pins.py (36- vs nine-term cumulant, exactness for
determinants, factored vs stored 3-RDM, descent identity).  Here the CUDA path (dense spin-orbital
GEMMs for the NY term, added to the V three-body term in the B kernel) must match it: FP64 within
1e-12 normwise, the split precisions within the tolerances of the V path.
"""
import numpy as np
import pytest

import acse_inputs as I
from oracle import acse_oracle as O
from tests.gpu_helpers import maxrel, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# split precisions: about five times the largest normwise error measured on a GB300 (9.7e-6, 1.4e-6)
TOL = {"fp64": 1e-12, "bf16x3": 5e-5, "tf32x3": 7e-6}


@pytest.fixture(scope="module")
def acse():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import api
    return api


def _problem(r, na, nb, seed, kind="state"):
    h, V = I.make_integrals(r, seed)
    if kind == "state":
        D = I.random_state_rdm_blocks(r, na, nb, seed + 1)
    else:
        D = I.random_pair_tensor_blocks(r, seed + 1, hermitian=1, scale=0.05)
    return I.Problem(f"ny_r{r}", r, na, nb, h, V, *D)


def _oracle_residual(p, mask=None):
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    sig = O.sigma_hf(p.r, p.n_alpha, p.n_beta)
    D = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
    A = O.residual(K, D, p.N, sigma=sig)
    n2 = O.norm2(A)
    if mask is not None:
        A = O.active_mask(A, p.r, *mask)
    return O.blocks_from_so(A), n2


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("r,na,nb,kind", [(3, 2, 1, "state"), (4, 2, 2, "state"), (5, 3, 2, "state"),
                                          (7, 3, 3, "pair")])
def test_ny_residual_parity(acse, prec, r, na, nb, kind):
    p = _problem(r, na, nb, 60 + r, kind)
    ctx = acse.ACSE(r, na, nb, p.h, p.V, prec, recon="NY")
    A, n2 = ctx.residual(ctx.to_blocks((p.Daa, p.Dab, p.Dbb)))
    want, n2w = _oracle_residual(p)
    err = maxrel(to_np(A), want)
    print(f"NY {prec} r={r}: max rel err {err:.3e}")
    assert err < TOL[prec]
    assert float(n2) == pytest.approx(n2w, rel=max(1e-12, 4 * TOL[prec]))
    # NY changes the residual: the V context gives something else
    cv = acse.ACSE(r, na, nb, p.h, p.V, "fp64")
    Av, _ = cv.residual(cv.to_blocks((p.Daa, p.Dab, p.Dbb)))
    assert maxrel(to_np(Av), want) > 1e-6
    ctx.close()
    cv.close()


@pytest.mark.parametrize("mask", [None, (1, 4)])
def test_ny_trajectory_fp64(acse, mask):
    """Five Euler steps with the NY reconstruction against the oracle's driver."""
    p = I.make_problem(6, 6, 21, "cas", core=[0], active=[1, 2, 3, 4], nelecas=4)
    eps, nsteps = 1e-3, 5
    ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "fp64", mask=mask, recon="NY")
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    sig = O.sigma_hf(p.r, p.n_alpha, p.n_beta)
    m = None if mask is None else (p.r, *mask)
    out = O.run_acse(p.h, p.V, p.N, O.so_from_blocks(p.Daa, p.Dab, p.Dbb), eps, nsteps, mask=m, sigma=sig)
    for k in range(nsteps):
        E, n2, _ = ctx.step(D, eps)
        assert float(E) == pytest.approx(out["E"][k + 1], abs=1e-10), f"step {k}"
        assert float(n2) == pytest.approx(out["norm2"][k], rel=1e-11)
    assert maxrel(to_np(D), O.blocks_from_so(out["D"])) < 1e-11
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_ny_invariants(acse, prec):
    """Tr(K U) = -||A||^2, Tr U = 0 and anti-Hermiticity with the NY reconstruction (r = 12)."""
    p = I.make_problem(12, 8, 5, "cas", core=[0, 1], active=[2, 3, 4, 5], nelecas=4)
    ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec, recon="NY")
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    D0 = to_np(D)
    A, n2 = ctx.residual(D)
    Aa = to_np(A)
    n2 = float(n2)
    eps = 1e-4
    ctx.step(D, eps)
    U = tuple((a - b) / eps for a, b in zip(to_np(D), D0))
    Kb = O.blocks_from_so(O.reduced_hamiltonian(p.h, p.V, p.N))
    trKU = np.sum(Kb[0] * U[0]) + np.sum(Kb[2] * U[2]) + 4 * np.sum(Kb[1] * U[1])
    assert trKU == pytest.approx(-n2, rel=1e-9 if prec == "fp64" else 2e-4)
    trU = sum(np.einsum("ijij->", u) * w for u, w in zip(U, (1, 2, 1)))
    assert abs(trU) < 1e-9 * max(np.abs(u).max() for u in U) * p.r ** 2
    sym = 1e-12 if prec == "fp64" else 1e-6
    for blk in Aa:
        assert np.abs(blk + blk.transpose(2, 3, 0, 1)).max() <= sym * np.abs(blk).max()
    ctx.close()


def test_ny_unsupported_paths(acse):
    from paper_2604_02550_gb300 import _lib
    p = _problem(4, 2, 2, 3)
    ctx = acse.ACSE(4, 2, 2, p.h, p.V, "fp64", recon="NY")
    with pytest.raises(_lib.AcseError):
        ctx.backward([ctx.to_blocks((p.Daa, p.Dab, p.Dbb))], 1, 1e-3)
    ctx.close()
