"""Spin-flip specialisation (opts.singlet) of the split-precision path vs the FP64 oracle.

For a state with n_alpha = n_beta whose 2-RDM is invariant under exchanging alpha and beta
(D_bb = D_aa, D_ab^{ij}_{kl} = D_ab^{ji}_{lk}; every singlet), the residual has A_bb = A_aa and the
bb-sector GEMMs, the beta-led particle-hole rows and the second spin-flip sector repeat alpha-led
work.  With singlet=True the context skips them.  On such inputs it must match the oracle within
the tolerances of the general split path, give A_bb equal to A_aa bit for bit, and keep the
symmetry along a trajectory.
"""
import numpy as np
import pytest

import acse_inputs as I
from tests.gpu_helpers import maxrel, oracle_residual_blocks, oracle_step_blocks, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# about five times the largest normwise error measured on a GB300 (1.2e-5, 4.9e-4, 3.4e-6)
TOL = {"bf16x3": 6e-5, "tf32": 2.5e-3, "tf32x3": 1.5e-5}


@pytest.fixture(scope="module")
def acse():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import api
    return api


def flip_symmetric(Daa, Dab, Dbb):
    """Average a spin-blocked 2-RDM with its alpha <-> beta image."""
    s = 0.5 * (Daa + Dbb)
    return s, 0.5 * (Dab + Dab.transpose(1, 0, 3, 2)), s.copy()


def _problem(r, n, seed, kind):
    h, V = I.make_integrals(r, seed)
    if kind == "state":
        D = I.random_state_rdm_blocks(r, n, n, seed + 1)
    else:
        D = I.random_pair_tensor_blocks(r, seed + 1, hermitian=1, scale=0.05)
    return I.Problem(f"singlet_r{r}", r, n, n, h, V, *flip_symmetric(*D))


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "tf32"])
@pytest.mark.parametrize("r,n,kind", [(4, 2, "state"), (6, 3, "state"), (9, 3, "pair"), (12, 4, "pair"),
                                      (16, 5, "pair"), (17, 5, "pair")])
def test_singlet_residual_parity(acse, prec, r, n, kind):
    p = _problem(r, n, 300 + r, kind)
    Db = (p.Daa, p.Dab, p.Dbb)
    ctx = acse.ACSE(r, n, n, p.h, p.V, prec, singlet=True)
    A, n2 = ctx.residual(ctx.to_blocks(Db))
    got = to_np(A)
    want, n2w = oracle_residual_blocks(p, Db)
    err = maxrel(got, want)
    print(f"singlet {prec} r={r}: max rel err {err:.3e}")
    assert err < TOL[prec]
    assert float(n2) == pytest.approx(n2w, rel=4 * TOL[prec])
    assert np.array_equal(got[0], got[2])                      # A_bb copied from A_aa
    # the alpha-beta block keeps the flip symmetry to working precision
    ab = got[1]
    assert np.abs(ab - ab.transpose(1, 0, 3, 2)).max() <= TOL[prec] * np.abs(ab).max()
    ctx.close()


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_singlet_matches_general_split_path(acse, prec):
    """Same input through singlet=True and singlet=False: both are the same approximation of A."""
    p = _problem(12, 4, 17, "state")
    Db = (p.Daa, p.Dab, p.Dbb)
    cs = acse.ACSE(p.r, 4, 4, p.h, p.V, prec, singlet=True)
    cg = acse.ACSE(p.r, 4, 4, p.h, p.V, prec)
    As, n2s = cs.residual(cs.to_blocks(Db))
    Ag, n2g = cg.residual(cg.to_blocks(Db))
    assert maxrel(to_np(As), to_np(Ag)) < TOL[prec]
    assert float(n2s) == pytest.approx(float(n2g), rel=2 * TOL[prec])
    cs.close()
    cg.close()


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_singlet_step_parity(acse, prec):
    p = _problem(6, 3, 7, "state")
    Db = (p.Daa, p.Dab, p.Dbb)
    ctx = acse.ACSE(6, 3, 3, p.h, p.V, prec, mask=(1, 4), singlet=True)
    D = ctx.to_blocks(Db)
    eps = 1e-3
    E, n2, _ = ctx.step(D, eps)
    Dw, Ew, n2w = oracle_step_blocks(p, Db, eps, (1, 4))
    Uw = tuple((a - b) / eps for a, b in zip(Dw, Db))
    Dg = to_np(D)
    Ug = tuple((a - b) / eps for a, b in zip(Dg, Db))
    assert maxrel(Ug, Uw) < 2 * TOL[prec]
    assert abs(float(E) - Ew) < {"bf16x3": 1e-6, "tf32x3": 1e-7}[prec]
    assert np.array_equal(Dg[0], Dg[2])
    ctx.close()


def test_singlet_trajectory_config2(acse):
    """r = 24 CAS(6e,6o) singlet reference: 10 BF16x3 steps with and without the specialisation
    track each other (both within the split path's per-step error of the FP64 trajectory)."""
    p = I.config_problem(2)
    assert p.n_alpha == p.n_beta
    Db = flip_symmetric(p.Daa, p.Dab, p.Dbb)
    # the CAS reference is a singlet: symmetrising changes it only at rounding level
    assert maxrel(Db, (p.Daa, p.Dab, p.Dbb)) < 1e-10
    cs = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "bf16x3", singlet=True)
    cg = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "bf16x3")
    c64 = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "fp64")
    Ds, Dg, D64 = cs.to_blocks(Db), cg.to_blocks(Db), c64.to_blocks(Db)
    for k in range(10):
        Es, _, _ = cs.step(Ds, 1e-3)
        Eg, _, _ = cg.step(Dg, 1e-3)
        E64, _, _ = c64.step(D64, 1e-3)
        assert abs(float(Es) - float(E64)) < 5e-4, f"step {k}"   # BF16x3 vs FP64: 8.4e-5 after 10 steps
        assert abs(float(Es) - float(Eg)) < 1e-4, f"step {k}"
    got = to_np(Ds)
    assert np.array_equal(got[0], got[2])
    for c in (cs, cg, c64):
        c.close()


def test_singlet_rejects_open_shell(acse):
    from paper_2604_02550_gb300 import _lib
    h, V = I.make_integrals(5, 1)
    with pytest.raises(_lib.AcseError):
        acse.ACSE(5, 3, 2, h, V, "bf16x3", singlet=True)


def test_singlet_ignored_in_fp64(acse):
    p = _problem(6, 3, 11, "state")
    Db = (p.Daa, p.Dab, p.Dbb)
    c1 = acse.ACSE(6, 3, 3, p.h, p.V, "fp64", singlet=True)
    c0 = acse.ACSE(6, 3, 3, p.h, p.V, "fp64")
    A1, _ = c1.residual(c1.to_blocks(Db))
    A0, _ = c0.residual(c0.to_blocks(Db))
    for x, y in zip(to_np(A1), to_np(A0)):
        assert np.array_equal(x, y)
    c1.close()
    c0.close()


def test_singlet_with_ny_reconstruction(acse):
    """The spin-flip specialisation with the NY 3-cumulant added (its sigma is flip-symmetric for
    n_alpha = n_beta): against the oracle's NY residual."""
    from oracle import acse_oracle as O
    p = _problem(6, 3, 41, "state")
    Db = (p.Daa, p.Dab, p.Dbb)
    ctx = acse.ACSE(6, 3, 3, p.h, p.V, "bf16x3", recon="NY", singlet=True)
    A, n2 = ctx.residual(ctx.to_blocks(Db))
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    sig = O.sigma_hf(p.r, 3, 3)
    Aw = O.residual(K, O.so_from_blocks(*Db), p.N, sigma=sig)
    want = O.blocks_from_so(Aw)
    got = to_np(A)
    err = maxrel(got, want)
    print(f"singlet NY bf16x3: max rel err {err:.3e}")
    assert err < TOL["bf16x3"]
    assert float(n2) == pytest.approx(O.norm2(Aw), rel=4 * TOL["bf16x3"])
    assert np.array_equal(got[0], got[2])
    ctx.close()
