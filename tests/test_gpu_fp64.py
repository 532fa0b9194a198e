"""FP64 CUDA path vs the FP64 oracle, through the C ABI (requires a GB300)."""
import numpy as np
import pytest

import acse_inputs as I
from oracle import acse_oracle as O
from tests.gpu_helpers import maxrel, oracle_residual_blocks, oracle_step_blocks, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_A = 1e-12      # max|dA| <= 1e-12 max|A| (normwise relative)
TOL_E = 1e-10      # Eh


@pytest.fixture(scope="module")
def acse():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import api
    return api


def _random_problem(r, na, nb, seed, kind="state"):
    """kind='state': 2-RDM of a random CI vector (all index paths populated, N-representable);
    kind='pair': a random antisymmetric pair-Hermitian tensor (any r)."""
    h, V = I.make_integrals(r, seed)
    if kind == "state":
        D = I.random_state_rdm_blocks(r, na, nb, seed + 1)
    else:
        D = I.random_pair_tensor_blocks(r, seed + 1, hermitian=1, scale=0.05)
    return I.Problem(f"rand_r{r}", r, na, nb, h, V, *D)


@pytest.mark.parametrize("r,na,nb,kind", [(3, 2, 1, "state"), (4, 2, 2, "state"), (5, 3, 2, "state"),
                                          (6, 2, 2, "state"), (9, 3, 3, "pair"), (12, 4, 3, "pair")])
def test_residual_parity(acse, r, na, nb, kind):
    p = _random_problem(r, na, nb, 10 + r, kind)
    ctx = acse.ACSE(r, na, nb, p.h, p.V, "fp64")
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    A, n2 = ctx.residual(D)
    torch.cuda.synchronize()
    want, n2w = oracle_residual_blocks(p, (p.Daa, p.Dab, p.Dbb))
    assert maxrel(to_np(A), want) < TOL_A
    assert float(n2) == pytest.approx(n2w, rel=1e-12)
    ctx.close()


@pytest.mark.parametrize("r,na,nb", [(4, 2, 2), (6, 3, 2)])
def test_energy_parity(acse, r, na, nb):
    p = _random_problem(r, na, nb, 40 + r)
    ctx = acse.ACSE(r, na, nb, p.h, p.V, "fp64")
    E = float(ctx.energy(ctx.to_blocks((p.Daa, p.Dab, p.Dbb))))
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    assert E == pytest.approx(O.energy(K, O.so_from_blocks(p.Daa, p.Dab, p.Dbb)), abs=TOL_E)
    ctx.close()


@pytest.mark.parametrize("r,na,nb,kind,mask", [(4, 2, 2, "state", None), (5, 2, 2, "state", (1, 4)),
                                               (10, 3, 3, "pair", (2, 7))])
def test_step_parity(acse, r, na, nb, kind, mask):
    p = _random_problem(r, na, nb, 60 + r, kind)
    ctx = acse.ACSE(r, na, nb, p.h, p.V, "fp64", mask=mask)
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    eps = 1e-3
    E, n2, e_used = ctx.step(D, eps)
    torch.cuda.synchronize()
    Dw, Ew, n2w = oracle_step_blocks(p, (p.Daa, p.Dab, p.Dbb), eps, mask)
    # compare the update itself: (D_new - D_old) / eps
    Uw = tuple((a - b) / eps for a, b in zip(Dw, (p.Daa, p.Dab, p.Dbb)))
    Ug = tuple((a - b) / eps for a, b in zip(to_np(D), (p.Daa, p.Dab, p.Dbb)))
    assert maxrel(Ug, Uw) < 1e-10
    assert maxrel(to_np(D), Dw) < TOL_A
    assert float(E) == pytest.approx(Ew, abs=TOL_E)
    assert float(n2) == pytest.approx(n2w, rel=1e-12)
    assert float(e_used) == eps
    ctx.close()


def test_mask_residual(acse):
    p = _random_problem(5, 2, 2, 77)
    mask = (1, 4)
    ctx = acse.ACSE(5, 2, 2, p.h, p.V, "fp64", mask=mask)
    A, n2 = ctx.residual(ctx.to_blocks((p.Daa, p.Dab, p.Dbb)))
    want, n2w = oracle_residual_blocks(p, (p.Daa, p.Dab, p.Dbb), mask)
    assert maxrel(to_np(A), want) < TOL_A
    assert float(n2) == pytest.approx(n2w, rel=1e-12)     # norm before the mask
    ctx.close()


def test_config1_trajectory(acse):
    """r = 8, N = 8, HF reference: one residual and 20 steps, E at every step.  eps = 1e-3 (the
    paper's default step); eps = 0.1 diverges to NaN within five steps on these integrals, on the
    oracle and on the GPU alike."""
    p = I.config_problem(1)
    ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "fp64")
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    A, _ = ctx.residual(D)
    want, _ = oracle_residual_blocks(p, (p.Daa, p.Dab, p.Dbb))
    assert maxrel(to_np(A), want) < TOL_A
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    Do = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
    for n in range(20):
        E, _, _ = ctx.step(D, 1e-3)
        Do, _, _ = O.step(K, Do, p.N, 1e-3)
        assert float(E) == pytest.approx(O.energy(K, Do), abs=TOL_E), f"step {n}"
    assert maxrel(to_np(D), O.blocks_from_so(Do)) < 1e-11
    ctx.close()


def test_line_search_steps(acse):
    p = I.make_problem(8, 6, 5, "cas", core=[0], active=[1, 2, 3, 4], nelecas=4)
    ctx = acse.ACSE(p.r, 3, 3, p.h, p.V, "fp64", line_search=True, eps0=1e-3)
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    out = O.run_acse(p.h, p.V, p.N, O.so_from_blocks(p.Daa, p.Dab, p.Dbb), None, 4, line_search=True, eps0=1e-3)
    for n in range(4):
        E, n2, e = ctx.step(D)
        assert float(e) == pytest.approx(out["eps"][n], rel=1e-10)
        assert float(E) == pytest.approx(out["E"][n + 1], abs=TOL_E)
        assert float(n2) == pytest.approx(out["norm2"][n], rel=1e-11)
    ctx.close()


def test_invariants_fp64(acse):
    """Tr(K U) = -||A||^2, Tr U = 0, A anti-Hermitian and antisymmetric (any size)."""
    p = _random_problem(7, 3, 3, 91)
    ctx = acse.ACSE(7, 3, 3, p.h, p.V, "fp64")
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    D0 = to_np(D)
    A, n2 = ctx.residual(D)
    E0 = float(ctx.energy(D))
    eps = 1e-3
    ctx.step(D, eps)
    E1 = float(ctx.energy(D))
    U = tuple((a - b) / eps for a, b in zip(to_np(D), D0))
    Aa = to_np(A)
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    Kb = O.blocks_from_so(K)
    trKU = np.sum(Kb[0] * U[0]) + np.sum(Kb[2] * U[2]) + 4 * np.sum(Kb[1] * U[1])
    assert trKU == pytest.approx(-float(n2), rel=1e-9)
    assert (E1 - E0) / eps == pytest.approx(trKU, rel=1e-9)
    trU = sum(np.einsum("ijij->", u) * w for u, w in zip(U, (1, 2, 1)))
    assert abs(trU) < 1e-9
    for blk in Aa:
        assert np.abs(blk + blk.transpose(2, 3, 0, 1)).max() < 1e-12 * np.abs(blk).max()
    for blk in (Aa[0], Aa[2]):
        assert np.abs(blk + blk.transpose(1, 0, 2, 3)).max() < 1e-12 * np.abs(blk).max()
    ctx.close()


def test_host_pointer_arguments(acse):
    """Host (numpy) buffers through the same C ABI: staged copies inside the call."""
    from paper_2604_02550_gb300 import _lib
    p = _random_problem(4, 2, 2, 5)
    ctx = _lib.acse_create(4, 2, 2, p.h, p.V, "fp64")
    A = [np.zeros_like(p.Daa) for _ in range(3)]
    n2 = np.zeros(1)
    _lib.acse_residual(ctx, p.Daa, p.Dab, p.Dbb, *A, n2)
    want, n2w = oracle_residual_blocks(p, (p.Daa, p.Dab, p.Dbb))
    assert maxrel(A, want) < TOL_A
    assert n2[0] == pytest.approx(n2w, rel=1e-12)
    D = [x.copy() for x in (p.Daa, p.Dab, p.Dbb)]
    E = np.zeros(1)
    _lib.acse_step(ctx, *D, 1e-3, E, None, None)
    Dw, Ew, _ = oracle_step_blocks(p, (p.Daa, p.Dab, p.Dbb), 1e-3)
    assert maxrel(D, Dw) < TOL_A
    assert E[0] == pytest.approx(Ew, abs=TOL_E)
    _lib.acse_destroy(ctx)


def test_error_codes(acse):
    from paper_2604_02550_gb300 import _lib
    p = _random_problem(4, 2, 2, 5)
    with pytest.raises(_lib.AcseError) as ei:
        _lib.acse_create(1, 1, 1, p.h, p.V)
    assert ei.value.status == -2
    with pytest.raises(_lib.AcseError):
        _lib.acse_create(4, 2, 2, p.h, p.V, "fp64", mask=(3, 2))
    ctx = _lib.acse_create(4, 2, 2, p.h, p.V, "fp64", check_inputs=True)
    bad = [x.copy() for x in (p.Daa, p.Dab, p.Dbb)]
    bad[0] *= 2.0                                     # wrong trace
    with pytest.raises(_lib.AcseError) as ei:
        _lib.acse_residual(ctx, *bad, None, None, None, None)
    assert ei.value.status == -4
    bad = [x.copy() for x in (p.Daa, p.Dab, p.Dbb)]
    bad[1][0, 0, 0, 0] = np.nan
    with pytest.raises(_lib.AcseError) as ei:
        _lib.acse_residual(ctx, *bad, None, None, None, None)
    assert ei.value.status == -3
    assert _lib.lib().acse_last_error(ctx) == -3
    _lib.acse_destroy(ctx)


def test_pinned_host_arguments(acse):
    """Pinned (page-locked) host buffers go through the SM copy path: same results as device ones."""
    from paper_2604_02550_gb300 import _lib
    p = _random_problem(6, 3, 2, 8)
    ctx = acse.ACSE(6, 3, 2, p.h, p.V, "fp64")
    Dd = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    Dh = [torch.from_numpy(x.copy()).pin_memory() for x in (p.Daa, p.Dab, p.Dbb)]
    Eh = torch.zeros(1, dtype=torch.float64).pin_memory()
    for _ in range(3):
        E, _, _ = ctx.step(Dd, 1e-3)
        _lib.acse_step(ctx.ctx, *Dh, 1e-3, Eh, None, None)
    torch.cuda.synchronize()
    assert maxrel([x.numpy() for x in Dh], to_np(Dd)) == 0.0
    assert float(Eh[0]) == float(E)
    ctx.close()
