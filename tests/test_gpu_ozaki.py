"""ACSE_OZAKI: FP64-accurate contractions with the O(r^6) GEMMs run by the modular Ozaki scheme on the
BF16 tensor cores (integer rows of min(6S, 53) bits, residue products modulo pairwise coprime moduli,
exact reconstruction by the Chinese remainder theorem), against the FP64 oracle (the FP64 tolerances:
1e-12 normwise on A, 1e-10 Eh on E) and against the FP64 FMA path on the GPU.

The GEMMs are exact on the integer rows, so their error is the rounding of the operands to 6S bits below
each row's leading bit: with the default S = 8 about 2^-48 |A||B| K, below the FP64 FMA path's own
rounding.  Fewer slices must make the error grow by about 2^6 a slice (the error is that rounding and
nothing else), which pins the scaling, the moduli count and the reconstruction.
"""
import numpy as np
import pytest

import acse_inputs as I
from oracle import acse_oracle as O
from tests.gpu_helpers import maxrel, oracle_residual_blocks, oracle_step_blocks, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_A = 1e-12
TOL_E = 1e-10


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
    return I.Problem(f"oz_r{r}", r, na, nb, h, V, *D)


@pytest.mark.parametrize("r,na,nb,kind", [(3, 2, 1, "state"), (4, 2, 2, "state"), (5, 3, 2, "state"),
                                          (6, 2, 2, "state"), (9, 3, 3, "pair"), (12, 4, 3, "pair"),
                                          (17, 5, 4, "pair")])
def test_ozaki_residual_parity(acse, r, na, nb, kind):
    p = _problem(r, na, nb, 10 + r, kind)
    Db = (p.Daa, p.Dab, p.Dbb)
    ctx = acse.ACSE(r, na, nb, p.h, p.V, "ozaki")
    A, n2 = ctx.residual(ctx.to_blocks(Db))
    want, n2w = oracle_residual_blocks(p, Db)
    err = maxrel(to_np(A), want)
    print(f"ozaki r={r}: max rel err {err:.3e}")
    assert err < TOL_A
    assert float(n2) == pytest.approx(n2w, rel=1e-12)
    ctx.close()


@pytest.mark.parametrize("r,na,nb,kind,mask", [(4, 2, 2, "state", None), (5, 2, 2, "state", (1, 4)),
                                               (10, 3, 3, "pair", (2, 7))])
def test_ozaki_step_parity(acse, r, na, nb, kind, mask):
    p = _problem(r, na, nb, 60 + r, kind)
    Db = (p.Daa, p.Dab, p.Dbb)
    ctx = acse.ACSE(r, na, nb, p.h, p.V, "ozaki", mask=mask)
    D = ctx.to_blocks(Db)
    eps = 1e-3
    E, n2, _ = ctx.step(D, eps)
    Dw, Ew, n2w = oracle_step_blocks(p, Db, eps, mask)
    Uw = tuple((a - b) / eps for a, b in zip(Dw, Db))
    Ug = tuple((a - b) / eps for a, b in zip(to_np(D), Db))
    assert maxrel(Ug, Uw) < 1e-10
    assert float(E) == pytest.approx(Ew, abs=TOL_E)
    assert float(n2) == pytest.approx(n2w, rel=1e-12)
    ctx.close()


def test_ozaki_config1_trajectory(acse):
    """r = 8 HF reference, one residual and 20 steps against the oracle (E at every step)."""
    p = I.config_problem(1)
    ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "ozaki")
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    Do = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
    for n in range(20):
        E, _, _ = ctx.step(D, 1e-3)
        Do, _, _ = O.step(K, Do, p.N, 1e-3)
        assert float(E) == pytest.approx(O.energy(K, Do), abs=TOL_E), f"step {n}"
    assert maxrel(to_np(D), O.blocks_from_so(Do)) < 1e-11
    ctx.close()


def test_ozaki_matches_fp64_gpu_config2(acse):
    """r = 24 CAS(6e,6o): Ozaki and FP64 FMA residuals agree to FP64 rounding, and so do ten steps."""
    p = I.config_problem(2)
    Db = (p.Daa, p.Dab, p.Dbb)
    c64 = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "fp64")
    coz = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "ozaki")
    D64, Doz = c64.to_blocks(Db), coz.to_blocks(Db)
    A64, n64 = c64.residual(D64)
    Aoz, noz = coz.residual(Doz)
    err = maxrel(to_np(Aoz), to_np(A64))
    print(f"config 2: Ozaki vs FP64 GPU residual max rel diff {err:.3e}")
    assert err < TOL_A
    assert float(noz) == pytest.approx(float(n64), rel=1e-12)
    for k in range(10):
        E64, _, _ = c64.step(D64, 1e-3)
        Eoz, _, _ = coz.step(Doz, 1e-3)
        assert abs(float(Eoz) - float(E64)) < TOL_E, f"step {k}"
    assert maxrel(to_np(Doz), to_np(D64)) < 1e-11
    c64.close()
    coz.close()


def test_ozaki_error_falls_with_slices(acse):
    """The error against the oracle falls by roughly 2^6 per added slice until it reaches FP64
    rounding: measured 1.7e-7, 4.1e-9, 5.5e-11 and 1.1e-14 for 4, 5, 6 and 8 slices."""
    p = _problem(9, 3, 3, 5, "pair")
    Db = (p.Daa, p.Dab, p.Dbb)
    want, _ = oracle_residual_blocks(p, Db)
    errs = {}
    for S in (4, 5, 6, 8):
        ctx = acse.ACSE(p.r, 3, 3, p.h, p.V, "ozaki", oz_slices=S)
        A, _ = ctx.residual(ctx.to_blocks(Db))
        errs[S] = maxrel(to_np(A), want)
        ctx.close()
    print("ozaki error by slices:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert errs[4] > 1e-10 and errs[4] < 1e-5
    assert errs[5] < errs[4] / 8 and errs[6] < errs[5] / 8
    assert errs[8] < TOL_A


def test_ozaki_options_and_errors(acse):
    from paper_2604_02550_gb300 import _lib
    h, V = I.make_integrals(4, 2)
    for bad in (3, 11):
        with pytest.raises(_lib.AcseError):
            acse.ACSE(4, 2, 2, h, V, "ozaki", oz_slices=bad)
    # a non-finite entry of D reaches the result as NaN (the row scale of its slices is NaN)
    p = _problem(4, 2, 2, 9)
    Daa = p.Daa.copy()
    Daa[0, 1, 0, 1] = np.nan
    Daa[1, 0, 1, 0] = np.nan
    ctx = acse.ACSE(4, 2, 2, p.h, p.V, "ozaki")
    A, n2 = ctx.residual(ctx.to_blocks((Daa, p.Dab, p.Dbb)))
    assert not np.isfinite(float(n2))
    ctx.close()


def test_ozaki_timeout_status_and_recovery(acse):
    """A bounded wait of the Ozaki GEMM that runs out (the MMA thread waits on a barrier nothing
    signals, 1 ms bound) ends the launch with ACSE_ERR_TIMEOUT and no fault; the next call is correct."""
    from paper_2604_02550_gb300 import _lib
    p = _problem(12, 4, 3, 3, "pair")
    Db = (p.Daa, p.Dab, p.Dbb)
    ctx = acse.ACSE(12, 4, 3, p.h, p.V, "ozaki")
    D = ctx.to_blocks(Db)
    _lib.acse_set_wait_bound_ns(ctx.ctx, 1_000_000, inject_stall=True)
    ctx.residual(D)
    with pytest.raises(_lib.AcseError) as ei:
        _lib.acse_sync_status(ctx.ctx)
    assert ei.value.status == -6
    _lib.acse_set_wait_bound_ns(ctx.ctx, 0, inject_stall=False)
    _lib.acse_clear_status(ctx.ctx)
    A, _ = ctx.residual(D)
    _lib.acse_sync_status(ctx.ctx)
    want, _ = oracle_residual_blocks(p, Db)
    assert maxrel(to_np(A), want) < TOL_A
    ctx.close()


def test_ozaki_adjoint_matches_fp64(acse):
    """The adjoint of an Ozaki context (its reverse sweep's GEMMs by the Ozaki scheme) equals an FP64
    context's gradient to 1e-10 relative."""
    p = _problem(5, 2, 2, 31)
    Db = (p.Daa, p.Dab, p.Dbb)
    grads = []
    for prec in ("fp64", "ozaki"):
        ctx = acse.ACSE(5, 2, 2, p.h, p.V, prec)
        D0 = ctx.to_blocks(Db)
        D = tuple(x.clone() for x in D0)
        ck = [tuple(x.clone() for x in D)]
        for _ in range(2):
            ctx.step(D, 1e-3)
            ck.append(tuple(x.clone() for x in D))
        grads.append([to_np(g) if isinstance(g, tuple) else g.detach().cpu().numpy()
                      for g in ctx.backward(ck, 2, 1e-3)])
        ctx.close()
    for a, b in zip(grads[0], grads[1]):
        if isinstance(a, tuple):
            for x, y in zip(a, b):
                assert np.abs(x - y).max() <= 1e-10 * max(np.abs(x).max(), 1e-300)
        else:
            assert np.abs(a - b).max() <= 1e-10 * max(np.abs(a).max(), 1e-300)
