"""Split-precision (BF16x3, TF32) tensor-core path vs the FP64 oracle and the FP64 GPU path.

Tolerances (normwise relative, max|dA| / max|A|), about five times the largest error measured on a
GB300 over these cases: BF16x3 represents each operand as hi + lo with about 16 significant bits and
drops the lo.lo product (about 2^-16 = 1.5e-5 relative per product before FP32 accumulation; measured
3.9e-6 ... 7.7e-6 on the residual, r = 4 ... 32): 3e-5.  TF32 (one product, 11 significant bits,
2^-11 = 4.9e-4 per product; measured 1.6e-4 ... 3.0e-4): 1.5e-3.  TF32x3 (hi + lo in tf32, about 2^-21
per product, then limited by the FP32 intermediates M, Z, w, B and the FP32 accumulation; measured
2.3e-7 ... 1.3e-5, growing with r): 5e-5.  ||A||^2 (relative; measured up to 9.5e-6, 4.8e-5 and
2.1e-5): NTOL.
"""
import numpy as np
import pytest

import acse_inputs as I
from oracle import acse_oracle as O
from tests.gpu_helpers import maxrel, oracle_residual_blocks, oracle_step_blocks, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 3e-5, "tf32": 1.5e-3, "tf32x3": 5e-5}
NTOL = {"bf16x3": 5e-5, "tf32": 2.5e-4, "tf32x3": 1e-4}


@pytest.fixture(scope="module")
def acse():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import api
    return api


def _problem(r, na, nb, seed, kind):
    h, V = I.make_integrals(r, seed)
    if kind == "state":
        D = I.random_state_rdm_blocks(r, na, nb, seed + 1)
    else:
        D = I.random_pair_tensor_blocks(r, seed + 1, hermitian=1, scale=0.05)
    return I.Problem(f"rand_r{r}", r, na, nb, h, V, *D)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "tf32x3"])
@pytest.mark.parametrize("r,na,nb,kind", [(4, 2, 2, "state"), (6, 3, 2, "state"), (9, 3, 3, "pair"),
                                          (12, 4, 3, "pair"), (16, 5, 4, "pair"), (17, 5, 4, "pair"),
                                          (32, 7, 6, "pair")])
def test_residual_parity_mixed(acse, prec, r, na, nb, kind):
    p = _problem(r, na, nb, 100 + r, kind)
    ctx = acse.ACSE(r, na, nb, p.h, p.V, prec)
    A, n2 = ctx.residual(ctx.to_blocks((p.Daa, p.Dab, p.Dbb)))
    from paper_2604_02550_gb300 import _lib
    _lib.acse_sync_status(ctx.ctx)
    want, n2w = oracle_residual_blocks(p, (p.Daa, p.Dab, p.Dbb))
    err = maxrel(to_np(A), want)
    print(f"{prec} r={r}: max rel err {err:.3e}, norm2 rel err {abs(float(n2) - n2w) / n2w:.3e}")
    assert err < TOL[prec]
    assert float(n2) == pytest.approx(n2w, rel=NTOL[prec])
    ctx.close()


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "tf32x3"])
def test_step_parity_mixed(acse, prec):
    p = _problem(6, 3, 3, 7, "state")
    ctx = acse.ACSE(6, 3, 3, p.h, p.V, prec, mask=(1, 4))
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    eps = 1e-3
    E, n2, _ = ctx.step(D, eps)
    Dw, Ew, n2w = oracle_step_blocks(p, (p.Daa, p.Dab, p.Dbb), eps, (1, 4))
    Uw = tuple((a - b) / eps for a, b in zip(Dw, (p.Daa, p.Dab, p.Dbb)))
    Ug = tuple((a - b) / eps for a, b in zip(to_np(D), (p.Daa, p.Dab, p.Dbb)))
    err = maxrel(Ug, Uw)
    print(f"{prec} step: U rel err {err:.3e}, E err {abs(float(E) - Ew):.3e}")
    assert err < 2 * TOL[prec]
    # measured 7.5e-9, 3.8e-9, 5.5e-8 Eh
    assert abs(float(E) - Ew) < {"bf16x3": 4e-8, "tf32x3": 2e-8, "tf32": 3e-7}[prec]
    ctx.close()


def test_mixed_vs_fp64_gpu_config2(acse):
    """r = 24, CAS(6e,6o): BF16x3 and FP64 GPU residuals on the same input, and energies over
    10 steps (mixed-precision error per iteration)."""
    p = I.config_problem(2)
    c64 = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "fp64")
    cmx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "bf16x3")
    D64 = c64.to_blocks((p.Daa, p.Dab, p.Dbb))
    Dmx = cmx.to_blocks((p.Daa, p.Dab, p.Dbb))
    A64, _ = c64.residual(D64)
    Amx, _ = cmx.residual(Dmx)
    err = maxrel(to_np(Amx), to_np(A64))
    print(f"config 2 residual: BF16x3 vs FP64 max rel err {err:.3e}")
    assert err < TOL["bf16x3"]
    dE = []
    for n in range(10):
        E64, _, _ = c64.step(D64, 1e-3)
        Emx, _, _ = cmx.step(Dmx, 1e-3)
        dE.append(abs(float(Emx) - float(E64)))
    print("per-step |E_bf16x3 - E_fp64|:", " ".join(f"{x:.2e}" for x in dE))
    # the split-precision error of E grows about linearly with the steps (measured 8.2e-7 after the first
    # step, 8.4e-5 after the tenth): a bound of about five times that per step
    for n, d in enumerate(dE):
        assert d < 5e-6 + 5e-5 * n, f"step {n}: {d:.2e}"
    c64.close()
    cmx.close()


def test_timeout_status_and_recovery(acse):
    """A bounded device wait that runs out (the MMA thread waits on a barrier that nothing
    signals, with a 1 ms bound set from the host) ends the GEMM with ACSE_ERR_TIMEOUT and no
    fault; with the knob off the next call is correct again."""
    from paper_2604_02550_gb300 import _lib
    p = _problem(12, 4, 3, 3, "pair")
    ctx = acse.ACSE(12, 4, 3, p.h, p.V, "bf16x3")
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    _lib.acse_set_wait_bound_ns(ctx.ctx, 1_000_000, inject_stall=True)
    ctx.residual(D)
    with pytest.raises(_lib.AcseError) as ei:
        _lib.acse_sync_status(ctx.ctx)
    assert ei.value.status == -6
    _lib.acse_set_wait_bound_ns(ctx.ctx, 0, inject_stall=False)
    _lib.acse_clear_status(ctx.ctx)
    A, _ = ctx.residual(D)
    _lib.acse_sync_status(ctx.ctx)
    want, _ = oracle_residual_blocks(p, (p.Daa, p.Dab, p.Dbb))
    assert maxrel(to_np(A), want) < TOL["bf16x3"]
    ctx.close()
