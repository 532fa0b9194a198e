"""The CTA-pair form of the tensor-core GEMMs (acse_opts.gemm_tile = 2: clusters of two CTAs share each
256 x 256 output tile through the pair MMA) against the FP64 oracle and against the one-SM form.

Both forms run the same products in the same K order into FP32 accumulators, so the residuals are
compared with each other exactly; against the oracle the split-precision tolerances of the one-SM form
apply (about five times the error measured on a GB300).  Shapes: r = 16 (the smallest r with 256-wide
tiles; same-spin pair GEMMs of 240 x 120, single ragged tiles), r = 20 (380 x 190: ragged in both M and
N), r = 32, and the r = 48 workload (every GEMM spanning many tiles, the persistent schedule in full)."""
import numpy as np
import pytest

import acse_inputs as I
from tests.gpu_helpers import maxrel, oracle_residual_blocks, to_np

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


def _problem(r, na, nb, seed):
    h, V = I.make_integrals(r, seed)
    D = I.random_pair_tensor_blocks(r, seed + 1, hermitian=1, scale=0.05)
    return I.Problem(f"rand_r{r}", r, na, nb, h, V, *D)


def _residual(acse, p, prec, tile, **kw):
    from paper_2604_02550_gb300 import _lib
    ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec, gemm_tile=tile, **kw)
    A, n2 = ctx.residual(ctx.to_blocks((p.Daa, p.Dab, p.Dbb)))
    _lib.acse_sync_status(ctx.ctx)
    out = to_np(A), float(n2)
    ctx.close()
    return out


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("r,na,nb", [(16, 5, 4), (20, 6, 5), (32, 7, 6)])
def test_pair_vs_oracle_and_one_sm(acse, prec, r, na, nb):
    p = _problem(r, na, nb, 300 + r)
    A2, n2 = _residual(acse, p, prec, 2)
    A1, n1 = _residual(acse, p, prec, 1)
    want, n2w = oracle_residual_blocks(p, (p.Daa, p.Dab, p.Dbb))
    err = maxrel(A2, want)
    d12 = max(float(np.max(np.abs(a - b))) for a, b in zip(A2, A1))
    print(f"{prec} r={r}: pair vs oracle {err:.3e}; pair vs one-SM max |dA| {d12:.3e}")
    assert err < TOL[prec]
    assert n2 == pytest.approx(n2w, rel=NTOL[prec])
    assert d12 == 0.0 and n2 == n1


def test_pair_singlet_and_r48(acse):
    """The r = 48 CAS(8e,8o) workload in BF16x3, general and spin-flip-specialised: the pair form
    gives the one-SM form's residual exactly."""
    p = I.config_problem(3)
    for singlet in (False, True):
        A2, n2 = _residual(acse, p, "bf16x3", 2, singlet=singlet)
        A1, n1 = _residual(acse, p, "bf16x3", 1, singlet=singlet)
        d12 = max(float(np.max(np.abs(a - b))) for a, b in zip(A2, A1))
        print(f"r=48 singlet={singlet}: pair vs one-SM max |dA| {d12:.3e}, norm2 {n2:.12e} vs {n1:.12e}")
        assert d12 == 0.0 and n2 == n1


def test_pair_steps_match_one_sm(acse):
    """Ten fixed steps at r = 24 (config 2): identical trajectories in both forms."""
    p = I.config_problem(2)
    runs = []
    for tile in (2, 1):
        ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "bf16x3", gemm_tile=tile)
        D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
        Es = [float(ctx.step(D, 1e-3)[0]) for _ in range(10)]
        runs.append(Es)
        ctx.close()
    print("pair:", runs[0][-1], "one-SM:", runs[1][-1])
    assert runs[0] == runs[1]


def test_pair_timeout_status_and_recovery(acse):
    """The bounded waits of the pair kernel: the MMA thread of the even CTA first waits on a barrier
    that nothing signals (1 ms bound set from the host); the launch ends with ACSE_ERR_TIMEOUT and no
    fault, and with the knob off the next call is correct again."""
    from paper_2604_02550_gb300 import _lib
    p = _problem(16, 5, 4, 5)
    ctx = acse.ACSE(16, 5, 4, p.h, p.V, "bf16x3", gemm_tile=2)
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


@pytest.mark.parametrize("r,na,nb", [(16, 5, 4), (20, 6, 5), (32, 7, 6)])
def test_pair_ozaki(acse, r, na, nb):
    """The Ozaki GEMMs on CTA pairs: the exact residue sums and the exact reconstruction make the
    residual identical to the one-SM form's; against the oracle the FP64-accurate bound (1e-12 relative)
    holds."""
    p = _problem(r, na, nb, 400 + r)
    A2, n2 = _residual(acse, p, "ozaki", 2)
    A1, n1 = _residual(acse, p, "ozaki", 1)
    want, n2w = oracle_residual_blocks(p, (p.Daa, p.Dab, p.Dbb))
    err = maxrel(A2, want)
    d12 = max(float(np.max(np.abs(a - b))) for a, b in zip(A2, A1))
    print(f"ozaki r={r}: pair vs oracle {err:.3e}; pair vs one-SM max |dA| {d12:.3e}")
    assert err < 1e-12
    assert d12 == 0.0 and n2 == n1


def test_pair_ozaki_adjoint(acse):
    """The adjoint's Ozaki GEMM lists run on CTA pairs too (r = 16: 256-wide tiles): gradients identical
    to the one-SM form's."""
    p = _problem(16, 5, 4, 77)
    grads = []
    for tile in (2, 1):
        ctx = acse.ACSE(16, 5, 4, p.h, p.V, "ozaki", gemm_tile=tile)
        D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
        dh, dV, dD = ctx.backward([D], 2, 1e-4, 1.0, 0.5)
        grads.append([dh.cpu().numpy(), dV.cpu().numpy()] + [x.cpu().numpy() for x in dD])
        ctx.close()
    d = max(float(np.max(np.abs(a - b))) for a, b in zip(*grads))
    print(f"ozaki adjoint: pair vs one-SM max |d grad| {d:.3e}")
    assert d == 0.0


def test_pair_ozaki_timeout_status_and_recovery(acse):
    from paper_2604_02550_gb300 import _lib
    p = _problem(16, 5, 4, 6)
    ctx = acse.ACSE(16, 5, 4, p.h, p.V, "ozaki", gemm_tile=2)
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
    assert maxrel(to_np(A), want) < 1e-12
    ctx.close()
