"""Adjoint of the ACSE trajectory (acse_residual_backward) vs the oracle and finite differences.

f = wE E(D_n) + wN ||A(D_n)||^2 after n fixed Euler steps.  The gradient is checked
(1) against the oracle's complex-step directional derivatives (exact to rounding, since the oracle
is polynomial in h, V and D_0) on a small problem, element-free (random symmetric directions), and
(2) on the r = 32, N = 14, CAS(6e,6o) system over 20 steps against central finite differences of the
GPU forward in the same precision with step 1e-5 on 64 random integral directions (agreement 1e-6
relative).  Both run for the FP64 FMA path and for the Ozaki path, whose reverse sweep runs every
GEMM (the forward-shaped passes and the transposed GEMM lists) on the BF16 tensor cores.
"""
import numpy as np
import pytest

import acse_inputs as I
from oracle import acse_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import api as a
    return a


def _sym_dirs(r, rng):
    dh = rng.normal(size=(r, r))
    dh = dh + dh.T
    dV = rng.normal(size=(r,) * 4)
    dV = dV + dV.transpose(1, 0, 2, 3)
    dV = dV + dV.transpose(0, 1, 3, 2)
    dV = dV + dV.transpose(2, 3, 0, 1)
    return dh, dV


def _sym_D(r, seed):
    return I.random_pair_tensor_blocks(r, seed, hermitian=1, scale=1.0)


def _gpu_forward_f(api, p, h, V, D0, eps, nsteps, wE, wN, mask=None, prec="fp64"):
    ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, h, V, prec, mask=mask)
    D = ctx.to_blocks(D0)
    for _ in range(nsteps):
        ctx.step(D, eps)
    E = float(ctx.energy(D))
    _, n2 = ctx.residual(D)
    ctx.close()
    return wE * E + wN * float(n2)


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
@pytest.mark.parametrize("mask", [None, (1, 3)])
def test_adjoint_matches_oracle_complex_step(api, mask, prec):
    p = I.make_problem(4, 4, 31, "cas", core=[0], active=[1, 2, 3], nelecas=2)
    eps, nsteps, wE, wN = 1e-3, 2, 1.0, 0.5
    ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec, mask=mask)
    D0 = (p.Daa, p.Dab, p.Dbb)
    dh, dV, dD = ctx.backward([ctx.to_blocks(D0)], nsteps, eps, wE, wN)
    dh, dV = dh.cpu().numpy(), dV.cpu().numpy()
    dD = [x.cpu().numpy() for x in dD]
    ctx.close()
    rng = np.random.default_rng(5)
    D0so = O.so_from_blocks(*D0)
    m = None if mask is None else (p.r, *mask)
    for k in range(6):
        eh, eV = _sym_dirs(p.r, rng)
        eD = _sym_D(p.r, 100 + k)
        want = O.complex_step_dir(p.h, p.V, p.N, D0so, eps, nsteps, eh, eV, O.so_from_blocks(*eD), wE, wN, m)
        got = np.sum(dh * eh) + np.sum(dV * eV) + sum(np.sum(a * b) for a, b in zip(dD, eD))
        assert got == pytest.approx(want, rel=1e-9, abs=1e-9 * abs(want)), f"direction {k}"


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_adjoint_config5_vs_central_differences(api, prec):
    """r = 32, N = 14, CAS(6e,6o): 20 steps, 64 random integral directions, step 1e-5.  eps = 1e-4:
    at eps = 1e-3 this trajectory diverges within two steps (||A||^2 = 1.2e4 at the reference)."""
    p = I.config_problem(5)
    eps, nsteps, wE, wN = 1e-4, 20, 1.0, 1e-3
    D0 = (p.Daa, p.Dab, p.Dbb)
    ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec)
    dh, dV, dD = ctx.backward([ctx.to_blocks(D0)], nsteps, eps, wE, wN)
    dh, dV = dh.cpu().numpy(), dV.cpu().numpy()
    ctx.close()
    rng = np.random.default_rng(17)
    t = 1e-5
    worst = 0.0
    for k in range(64):
        eh, eV = _sym_dirs(p.r, rng)
        # scale directions like the integrals themselves
        eh *= 0.05
        eV *= 0.01
        fp = _gpu_forward_f(api, p, p.h + t * eh, p.V + t * eV, D0, eps, nsteps, wE, wN, prec=prec)
        fm = _gpu_forward_f(api, p, p.h - t * eh, p.V - t * eV, D0, eps, nsteps, wE, wN, prec=prec)
        fd = (fp - fm) / (2 * t)
        ad = np.sum(dh * eh) + np.sum(dV * eV)
        rel = abs(ad - fd) / max(abs(fd), 1e-12)
        worst = max(worst, rel)
        assert rel < 1e-6, f"direction {k}: adjoint {ad} vs FD {fd}"
    print(f"config 5 {prec}: worst relative adjoint/FD mismatch over 64 directions {worst:.2e}")


def test_autograd_function_matches_oracle(api):
    """torch.autograd through ACSEObjective: gradients of f with respect to h, V and D_0 tensors equal
    the oracle's complex-step directional derivatives."""
    p = I.make_problem(4, 4, 33, "cas", core=[0], active=[1, 2, 3], nelecas=2)
    eps, nsteps, wE, wN = 1e-3, 3, 1.0, 0.25
    dev = torch.device("cuda")
    h = torch.tensor(p.h, device=dev, requires_grad=True)
    V = torch.tensor(p.V, device=dev, requires_grad=True)
    D = [torch.tensor(x, device=dev, requires_grad=True) for x in (p.Daa, p.Dab, p.Dbb)]
    f = api.acse_objective(h, V, D, p.n_alpha, p.n_beta, "fp64", nsteps, eps, wE, wN)
    f.backward()
    f_or = O.objective(p.h, p.V, p.N, O.so_from_blocks(p.Daa, p.Dab, p.Dbb), eps, nsteps, wE, wN)
    assert float(f) == pytest.approx(f_or, rel=1e-12)
    rng = np.random.default_rng(9)
    for k in range(4):
        eh, eV = _sym_dirs(p.r, rng)
        eD = _sym_D(p.r, 200 + k)
        want = O.complex_step_dir(p.h, p.V, p.N, O.so_from_blocks(p.Daa, p.Dab, p.Dbb), eps, nsteps, eh, eV,
                                  O.so_from_blocks(*eD), wE, wN)
        got = (np.sum(h.grad.cpu().numpy() * eh) + np.sum(V.grad.cpu().numpy() * eV)
               + sum(np.sum(d.grad.cpu().numpy() * e) for d, e in zip(D, eD)))
        assert got == pytest.approx(want, rel=1e-9, abs=1e-9 * abs(want)), f"direction {k}"


def test_split_precision_adjoint(api):
    """A BF16x3 context's adjoint is the FP64-accurate reverse sweep (its Ozaki companion) along the BF16x3
    forward trajectory: with the same checkpoints it equals an FP64 context's adjoint to FP64 accuracy,
    and it differs from the gradient of the FP64 trajectory only by the split-precision error of the
    forward steps."""
    p = I.config_problem(2)
    eps, nsteps, wE, wN = 1e-3, 3, 1.0, 1e-3
    D0 = (p.Daa, p.Dab, p.Dbb)
    cm = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "bf16x3")
    D = cm.to_blocks(D0)
    ck = [tuple(x.clone() for x in D)]
    for _ in range(nsteps):
        cm.step(D, eps)
        ck.append(tuple(x.clone() for x in D))
    gm = cm.backward(ck, nsteps, eps, wE, wN)
    c64 = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "fp64")
    g64_same = c64.backward(ck, nsteps, eps, wE, wN)
    g64_own = c64.backward([c64.to_blocks(D0)], nsteps, eps, wE, wN)
    flat = lambda g: np.concatenate([g[0].cpu().numpy().ravel(), g[1].cpu().numpy().ravel()]
                                    + [x.cpu().numpy().ravel() for x in g[2]])
    a, b, c = flat(gm), flat(g64_same), flat(g64_own)
    same = np.abs(a - b).max() / np.abs(b).max()
    print(f"BF16x3 context (Ozaki reverse sweep) vs FP64 context, same checkpoints: max rel diff {same:.2e}")
    assert same <= 1e-11
    rel = np.abs(a - c).max() / np.abs(c).max()
    print(f"BF16x3-trajectory adjoint vs FP64-trajectory adjoint: max rel diff {rel:.2e}")
    assert rel < 1e-3
    cm.close()
    c64.close()
