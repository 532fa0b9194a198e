"""Batched propagation (acse_batch_*): one grouped GEMM launch per pass over all instances, forked
elementwise streams, a graph-captured step and the device-side stopping rule."""
import numpy as np
import pytest

import acse_inputs as I
from oracle import acse_oracle as O
from tests.gpu_helpers import maxrel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import _lib, api
    return _lib, api


def _mixed_set():
    out = []
    h, V = I.make_integrals(5, 3)
    out.append(I.Problem("rs5", 5, 2, 2, h, V, *I.random_state_rdm_blocks(5, 2, 2, 4)))
    out.append(I.make_problem(8, 8, 7, "hf"))
    out.append(I.make_problem(12, 6, 9, "cas", core=[0], active=[1, 2, 3, 4], nelecas=4))
    h, V = I.make_integrals(17, 5)
    out.append(I.Problem("pair17", 17, 5, 4, h, V, *I.random_pair_tensor_blocks(17, 6, hermitian=1, scale=0.05)))
    return out


def _get_D(_lib, b, i, r):
    D = [np.zeros((r,) * 4) for _ in range(3)]
    _lib.acse_batch_get_D(b, i, *D)
    return D


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
def test_batch_matches_single_contexts(libs, prec):
    _lib, api = libs
    probs = _mixed_set()
    eps, nsteps = 1e-4, 4
    b = _lib.acse_batch_create(probs, prec)
    for i, p in enumerate(probs):
        _lib.acse_batch_set_D(b, i, p.Daa, p.Dab, p.Dbb, eps)
    E, N2, S, R = _lib.acse_batch_run(b, len(probs), nsteps, stop_rule=False)
    assert list(S) == [nsteps] * len(probs) and list(R) == [0] * len(probs)
    for i, p in enumerate(probs):
        ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec)
        D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
        for _ in range(nsteps):
            Es, _, _ = ctx.step(D, eps)
        torch.cuda.synchronize()
        Db = _get_D(_lib, b, i, p.r)
        assert maxrel(Db, [x.cpu().numpy() for x in D]) < 1e-12, p.name
        assert E[i] == pytest.approx(float(Es), rel=1e-12)
        ctx.close()
    tune, split, launches = _lib.acse_batch_info(b)
    assert launches > 0 and tune in (0, 1, 2)
    # every replay counts the kernels it runs, the same number each time
    _lib.acse_batch_run(b, len(probs), 1, stop_rule=False)
    _, _, l1 = _lib.acse_batch_info(b)
    _lib.acse_batch_run(b, len(probs), 2, stop_rule=False)
    _, _, l2 = _lib.acse_batch_info(b)
    assert l1 > launches and l2 - l1 == 2 * (l1 - launches)
    _lib.acse_batch_destroy(b)


def test_batch_stop_rule_matches_oracle_driver(libs):
    """FP64 batch of two instances: a large step that makes E or ||A|| rise (the previous D is kept and
    the instance freezes) and a small one that keeps going; both against the oracle's driver."""
    _lib, api = libs
    p0 = I.make_problem(4, 4, 2, "cas", core=[0], active=[1, 2, 3], nelecas=2)
    p1 = I.make_problem(4, 4, 5, "cas", core=[0], active=[1, 2, 3], nelecas=2)
    runs = [(p0, 0.5), (p1, 1e-3)]
    b = _lib.acse_batch_create([p for p, _ in runs], "fp64")
    for i, (p, eps) in enumerate(runs):
        _lib.acse_batch_set_D(b, i, p.Daa, p.Dab, p.Dbb, eps)
    nrep = 8
    E, N2, S, R = _lib.acse_batch_run(b, 2, nrep, stop_rule=True)
    for i, (p, eps) in enumerate(runs):
        D0 = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
        want = O.run_acse(p.h, p.V, p.N, D0, eps, nrep - 1 if i == 0 else nrep, stop_rule=True)
        if i == 0:
            assert want["steps"] < nrep - 1 and R[i] == 1        # stopped on an increase
        else:
            assert want["steps"] == nrep and R[i] == 0
        assert S[i] == want["steps"]
        Db = _get_D(_lib, b, i, p.r)
        assert maxrel(Db, O.blocks_from_so(want["D"])) < 1e-12
        assert E[i] == pytest.approx(want["E"][-1], abs=1e-10)
    _lib.acse_batch_destroy(b)


def test_batch_config4_sixteen_instances(libs):
    """16 instances, r in {12, 16, ..., 40}, N = r/2, CAS(4e,4o) ground state and second root each,
    BF16x3, stopping rule on: energies agree with each instance stepped alone."""
    _lib, api = libs
    probs = I.batch_problems(0)
    assert len(probs) == 16
    eps, nrep = 1e-4, 6
    b = _lib.acse_batch_create(probs, "bf16x3")
    for i, p in enumerate(probs):
        _lib.acse_batch_set_D(b, i, p.Daa, p.Dab, p.Dbb, eps)
    E, N2, S, R = _lib.acse_batch_run(b, len(probs), nrep, stop_rule=True)
    assert np.all(np.isfinite(E))
    for i in (0, 5, 14, 15):
        p = probs[i]
        ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "bf16x3")
        D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
        for _ in range(int(S[i])):
            Es, _, _ = ctx.step(D, eps)
        assert E[i] == pytest.approx(float(Es), rel=1e-11), p.name
        ctx.close()
    # the two r = 12 instances (ground state and second root) against the FP64 oracle's own trajectory:
    # the split-precision error of a step is about 1e-5 of what the step changes (E and D)
    for i in (0, 1):
        p = probs[i]
        K = O.reduced_hamiltonian(p.h, p.V, p.N)
        D0 = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
        want = O.run_acse(p.h, p.V, p.N, D0, eps, int(S[i]))
        got = tuple(np.zeros_like(p.Daa) for _ in range(3))
        _lib.acse_batch_get_D(b, i, *got)
        Dw = O.blocks_from_so(want["D"])
        dD = max(np.abs(g - w).max() for g, w in zip(got, Dw))
        moved = max(np.abs(w - d).max() for w, d in zip(Dw, (p.Daa, p.Dab, p.Dbb)))
        drop = abs(want["E"][-1] - want["E"][0])
        print(f"{p.name}: |E - E_oracle| {abs(E[i] - want['E'][-1]):.2e} of a drop {drop:.3f}; "
              f"max |D - D_oracle| {dD:.2e} of a change {moved:.3e}")
        assert abs(E[i] - want["E"][-1]) < 1e-5 * drop
        assert dD < 1e-5 * moved
        assert O.energy(K, O.so_from_blocks(*got)) == pytest.approx(E[i], abs=1e-9)
    tune, split, launches = _lib.acse_batch_info(b)
    print(f"config 4 batch: tile choice {tune} (split r^2 {split}), steps {list(S)}, reasons {list(R)}")
    _lib.acse_batch_destroy(b)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_batch_instance_adjoint(libs, prec):
    """acse_batch_residual_backward: the gradient of one instance, from checkpoints read off the batch
    after one-step runs, equals that of a single context with the same checkpoints; the batch's
    trajectory continues unchanged after it."""
    _lib, api = libs
    probs = _mixed_set()
    eps, nsteps, wE, wN, i = 1e-4, 2, 1.0, 0.5, 2
    b = _lib.acse_batch_create(probs, prec)
    for k, p in enumerate(probs):
        _lib.acse_batch_set_D(b, k, p.Daa, p.Dab, p.Dbb, eps)
    p = probs[i]
    ck = [[p.Daa.copy(), p.Dab.copy(), p.Dbb.copy()]]
    for _ in range(nsteps):
        _lib.acse_batch_run(b, len(probs), 1, stop_rule=False)
        ck.append(_get_D(_lib, b, i, p.r))
    r = p.r
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), device="cuda")
    ckd = [dev(x) for blk in ck for x in blk]
    out_b = [torch.zeros((r, r), dtype=torch.float64, device="cuda"), torch.zeros((r,) * 4, dtype=torch.float64, device="cuda")]
    out_b += [torch.zeros((r,) * 4, dtype=torch.float64, device="cuda") for _ in range(3)]
    _lib.acse_batch_residual_backward(b, i, ckd, nsteps, eps, wE, wN, *out_b)
    ctx = api.ACSE(r, p.n_alpha, p.n_beta, p.h, p.V, prec)
    dh, dV, dD = ctx.backward([tuple(ckd[3 * k:3 * k + 3]) for k in range(nsteps + 1)], nsteps, eps, wE, wN)
    torch.cuda.synchronize()
    for a, c in zip(out_b, [dh, dV, *dD]):
        a, c = a.cpu().numpy(), c.cpu().numpy()
        assert np.abs(c).max() > 0
        assert np.abs(a - c).max() <= 1e-13 * np.abs(c).max()
    ctx.close()
    # the batch goes on from where it was: one more step equals a single context's third step
    E, _, _, _ = _lib.acse_batch_run(b, len(probs), 1, stop_rule=False)
    c2 = api.ACSE(r, p.n_alpha, p.n_beta, p.h, p.V, prec)
    D = c2.to_blocks((p.Daa, p.Dab, p.Dbb))
    for _ in range(nsteps + 1):
        Es, _, _ = c2.step(D, eps)
    assert E[i] == pytest.approx(float(Es), rel=1e-12)
    c2.close()
    _lib.acse_batch_destroy(b)
