"""The allocation-free energy entry point (acse_energy_noalloc) against acse_energy.

acse_energy_noalloc serves callers that cannot allocate device memory when they need an energy
(a framework that owns the whole device heap, a latency-critical path that must not risk the
implicit synchronisation of cudaMalloc/cudaFree, or a caller without an ACSE context): it keeps
its scratch in a static device array instead.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import acse_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_energy_noalloc_matches_context_energy_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import _lib
    from paper_2604_02550_gb300.api import ACSE
    p = I.make_problem(10, 8, 21, "cas", core=[0, 1], active=[2, 3, 4, 5], nelecas=4)
    dev = torch.device("cuda")
    h = torch.from_numpy(p.h).to(dev)
    V = torch.from_numpy(p.V).to(dev)
    D = [torch.from_numpy(x).to(dev) for x in (p.Daa, p.Dab, p.Dbb)]
    ctx = ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "fp64")
    E_ref = float(ctx.energy(D))
    ctx.close()
    # a second, different 2-RDM for the second call (the scratch keeps the first call's contents)
    q = I.make_problem(10, 8, 21, "cas", core=[0, 1], active=[2, 3, 4, 5], nelecas=4, root=1)
    # both calls pass p's integrals: q must share them (same seed), so that E2_ref is their energy
    assert np.array_equal(p.h, q.h) and np.array_equal(p.V, q.V)
    D2 = [torch.from_numpy(x).to(dev) for x in (q.Daa, q.Dab, q.Dbb)]
    ctx2 = ACSE(q.r, q.n_alpha, q.n_beta, q.h, q.V, "fp64")
    E2_ref = float(ctx2.energy(D2))
    ctx2.close()
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    for Dx, want in ((D, E_ref), (D2, E2_ref)):
        _lib.acse_energy_noalloc(p.r, p.n_alpha, p.n_beta, h, V, *Dx, E)
        torch.cuda.synchronize()
        assert float(E) == pytest.approx(want, rel=1e-12, abs=1e-10)
    assert abs(E_ref - E2_ref) > 1e-3          # the two calls really computed different things


def test_energy_noalloc_rejects_oversize_and_host_pointers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import _lib
    dev = torch.device("cuda")
    r = 65
    t = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(_lib.AcseError) as ei:
        _lib.acse_energy_noalloc(r, 2, 2, t, t, t, t, t, t)
    assert ei.value.status == -9
    host = np.zeros(16)
    with pytest.raises(_lib.AcseError) as ei:
        _lib.acse_energy_noalloc(2, 1, 1, host, t, t, t, t, t)
    assert ei.value.status == -1
