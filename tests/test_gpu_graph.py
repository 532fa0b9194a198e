"""acse_step as a CUDA graph: a call whose arguments repeat those of the previous call is captured once and
replayed.  Replays launch the same kernels with the same arguments in the same order as direct calls, so
trajectories are compared bit for bit with a context that runs directly (profiling on keeps a context on
direct calls)."""
import numpy as np
import pytest

import acse_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import _lib, api
    return _lib, api


def _run(api, _lib, p, prec, nsteps, direct, line_search=False, alternate=False):
    stream = torch.cuda.Stream()
    ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec, stream=stream, line_search=line_search, eps0=1e-4)
    _lib.acse_profile(ctx.ctx, 1 if direct else 0)
    outs = [torch.zeros(3, dtype=torch.float64, device="cuda") for _ in range(2)]
    Es = []
    with torch.cuda.stream(stream):
        D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
        for k in range(nsteps):
            s = outs[k % 2] if alternate else outs[0]
            _lib.acse_step(ctx.ctx, *D, 1e-4, s[0:1], s[1:2], s[2:3])
            Es.append(s.clone())
    stream.synchronize()
    _, _, launches = _lib.acse_profile_read(ctx.ctx)
    out = [x.cpu().numpy() for x in D], [e.cpu().numpy() for e in Es], launches
    ctx.close()
    return out


@pytest.mark.parametrize("prec,line_search", [("bf16x3", False), ("bf16x3", True), ("fp64", False),
                                              ("ozaki", False), ("tf32x3", False)])
def test_graph_steps_match_direct(libs, prec, line_search):
    _lib, api = libs
    p = I.config_problem(2) if prec != "fp64" else I.config_problem(1)
    Dg, Eg, lg = _run(api, _lib, p, prec, 6, direct=False, line_search=line_search)
    Dd, Ed, ld = _run(api, _lib, p, prec, 6, direct=True, line_search=line_search)
    Da, Ea, la = _run(api, _lib, p, prec, 6, direct=False, line_search=line_search, alternate=True)
    for a, b, c in zip(Dg, Dd, Da):
        assert np.array_equal(a, b) and np.array_equal(c, b)
    for a, b in zip(Eg, Ed):
        assert np.array_equal(a, b)
    # the launch counter counts the kernels of every replay
    assert lg == ld == la and lg > 0


def test_step_inside_a_callers_graph(libs):
    """A caller capturing its own graph around acse_step gets the direct launches inside it."""
    _lib, api = libs
    p = I.config_problem(2)
    stream = torch.cuda.Stream()
    ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "bf16x3", stream=stream)
    s = torch.zeros(3, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        D0 = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
        D = tuple(x.clone() for x in D0)
        for _ in range(2):   # warm up (first-use allocations happen outside the capture)
            _lib.acse_step(ctx.ctx, *D, 1e-4, s[0:1], s[1:2], s[2:3])
        for dst, src in zip(D, D0):
            dst.copy_(src)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        _lib.acse_step(ctx.ctx, *D, 1e-4, s[0:1], s[1:2], s[2:3])
    with torch.cuda.stream(stream):
        for dst, src in zip(D, D0):
            dst.copy_(src)
        for _ in range(3):
            g.replay()
        Dg = [x.clone() for x in D]
        for dst, src in zip(D, D0):
            dst.copy_(src)
        for _ in range(3):
            _lib.acse_step(ctx.ctx, *D, 1e-4, s[0:1], s[1:2], s[2:3])
    stream.synchronize()
    for a, b in zip(Dg, D):
        assert torch.equal(a, b)
    ctx.close()


def test_host_outputs_run_directly(libs):
    """Host outputs need a synchronisation: such calls run directly and return the same values."""
    _lib, api = libs
    p = I.config_problem(1)
    ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "bf16x3")
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    E = np.zeros(1)
    vals = []
    for _ in range(3):
        _lib.acse_step(ctx.ctx, *D, 1e-4, E, None, None)
        vals.append(float(E[0]))
    Dd, Ed, _ = _run(api, _lib, p, "bf16x3", 3, direct=True)
    assert vals == [float(e[0]) for e in Ed]
    ctx.close()
