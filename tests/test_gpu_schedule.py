"""Precision schedule (acse_opts.refine) and the time-to-E bar.

The schedule starts a context in one precision and, from the first step at which ||A||^2 falls by less than
refine_tol (relative), continues in the FP64-accurate Ozaki precision from the same D and line-search state:
after the switch its steps are those of an Ozaki context started there.  The bar is that of the Methods
stopping rule (E or ||A|| rises, or |dE| < 1e-6 Eh; a rise counts beyond the rounding level of the values
compared): the stopping energy within 1e-6 Eh of the FP64 path's, on the r = 24 CAS(6e,6o) and the r = 32
CAS(6e,6o) systems, for the Ozaki precision and the Ozaki 6-slice -> 8-slice schedule, in less wall time."""
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


def test_schedule_continues_as_an_ozaki_context(libs):
    _lib, api = libs
    p = I.config_problem(2)
    ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "bf16x3", line_search=True, eps0=1e-3, refine=True,
                   refine_tol=0.1)
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    last_eps = None
    for k in range(30):
        _, _, e = ctx.step(D)
        last_eps = float(e)
        switched, nsteps = _lib.acse_schedule_state(ctx.ctx)
        if switched:
            break
    assert switched and nsteps == k + 1, "the schedule switches within 30 steps"
    print(f"switched after {nsteps} steps")
    oz = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "ozaki", line_search=True, eps0=last_eps)
    D2 = tuple(x.clone() for x in D)
    for k in range(5):
        Ea, na, ea = ctx.step(D)
        Eb, nb, eb = oz.step(D2)
        assert float(Ea) == float(Eb) and float(na) == float(nb) and float(ea) == float(eb), f"step {k}"
    assert _lib.acse_schedule_state(ctx.ctx) == (True, nsteps)
    ctx.close()
    oz.close()


@pytest.mark.parametrize("cfg", [2, 5])
def test_time_to_e_bar(libs, cfg):
    import time
    _lib, api = libs
    p = I.config_problem(cfg)
    runs = {}
    for label, prec, kw in (("fp64", "fp64", {}), ("ozaki", "ozaki", {}),
                            ("ozaki6->ozaki", "ozaki", dict(oz_slices=6, refine=True, refine_tol=0.1))):
        ctx = api.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec, line_search=True, eps0=1e-3, **kw)
        D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.run_until_stop(D, 100)
        res["seconds"] = time.perf_counter() - t0
        runs[label] = res
        ctx.close()
    ref = runs["fp64"]
    for label, res in runs.items():
        dE = abs(res["E_stop"] - ref["E_stop"])
        print(f"config {cfg} {label}: {res['reason']} at {res['accepted']}, |E_stop - E_stop(fp64)| {dE:.2e} Eh, "
              f"{res['seconds']:.3f} s (fp64 {ref['seconds']:.3f} s)")
        assert dE <= 1e-6
        if label != "fp64":
            assert res["seconds"] < ref["seconds"]
