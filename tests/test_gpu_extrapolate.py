"""The E(lambda) fit on the device (acse_extrapolate, acse_batch_extrapolate) against oracle/extrapolate.py
on the same trajectory points: exact synthetic trajectories, the stored 50-step line-searched oracle
trajectory of the r = 24 CAS(6e,6o) system, and the FP64 batch's own record of that system at a fixed step.

Tolerance: both sides solve dF/dkappa = 0 to about four ulps of kappa and form the linear coefficients by
orthogonal projections, so the intercept a agrees to rounding of the sums (1e-10 Eh absolute)."""
import json
import os

import numpy as np
import pytest

import acse_inputs as I
from oracle import extrapolate as X

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cfg2_line_search_50.json")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import _lib
    return _lib


def _gpu_fit(lib, lam, E, n_skip=0):
    dev = torch.device("cuda")
    lt = torch.tensor(np.asarray(lam, dtype=np.float64), device=dev)
    Et = torch.tensor(np.asarray(E, dtype=np.float64), device=dev)
    out = torch.zeros(6, dtype=torch.float64, device=dev)
    lib.acse_extrapolate(lt, Et, out, n_skip)
    torch.cuda.synchronize()
    return dict(zip(lib.FIT_KEYS, out.cpu().numpy()))


def _compare(g, o, tol_a=1e-10):
    print(f"a gpu {g['a']:.15f} oracle {o['a']:.15f} |d| {abs(g['a'] - o['a']):.2e}; k {g['k']:.10g} vs "
          f"{o['k']:.10g}; flag {g['flag']:.0f}/{o['flag']}")
    assert int(g["flag"]) == o["flag"]
    assert abs(g["a"] - o["a"]) <= tol_a
    assert g["k"] == pytest.approx(o["k"], rel=1e-7)
    assert g["b"] == pytest.approx(o["b"], rel=1e-7, abs=1e-10)
    assert g["rss"] == pytest.approx(o["rss"], rel=1e-6, abs=1e-20)


@pytest.mark.parametrize("a,b,c,k,noise", [(-107.3, -0.634, 2.5, 300.0, 0.0), (-12.0, -8e-3, 0.4, 30.0, 1e-6),
                                           (5.0, 1.5, -3.0, 40.0, 1e-3)])
def test_fit_synthetic_matches_oracle(lib, a, b, c, k, noise):
    rng = np.random.default_rng(7)
    lam = 1e-3 * np.arange(150)
    E = a + b * lam + c * np.exp(-k * lam) + noise * rng.standard_normal(lam.size)
    _compare(_gpu_fit(lib, lam, E), X.fit(lam, E))
    _compare(_gpu_fit(lib, lam, E, 9), X.fit(lam, E, 9))


def test_fit_edge_and_argument_checks(lib):
    lam = 1e-3 * np.arange(60)
    g = _gpu_fit(lib, lam, -4.0 - 0.7 * lam + np.exp(-1e6 * lam))
    assert int(g["flag"]) == 1
    g = _gpu_fit(lib, np.zeros(8), np.arange(8.0))
    assert int(g["flag"]) == 3 and np.isnan(g["a"])
    with pytest.raises(lib.AcseError) as ei:
        _gpu_fit(lib, lam[:5], lam[:5], n_skip=2)
    assert ei.value.status == -2
    with pytest.raises(lib.AcseError) as ei:            # host memory is refused
        lib.acse_extrapolate(torch.zeros(8, dtype=torch.float64), torch.zeros(8, dtype=torch.float64),
                             torch.zeros(6, dtype=torch.float64), 0)
    assert ei.value.status == -1


def test_fit_of_stored_line_search_trajectory(lib):
    """lambda_n = sum of the accepted steps before n (the oracle's 50 line-searched steps of config 2)."""
    d = json.load(open(GOLDEN))
    lam = np.concatenate([[0.0], np.cumsum(d["eps"])])
    E = np.array(d["E"])
    for skip in (0, 10):
        _compare(_gpu_fit(lib, lam, E, skip), X.fit(lam, E, skip))


def test_batch_record_and_fit_fp64(lib):
    """FP64 batch of the config-2 system and a second seed at eps = 3e-4 for 30 steps (no stopping rule; the
    second seed diverges at 1e-3):
    the record is the trajectory of the batch's own energies, and the device fit of every record matches
    the oracle's fit of the same points."""
    probs = [I.config_problem(2, 0), I.config_problem(2, 1)]
    b = lib.acse_batch_create(probs, "fp64")
    for i, p in enumerate(probs):
        lib.acse_batch_set_D(b, i, p.Daa, p.Dab, p.Dbb, 3e-4)
    E_last = None
    for _ in range(30):
        E_last, _, _, _ = lib.acse_batch_run(b, len(probs), 1, stop_rule=False)
    fits = lib.acse_batch_extrapolate(b, len(probs), n_skip=2)
    for i in range(len(probs)):
        lam, E = lib.acse_batch_history(b, i)
        assert lam.size == 31
        assert np.allclose(lam, 3e-4 * np.arange(31), rtol=0, atol=1e-15)
        assert E[-1] == E_last[i]
        _compare(fits[i], X.fit(lam, E, 2))
    lib.acse_batch_destroy(b)


def test_batch_record_drops_undone_step(lib):
    """With the stopping rule, a step that raised E or ||A|| is undone and its point leaves the record:
    the record ends at the accepted steps."""
    p = I.config_problem(2, 0)
    b = lib.acse_batch_create([p], "fp64")
    lib.acse_batch_set_D(b, 0, p.Daa, p.Dab, p.Dbb, 1e-3)
    E, N2, S, R = lib.acse_batch_run(b, 1, 60, stop_rule=True)
    lam, Eh = lib.acse_batch_history(b, 0)
    print(f"stopped after {S[0]} steps, reason {R[0]}, record of {lam.size} points")
    assert lam.size == S[0] + 1
    assert Eh[-1] == E[0]
    lib.acse_batch_destroy(b)
