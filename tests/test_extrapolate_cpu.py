"""Pins of the E(lambda) fit of oracle/extrapolate.py (reading R17 of the Results section's damped-then-linear
trajectory): exact recovery of known parameters, the least-squares minimum against a brute-force scan, and
the invariances the model has."""
import numpy as np
import pytest

from oracle import extrapolate as X


def _traj(a, b, c, k, lam):
    return a + b * lam + c * np.exp(-k * lam)


@pytest.mark.parametrize("a,b,c,k", [(-107.3, -0.634, 2.5, 300.0), (-12.0, -8e-3, 0.4, 30.0), (5.0, 1.5, -3.0, 40.0)])
def test_exact_data_recovers_parameters(a, b, c, k):
    lam = 1e-3 * np.arange(120)
    f = X.fit(lam, _traj(a, b, c, k, lam))
    assert f["flag"] == 0
    assert f["a"] == pytest.approx(a, rel=1e-11, abs=1e-11)
    assert f["b"] == pytest.approx(b, rel=1e-8)
    assert f["c"] == pytest.approx(c, rel=1e-8)
    assert f["k"] == pytest.approx(k, rel=1e-8)
    assert f["rss"] < 1e-20 * (1 + a * a)


def test_uneven_steps_and_skip():
    """A line-searched trajectory: lambda is the running sum of uneven steps; dropping the first points
    leaves the parameters of exact data unchanged."""
    rng = np.random.default_rng(3)
    eps = 1e-3 * rng.uniform(0.25, 2.0, size=80)
    lam = np.concatenate([[0.0], np.cumsum(eps)])
    E = _traj(-50.0, -0.2, 1.3, 60.0, lam)
    for skip in (0, 5, 17):
        f = X.fit(lam, E, n_skip=skip)
        assert f["flag"] == 0
        assert f["a"] == pytest.approx(-50.0, abs=1e-10)
        assert f["k"] == pytest.approx(60.0, rel=1e-7)


def test_noisy_fit_is_the_least_squares_minimum():
    """With noise, no kappa of a dense brute-force scan gives a smaller residual than the fit, and the fit's
    residual is no larger than that of the generating parameters."""
    rng = np.random.default_rng(11)
    lam = 2e-3 * np.arange(100)
    E_true = _traj(-30.0, -0.05, 0.8, 25.0, lam)
    E = E_true + 1e-4 * rng.standard_normal(lam.size)
    f = X.fit(lam, E)
    r_fit = np.sum((E - X.model(lam, f["a"], f["b"], f["c"], f["k"])) ** 2)
    assert r_fit == pytest.approx(f["rss"], rel=1e-9)
    assert f["rss"] <= np.sum((E - E_true) ** 2) * (1 + 1e-12)
    t = (lam - lam[0]) / (lam[-1] - lam[0])
    dense = np.exp(np.linspace(np.log(X.KAPPA_MIN), np.log(X.KAPPA_STEPS * (lam.size - 1)), 20000))
    best = min(X.rss(t, E, kp) for kp in dense)
    assert f["rss"] <= best * (1 + 1e-12)


def test_invariances():
    """E -> E + s shifts a by s; lambda -> s lambda divides k and b by s."""
    lam = 1e-3 * np.arange(90)
    E = _traj(-7.0, -0.3, 0.9, 80.0, lam) + 1e-5 * np.sin(37 * np.arange(90))
    f = X.fit(lam, E)
    g = X.fit(lam, E + 3.25)
    assert g["a"] - f["a"] == pytest.approx(3.25, abs=1e-10)
    assert g["k"] == pytest.approx(f["k"], rel=1e-9)
    h = X.fit(4.0 * lam, E)
    assert h["a"] == pytest.approx(f["a"], abs=1e-10)
    assert h["k"] == pytest.approx(f["k"] / 4.0, rel=1e-9)
    assert h["b"] == pytest.approx(f["b"] / 4.0, rel=1e-9)


def test_pure_line_and_edge_of_grid():
    """Exact data without a damped part: the line is recovered whatever kappa is chosen; a decay faster than
    the grid reaches ends on the grid's edge with flag 1."""
    lam = 1e-3 * np.arange(60)
    f = X.fit(lam, -4.0 - 0.7 * lam)
    assert f["a"] + f["c"] * np.exp(-f["k"] * 1.0) == pytest.approx(-4.0, abs=1e-6) or abs(f["c"]) < 1e-8
    assert np.max(np.abs(X.model(lam, f["a"], f["b"], f["c"], f["k"]) - (-4.0 - 0.7 * lam))) < 1e-10
    E = _traj(-4.0, -0.7, 1.0, 1e6, lam)          # decays within a small fraction of the first step
    g = X.fit(lam, E)
    assert g["flag"] == 1


def test_too_few_points_and_flat_lambda():
    with pytest.raises(ValueError):
        X.fit([0.0, 1.0, 2.0], [1.0, 2.0, 3.0])
    with pytest.raises(ValueError):
        X.fit(np.zeros(6), np.arange(6.0))
