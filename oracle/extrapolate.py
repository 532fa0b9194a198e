"""FP64 reference fit of the asymptotic regime of an ACSE energy trajectory.  TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg may import this
module.  The CUDA library never calls it and shares no code with it.

What the paper fixes (Results, the ethylene convergence discussion; Conclusions):
  * the trajectory coordinate is lambda = eps * n (eps the Euler step of Eq. update, n the iteration;
    with a varying step, reading R17b, lambda_n is the sum of the steps taken before iteration n);
  * the energy along a trajectory is an exponentially damped region followed by an asymptotic regime
    in which E changes approximately linearly in lambda (slopes of a few mH per unit lambda quoted);
  * future work is to estimate the solution by extrapolation and fitting once the trajectory stably
    enters that asymptotic regime.
The paper gives no fit.  Reading R17 (this module and the library implement it independently):
  model   E(lambda) = a + b lambda + c exp(-k lambda),  k > 0,
  fitted by least squares over the points n >= n_skip, in the scaled coordinate
  t = (lambda - lambda_first) / (lambda_last - lambda_first) in [0, 1] (kappa = k (lambda_last - lambda_first));
  the extrapolated energy is a, the intercept of the asymptote at lambda = 0, b its slope.
  Search over kappa: for each kappa the optimal (a, b, c) solve a linear least-squares problem; F(kappa)
  is its residual sum of squares.  kappa is scanned on NGRID points spaced evenly in log kappa over
  [KAPPA_MIN, kappa_max = KAPPA_STEPS * (m - 1)] (m fitted points: the fastest decay spans a fraction
  of one step), the best grid point j is taken (the first one on ties), and when 0 < j < NGRID - 1 the
  stationarity condition dF/dkappa = 0 is solved in [kappa_{j-1}, kappa_{j+1}] by a bracketing root
  finder; dF/dkappa = 2 c_t sum_n r_n t_n exp(-kappa t_n) (the variable-projection derivative: at the
  optimal linear coefficients only the explicit kappa dependence of the exponential column remains;
  r = E - fit, c_t the exponential coefficient).  A minimum on the edge of the grid is reported with
  flag 1 and no refinement.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq

NGRID = 256
KAPPA_MIN = 0.25
KAPPA_STEPS = 4.0


def _columns(t, kappa):
    return np.stack([np.ones_like(t), t, np.exp(-kappa * t)], axis=1)


def linear_part(t, E, kappa):
    """Least-squares (a_t, b_t, c_t) of E ~ a_t + b_t t + c_t exp(-kappa t) and its residual vector."""
    Phi = _columns(t, kappa)
    coef, *_ = np.linalg.lstsq(Phi, E, rcond=None)
    return coef, E - Phi @ coef


def rss(t, E, kappa):
    _, res = linear_part(t, E, kappa)
    return float(res @ res)


def drss(t, E, kappa):
    """dF/dkappa at the optimal linear coefficients (variable projection)."""
    coef, res = linear_part(t, E, kappa)
    return float(2.0 * coef[2] * np.sum(res * t * np.exp(-kappa * t)))


def kappa_grid(m):
    kmax = KAPPA_STEPS * (m - 1)
    return np.exp(np.linspace(np.log(KAPPA_MIN), np.log(kmax), NGRID))


def fit(lam, E, n_skip=0):
    """Fit of reading R17 to the trajectory points (lam[n], E[n]), n >= n_skip.

    Returns dict(a, b, c, k, rss, flag): E(lambda) ~ a + b lambda + c exp(-k lambda); flag 0 for an
    interior minimum refined to dF/dkappa = 0, 1 for a minimum on the edge of the kappa grid."""
    lam = np.asarray(lam, dtype=np.float64)[n_skip:]
    E = np.asarray(E, dtype=np.float64)[n_skip:]
    m = lam.size
    if m < 4:
        raise ValueError("the fit needs at least four points")
    l0, span = lam[0], lam[-1] - lam[0]
    if not span > 0:
        raise ValueError("lambda must increase along the trajectory")
    t = (lam - l0) / span
    grid = kappa_grid(m)
    F = np.array([rss(t, E, kp) for kp in grid])
    j = int(np.argmin(F))
    flag = 1
    kappa = grid[j]
    if 0 < j < NGRID - 1:
        lo, hi = grid[j - 1], grid[j + 1]
        glo, ghi = drss(t, E, lo), drss(t, E, hi)
        if glo < 0.0 < ghi:
            kappa = brentq(lambda x: drss(t, E, x), lo, hi, xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=200)
            flag = 0
    (at, bt, ct), res = linear_part(t, E, kappa)
    # back to lambda: a_t + b_t t + c_t e^{-kappa t} with t = (lambda - l0) / span
    k = kappa / span
    b = bt / span
    c = ct * np.exp(kappa * l0 / span)
    a = at - bt * l0 / span
    return dict(a=float(a), b=float(b), c=float(c), k=float(k), rss=float(res @ res), flag=flag)


def model(lam, a, b, c, k):
    lam = np.asarray(lam, dtype=np.float64)
    return a + b * lam + c * np.exp(-k * lam)
