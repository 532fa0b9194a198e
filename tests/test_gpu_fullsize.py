"""Parity at the full benchmark size (r = 48, 96 spin orbitals) and along a stored trajectory.

The full r = 48 residual is out of reach of the oracle in a test (one FP64 contraction takes tens of
seconds of host time and its 3-RDM would not fit), so the CUDA result is compared entry by entry with
the oracle's term-by-term evaluation of sampled entries (each 3-RDM element rebuilt from the
cumulant reconstruction on the fly), and through identities that hold at any size:

* Tr(K U) = -||A||^2: the update is the adjoint image of the residual,
* dE/deps = Tr(K U) for the Euler step D + eps U (energy is linear in D),
* Tr U = 0 (the step conserves the particle number) and A^{ij}_{kl} = -A^{kl}_{ij}.

The stored trajectory (tests/golden/cfg2_line_search_50.json, written by make_golden.py from the
oracle alone) is 50 line-searched steps of the r = 24 CAS(6e,6o) system.
"""
import json
import os

import numpy as np
import pytest

import acse_inputs as I
from oracle import acse_oracle as O
from tests.gpu_helpers import to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
R = 48
# normwise relative tolerances on sampled entries: FP64 sums of ~r^3 terms per entry; BF16x3 as in
# the small-size tests (about 2^-16 per product, some cancellation between GEMM outputs)
# BF16x3: about five times the largest error measured on a GB300 (1.1e-5 on the random pair tensor)
TOL_ENT = {"fp64": 1e-11, "ozaki": 1e-11, "bf16x3": 5e-5}


@pytest.fixture(scope="module")
def acse():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02550_gb300 import api
    return api


def _inputs():
    """The r = 48 CAS(8e,8o) state the benchmark starts from, and a random pair-Hermitian tensor of the
    same size (every index path of the reconstruction populated)."""
    p3 = I.config_problem(3)
    h, V = I.make_integrals(R, 77)
    pr = I.Problem("pair48", R, 10, 10, h, V, *I.random_pair_tensor_blocks(R, 78, hermitian=1, scale=0.02))
    return [p3, pr]


def _entries(p, seed, per_sector=8):
    """Seeded entries of the aa, ab and bb blocks: (spin-orbital index, block, block index).  For the CAS
    state the four draws cycle through excitation-type pairs (ij above the core, kl in core + active),
    their transposes, core + active only and unrestricted, so that large entries are sampled."""
    rng = np.random.default_rng(seed)
    lo, hi = (p.act_lo, p.act_hi) if p.act_hi > 0 else (0, R)
    ranges = [((lo, R), (0, hi)), ((0, hi), (lo, R)), ((0, hi), (0, hi)), ((0, R), (0, R))]
    out = []
    for blk, sector in enumerate(("aa", "ab", "bb")):
        for n in range(per_sector):
            (a0, a1), (b0, b1) = ranges[n % 4]
            while True:
                i, j = (int(x) for x in rng.integers(a0, a1, 2))
                k, l = (int(x) for x in rng.integers(b0, b1, 2))
                if sector == "ab" or (i != j and k != l):
                    break
            off = {"aa": (0, 0, 0, 0), "ab": (0, R, 0, R), "bb": (R, R, R, R)}[sector]
            so = tuple(x + o for x, o in zip((i, j, k, l), off))
            out.append((so, blk, (i, j, k, l)))
    return out


@pytest.fixture(scope="module")
def oracle_samples():
    """Expected sampled entries, computed once for both precisions (oracle only)."""
    out = []
    for t, p in enumerate(_inputs()):
        ent = _entries(p, 500 + t)
        vals = O.residual_entries(p.h, p.V, p.N, p.Daa, p.Dab, p.Dbb, [so for so, _, _ in ent])
        out.append((p, ent, vals))
    return out


@pytest.mark.parametrize("prec", ["bf16x3", "fp64", "ozaki"])
def test_fullsize_sampled_entries(acse, oracle_samples, prec):
    for p, ent, want in oracle_samples:
        ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec)
        A, n2 = ctx.residual(ctx.to_blocks((p.Daa, p.Dab, p.Dbb)))
        Ab = to_np(A)
        got = np.array([Ab[blk][idx] for _, blk, idx in ent])
        scale = np.abs(want).max()
        err = np.abs(got - want).max() / scale
        print(f"{p.name} {prec}: sampled max |A| {scale:.3e}, max rel err {err:.3e}")
        assert scale > 0
        assert err < TOL_ENT[prec], p.name
        ctx.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp64", "ozaki"])
def test_fullsize_invariants(acse, prec):
    """The benchmark's call (one context, default plan, step with eps = 1e-4) at r = 48."""
    p = I.config_problem(3)
    ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec)
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    E0 = float(ctx.energy(D))
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    assert E0 == pytest.approx(O.energy(K, O.so_from_blocks(p.Daa, p.Dab, p.Dbb)), abs=1e-9)
    Kb = O.blocks_from_so(K)
    del K
    A, n2 = ctx.residual(D)
    Aa = to_np(A)
    n2 = float(n2)
    assert n2 == pytest.approx(np.sum(Aa[0] ** 2) + np.sum(Aa[2] ** 2) + 4 * np.sum(Aa[1] ** 2), rel=1e-12)
    f64 = prec in ("fp64", "ozaki")
    sym = 1e-12 if f64 else 1e-6
    for blk in Aa:
        assert np.abs(blk + blk.transpose(2, 3, 0, 1)).max() <= sym * np.abs(blk).max()
    for blk in (Aa[0], Aa[2]):
        assert np.abs(blk + blk.transpose(1, 0, 2, 3)).max() <= sym * np.abs(blk).max()
    eps = 1e-4
    E1, n2s, _ = ctx.step(D, eps)
    E1 = float(E1)
    assert float(n2s) == pytest.approx(n2, rel=1e-12)
    U = tuple((a - b) / eps for a, b in zip(to_np(D), (p.Daa, p.Dab, p.Dbb)))
    trKU = np.sum(Kb[0] * U[0]) + np.sum(Kb[2] * U[2]) + 4 * np.sum(Kb[1] * U[1])
    tol = 1e-9 if f64 else 1e-6        # BF16x3: Tr(KU) + ||A||^2 measured 1.7e-7 relative
    print(f"r=48 {prec}: ||A||^2 {n2:.6e}, Tr(KU) {trKU:.6e}, dE/eps {(E1 - E0) / eps:.6e}")
    assert trKU == pytest.approx(-n2, rel=tol)
    assert (E1 - E0) / eps == pytest.approx(trKU, rel=1e-6)
    trU = sum(np.einsum("ijij->", u) * w for u, w in zip(U, (1, 2, 1)))
    assert abs(trU) < 1e-9 * max(np.abs(u).max() for u in U) * R * R
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "ozaki"])
def test_golden_line_search_trajectory(acse, prec):
    """50 line-searched Euler steps of the r = 24 CAS(6e,6o) system against the stored oracle
    trajectory: accepted eps, ||A||^2 before each step and E after it.

    ||A||^2 falls to a floor near 633.6 by step 19 (the reconstructed residual does not vanish);
    from there f(eps) = ||A(D + eps U)||^2 is flat to rounding at the three trial points, the curvature
    test of the line search compares differences of about 1e-13 relative, and either side may take
    either branch (the trial step then shrinks fourfold per step on both, and D no longer moves).  The
    accepted eps is therefore compared only on the steps where the merit still falls by more than
    1e-3 relative; E and ||A||^2 are compared on every step."""
    g = json.load(open(os.path.join(HERE, "golden", "cfg2_line_search_50.json")))
    p = I.config_problem(2)
    assert p.name == g["system"]
    ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec, line_search=True, eps0=g["eps0"])
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    assert float(ctx.energy(D)) == pytest.approx(g["E"][0], abs=1e-10)
    got_e, got_n2, got_E = [], [], []
    for _ in range(g["nsteps"]):
        E, n2, e = ctx.step(D)
        got_e.append(e)
        got_n2.append(n2)
        got_E.append(E)
    got_e = np.array([float(x) for x in got_e])
    got_n2 = np.array([float(x) for x in got_n2])
    got_E = np.array([float(x) for x in got_E])
    n2w = np.array(g["norm2"])
    cond = (n2w[:-1] - n2w[1:]) / n2w[:-1] > 1e-3
    assert cond[:19].all() and cond.sum() == 19
    de = np.abs(got_e / np.array(g["eps"]) - 1)[cond].max()
    dn = np.abs(got_n2 / n2w[:g["nsteps"]] - 1).max()
    Ew = np.array(g["E"][1:])
    dE_all = np.abs(got_E - Ew)
    dE = dE_all[:cond.sum() + 1].max()
    drop = abs(Ew[-1] - g["E"][0])
    print(f"{prec}: max rel eps (conditioned steps) {de:.2e}, max rel ||A||^2 {dn:.2e}, "
          f"max |dE| conditioned {dE:.2e}, all steps {dE_all.max():.2e} (E drop {drop:.1f})")
    if prec in ("fp64", "ozaki"):
        # FP64-accurate paths: exact agreement while the merit falls; in the flat regime a flipped
        # curvature branch changes one step's eps, so E may move by a step's eps ||A||^2 (about 1e-7 Eh
        # here), below the 1e-6 Eh stopping threshold
        # (measured: eps 9.6e-13, ||A||^2 3.0e-10, E 1.3e-12 Eh on the conditioned steps)
        assert de < 1e-11 and dn < 2e-9 and dE < 1e-10 and dE_all.max() < 1e-6
    else:
        # BF16x3 noise in f (about 3e-5 relative) moves the accepted eps by about 1e-4 relative, and
        # each step changes E by eps ||A||^2 (up to 4 Eh here): E may drift by about 1e-4 of the total
        # drop over the conditioned steps; in the flat regime the mixed run may keep stepping
        # (measured: eps 8.9e-5, ||A||^2 2.2e-5, E 9.3e-5 Eh conditioned, 5.5e-3 Eh over all steps)
        assert de < 5e-4 and dn < 1e-4
        assert dE < 5e-4 and dE_all.max() < 1e-3 * drop
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "ozaki", "bf16x3", "ozaki6->ozaki"])
def test_golden_config3_fixed_step_trajectory(acse, prec):
    """The headline r = 48 CAS(8e,8o) workload: five Euler steps at eps = 1e-4 against the stored oracle
    trajectory (tests/golden/cfg3_fixed_eps_5.json, written by make_golden.py from the oracle alone):
    E and ||A||^2 at every step and 64 seeded entries of each block of D_5.  FP64-accurate paths: 1e-10 Eh
    on E and 1e-12 relative on ||A||^2 and D; BF16x3: its error grows with what the steps change, a bound
    of 3e-5 of the energy drop so far (measured 1.0e-5, 7.1e-5, 1.1e-4, 1.5e-4, 1.8e-4 Eh after the five
    steps, whose drops are 6.0, 11.1, 15.7, 20.0, 23.9 Eh: four to eighteen times below the bound); the
    Ozaki 6 -> 8 slice schedule: 1e-7 Eh (its 6-slice steps carry about 2^-30 relative error)."""
    g = json.load(open(os.path.join(HERE, "golden", "cfg3_fixed_eps_5.json")))
    p = I.config_problem(3)
    assert p.name == g["system"] and p.r == R
    if prec == "ozaki6->ozaki":   # the precision schedule: 6 slices until ||A||^2 falls by < 10 % a step
        ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, "ozaki", oz_slices=6, refine=True, refine_tol=0.1)
    else:
        ctx = acse.ACSE(p.r, p.n_alpha, p.n_beta, p.h, p.V, prec)
    D = ctx.to_blocks((p.Daa, p.Dab, p.Dbb))
    E0 = float(ctx.energy(D))
    assert E0 == pytest.approx(g["E"][0], abs=1e-10)
    dEs, dNs = [], []
    for k in range(g["nsteps"]):
        E, n2, _ = ctx.step(D, g["eps"])
        dEs.append(abs(float(E) - g["E"][k + 1]))
        dNs.append(abs(float(n2) / g["norm2"][k] - 1.0))
    idx = np.array(g["D_final_index"])
    got = to_np(D)
    dD = max(np.abs(got[s][tuple(idx[s].T)] - np.array(g["D_final_aa_ab_bb"][s])).max() for s in range(3))
    scale = max(np.abs(np.array(v)).max() for v in g["D_final_aa_ab_bb"])
    print(f"{prec} config 3: per-step |dE| " + " ".join(f"{x:.2e}" for x in dEs) +
          f"; max rel ||A||^2 {max(dNs):.2e}; sampled D_5 {dD / scale:.2e}")
    if prec in ("fp64", "ozaki"):
        assert max(dEs) < 1e-10 and max(dNs) < 1e-12 and dD < 1e-12 * scale
    elif prec == "ozaki6->ozaki":
        # 6 slices carry about 2^-30 relative per GEMM product (measured 3e-9 Eh per step over 100 steps)
        assert max(dEs) < 1e-7 and max(dNs) < 1e-8 and dD < 1e-8 * scale
    else:
        for k, d in enumerate(dEs):
            assert d < 3e-5 * abs(g["E"][k + 1] - g["E"][0]), f"step {k}"
        assert max(dNs) < 1e-4 and dD < 1e-4 * scale
    ctx.close()
