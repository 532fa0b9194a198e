"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks one oracle function against what the mathematics or the paper fixes:
brute-force Fock-space expectation values (Jordan-Wigner matrices, n <= 8 spin orbitals),
exact eigenstates, single determinants, the textbook cumulant expansion of the 3-RDM,
closed forms and exact identities.  A dropped term, a wrong sign, index or transposed
operand anywhere in the oracle makes at least one of them fail.
"""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.linalg import expm

import acse_inputs as I
from oracle import acse_oracle as O
from oracle import fock as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _antisym_W(n, seed, herm=0):
    rng = np.random.default_rng(seed)
    W = rng.normal(size=(n,) * 4)
    W = W - W.transpose(1, 0, 2, 3)
    W = W - W.transpose(0, 1, 3, 2)
    if herm:
        W = 0.5 * (W + herm * W.transpose(2, 3, 0, 1))
    return W


@pytest.fixture(scope="module")
def sys3():
    """r = 3 spatial orbitals (6 spin orbitals), N = 3 (2 alpha, 1 beta), random state."""
    r, N, na = 3, 3, 2
    n = 2 * r
    a = F.annihilators(n)
    h, V = I.make_integrals(r, 11)
    psi = F.random_state(n, N, 5, n_alpha=na, r=r)
    hs, gs = F.so_integrals(h, V)
    return dict(r=r, n=n, N=N, na=na, a=a, h=h, V=V, psi=psi,
                D=F.rdm2(a, psi), D3=F.rdm3(a, psi), g1=F.rdm1(a, psi),
                H=F.hamiltonian_matrix(a, hs, gs), K=O.reduced_hamiltonian(h, V, N))


@pytest.fixture(scope="module")
def sys4():
    """r = 4 (8 spin orbitals), N = 4 (2 alpha, 2 beta)."""
    r, N, na = 4, 4, 2
    n = 2 * r
    a = F.annihilators(n)
    h, V = I.make_integrals(r, 12)
    psi = F.random_state(n, N, 6, n_alpha=na, r=r)
    hs, gs = F.so_integrals(h, V)
    return dict(r=r, n=n, N=N, na=na, a=a, h=h, V=V, psi=psi,
                D=F.rdm2(a, psi), D3=F.rdm3(a, psi),
                H=F.hamiltonian_matrix(a, hs, gs), K=O.reduced_hamiltonian(h, V, N))


# ---------------------------------------------------------------------------------- RDMs

def test_trace_and_gamma(sys3):
    s = sys3
    N = s["N"]
    assert O.trace2(s["D"]) == pytest.approx(N * (N - 1) / 2, abs=1e-13)
    np.testing.assert_allclose(O.gamma(s["D"], N), s["g1"], atol=1e-14)
    assert np.trace(s["g1"]) == pytest.approx(N, abs=1e-13)


def test_spin_block_traces_appendix_A():
    """Appendix A normalisations: Tr D_aa = Na(Na-1)/2, Tr D_ab = Na Nb/2, Tr D_bb = Nb(Nb-1)/2
    (the three printed labels all read 'aa'; reading: aa, ab, bb) and the 3-RDM blocks
    Tr D_aaa = Na(Na-1)(Na-2)/6, Tr D_aab = Na(Na-1)Nb/6, Tr D_abb = Na Nb(Nb-1)/6."""
    fx = json.load(open(os.path.join(GOLDEN, "spin_block_traces.json")))
    r = 4
    n = 2 * r
    a = F.annihilators(n)
    for case in fx["cases"]:
        na, nb = case["n_alpha"], case["n_beta"]
        psi = F.random_state(n, na + nb, 3 + na, n_alpha=na, r=r)
        D = F.rdm2(a, psi)
        Daa, Dab, Dbb = O.blocks_from_so(D)
        assert np.einsum("ijij->", Daa) == pytest.approx(case["tr_aa"], abs=1e-12)
        assert np.einsum("ijij->", Dab) == pytest.approx(case["tr_ab"], abs=1e-12)
        assert np.einsum("ijij->", Dbb) == pytest.approx(case["tr_bb"], abs=1e-12)
        D3 = F.rdm3(a, psi)
        al, be = slice(0, r), slice(r, n)
        assert np.einsum("ijkijk->", D3[al, al, al, al, al, al]) == pytest.approx(case["tr_aaa"], abs=1e-12)
        assert np.einsum("ijkijk->", D3[al, al, be, al, al, be]) == pytest.approx(case["tr_aab"], abs=1e-12)
        assert np.einsum("ijkijk->", D3[al, be, be, al, be, be]) == pytest.approx(case["tr_abb"], abs=1e-12)


def test_block_mapping_matches_fock_state():
    """The inputs' spin-block 2-RDM of a CI vector equals the brute-force spin-orbital 2-RDM
    of the same state under the oracle's block -> spin-orbital map."""
    r, na, nb = 4, 2, 1
    n = 2 * r
    a = F.annihilators(n)
    sa, sb, c = I.random_ci_vector(r, na, nb, 7)
    psi = np.zeros(1 << n)
    for ia, A in enumerate(sa):
        for ib, B in enumerate(sb):
            psi[A | (B << r)] = c[ia, ib]
    Dbf = F.rdm2(a, psi)
    D = O.so_from_blocks(*I.rdm_blocks_from_ci(r, sa, sb, c))
    np.testing.assert_allclose(D, Dbf, atol=1e-15)
    np.testing.assert_allclose(np.stack(O.blocks_from_so(Dbf)), np.stack(I.rdm_blocks_from_ci(r, sa, sb, c)), atol=1e-15)


def test_hf_blocks_are_the_determinant():
    r, na, nb = 4, 2, 2
    n = 2 * r
    a = F.annihilators(n)
    psi = F.determinant(n, [0, 1, r, r + 1])
    np.testing.assert_allclose(O.so_from_blocks(*I.hf_rdm_blocks(r, na, nb)), F.rdm2(a, psi), atol=1e-15)


# --------------------------------------------------------------------------- Hamiltonian

def test_energy_is_expectation_of_H(sys4):
    """Reading R1 of Eq. (2): with that K, E = sum K.D equals <psi|H|psi>."""
    s = sys4
    assert O.energy(s["K"], s["D"]) == pytest.approx(s["psi"] @ s["H"] @ s["psi"], abs=1e-12)


def test_hf_energy_closed_form():
    p = I.make_problem(6, 6, 4, "hf")
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    D = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
    occ = range(3)
    e = sum(2 * p.h[i, i] for i in occ) + sum(2 * p.V[i, i, j, j] - p.V[i, j, j, i] for i in occ for j in occ)
    assert O.energy(K, D) == pytest.approx(e, abs=1e-12)


def test_cas_energy_and_rdm_vs_bruteforce():
    r, n, N = 4, 8, 4
    h, V = I.make_integrals(r, 3)
    a = F.annihilators(n)
    hs, gs = F.so_integrals(h, V)
    H = F.hamiltonian_matrix(a, hs, gs)
    m = F.sector_mask(n, N, 2, r)
    idx = [s for s in np.nonzero(m)[0] if (s & 1) and (s >> r) & 1]
    w, v = np.linalg.eigh(H[np.ix_(idx, idx)])
    K = O.reduced_hamiltonian(h, V, N)
    for root in (0, 1):
        res = I.cas_rdm_blocks(h, V, [0], [1, 2, 3], 2, root=root)
        D = O.so_from_blocks(res.Daa, res.Dab, res.Dbb)
        psi = np.zeros(1 << n)
        psi[idx] = v[:, root]
        np.testing.assert_allclose(D, F.rdm2(a, psi), atol=1e-13)
        assert O.energy(K, D) == pytest.approx(res.e_core + res.e_cas, abs=1e-12)
        assert res.e_core + res.e_cas == pytest.approx(w[root], abs=1e-12)


def test_block_energy_and_norm_formulas(sys4):
    """E = sum K_aa D_aa + sum K_bb D_bb + 4 sum K_ab D_ab and ||X||^2 = ||X_aa||^2 +
    ||X_bb||^2 + 4 ||X_ab||^2 for spin-conserving pair tensors."""
    s = sys4
    Kb = O.blocks_from_so(s["K"])
    Db = O.blocks_from_so(s["D"])
    e = np.sum(Kb[0] * Db[0]) + np.sum(Kb[2] * Db[2]) + 4 * np.sum(Kb[1] * Db[1])
    assert e == pytest.approx(O.energy(s["K"], s["D"]), abs=1e-12)
    A = O.residual(s["K"], s["D"], s["N"])
    Ab = O.blocks_from_so(A)
    np.testing.assert_allclose(O.so_from_blocks(*Ab), A, atol=1e-14)
    assert np.sum(Ab[0] ** 2) + np.sum(Ab[2] ** 2) + 4 * np.sum(Ab[1] ** 2) == pytest.approx(O.norm2(A), rel=1e-13)


# ------------------------------------------------------------------------------ residual

def test_G_explicit_is_the_commutator(sys3, sys4):
    """G_explicit(W, 2D, 3D) with the exact 3-RDM equals <[a+a+aa, W^]> for general W
    (pair-Hermitian, pair-anti-Hermitian and neither)."""
    for s in (sys3, sys4):
        for k, herm in enumerate((1, -1, 0)):
            W = _antisym_W(s["n"], 100 + k, herm)
            C = F.commutator_expectation(s["a"], W, s["psi"])
            G = O.G_explicit(W, s["D"], s["D3"])
            np.testing.assert_allclose(G, C, atol=1e-12 * np.abs(C).max())


def test_printed_residual_is_minus_commutator(sys4):
    """Reading R2: Eq. (residual) as printed equals -<[a+_i a+_j a_l a_k, H]>."""
    s = sys4
    C = F.commutator_expectation(s["a"], 0.5 * s["K"], s["psi"])
    # 1/2 K as two-body operator is H on N-electron states
    Hpsi = s["H"] @ s["psi"]
    np.testing.assert_allclose(F.two_body_op_apply(s["a"], 0.5 * s["K"], s["psi"]), Hpsi, atol=1e-12)
    R = O.residual_paper_form(s["K"], s["D"], s["D3"])
    np.testing.assert_allclose(R, -C, atol=1e-12 * np.abs(C).max())


def test_residual_vanishes_at_eigenstates(sys4):
    s = sys4
    m = F.sector_mask(s["n"], s["N"], s["na"], s["r"])
    w, v = np.linalg.eigh(s["H"][np.ix_(m, m)])
    for root in (0, 3):
        psi = np.zeros(1 << s["n"])
        psi[m] = v[:, root]
        A = O.G_explicit(0.5 * s["K"], F.rdm2(s["a"], psi), F.rdm3(s["a"], psi))
        assert np.abs(A).max() < 1e-12


def test_residual_symmetries(sys4):
    s = sys4
    A = O.residual(s["K"], s["D"], s["N"])
    assert np.abs(A + A.transpose(1, 0, 2, 3)).max() < 1e-13
    assert np.abs(A + A.transpose(0, 1, 3, 2)).max() < 1e-13
    assert np.abs(A + A.transpose(2, 3, 0, 1)).max() < 1e-13


# ------------------------------------------------------------------------ reconstruction

def _textbook_3rdm(D, N):
    """Standard cumulant expansion written independently of the paper's nine M.1D terms:
    Gamma3 = sum_pi sgn(pi) g g g + (1/4) sum_{sigma,pi} sgn sgn lambda2^{..}_{..} g^._.
    with Gamma2 = 2 D, lambda2 = Gamma2 - (g g - g g);  3D = Gamma3 / 6."""
    n = D.shape[0]
    g = O.gamma(D, N)
    G2 = 2.0 * D
    lam = G2 - (np.einsum("pr,qs->pqrs", g, g) - np.einsum("ps,qr->pqrs", g, g))
    perms = list(itertools.permutations(range(3)))

    def sgn(p):
        return np.linalg.det(np.eye(3)[list(p)])

    up = "abc"
    lo = "def"
    G3 = np.zeros((n,) * 6)
    for pi in perms:
        lo_p = "".join(lo[i] for i in pi)
        G3 += sgn(pi) * np.einsum(f"{up[0]}{lo_p[0]},{up[1]}{lo_p[1]},{up[2]}{lo_p[2]}->abcdef", g, g, g)
    F_ = np.einsum("abde,cf->abcdef", lam, g)
    acc = np.zeros_like(G3)
    for s1 in perms:
        for s2 in perms:
            axes = list(s1) + [3 + i for i in s2]
            acc += sgn(s1) * sgn(s2) * F_.transpose(np.argsort(axes))
    return (G3 + 0.25 * acc) / 6.0


def test_valdemoro_equals_textbook_cumulant_form(sys3):
    s = sys3
    np.testing.assert_allclose(O.recon_3rdm_V(s["D"], s["N"]), _textbook_3rdm(s["D"], s["N"]), atol=1e-14)


def test_valdemoro_exact_for_determinants():
    r = 4
    n = 2 * r
    a = F.annihilators(n)
    for occ in ([0, 1, r], [0, 2, r + 1, r + 3], [1, 2, 3, r, r + 2]):
        psi = F.determinant(n, occ)
        D = F.rdm2(a, psi)
        np.testing.assert_allclose(O.recon_3rdm_V(D, len(occ)), F.rdm3(a, psi), atol=1e-15)


def test_valdemoro_not_exact_for_correlated_state(sys3):
    """Guard that the determinant test is not vacuous: 3Delta != 0 for a random state."""
    s = sys3
    assert np.abs(O.recon_3rdm_V(s["D"], s["N"]) - s["D3"]).max() > 1e-3


def test_factored_equals_explicit(sys3, sys4):
    """App. C (V): G without storing 3D equals G with the stored Valdemoro 3D."""
    for s in (sys3, sys4):
        D3v = O.recon_3rdm_V(s["D"], s["N"])
        for k, herm in enumerate((1, -1)):
            W = _antisym_W(s["n"], 200 + k, herm)
            np.testing.assert_allclose(O.G_factored(W, s["D"], s["N"]), O.G_explicit(W, s["D"], D3v),
                                       atol=1e-12 * np.abs(O.G_explicit(W, s["D"], D3v)).max())


# -------------------------------------------------------------------------------- update

def test_update_is_first_order_flow(sys3):
    """Reading R3: with the exact 3-RDM, D(e^{lam A^} psi) - D - lam U = O(lam^2)."""
    s = sys3
    a, psi, K, D, D3 = s["a"], s["psi"], s["K"], s["D"], s["D3"]
    A = O.G_explicit(0.5 * K, D, D3)
    U = 0.5 * O.G_explicit(A, D, D3)
    Ahat = F.hamiltonian_matrix(a, np.zeros((s["n"], s["n"])), 2.0 * A)   # sum A a+a+aa
    errs = []
    for lam in (1e-3, 1e-4):
        pl = expm(lam * Ahat) @ psi
        errs.append(np.abs(F.rdm2(a, pl) - D - lam * U).max())
    assert 60 < errs[0] / errs[1] < 140
    assert errs[1] < 1e-6


def test_energy_descent_identity_with_reconstruction(sys4):
    """Tr(K U) = -||A||^2 and Tr U = 0 hold exactly with the reconstructed 3-RDM."""
    s = sys4
    A = O.residual(s["K"], s["D"], s["N"])
    U = O.update(A, s["D"], s["N"])
    assert np.sum(s["K"] * U) == pytest.approx(-O.norm2(A), rel=1e-12)
    assert abs(O.trace2(U)) < 1e-12
    # and the same for the explicit-3D path (independent of the factorisation)
    Ue = O.update(A, s["D"], s["N"], explicit=True)
    np.testing.assert_allclose(Ue, U, atol=1e-12 * np.abs(U).max())


def test_active_mask():
    r = 3
    A = np.ones((6,) * 4)
    Am = O.active_mask(A, r, 1, 3)
    for idx in itertools.product(range(6), repeat=4):
        act = all(1 <= (p % r) < 3 for p in idx)
        assert Am[idx] == (0.0 if act else 1.0)


# ---------------------------------------------------------------- line search and driver

def test_line_search_parabola():
    c0, b, c = 5.0, -3.0, 2.0
    f = lambda x: c0 + b * x + c * x * x
    e0 = 0.4
    x = O.line_search_eps(f(0), f(e0), f(2 * e0), e0)
    assert x == pytest.approx(0.75, abs=1e-14)          # -b/(2c) inside [e0/4, 2e0]
    x = O.line_search_eps(f(0), f(0.1), f(0.2), 0.1)
    assert x == pytest.approx(0.2, abs=1e-14)           # clamped to 2 e0
    x = O.line_search_eps(f(0), f(10), f(20), 10.0)
    assert x == pytest.approx(2.5, abs=1e-14)           # clamped to e0/4
    g = lambda x: 1.0 - x * x                           # concave: better of e0, 2e0
    assert O.line_search_eps(g(0), g(0.3), g(0.6), 0.3) == pytest.approx(0.6)
    # a merit flat to rounding (trial values within 1e-10 of f(0), either curvature sign): e0 / 4
    f0 = 7937.055219104771
    assert O.line_search_eps(f0, f0 * (1 + 3e-14), f0 * (1 - 2e-14), 1e-9) == 0.25e-9
    assert O.line_search_eps(f0, f0 * (1 - 3e-14), f0 * (1 + 2e-14), 1e-9) == 0.25e-9
    # just outside the flat band the parabola decides again
    assert O.line_search_eps(f0, f0 * (1 - 4e-10), f0 * (1 - 6e-10), 1e-9) != 0.25e-9


def test_driver_fixed_steps_and_descent():
    p = I.make_problem(4, 4, 2, "cas", core=[0], active=[1, 2, 3], nelecas=2)
    D0 = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
    K = O.reduced_hamiltonian(p.h, p.V, p.N)
    out = O.run_acse(p.h, p.V, p.N, D0, 0.02, 3)
    D = D0
    for _ in range(3):
        D, _, _ = O.step(K, D, p.N, 0.02)
    np.testing.assert_allclose(out["D"], D, atol=1e-15)
    assert out["steps"] == 3 and len(out["E"]) == 4
    # small eps: energy decreases at first order by eps ||A||^2
    A = O.residual(K, D0, p.N)
    D1, _, _ = O.step(K, D0, p.N, 1e-6)
    assert (O.energy(K, D1) - O.energy(K, D0)) / 1e-6 == pytest.approx(-O.norm2(A), rel=1e-4)


def test_driver_stop_rule():
    p = I.make_problem(4, 4, 2, "cas", core=[0], active=[1, 2, 3], nelecas=2)
    D0 = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
    out = O.run_acse(p.h, p.V, p.N, D0, 5.0, 10, stop_rule=True)   # huge eps: E or ||A|| rises
    assert out["steps"] < 10
    assert all(np.diff(out["E"]) <= 0)


def test_complex_step_matches_central_difference():
    p = I.make_problem(3, 2, 5, "hf")
    rng = np.random.default_rng(1)
    dh = rng.normal(size=p.h.shape); dh = dh + dh.T
    dV = rng.normal(size=p.V.shape)
    dV = dV + dV.transpose(1, 0, 2, 3); dV = dV + dV.transpose(0, 1, 3, 2); dV = dV + dV.transpose(2, 3, 0, 1)
    D0 = O.so_from_blocks(p.Daa, p.Dab, p.Dbb)
    dD = O.so_from_blocks(*I.random_pair_tensor_blocks(3, 9, hermitian=1))
    cs = O.complex_step_dir(p.h, p.V, p.N, D0, 0.05, 2, dh, dV, dD, wE=1.0, wN=0.5)
    t = 1e-5
    fp = O.objective(p.h + t * dh, p.V + t * dV, p.N, D0 + t * dD, 0.05, 2, 1.0, 0.5)
    fm = O.objective(p.h - t * dh, p.V - t * dV, p.N, D0 - t * dD, 0.05, 2, 1.0, 0.5)
    assert cs == pytest.approx((fp - fm) / (2 * t), rel=1e-7)


def test_residual_entries_match_full_residual(sys4):
    """The entry-wise evaluation (printed Eq. residual, 3D elements on the fly) used for sampled
    parity at full size agrees with the brute-force-pinned full residual."""
    s = sys4
    r = s["r"]
    Db = O.blocks_from_so(s["D"])
    A = O.residual(s["K"], s["D"], s["N"])
    rng = np.random.default_rng(3)
    ent = [tuple(int(x) for x in rng.integers(0, 2 * r, 4)) for _ in range(12)]
    e = O.residual_entries(s["h"], s["V"], s["N"], *Db, ent)
    np.testing.assert_allclose(e, [A[t] for t in ent], atol=1e-14)


# ----------------------------------------------------------------------- NY reconstruction

def _sig(s):
    return O.sigma_hf(s["r"], s["na"], s["N"] - s["na"])


def test_ny_cumulant_36_terms_equal_printed_nine(sys3, sys4):
    """Eq. (NY): the 36-term antisymmetrised definition equals the nine-term form printed in the
    appendix (the two printed forms of the same cumulant, read independently)."""
    for s in (sys3, sys4):
        g = O.gamma(s["D"], s["N"])
        _, delta = O.cumulant_M(s["D"], g)
        sig = _sig(s)
        full = O.cumulant3_NY(delta, sig)
        nine = O.cumulant3_NY_simplified(delta, sig)
        assert np.abs(full).max() > 1e-4
        np.testing.assert_allclose(full, nine, atol=1e-14 * np.abs(full).max() * 100)


def test_ny_sigma_is_the_hf_occupation():
    sig = O.sigma_hf(4, 2, 1)
    np.testing.assert_array_equal(sig, [1, 1, -1, -1, 1, -1, -1, -1])


def test_ny_exact_for_determinants():
    """For a determinant the 2-cumulant vanishes, so the NY cumulant does too and the NY 3-RDM equals
    the exact one (as the V one does)."""
    r = 4
    n = 2 * r
    a = F.annihilators(n)
    for occ in ([0, 1, r], [0, 2, r + 1, r + 3]):
        psi = F.determinant(n, occ)
        D = F.rdm2(a, psi)
        na = sum(1 for o in occ if o < r)
        sig = O.sigma_hf(r, na, len(occ) - na)
        np.testing.assert_allclose(O.recon_3rdm_NY(D, len(occ), sig), F.rdm3(a, psi), atol=1e-15)


def test_ny_cumulant_symmetries(sys4):
    """Antisymmetric in the upper and in the lower indices, Hermitian (upper <-> lower), and not
    the exact cumulant of a correlated state (it is an approximation)."""
    s = sys4
    g = O.gamma(s["D"], s["N"])
    _, delta = O.cumulant_M(s["D"], g)
    C = O.cumulant3_NY(delta, _sig(s))
    scale = np.abs(C).max()
    for ax in ((1, 0, 2, 3, 4, 5), (0, 2, 1, 3, 4, 5), (0, 1, 2, 4, 3, 5), (0, 1, 2, 3, 5, 4)):
        assert np.abs(C + C.transpose(ax)).max() < 1e-15 * 100 * scale
    assert np.abs(C - C.transpose(3, 4, 5, 0, 1, 2)).max() < 1e-15 * 100 * scale
    exact = s["D3"] - O.recon_3rdm_V(s["D"], s["N"])
    assert np.abs(exact - C).max() > 1e-3 * np.abs(exact).max()


def test_ny_factored_equals_explicit(sys3, sys4):
    """The NY contraction without storing 3D equals G with the stored NY 3-RDM, for pair-Hermitian
    and anti-Hermitian W (residual and update)."""
    for s in (sys3, sys4):
        sig = _sig(s)
        D3 = O.recon_3rdm_NY(s["D"], s["N"], sig)
        for k, herm in enumerate((1, -1)):
            W = _antisym_W(s["n"], 300 + k, herm)
            want = O.G_explicit(W, s["D"], D3)
            np.testing.assert_allclose(O.G_factored(W, s["D"], s["N"], sig), want, atol=1e-12 * np.abs(want).max())


def test_ny_residual_is_commutator_with_ny_3rdm_and_descent_identity(sys4):
    """With the NY 3-RDM: the printed Eq. (residual) is minus the factored residual, A is
    anti-Hermitian, and Tr(K U) = -||A||^2 (the descent identity needs only a Hermitian 3-RDM)."""
    s = sys4
    sig = _sig(s)
    K, D, N = s["K"], s["D"], s["N"]
    A = O.residual(K, D, N, sigma=sig)
    np.testing.assert_allclose(O.residual_paper_form(K, D, O.recon_3rdm_NY(D, N, sig)), -A,
                               atol=1e-12 * np.abs(A).max())
    assert np.abs(A + A.transpose(2, 3, 0, 1)).max() < 1e-12 * np.abs(A).max()
    U = O.update(A, D, N, sigma=sig)
    assert np.sum(K * U) == pytest.approx(-O.norm2(A), rel=1e-10)
    Av = O.residual(K, D, N)
    assert np.abs(A - Av).max() > 1e-4 * np.abs(Av).max()     # NY changes the residual
