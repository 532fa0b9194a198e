"""Seeded synthetic inputs for the ACSE hot path.

This module is shared by the CUDA library's tests and benchmark and by the FP64
oracle's tests. It draws the one- and two-electron integrals and builds the
reference 2-RDMs (Hartree-Fock determinants and exact CAS-CI states embedded in
a doubly occupied core). It contains none of the ACSE arithmetic itself: no
reduced Hamiltonian, no residual, no reconstruction, no update.

Workload shapes follow the paper's systems (Methods section: CASSCF or HF
references, spatial-orbital spin blocks); the integrals are synthetic because no
molecular integral code is available.

Spin-block layout used everywhere (spatial indices 0..r-1, row-major, full square):
    X_aa[i,j,k,l] = X^{i a, j a}_{k a, l a}
    X_ab[i,j,k,l] = X^{i a, j b}_{k a, l b}
    X_bb[i,j,k,l] = X^{i b, j b}_{k b, l b}
with 2-RDM normalisation D^{pq}_{rs} = 1/2 <a+_p a+_q a_s a_r>.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "rng_for", "make_integrals", "hf_rdm_blocks", "cas_rdm_blocks", "CASResult",
    "random_pair_tensor_blocks", "random_state_rdm_blocks", "random_ci_vector",
    "rdm_blocks_from_ci", "Problem", "make_problem",
    "config_problem", "batch_problems",
]


def rng_for(seed: int) -> np.random.Generator:
    """numpy PCG64 generator for a seed (every drawn array comes from one of these)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def make_integrals(r: int, seed: int):
    """Synthetic integrals shaped like molecular ones.

    h: symmetric r x r; diagonal U(-2, 1) sorted ascending; off-diagonal N(0, 0.05^2).
    V: chemist's notation (pq|rs) = sum_Q B^Q_pq B^Q_rs with 3r factors
       B^Q = 0.5^Q (G_Q + G_Q^T)/2, G_Q ~ N(0, 0.5^2) -> 8-fold symmetric, PSD.
    Returns (h, V) as float64 arrays of shapes (r, r) and (r, r, r, r).
    """
    rng = rng_for(seed)
    diag = np.sort(rng.uniform(-2.0, 1.0, size=r))
    off = rng.normal(0.0, 0.05, size=(r, r))
    h = np.triu(off, 1)
    h = h + h.T
    h[np.arange(r), np.arange(r)] = diag
    nq = 3 * r
    g = rng.normal(0.0, 0.5, size=(nq, r, r))
    scale = 0.5 ** np.arange(nq, dtype=np.float64)
    b = scale[:, None, None] * 0.5 * (g + g.transpose(0, 2, 1))
    bf = b.reshape(nq, r * r)
    V = (bf.T @ bf).reshape(r, r, r, r)
    return np.ascontiguousarray(h), np.ascontiguousarray(V)


def _det_blocks(occ_a, occ_b, r):
    ga = np.zeros((r, r)); ga[list(occ_a), list(occ_a)] = 1.0
    gb = np.zeros((r, r)); gb[list(occ_b), list(occ_b)] = 1.0
    daa = 0.5 * (np.einsum("ik,jl->ijkl", ga, ga) - np.einsum("jk,il->ijkl", ga, ga))
    dbb = 0.5 * (np.einsum("ik,jl->ijkl", gb, gb) - np.einsum("jk,il->ijkl", gb, gb))
    dab = 0.5 * np.einsum("ik,jl->ijkl", ga, gb)
    return tuple(np.ascontiguousarray(x) for x in (daa, dab, dbb))


def hf_rdm_blocks(r: int, n_alpha: int, n_beta: int):
    """2-RDM blocks of the determinant occupying orbitals 0..n_sigma-1 of each spin."""
    return _det_blocks(range(n_alpha), range(n_beta), r)


# ----------------------------------------------------------------------------------------
# Determinant CAS-CI (string-based), used only to produce reference 2-RDMs.
# ----------------------------------------------------------------------------------------

def _strings(norb, nel):
    return [sum(1 << o for o in c) for c in itertools.combinations(range(norb), nel)]


def _excitation_mats(norb, strs):
    """E[p, q] as dense (nstr, nstr) matrices for a+_p a_q within one spin."""
    index = {s: i for i, s in enumerate(strs)}
    ns = len(strs)
    E = np.zeros((norb, norb, ns, ns))
    for i, s in enumerate(strs):
        for q in range(norb):
            if not (s >> q) & 1:
                continue
            s1 = s & ~(1 << q)
            sg1 = -1.0 if bin(s & ((1 << q) - 1)).count("1") % 2 else 1.0
            for p in range(norb):
                if (s1 >> p) & 1:
                    continue
                s2 = s1 | (1 << p)
                sg2 = -1.0 if bin(s1 & ((1 << p) - 1)).count("1") % 2 else 1.0
                E[p, q, index[s2], i] = sg1 * sg2
    return E


@dataclass
class CASResult:
    Daa: np.ndarray
    Dab: np.ndarray
    Dbb: np.ndarray
    e_core: float
    e_cas: float
    energies: np.ndarray = field(repr=False)
    s2: float = 0.0


def cas_rdm_blocks(h, V, core, active, nelecas, root=0, nroots=None) -> CASResult:
    """Exact CAS-CI (Ms = 0) state `root` in orbitals `active` with `core` doubly occupied,
    its 2-RDM embedded into the full r-orbital space as spin blocks.

    The frozen-core CAS Hamiltonian uses h_eff = h + sum_c [2 (tu|cc) - (tc|cu)] and
    E_core = sum_c 2 h_cc + sum_cd [2 (cc|dd) - (cd|dc)].
    """
    r = h.shape[0]
    core = list(core); act = list(active)
    ncas = len(act)
    assert nelecas % 2 == 0, "Ms = 0 CAS only"
    nel_s = nelecas // 2
    hc = h[np.ix_(act, act)].copy()
    e_core = 0.0
    for c in core:
        hc += 2.0 * V[np.ix_(act, act, [c], [c])][:, :, 0, 0] - V[np.ix_(act, [c], [c], act)][:, 0, 0, :]
        e_core += 2.0 * h[c, c]
    for c in core:
        for d in core:
            e_core += 2.0 * V[c, c, d, d] - V[c, d, d, c]
    va = V[np.ix_(act, act, act, act)]
    strs = _strings(ncas, nel_s)
    ns = len(strs)
    E = _excitation_mats(ncas, strs)               # [p, q, J, I]
    # H = sum_ps h'_ps E_ps + 1/2 sum (pq|rs) E_pq E_rs with h' = h - 1/2 sum_q (pq|qs)
    hp = hc - 0.5 * np.einsum("pqqs->ps", va)
    Ef = E.reshape(ncas * ncas, ns, ns)
    vf = va.reshape(ncas * ncas, ncas * ncas)
    F = np.einsum("ab,bJI->aJI", vf, Ef)
    H1 = np.einsum("ps,psJI->JI", hp, E) + 0.5 * np.einsum("aJK,aKI->JI", Ef, F)
    # full matrix over (Ia, Ib): H1 (x) 1 + 1 (x) H1 + sum_{a,b} v_ab E_a (x) E_b
    eye = np.eye(ns)
    H = np.kron(H1, eye) + np.kron(eye, H1)
    Efl = Ef.reshape(ncas * ncas, ns * ns)
    cross = (Efl.T @ vf @ Efl).reshape(ns, ns, ns, ns)      # [Ja, Ia, Jb, Ib]
    H += cross.transpose(0, 2, 1, 3).reshape(ns * ns, ns * ns)
    H = 0.5 * (H + H.T)
    w, vecs = np.linalg.eigh(H)
    c = vecs[:, root].reshape(ns, ns)
    # active RDMs: gamma_a[p,q] = <E^a_pq>, D_aa = 1/2(<E_pr E_qs> - d_qr <E_ps>), D_ab = 1/2 <E^a_pr E^b_qs>
    T_a = np.einsum("pqJI,IB->pqJB", E, c)         # E^a_pq C
    T_b = np.einsum("AI,pqJI->pqAJ", c, E)         # C E^b_pq^T
    ga = np.einsum("JB,pqJB->pq", c, T_a)
    gb = np.einsum("AJ,pqAJ->pq", c, T_b)
    ee_a = np.einsum("rpJB,qsJB->pqrs", T_a, T_a)  # <E_rp C, E_qs C> = <E_pr E_qs>
    ee_b = np.einsum("rpAJ,qsAJ->pqrs", T_b, T_b)
    # <E^a_pr E^b_qs> = <E^a_rp C, C E^b_qs^T>
    ee_ab = np.einsum("rpJB,qsJB->pqrs", T_a, T_b)
    dl = np.eye(ncas)
    daa_act = 0.5 * (ee_a - np.einsum("qr,ps->pqrs", dl, ga))
    dbb_act = 0.5 * (ee_b - np.einsum("qr,ps->pqrs", dl, gb))
    dab_act = 0.5 * ee_ab
    # embed: Gamma2_full = Gamma2_act + wedge(g, g) - wedge(g_act, g_act), g = g_core + g_act
    gfa = np.zeros((r, r)); gfb = np.zeros((r, r))
    gfa[core, core] = 1.0; gfb[core, core] = 1.0
    gaa = np.zeros((r, r)); gbb = np.zeros((r, r))
    gaa[np.ix_(act, act)] = ga; gbb[np.ix_(act, act)] = gb
    ta = gfa + gaa; tb = gfb + gbb

    def wedge_same(x, y):
        return 0.5 * (np.einsum("ik,jl->ijkl", x, y) - np.einsum("jk,il->ijkl", x, y))

    Daa = wedge_same(ta, ta) - wedge_same(gaa, gaa)
    Dbb = wedge_same(tb, tb) - wedge_same(gbb, gbb)
    Dab = 0.5 * (np.einsum("ik,jl->ijkl", ta, tb) - np.einsum("ik,jl->ijkl", gaa, gbb))
    ix = np.ix_(act, act, act, act)
    Daa[ix] += daa_act; Dbb[ix] += dbb_act; Dab[ix] += dab_act
    Daa, Dab, Dbb = (np.ascontiguousarray(x) for x in (Daa, Dab, Dbb))
    # <S^2> = Ms^2 + Ms + N_beta - sum_pq <a+_pa a_qa a+_qb a_pb>; for Ms = 0 (spin-flip term)
    # <a+_pa a_qa a+_qb a_pb> = <E^a_pq E^b_qp>
    ee_ab_pq = np.einsum("qpJB,qpJB->", T_a, T_b)
    s2 = float(nel_s - ee_ab_pq)
    return CASResult(Daa, Dab, Dbb, float(e_core), float(w[root]), w, s2)


def random_pair_tensor_blocks(r: int, seed: int, hermitian: int = 1, scale: float = 1.0):
    """Random spin blocks of a pair tensor X^{pq}_{rs}: antisymmetric within each index pair
    (aa, bb blocks), and pair-Hermitian (hermitian=1), anti-Hermitian (-1) or neither (0).
    The ab block carries no intra-block antisymmetry."""
    rng = rng_for(seed)
    out = []
    for blk in ("aa", "ab", "bb"):
        x = rng.normal(0.0, scale, size=(r, r, r, r))
        if blk != "ab":
            x = 0.5 * (x - x.transpose(1, 0, 2, 3))
            x = 0.5 * (x - x.transpose(0, 1, 3, 2))
        if hermitian:
            x = 0.5 * (x + hermitian * x.transpose(2, 3, 0, 1))
        out.append(np.ascontiguousarray(x))
    return tuple(out)


def random_ci_vector(r: int, n_alpha: int, n_beta: int, seed: int):
    """A random normalised CI vector c[I_alpha, I_beta] over all determinants with
    (n_alpha, n_beta) electrons in r orbitals, with its alpha and beta occupation strings
    (bit p set = orbital p occupied; determinant = alpha string then beta string, each in
    ascending orbital order)."""
    sa = _strings(r, n_alpha); sb = _strings(r, n_beta)
    rng = rng_for(seed)
    c = rng.normal(size=(len(sa), len(sb)))
    return sa, sb, c / np.linalg.norm(c)


def rdm_blocks_from_ci(r, sa, sb, c):
    """2-RDM spin blocks of the state sum c[Ia, Ib] |Ia Ib>:
    D_aa = 1/2(<E^a_pr E^a_qs> - d_qr <E^a_ps>), D_ab = 1/2 <E^a_pr E^b_qs>, D_bb like D_aa."""
    Ea = _excitation_mats(r, sa); Eb = _excitation_mats(r, sb)
    T_a = np.einsum("pqJI,IB->pqJB", Ea, c)
    T_b = np.einsum("AI,pqJI->pqAJ", c, Eb)
    ga = np.einsum("JB,pqJB->pq", c, T_a)
    gb = np.einsum("AJ,pqAJ->pq", c, T_b)
    dl = np.eye(r)
    Daa = 0.5 * (np.einsum("rpJB,qsJB->pqrs", T_a, T_a) - np.einsum("qr,ps->pqrs", dl, ga))
    Dbb = 0.5 * (np.einsum("rpAJ,qsAJ->pqrs", T_b, T_b) - np.einsum("qr,ps->pqrs", dl, gb))
    Dab = 0.5 * np.einsum("rpJB,qsJB->pqrs", T_a, T_b)
    return tuple(np.ascontiguousarray(x) for x in (Daa, Dab, Dbb))


def random_state_rdm_blocks(r: int, n_alpha: int, n_beta: int, seed: int):
    """2-RDM blocks of a random normalised state with fixed (n_alpha, n_beta) spread over
    all r orbitals (a correlated, N-representable 2-RDM).  Feasible for r <= 8 or so."""
    sa, sb, c = random_ci_vector(r, n_alpha, n_beta, seed)
    return rdm_blocks_from_ci(r, sa, sb, c)


@dataclass
class Problem:
    """One ACSE instance: integrals, electron counts and an initial 2-RDM."""
    name: str
    r: int
    n_alpha: int
    n_beta: int
    h: np.ndarray
    V: np.ndarray
    Daa: np.ndarray
    Dab: np.ndarray
    Dbb: np.ndarray
    act_lo: int = 0
    act_hi: int = 0
    e_ref: float | None = None     # E_core + E_CAS (or HF closed form) of the reference

    @property
    def N(self):
        return self.n_alpha + self.n_beta


def make_problem(r, n_elec, seed, kind="hf", core=None, active=None, nelecas=None, root=0,
                 name=None):
    h, V = make_integrals(r, seed)
    if kind == "hf":
        na = nb = n_elec // 2
        Daa, Dab, Dbb = hf_rdm_blocks(r, na, nb)
        occ = range(na)
        e_ref = sum(2 * h[i, i] for i in occ) + sum(2 * V[i, i, j, j] - V[i, j, j, i] for i in occ for j in occ)
        return Problem(name or f"hf_r{r}_n{n_elec}_s{seed}", r, na, nb, h, V, Daa, Dab, Dbb, 0, 0, float(e_ref))
    res = cas_rdm_blocks(h, V, core, active, nelecas, root=root)
    na = nb = n_elec // 2
    return Problem(name or f"cas_r{r}_n{n_elec}_s{seed}_root{root}", r, na, nb, h, V,
                   res.Daa, res.Dab, res.Dbb, min(active), max(active) + 1,
                   res.e_core + res.e_cas)


def config_problem(idx: int, seed: int = 0) -> Problem:
    """The five benchmark systems (synthetic stand-ins for the paper's molecules).

    1: r=8,  N=8,  HF determinant, orbitals 0-3 doubly occupied.
    2: r=24, N=12, CAS(6e,6o) ground state in orbitals 4-9, core 0-2 (orbital 3 empty).
    3: r=48, N=20, CAS(8e,8o) ground state in orbitals 6-13, core 0-5.
    5: r=32, N=14, CAS(6e,6o) ground state in orbitals 4-9, core 0-3.
    (4 is the batch; see batch_problems.)
    """
    if idx == 1:
        return make_problem(8, 8, seed, "hf", name="cfg1_r8_hf")
    if idx == 2:
        return make_problem(24, 12, seed, "cas", core=range(0, 3), active=range(4, 10), nelecas=6,
                            name="cfg2_r24_cas66")
    if idx == 3:
        return make_problem(48, 20, seed, "cas", core=range(0, 6), active=range(6, 14), nelecas=8,
                            name="cfg3_r48_cas88")
    if idx == 5:
        return make_problem(32, 14, seed, "cas", core=range(0, 4), active=range(4, 10), nelecas=6,
                            name="cfg5_r32_cas66")
    raise ValueError(f"no single-instance config {idx}")


def batch_problems(seed: int = 0, rs=(12, 16, 20, 24, 28, 32, 36, 40)):
    """The batch: for each r, N = r/2, CAS(4e,4o) just above a doubly occupied core of
    (N-4)/2 orbitals; instance 2k is the ground state, 2k+1 the second Ms=0 root."""
    out = []
    for k, r in enumerate(rs):
        n = r // 2
        nc = (n - 4) // 2
        for root in (0, 1):
            out.append(make_problem(r, n, seed + k, "cas", core=range(0, nc),
                                    active=range(nc, nc + 4), nelecas=4, root=root,
                                    name=f"batch_r{r}_root{root}"))
    return out
