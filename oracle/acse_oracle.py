"""FP64 reference oracle for the ACSE hot path.  TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg may
import this module.  The CUDA library never calls it and shares no code with it.

Everything here is plain numpy in the spin-orbital basis (n = 2r spin orbitals,
index P = p for alpha and P = r + p for beta), written from the paper's equations:

  * Eq. (1)-(2)       reduced two-body Hamiltonian K                 -> `reduced_hamiltonian`
  * RDM definitions    2D = 1/2 <a+a+aa>, 3D = 1/6 <a+a+a+aaa>
  * Appendix C         1D from 2D, cumulant 2Delta, M, Valdemoro 3D    -> `gamma`, `cumulant_M`, `recon_3rdm_V`
  * Eq. (residual)     six-term residual in 2D and 3D                  -> `residual_paper_form`
  * Appendix B         the same terms for a general pair operator W   -> `G_explicit`
  * Appendix C (V)     3D inserted into the residual without storing
                       it, with the intermediate E^{ij}_{kl}           -> `G_factored`
  * Eq. (update)       Euler step D <- D + eps U                       -> `update`, `step`
  * Methods            stopping rule on E, ||R|| and |dE| < 1e-6       -> `run_acse`
  * Eq. (NY), App. (NY) Nakatsuji-Yasuda 3-cumulant added to the V terms -> `sigma_hf`,
                       `cumulant3_NY`, `recon_3rdm_NY`, `_three_body_NY` (every driver
                       function takes sigma=None for V, the HF occupation signs for NY)

Readings of places where the paper is garbled or silent (each also pinned by tests):
  R1  K = 1/2(<pq|rs> - <pq|sr>) + (h_pr d_qs + h_qs d_pr - h_ps d_qr - h_qr d_ps)/(2(N-1)),
      <pq|rs> = (pr|qs); then H = 1/2 sum K a+_p a+_q a_s a_r and E = sum K.D   (Eq. 2)
  R2  A := <[a+_i a+_j a_l a_k, H]> equals MINUS the printed Eq. (residual)       (Eq. residual)
  R3  U := 1/2 <[a+_i a+_j a_l a_k, A^]>, A^ = sum A^{pq}_{rs} a+_p a+_q a_s a_r  (Eq. update)
  R4  1D = 2/(N-1) sum_q 2D^{pq}_{rq} over the full spin-orbital space             (App. C)
  R5  ||A||^2 is the spin-orbital Frobenius norm taken before the active mask      (Results)
  R6  the active mask zeroes A where all four spatial indices lie in [act_lo, act_hi)
  R7  spin blocks aa, ab, bb (Appendix A's labels all read aa); Tr D_ab = N_a N_b / 2     (App. A)
  R8  line search (not in the paper): f(eps) = ||A(D + eps U)||^2 at {0, e0, 2 e0};
      a merit flat to rounding (both trial values within 1e-10 f(0) of f(0)) -> e0/4; otherwise a
      convex parabola -> its minimiser clamped to [e0/4, 2 e0], else the better of e0, 2 e0;
      next e0 = accepted eps.
  R13 sigma_a of the NY cumulant: +1 for the first n_alpha alpha and the first n_beta beta spatial
      orbitals (aufbau by orbital index), -1 for the others.
All functions accept complex arrays too (complex-step derivatives): no abs(), no conj().
"""
from __future__ import annotations

import numpy as np

_EIN = dict(optimize=True)


# ----------------------------------------------------------------------------------------
# spin blocks <-> spin-orbital tensors (the oracle's own mapping)
# ----------------------------------------------------------------------------------------

def so_from_blocks(Xaa, Xab, Xbb):
    """Spin-orbital pair tensor X^{PQ}_{RS} from its aa, ab, bb blocks; the ba-ordered
    pieces follow from antisymmetry within each index pair."""
    r = Xaa.shape[0]
    n = 2 * r
    X = np.zeros((n, n, n, n), dtype=np.result_type(Xaa, Xab, Xbb))
    a = slice(0, r)
    b = slice(r, n)
    X[a, a, a, a] = Xaa
    X[b, b, b, b] = Xbb
    X[a, b, a, b] = Xab
    X[b, a, b, a] = Xab.transpose(1, 0, 3, 2)
    X[a, b, b, a] = -Xab.transpose(0, 1, 3, 2)
    X[b, a, a, b] = -Xab.transpose(1, 0, 2, 3)
    return X


def blocks_from_so(X):
    n = X.shape[0]
    r = n // 2
    a = slice(0, r)
    b = slice(r, n)
    return (np.ascontiguousarray(X[a, a, a, a]), np.ascontiguousarray(X[a, b, a, b]),
            np.ascontiguousarray(X[b, b, b, b]))


def so_one_body(xa, xb=None):
    """Block-diagonal spin-orbital one-body matrix from alpha (and beta) blocks."""
    xb = xa if xb is None else xb
    r = xa.shape[0]
    out = np.zeros((2 * r, 2 * r), dtype=np.result_type(xa, xb))
    out[:r, :r] = xa
    out[r:, r:] = xb
    return out


# ----------------------------------------------------------------------------------------
# Hamiltonian, RDMs, reconstruction
# ----------------------------------------------------------------------------------------

def reduced_hamiltonian(h, V, N):
    """Spin-orbital reduced Hamiltonian K (reading R1 of Eq. 2).

    h: (r, r) one-electron integrals; V: (r,r,r,r) chemist's (pq|rs); N electrons.
    """
    r = h.shape[0]
    n = 2 * r
    hs = so_one_body(h)
    sp = np.zeros(n, dtype=int)
    sp[r:] = 1
    orb = np.arange(n) % r
    same = (sp[:, None] == sp[None, :]).astype(float)
    # <PQ|RS> = (pr|qs) d(sP,sR) d(sQ,sS)
    Vsp = V[np.ix_(orb, orb, orb, orb)]                      # (pr|qs) indexed [P,R,Q,S]
    g = Vsp.transpose(0, 2, 1, 3) * same[:, None, :, None] * same[None, :, None, :]   # [P,Q,R,S]
    I = np.eye(n)
    one = (np.einsum("pr,qs->pqrs", hs, I) + np.einsum("qs,pr->pqrs", hs, I)
           - np.einsum("ps,qr->pqrs", hs, I) - np.einsum("qr,ps->pqrs", hs, I)) / (2.0 * (N - 1))
    return 0.5 * (g - g.transpose(0, 1, 3, 2)) + one


def energy(K, D):
    """E = sum_{pqrs} K^{pq}_{rs} 2D^{pq}_{rs} (Eq. 2 with reading R1)."""
    return np.sum(K * D)


def trace2(D):
    return np.einsum("pqpq->", D)


def gamma(D, N):
    """1-RDM from the 2-RDM: 1D^p_r = 2/(N-1) sum_q 2D^{pq}_{rq} (reading R4)."""
    return (2.0 / (N - 1)) * np.einsum("pqrq->pr", D)


def wedge11(g):
    """(1D ^ 1D)^{ij}_{rq} = 1/2 (1D^i_r 1D^j_q - 1D^j_r 1D^i_q)  (App. C expansion)."""
    return 0.5 * (np.einsum("ir,jq->ijrq", g, g) - np.einsum("jr,iq->ijrq", g, g))


def cumulant_M(D, g):
    """2-cumulant 2Delta = 2D - 1D^1D and M = 3 2Delta + 1D^1D  (App. C)."""
    gg = wedge11(g)
    delta = D - gg
    return 3.0 * delta + gg, delta


def recon_3rdm_V(D, N):
    """Valdemoro 3-RDM, 3D^{ijp}_{rql} stored as D3[i,j,p,r,q,l]: the nine signed M.1D
    terms of Eq. (3rdm_recon) divided by 9, with 3Delta = 0.  O(n^6) memory: tiny n only."""
    g = gamma(D, N)
    M, _ = cumulant_M(D, g)
    e = np.einsum
    D3 = (e("ijrq,pl->ijprql", M, g) - e("ijlq,pr->ijprql", M, g) - e("ijrl,pq->ijprql", M, g)
          - e("iprq,jl->ijprql", M, g) + e("iplq,jr->ijprql", M, g) + e("iprl,jq->ijprql", M, g)
          + e("jprq,il->ijprql", M, g) - e("jplq,ir->ijprql", M, g) - e("jprl,iq->ijprql", M, g))
    return D3 / 9.0


def sigma_hf(r, n_alpha, n_beta):
    """sigma_a of the NY functional (Eq. NY): +1 for spin orbitals occupied in the Hartree-Fock
    reference, -1 otherwise; reading R13: aufbau by orbital index, the first n_alpha alpha and the first
    n_beta beta spatial orbitals occupied."""
    sig = -np.ones(2 * r)
    sig[:n_alpha] = 1.0
    sig[r:r + n_beta] = 1.0
    return sig


def _perm_sign(p):
    s = 1
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if p[i] > p[j]:
                s = -s
    return s


def cumulant3_NY(delta, sig):
    """NY 3-cumulant (Eq. NY, stored as C3[i,j,p,r,q,l] = 3Delta^{ijp}_{rql}): 1/6 sum_a sigma_a A(...)
    with A the antisymmetriser over the upper (i,j,p) and the lower (r,q,l) indices of
    2Delta^{ia}_{rq} 2Delta^{jp}_{al} (all 36 signed permutations, a fixed).  O(n^6) memory: tiny n only."""
    from itertools import permutations
    X = np.einsum("a,iarq,jpal->ijprql", sig, delta, delta)
    out = np.zeros_like(X)
    for pu in permutations(range(3)):
        for pl in permutations(range(3)):
            out = out + _perm_sign(pu) * _perm_sign(pl) * X.transpose(list(pu) + [3 + x for x in pl])
    return out / 6.0


def cumulant3_NY_simplified(delta, sig):
    """The nine-term form of the same cumulant printed in the appendix (pair antisymmetry of 2Delta
    collapses the 36 terms four by four)."""
    e = np.einsum
    t = (4 * e("a,iarq,jpal->ijprql", sig, delta, delta) - 4 * e("a,jarq,ipal->ijprql", sig, delta, delta)
         - 4 * e("a,parq,jial->ijprql", sig, delta, delta) - 4 * e("a,ialq,jpar->ijprql", sig, delta, delta)
         + 4 * e("a,jalq,ipar->ijprql", sig, delta, delta) + 4 * e("a,palq,jiar->ijprql", sig, delta, delta)
         - 4 * e("a,iarl,jpaq->ijprql", sig, delta, delta) + 4 * e("a,jarl,ipaq->ijprql", sig, delta, delta)
         + 4 * e("a,parl,jiaq->ijprql", sig, delta, delta))
    return t / 6.0


def recon_3rdm_NY(D, N, sig):
    """NY 3-RDM: the Valdemoro terms plus the NY 3-cumulant (tiny n only)."""
    g = gamma(D, N)
    _, delta = cumulant_M(D, g)
    return recon_3rdm_V(D, N) + cumulant3_NY(delta, sig)


def _three_body_NY(W, delta, sig):
    """sum_{pqr} W^{kp}_{rq} 3Delta^{ijp}_{rql} with the nine-term NY cumulant, each term contracted
    directly (numpy chooses the pairwise order; 3Delta is never formed)."""
    e = lambda s_, *a: np.einsum(s_, *a, **_EIN)
    d = delta
    t = (4 * e("kprq,a,iarq,jpal->ijkl", W, sig, d, d) - 4 * e("kprq,a,jarq,ipal->ijkl", W, sig, d, d)
         - 4 * e("kprq,a,parq,jial->ijkl", W, sig, d, d) - 4 * e("kprq,a,ialq,jpar->ijkl", W, sig, d, d)
         + 4 * e("kprq,a,jalq,ipar->ijkl", W, sig, d, d) + 4 * e("kprq,a,palq,jiar->ijkl", W, sig, d, d)
         - 4 * e("kprq,a,iarl,jpaq->ijkl", W, sig, d, d) + 4 * e("kprq,a,jarl,ipaq->ijkl", W, sig, d, d)
         + 4 * e("kprq,a,parl,jiaq->ijkl", W, sig, d, d))
    return t / 6.0


# ----------------------------------------------------------------------------------------
# residual and update contractions
# ----------------------------------------------------------------------------------------

def residual_paper_form(K, D, D3):
    """Eq. (residual) exactly as printed (with the K of reading R1):
    R = sum 2K^{ij}_{qp}D^{kl}_{qp} + 6K^{kp}_{rq}D3^{ijp}_{rql} - 6K^{lp}_{rq}D3^{ijp}_{rqk}
        - 2K^{kl}_{qp}D^{ij}_{qp} - 6K^{pq}_{ri}D3^{jpq}_{rlk} + 6K^{pq}_{rj}D3^{ipq}_{rlk}.
    Reading R2: the commutator <[O, H]> is -R."""
    e = lambda s, *a: np.einsum(s, *a, **_EIN)
    return (2 * e("ijqp,klqp->ijkl", K, D) + 6 * e("kprq,ijprql->ijkl", K, D3)
            - 6 * e("lprq,ijprqk->ijkl", K, D3) - 2 * e("klqp,ijqp->ijkl", K, D)
            - 6 * e("pqri,jpqrlk->ijkl", K, D3) + 6 * e("pqrj,ipqrlk->ijkl", K, D3))


def G_explicit(W, D, D3):
    """<[a+_i a+_j a_l a_k, sum W^{pq}_{rs} a+_p a+_q a_s a_r]> from 2D and a stored 3D.

    The Appendix B form that precedes the use of K's Hermiticity (terms 2W^{pq}_{ji}2D^{pq}_{lk}
    and -6W^{pq}_{ri}3D^{jpq}_{rlk} keep W's own index order), with K -> 2W and the overall
    sign of reading R2; valid for any W antisymmetric within each index pair."""
    e = lambda s, *a: np.einsum(s, *a, **_EIN)
    R = (2 * e("pqji,pqlk->ijkl", W, D) + 6 * e("kprq,ijprql->ijkl", W, D3)
         - 6 * e("lprq,ijprqk->ijkl", W, D3) - 2 * e("klqp,ijqp->ijkl", W, D)
         - 6 * e("pqri,jpqrlk->ijkl", W, D3) + 6 * e("pqrj,ipqrlk->ijkl", W, D3))
    return -2.0 * R


def _three_body_V(W, M, g):
    """sum_{pqr} W^{kp}_{rq} 3D^{ijp}_{rql} with the Valdemoro 3D inserted (App. C, V):
    1/9 [ sum W^{kp}_{rq} M^{ij}_{rq} 1D^p_l - (W^{kp}_{rq} - W^{kp}_{qr}) M^{ij}_{lq} 1D^p_r
          + E^{ij}_{kl} - E^{ji}_{kl} ],
    E^{ij}_{kl} = sum (W^{kp}_{rq} - W^{kp}_{qr}) M^{ip}_{lq} 1D^j_r - W^{kp}_{rq} M^{ip}_{rq} 1D^j_l.
    Never forms 3D."""
    e = lambda s, *a: np.einsum(s, *a, **_EIN)
    Wd = W - W.transpose(0, 1, 3, 2)
    t1 = e("kprq,ijrq,pl->ijkl", W, M, g)
    t2 = e("kprq,ijlq,pr->ijkl", Wd, M, g)
    E = e("kprq,iplq,jr->ijkl", Wd, M, g) - e("kprq,iprq,jl->ijkl", W, M, g)
    return (t1 - t2 + E - E.transpose(1, 0, 2, 3)) / 9.0


def G_factored(W, D, N, sigma=None):
    """Same value as G_explicit(W, D, recon_3rdm_V(D, N)) without ever holding 3D; with sigma given,
    the same with the NY 3-RDM (recon_3rdm_NY(D, N, sigma)), whose cumulant is Hermitian too.

    The six terms of G_explicit: two 2D terms and four 3D terms; each 3D term is a relabelling
    of sum W^{kp}_{rq} 3D^{ijp}_{rql} (for W^{pq}_{ri} 3D^{jpq}_{rlk} by the Hermiticity of
    3D, which holds for the reconstruction because M and 1D are Hermitian)."""
    e = lambda s, *a: np.einsum(s, *a, **_EIN)
    g = gamma(D, N)
    M, delta = cumulant_M(D, g)
    two = 2 * e("pqji,pqlk->ijkl", W, D) - 2 * e("klqp,ijqp->ijkl", W, D)
    T = _three_body_V(W, M, g)                     # T^{ij}_{kl} = sum W^{kp}_{rq} 3D^{ijp}_{rql}
    if sigma is not None:
        T = T + _three_body_NY(W, delta, sigma)
    # sum W^{pq}_{ri} 3D^{jpq}_{rlk}: 3D^{jpq}_{rlk} = 3D^{rlk}_{jpq} = 3D^{lkr}_{pqj} (cyclic)
    # so the sum equals  sum_{pqr} Wt^{ir}_{pq} 3D^{lkr}_{pqj} = T'(Wt)^{lk}_{ij}, Wt^{ir}_{pq} = W^{pq}_{ri}
    Wt = W.transpose(3, 2, 0, 1)                   # Wt[i,r,p,q] = W[p,q,r,i]
    Tt = _three_body_V(Wt, M, g)                   # Tt^{ab}_{cd} = sum Wt^{cp}_{rq} 3D^{abp}_{rqd}
    if sigma is not None:
        Tt = Tt + _three_body_NY(Wt, delta, sigma)
    # term5:  sum W^{pq}_{ri} 3D^{jpq}_{rlk} = Tt^{lk}_{ij}
    t5 = Tt.transpose(2, 3, 1, 0)                  # [i,j,k,l] <- Tt[l,k,i,j]
    t6 = Tt.transpose(3, 2, 1, 0)                  # [i,j,k,l] <- Tt[l,k,j,i]
    R = two + 6 * T - 6 * T.transpose(0, 1, 3, 2) - 6 * t5 + 6 * t6
    return -2.0 * R


def _recon(D, N, sigma):
    return recon_3rdm_V(D, N) if sigma is None else recon_3rdm_NY(D, N, sigma)


def residual(K, D, N, explicit=False, sigma=None):
    """A = <[a+_i a+_j a_l a_k, H]> = G(K/2) (readings R1, R2); V reconstruction, or NY when the
    HF occupation signs sigma are given."""
    if explicit:
        return G_explicit(0.5 * K, D, _recon(D, N, sigma))
    return G_factored(0.5 * K, D, N, sigma)


def update(A, D, N, explicit=False, sigma=None):
    """U = 1/2 <[a+_i a+_j a_l a_k, A^]> with the same reconstructed 3D (reading R3, Eq. update)."""
    if explicit:
        return 0.5 * G_explicit(A, D, _recon(D, N, sigma))
    return 0.5 * G_factored(A, D, N, sigma)


def norm2(A):
    """Spin-orbital ||A||^2 = sum A*A (complex-step safe; reading R5)."""
    return np.sum(A * A)


def active_mask(A, r, act_lo, act_hi):
    """Zero A^{ij}_{kl} where all four spatial indices are active (reading R6)."""
    n = A.shape[0]
    act = np.zeros(n, dtype=bool)
    for p in range(n):
        act[p] = act_lo <= (p % r) < act_hi
    m = act[:, None, None, None] & act[None, :, None, None] & act[None, None, :, None] & act[None, None, None, :]
    out = A.copy()
    out[m] = 0.0
    return out


# ----------------------------------------------------------------------------------------
# step, line search, driver
# ----------------------------------------------------------------------------------------

def step(K, D, N, eps, mask=None, sigma=None):
    """One Euler step of Eq. (update): returns (D_next, A, U) with A evaluated at D."""
    A = residual(K, D, N, sigma=sigma)
    Am = A if mask is None else active_mask(A, *mask)
    U = update(Am, D, N, sigma=sigma)
    return D + eps * U, A, U


LS_FLAT = 1e-10   # reading R8: trial values this close to f(0) (relative) are rounding, not a slope


def line_search_eps(f0, f1, f2, e0):
    """Reading R8: choose eps from f at {0, e0, 2 e0}."""
    if abs(f1 - f0) <= LS_FLAT * abs(f0) and abs(f2 - f0) <= LS_FLAT * abs(f0):
        return 0.25 * e0
    c = (f2 - 2.0 * f1 + f0) / (2.0 * e0 * e0)
    if c > 0.0:
        b = (f1 - f0) / e0 - c * e0
        x = -b / (2.0 * c)
        return min(max(x, 0.25 * e0), 2.0 * e0)
    return e0 if f1 <= f2 else 2.0 * e0


def run_acse(h, V, N, D0, eps, nsteps, line_search=False, mask=None, stop_rule=False,
             eps0=1e-3, log=None, sigma=None):
    """The Euler-step driver.  Returns dict(D, E[list], norm2[list], eps[list], steps).

    E[n], norm2[n] are at D_n (E[0] at the reference).  With stop_rule the loop ends when E
    or ||A|| increases (returning the previous D) or |dE| < 1e-6 Eh (Methods)."""
    K = reduced_hamiltonian(h, V, N)
    D = D0
    Es = [energy(K, D)]
    ns = []
    epss = []
    e_ls = eps0
    A = residual(K, D, N, sigma=sigma)
    for n in range(nsteps):
        ns.append(norm2(A))
        Am = A if mask is None else active_mask(A, *mask)
        U = update(Am, D, N, sigma=sigma)
        if line_search:
            f0 = ns[-1]
            A1 = residual(K, D + e_ls * U, N, sigma=sigma)
            A2 = residual(K, D + 2 * e_ls * U, N, sigma=sigma)
            e_use = line_search_eps(f0, norm2(A1), norm2(A2), e_ls)
            e_ls = e_use
        else:
            e_use = eps
        Dn = D + e_use * U
        En = energy(K, Dn)
        An = residual(K, Dn, N, sigma=sigma)
        if stop_rule:
            if En > Es[-1] or norm2(An) > ns[-1]:
                break
            conv = abs(En - Es[-1]) < 1e-6
        D, A = Dn, An
        Es.append(En)
        epss.append(e_use)
        if log is not None:
            log(n, En, ns[-1], e_use)
        if stop_rule and conv:
            break
    ns.append(norm2(A))
    return dict(D=D, E=Es, norm2=ns, eps=epss, steps=len(epss))


def objective(h, V, N, D0, eps, nsteps, wE=1.0, wN=0.0, mask=None, sigma=None):
    """wE * E(D_n) + wN * ||A(D_n)||^2 after n fixed Euler steps from D0 (the function the
    adjoint differentiates).  Polynomial in (h, V, D0): complex-step exact."""
    K = reduced_hamiltonian(h, V, N)
    D = D0
    for _ in range(nsteps):
        D, _, _ = step(K, D, N, eps, mask, sigma)
    A = residual(K, D, N, sigma=sigma)
    return wE * energy(K, D) + wN * norm2(A)


def complex_step_dir(h, V, N, D0, eps, nsteps, dh, dV, dD0, wE=1.0, wN=0.0, mask=None, t=1e-30, sigma=None):
    """Directional derivative of `objective` along (dh, dV, dD0), exact to rounding
    (complex step: Im f(x + i t d) / t)."""
    f = objective(h + 1j * t * dh, V + 1j * t * dV, N, D0 + 1j * t * dD0, eps, nsteps, wE, wN, mask, sigma)
    return float(np.imag(f) / t)


# ----------------------------------------------------------------------------------------
# single entries at any size (sampled parity)
# ----------------------------------------------------------------------------------------

def d3_elements(M, g, a, b, c, d, e, f):
    """3D^{abc}_{def} from Eq. (3rdm_recon) with 3Delta = 0, for integer or broadcastable index
    arrays; (a,b,c,d,e,f) play the roles of (i,j,p,r,q,l) there."""
    return (M[a, b, d, e] * g[c, f] - M[a, b, f, e] * g[c, d] - M[a, b, d, f] * g[c, e]
            - M[a, c, d, e] * g[b, f] + M[a, c, f, e] * g[b, d] + M[a, c, d, f] * g[b, e]
            + M[b, c, d, e] * g[a, f] - M[b, c, f, e] * g[a, d] - M[b, c, d, f] * g[a, e]) / 9.0


def residual_entries(h, V, N, Daa, Dab, Dbb, entries):
    """A^{ij}_{kl} (spin-orbital indices) for each (i, j, k, l) in `entries`: the printed
    Eq. (residual) term by term, with each 3D element evaluated from the nine M.1D terms and
    the overall sign of reading R2.  Holds K, 2D and M (n^4 each) but never 3D."""
    K = reduced_hamiltonian(h, V, N)
    D = so_from_blocks(Daa, Dab, Dbb)
    g = gamma(D, N)
    M, _ = cumulant_M(D, g)
    n = D.shape[0]
    P = np.arange(n)[:, None, None]
    Rr = np.arange(n)[None, :, None]
    Qq = np.arange(n)[None, None, :]
    out = []
    for (i, j, k, l) in entries:
        t = 2.0 * np.sum(K[i, j] * D[k, l]) - 2.0 * np.sum(K[k, l] * D[i, j])
        t += 6.0 * np.sum(K[k][P, Rr, Qq] * d3_elements(M, g, i, j, P, Rr, Qq, l))
        t -= 6.0 * np.sum(K[l][P, Rr, Qq] * d3_elements(M, g, i, j, P, Rr, Qq, k))
        # (p, q, r) grids for the last two terms: K^{pq}_{ri} 3D^{jpq}_{rlk}
        t -= 6.0 * np.sum(K[P, Rr, Qq, i] * d3_elements(M, g, j, P, Rr, Qq, l, k))
        t += 6.0 * np.sum(K[P, Rr, Qq, j] * d3_elements(M, g, i, P, Rr, Qq, l, k))
        out.append(-t)
    return np.array(out)
