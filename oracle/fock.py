"""Brute-force Fock-space tools (Jordan-Wigner matrices) for pinning the oracle.
TEST INFRASTRUCTURE ONLY: imported by tests/, never by the CUDA library.

For n <= 8 spin orbitals the whole 2^n Fock space is held as dense matrices, so RDMs and
commutator expectations are computed straight from their definitions:
    2D^{pq}_{rs}   = 1/2 <psi| a+_p a+_q a_s a_r |psi>
    3D^{pqt}_{rsu} = 1/6 <psi| a+_p a+_q a+_t a_u a_s a_r |psi>
    <[a+_i a+_j a_l a_k, W^]>,   W^ = sum W^{pq}_{rs} a+_p a+_q a_s a_r
"""
from __future__ import annotations

import numpy as np


def annihilators(n):
    """a_p (p = 0..n-1) as dense 2^n x 2^n matrices; basis state bit p = occupation of p,
    Jordan-Wigner sign (-1)^(number of occupied q < p)."""
    dim = 1 << n
    ops = []
    for p in range(n):
        a = np.zeros((dim, dim))
        for s in range(dim):
            if (s >> p) & 1:
                sign = -1.0 if bin(s & ((1 << p) - 1)).count("1") % 2 else 1.0
                a[s & ~(1 << p), s] = sign
        ops.append(a)
    return ops


def sector_mask(n, N, n_alpha=None, r=None):
    """Basis states with N electrons (and n_alpha alpha electrons among the first r)."""
    s = np.arange(1 << n)
    cnt = np.array([bin(x).count("1") for x in s])
    m = cnt == N
    if n_alpha is not None:
        ca = np.array([bin(x & ((1 << r) - 1)).count("1") for x in s])
        m &= ca == n_alpha
    return m


def random_state(n, N, seed, n_alpha=None, r=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    m = sector_mask(n, N, n_alpha, r)
    psi = np.zeros(1 << n)
    psi[m] = rng.normal(size=int(m.sum()))
    return psi / np.linalg.norm(psi)


def determinant(n, occ):
    psi = np.zeros(1 << n)
    psi[sum(1 << o for o in occ)] = 1.0
    return psi


def rdm1(a, psi):
    n = len(a)
    v = np.array([a[r] @ psi for r in range(n)])         # a_r psi
    return v @ v.T                                        # <a+_p a_r> = <a_p psi, a_r psi>


def rdm2(a, psi):
    n = len(a)
    v = np.array([[a[s] @ (a[r] @ psi) for s in range(n)] for r in range(n)])   # v[r,s] = a_s a_r psi
    vf = v.reshape(n * n, -1)
    return 0.5 * (vf @ vf.T).reshape(n, n, n, n)


def rdm3(a, psi):
    n = len(a)
    w = np.zeros((n, n, n, psi.size))
    for r in range(n):
        x = a[r] @ psi
        for s in range(n):
            y = a[s] @ x
            for u in range(n):
                w[r, s, u] = a[u] @ y                      # a_u a_s a_r psi
    wf = w.reshape(n ** 3, -1)
    return (wf @ wf.T).reshape((n,) * 6) / 6.0


def two_body_op_apply(a, W, psi):
    """W^ psi with W^ = sum W^{pq}_{rs} a+_p a+_q a_s a_r."""
    n = len(a)
    out = np.zeros_like(psi)
    v = np.array([[a[s] @ (a[r] @ psi) for s in range(n)] for r in range(n)])
    t = np.einsum("pqrs,rsx->pqx", W, v)
    for p in range(n):
        for q in range(n):
            out += a[p].T @ (a[q].T @ t[p, q])
    return out


def two_body_op_apply_adj(a, W, psi):
    """W^+ psi = sum W^{pq}_{rs} a+_r a+_s a_q a_p psi (real W)."""
    return two_body_op_apply(a, W.transpose(2, 3, 0, 1), psi)


def commutator_expectation(a, W, psi):
    """C[i,j,k,l] = <psi|[a+_i a+_j a_l a_k, W^]|psi> for every i, j, k, l."""
    n = len(a)
    phi = two_body_op_apply(a, W, psi)        # W^ psi
    chi = two_body_op_apply_adj(a, W, psi)    # W^+ psi

    def pairs(x):
        return np.array([[a[j] @ (a[i] @ x) for j in range(n)] for i in range(n)]).reshape(n * n, -1)

    v = pairs(psi)     # v[ij] = a_j a_i psi
    u = pairs(phi)
    t = pairs(chi)
    # <psi|O W|psi> = <a_j a_i psi, a_l a_k W psi>;  <psi|W O|psi> = <a_j a_i W+ psi, a_l a_k psi>
    return (v @ u.T - t @ v.T).reshape(n, n, n, n)


def hamiltonian_matrix(a, h_so, g_so):
    """H = sum h_pr a+_p a_r + 1/2 sum g^{pq}_{rs} a+_p a+_q a_s a_r on the full Fock space
    (g^{pq}_{rs} = <pq|rs>, spin-orbital)."""
    n = len(a)
    dim = a[0].shape[0]
    H = np.zeros((dim, dim))
    for p in range(n):
        for r in range(n):
            if h_so[p, r] != 0.0:
                H += h_so[p, r] * (a[p].T @ a[r])
    P = np.array([[a[q] @ a[p] for q in range(n)] for p in range(n)])   # P[p,q] = a_q a_p
    F = np.tensordot(g_so, P, axes=([2, 3], [0, 1]))                    # sum_rs g^{pq}_{rs} a_s a_r
    Pt = P.transpose(0, 1, 3, 2)                                        # (a_q a_p)^T = a+_p a+_q
    H += 0.5 * np.tensordot(Pt, F, axes=([0, 1, 3], [0, 1, 2]))
    return H


def so_integrals(h, V):
    """Spin-orbital h and <PQ|RS> = (pr|qs) d(sP,sR) d(sQ,sS) from spatial (h, V)."""
    r = h.shape[0]
    n = 2 * r
    hs = np.zeros((n, n))
    hs[:r, :r] = h
    hs[r:, r:] = h
    g = np.zeros((n, n, n, n))
    for P in range(n):
        for Q in range(n):
            for R in range(n):
                for S in range(n):
                    if (P < r) == (R < r) and (Q < r) == (S < r):
                        g[P, Q, R, S] = V[P % r, R % r, Q % r, S % r]
    return hs, g
